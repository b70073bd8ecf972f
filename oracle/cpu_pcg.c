/*
 * Same-method CPU statement of the BURA solve (oracle) -- TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, the smoke check and the CPU-baseline legs of bench.py load this file's library; the
 * CUDA product path never does, and it shares no code with it.
 *
 * What it computes (eq. (Rgeneral), Sec. 2.2): for weights c_j and shifts d_j <= 0,
 *     u = sum_j c_j v_j,    (A - d_j I) v_j = f,
 * A = Atilde / Lambda the scaled finite-difference matrix of -div(a grad u) on a uniform interior grid
 * of the unit square / cube with homogeneous Dirichlet data (eq. (algebraic), Sec. 1.4).  Each shifted
 * system is solved on its own, one after the other, by the preconditioned conjugate gradient method
 * (the paper solves the k+1 systems by PCG with an algebraic multigrid preconditioner, Sec. 5.4; here
 * the preconditioner is a plain geometric multigrid V-cycle), in FP64, to a relative residual rtol.
 *
 * Operator.  Points are numbered lexicographically, x fastest.  With face coefficients a (arrays of the
 * shapes (nz, ny, nx+1), (nz, ny+1, nx), (nz+1, ny, nx); NULL means a = 1) and h_x = 1/(nx+1):
 *     (Atilde x)_P = sum over the faces F of P:  a_F (x_P - x_Q(F)) / h_F^2,   x_Q = 0 outside the grid.
 * Multigrid.  Levels n -> (n-1)/2 per axis while every n is odd and >= 3 (coarse node I is fine node
 * 2I+1).  Coarse face coefficients: the two fine faces on the line through the coarse nodes in series
 * (harmonic mean); each level is the rediscretised operator with its own mesh size, scaled by the same
 * Lambda, shifted by the same d.  Restriction: full weighting (1/4, 1/2, 1/4 per axis); prolongation:
 * its transpose times 2^dim (linear interpolation).  Smoother: damped Jacobi, weight 2/(2 + 1/dim),
 * two sweeps before and two after (a symmetric V-cycle, so the preconditioner is SPD).  Coarsest
 * level: a dense Cholesky factorisation when it has at most 1024 points, else 40 Jacobi sweeps.
 * Threads: OpenMP over the two slowest grid axes; dot products in a fixed per-thread order.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int nx, ny, nz;
    long N;
    double *fx, *fy, *fz;  /* scaled face weights a_F / (h_F^2 Lambda); fz NULL in 2D */
    double *x, *b, *r;     /* level vectors (x, b unused on the finest level of a V-cycle's caller) */
    double *chol;          /* coarsest level: dense Cholesky factor (lower, row major), or NULL */
} level;

typedef struct {
    int dim, nlev;
    level lev[32];
    double shift;          /* the d of the system being solved */
} hierarchy;

static long idx3(const level* L, int i, int j, int l) { return ((long)l * L->ny + j) * L->nx + i; }

/* face weight arrays of one axis, with their index helpers */
static double xface(const level* L, int i, int j, int l) { return L->fx[((long)l * L->ny + j) * (L->nx + 1) + i]; }
static double yface(const level* L, int i, int j, int l) { return L->fy[((long)l * (L->ny + 1) + j) * L->nx + i]; }
static double zface(const level* L, int i, int j, int l) { return L->fz[((long)l * L->ny + j) * L->nx + i]; }

static double diag_at(const level* L, int i, int j, int l, double d) {
    double s = xface(L, i, j, l) + xface(L, i + 1, j, l) + yface(L, i, j, l) + yface(L, i, j + 1, l);
    if (L->fz) s += zface(L, i, j, l) + zface(L, i, j, l + 1);
    return s - d;
}

/* ((A - d I) x)_P */
static double apply_at(const level* L, const double* x, int i, int j, int l, double d) {
    const long P = idx3(L, i, j, l);
    double s = diag_at(L, i, j, l, d) * x[P];
    if (i > 0) s -= xface(L, i, j, l) * x[P - 1];
    if (i < L->nx - 1) s -= xface(L, i + 1, j, l) * x[P + 1];
    if (j > 0) s -= yface(L, i, j, l) * x[P - L->nx];
    if (j < L->ny - 1) s -= yface(L, i, j + 1, l) * x[P + L->nx];
    if (L->fz) {
        const long pl = (long)L->nx * L->ny;
        if (l > 0) s -= zface(L, i, j, l) * x[P - pl];
        if (l < L->nz - 1) s -= zface(L, i, j, l + 1) * x[P + pl];
    }
    return s;
}

static void apply(const level* L, const double* x, double* y, double d) {
    int l, j;
#pragma omp parallel for collapse(2) schedule(static)
    for (l = 0; l < L->nz; ++l)
        for (j = 0; j < L->ny; ++j)
            for (int i = 0; i < L->nx; ++i) y[idx3(L, i, j, l)] = apply_at(L, x, i, j, l, d);
}

/* x_new = x + w D^{-1} (b - (A - dI) x), Jacobi (reads x, writes tmp, then copies) */
static void jacobi(const level* L, const double* b, double* x, double* tmp, double d, double w) {
    int l, j;
#pragma omp parallel for collapse(2) schedule(static)
    for (l = 0; l < L->nz; ++l)
        for (j = 0; j < L->ny; ++j)
            for (int i = 0; i < L->nx; ++i) {
                const long P = idx3(L, i, j, l);
                tmp[P] = x[P] + w * (b[P] - apply_at(L, x, i, j, l, d)) / diag_at(L, i, j, l, d);
            }
    long q;
#pragma omp parallel for schedule(static)
    for (q = 0; q < L->N; ++q) x[q] = tmp[q];
}

/* bc = R (b - (A - dI) x): full weighting of the residual onto the coarse level */
static void restrict_residual(const level* F, const level* Cl, const double* x, const double* b, double* bc,
                              double d, int dim) {
    static const double w1[3] = {0.25, 0.5, 0.25};
    int L, J;
#pragma omp parallel for collapse(2) schedule(static)
    for (L = 0; L < Cl->nz; ++L)
        for (J = 0; J < Cl->ny; ++J)
            for (int I = 0; I < Cl->nx; ++I) {
                double s = 0.0;
                const int zl = dim == 3 ? -1 : 0, zh = dim == 3 ? 1 : 0;
                for (int dz = zl; dz <= zh; ++dz)
                    for (int dy = -1; dy <= 1; ++dy)
                        for (int dx = -1; dx <= 1; ++dx) {
                            const int i = 2 * I + 1 + dx, j = 2 * J + 1 + dy, l = dim == 3 ? 2 * L + 1 + dz : 0;
                            const double wt = w1[dx + 1] * w1[dy + 1] * (dim == 3 ? w1[dz + 1] : 1.0);
                            s += wt * (b[idx3(F, i, j, l)] - apply_at(F, x, i, j, l, d));
                        }
                bc[idx3(Cl, I, J, L)] = s;
            }
}

/* x += P xc: linear interpolation of the coarse correction (coarse node I at fine node 2I+1) */
static double coarse_val(const level* Cl, const double* xc, int I, int J, int L) {
    if (I < 0 || J < 0 || L < 0 || I >= Cl->nx || J >= Cl->ny || L >= Cl->nz) return 0.0;
    return xc[idx3(Cl, I, J, L)];
}

static void prolong_add(const level* F, const level* Cl, const double* xc, double* x, int dim) {
    int l, j;
#pragma omp parallel for collapse(2) schedule(static)
    for (l = 0; l < F->nz; ++l)
        for (j = 0; j < F->ny; ++j)
            for (int i = 0; i < F->nx; ++i) {
                /* per axis: an odd fine index sits on a coarse node, an even one between two */
                int lo[3], hi[3];
                double wl[3], wh[3];
                const int f[3] = {i, j, l};
                for (int a = 0; a < 3; ++a) {
                    if (a >= dim) { lo[a] = hi[a] = 0; wl[a] = 1.0; wh[a] = 0.0; continue; }
                    if (f[a] % 2 == 1) { lo[a] = hi[a] = (f[a] - 1) / 2; wl[a] = 1.0; wh[a] = 0.0; }
                    else { lo[a] = f[a] / 2 - 1; hi[a] = f[a] / 2; wl[a] = 0.5; wh[a] = 0.5; }
                }
                double s = 0.0;
                for (int cz = 0; cz < 2; ++cz)
                    for (int cy = 0; cy < 2; ++cy)
                        for (int cx = 0; cx < 2; ++cx) {
                            const double wt = (cx ? wh[0] : wl[0]) * (cy ? wh[1] : wl[1]) * (cz ? wh[2] : wl[2]);
                            if (wt == 0.0) continue;
                            s += wt * coarse_val(Cl, xc, cx ? hi[0] : lo[0], cy ? hi[1] : lo[1], cz ? hi[2] : lo[2]);
                        }
                x[idx3(F, i, j, l)] += s;
            }
}

/* dense (A - dI) of a small level, then its Cholesky factor in place (lower triangle) */
static int coarse_factor(level* L, double d) {
    const long n = L->N;
    double* M = L->chol;
    double* e = (double*)calloc((size_t)n, sizeof(double));
    double* col = (double*)malloc(sizeof(double) * (size_t)n);
    if (!e || !col) { free(e); free(col); return -1; }
    for (long q = 0; q < n; ++q) {  /* column q of A - dI */
        e[q] = 1.0;
        for (int l = 0; l < L->nz; ++l)
            for (int j = 0; j < L->ny; ++j)
                for (int i = 0; i < L->nx; ++i) col[idx3(L, i, j, l)] = apply_at(L, e, i, j, l, d);
        for (long p = 0; p < n; ++p) M[p * n + q] = col[p];
        e[q] = 0.0;
    }
    free(e);
    free(col);
    for (long k = 0; k < n; ++k) {
        double s = M[k * n + k];
        for (long m = 0; m < k; ++m) s -= M[k * n + m] * M[k * n + m];
        if (!(s > 0)) return -2;
        M[k * n + k] = sqrt(s);
        for (long p = k + 1; p < n; ++p) {
            double t = M[p * n + k];
            for (long m = 0; m < k; ++m) t -= M[p * n + m] * M[k * n + m];
            M[p * n + k] = t / M[k * n + k];
        }
    }
    return 0;
}

static void coarse_solve(const level* L, const double* b, double* x) {
    const long n = L->N;
    const double* M = L->chol;
    for (long p = 0; p < n; ++p) {  /* forward: G y = b */
        double s = b[p];
        for (long m = 0; m < p; ++m) s -= M[p * n + m] * x[m];
        x[p] = s / M[p * n + p];
    }
    for (long p = n - 1; p >= 0; --p) {  /* backward: G^T x = y */
        double s = x[p];
        for (long m = p + 1; m < n; ++m) s -= M[m * n + p] * x[m];
        x[p] = s / M[p * n + p];
    }
}

/* x = V-cycle(b) on level k with a zero initial guess */
static void vcycle(hierarchy* H, int k, const double* b, double* x) {
    level* L = &H->lev[k];
    const double d = H->shift;
    const double w = 2.0 / (2.0 + 1.0 / H->dim);
    memset(x, 0, sizeof(double) * L->N);
    if (k == H->nlev - 1) {
        if (L->chol) coarse_solve(L, b, x);
        else
            for (int s = 0; s < 40; ++s) jacobi(L, b, x, L->r, d, w);
        return;
    }
    level* Cl = &H->lev[k + 1];
    jacobi(L, b, x, L->r, d, w);
    jacobi(L, b, x, L->r, d, w);
    restrict_residual(L, Cl, x, b, Cl->b, d, H->dim);
    vcycle(H, k + 1, Cl->b, Cl->x);
    prolong_add(L, Cl, Cl->x, x, H->dim);
    jacobi(L, b, x, L->r, d, w);
    jacobi(L, b, x, L->r, d, w);
}

static double dot(const double* a, const double* b, long n) {
    double s = 0.0;
    long i;
#pragma omp parallel for schedule(static) reduction(+ : s)
    for (i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

static double harm(double a, double b) { return 2.0 / (1.0 / a + 1.0 / b); }

static void free_hierarchy(hierarchy* H) {
    for (int k = 0; k < H->nlev; ++k) {
        level* L = &H->lev[k];
        free(L->fx); free(L->fy); free(L->fz); free(L->x); free(L->b); free(L->r); free(L->chol);
    }
}

/* levels, scaled face weights and work vectors; faces may be NULL (a = 1) */
static int build_hierarchy(hierarchy* H, int dim, const int* n, const double* ax, const double* ay,
                           const double* az, double Lambda) {
    memset(H, 0, sizeof(*H));
    H->dim = dim;
    int m[3] = {n[0], n[1], dim == 3 ? n[2] : 1};
    double* raw[3] = {NULL, NULL, NULL};  /* unscaled faces of the current level */
    for (int k = 0; k < 32; ++k) {
        level* L = &H->lev[k];
        L->nx = m[0]; L->ny = m[1]; L->nz = m[2];
        L->N = (long)m[0] * m[1] * m[2];
        const long sx = (long)m[2] * m[1] * (m[0] + 1), sy = (long)m[2] * (m[1] + 1) * m[0],
                   sz = (long)(m[2] + 1) * m[1] * m[0];
        double* nr[3] = {(double*)malloc(sizeof(double) * sx), (double*)malloc(sizeof(double) * sy),
                         dim == 3 ? (double*)malloc(sizeof(double) * sz) : NULL};
        if (!nr[0] || !nr[1] || (dim == 3 && !nr[2])) return -1;
        if (k == 0) {
            for (long q = 0; q < sx; ++q) nr[0][q] = ax ? ax[q] : 1.0;
            for (long q = 0; q < sy; ++q) nr[1][q] = ay ? ay[q] : 1.0;
            if (dim == 3) for (long q = 0; q < sz; ++q) nr[2][q] = az ? az[q] : 1.0;
        } else {  /* the two fine faces on the line through the coarse nodes, in series */
            const level* F = &H->lev[k - 1];
            const int fx = F->nx, fy = F->ny;
            for (int l = 0; l < m[2]; ++l)
                for (int j = 0; j < m[1]; ++j) {
                    const int fl = dim == 3 ? 2 * l + 1 : 0, fj = 2 * j + 1;
                    for (int i = 0; i <= m[0]; ++i)
                        nr[0][((long)l * m[1] + j) * (m[0] + 1) + i] =
                            harm(raw[0][((long)fl * fy + fj) * (fx + 1) + 2 * i], raw[0][((long)fl * fy + fj) * (fx + 1) + 2 * i + 1]);
                }
            for (int l = 0; l < m[2]; ++l)
                for (int j = 0; j <= m[1]; ++j) {
                    const int fl = dim == 3 ? 2 * l + 1 : 0;
                    for (int i = 0; i < m[0]; ++i)
                        nr[1][((long)l * (m[1] + 1) + j) * m[0] + i] =
                            harm(raw[1][((long)fl * (fy + 1) + 2 * j) * fx + 2 * i + 1],
                                 raw[1][((long)fl * (fy + 1) + 2 * j + 1) * fx + 2 * i + 1]);
                }
            if (dim == 3)
                for (int l = 0; l <= m[2]; ++l)
                    for (int j = 0; j < m[1]; ++j)
                        for (int i = 0; i < m[0]; ++i)
                            nr[2][((long)l * m[1] + j) * m[0] + i] =
                                harm(raw[2][((long)(2 * l) * fy + 2 * j + 1) * fx + 2 * i + 1],
                                     raw[2][((long)(2 * l + 1) * fy + 2 * j + 1) * fx + 2 * i + 1]);
            for (int a = 0; a < 3; ++a) free(raw[a]);
        }
        for (int a = 0; a < 3; ++a) raw[a] = nr[a];
        /* scaled weights a / (h^2 Lambda) of this level */
        const double hx = 1.0 / (m[0] + 1), hy = 1.0 / (m[1] + 1), hz = 1.0 / (m[2] + 1);
        L->fx = (double*)malloc(sizeof(double) * sx);
        L->fy = (double*)malloc(sizeof(double) * sy);
        L->fz = dim == 3 ? (double*)malloc(sizeof(double) * sz) : NULL;
        if (!L->fx || !L->fy || (dim == 3 && !L->fz)) return -1;
        for (long q = 0; q < sx; ++q) L->fx[q] = raw[0][q] / (hx * hx * Lambda);
        for (long q = 0; q < sy; ++q) L->fy[q] = raw[1][q] / (hy * hy * Lambda);
        if (dim == 3) for (long q = 0; q < sz; ++q) L->fz[q] = raw[2][q] / (hz * hz * Lambda);
        L->x = (double*)malloc(sizeof(double) * L->N);
        L->b = (double*)malloc(sizeof(double) * L->N);
        L->r = (double*)malloc(sizeof(double) * L->N);
        if (!L->x || !L->b || !L->r) return -1;
        H->nlev = k + 1;
        int more = 1;
        for (int a = 0; a < dim; ++a) more = more && m[a] >= 3 && m[a] % 2 == 1;
        if (!more) break;
        for (int a = 0; a < dim; ++a) m[a] = (m[a] - 1) / 2;
    }
    for (int a = 0; a < 3; ++a) free(raw[a]);
    level* C = &H->lev[H->nlev - 1];
    if (C->N <= 1024) {
        C->chol = (double*)malloc(sizeof(double) * (size_t)C->N * (size_t)C->N);
        if (!C->chol) return -1;
    }
    return 0;
}

/* v = (A - d I)^{-1} f by PCG to ||f - (A - dI) v|| <= rtol ||f||; returns iterations, -1 on breakdown or
   no convergence within max_iter */
static int pcg_one(hierarchy* H, double d, const double* f, double* v, double rtol, int max_iter) {
    level* L = &H->lev[0];
    const long N = L->N;
    H->shift = d;
    if (H->lev[H->nlev - 1].chol && coarse_factor(&H->lev[H->nlev - 1], d) != 0) return -1;
    double* r = (double*)malloc(sizeof(double) * N);
    double* z = (double*)malloc(sizeof(double) * N);
    double* p = (double*)malloc(sizeof(double) * N);
    double* q = (double*)malloc(sizeof(double) * N);
    if (!r || !z || !p || !q) { free(r); free(z); free(p); free(q); return -1; }
    memset(v, 0, sizeof(double) * N);
    memcpy(r, f, sizeof(double) * N);
    const double fn = sqrt(dot(f, f, N));
    int it = 0, rc = -1;
    if (fn == 0.0) { rc = 0; goto done; }
    vcycle(H, 0, r, z);
    memcpy(p, z, sizeof(double) * N);
    double rz = dot(r, z, N);
    for (it = 1; it <= max_iter; ++it) {
        apply(L, p, q, d);
        const double pq = dot(p, q, N);
        if (!(pq > 0)) break;
        const double a = rz / pq;
        long i;
#pragma omp parallel for schedule(static)
        for (i = 0; i < N; ++i) { v[i] += a * p[i]; r[i] -= a * q[i]; }
        if (sqrt(dot(r, r, N)) <= rtol * fn) { rc = it; break; }
        vcycle(H, 0, r, z);
        const double rz2 = dot(r, z, N);
        const double beta = rz2 / rz;
        rz = rz2;
#pragma omp parallel for schedule(static)
        for (i = 0; i < N; ++i) p[i] = z[i] + beta * p[i];
    }
done:
    free(r); free(z); free(p); free(q);
    return rc;
}

/*
 * u = sum_j c[j] (A - d[j] I)^{-1} f for K systems (host arrays; u and f of N = nx*ny*nz doubles).
 *   dim 2 or 3; n = {nx, ny, nz}; ax, ay, az face coefficients or NULL (a = 1); Lambda the scale of A.
 *   rtol: K relative residual targets, one per system.
 *   V: if not NULL, receives the K solutions, system-major (V[j*N + i]).
 *   iters: K entries, PCG iterations per system.  nthreads <= 0: the OpenMP default.
 * Returns 0, -1 (allocation / factorisation failure), -2 (a system did not converge within max_iter).
 */
int op_bura_solve(int dim, const int* n, const double* ax, const double* ay, const double* az, double Lambda, int K,
                  const double* c, const double* d, const double* f, double* u, double* V, const double* rtol,
                  int max_iter, int* iters, int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    hierarchy H;
    if (build_hierarchy(&H, dim, n, ax, ay, az, Lambda) != 0) { free_hierarchy(&H); return -1; }
    const long N = H.lev[0].N;
    double* v = (double*)malloc(sizeof(double) * N);
    if (!v) { free_hierarchy(&H); return -1; }
    memset(u, 0, sizeof(double) * N);
    int rc = 0;
    for (int j = 0; j < K && rc == 0; ++j) {
        const int it = pcg_one(&H, d[j], f, v, rtol[j], max_iter);
        if (iters) iters[j] = it;
        if (it < 0) { rc = -2; break; }
        long i;
#pragma omp parallel for schedule(static)
        for (i = 0; i < N; ++i) u[i] += c[j] * v[i];
        if (V) memcpy(V + (size_t)j * N, v, sizeof(double) * N);
    }
    free(v);
    free_hierarchy(&H);
    return rc;
}

/* threads the OpenMP runtime would use */
int op_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
