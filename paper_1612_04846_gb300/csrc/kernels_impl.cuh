// Kernel templates of the multi-shift MG-PCG; instantiated for float and double in
// kernels_f32.cu / kernels_f64.cu.  See kernels.cuh for the data layout.
#pragma once
#include "kernels.cuh"

namespace bura {

template <class T>
__device__ __forceinline__ void vld(const T* p, T (&o)[VecT<T>::W]) {
    typename VecT<T>::V v = *reinterpret_cast<const typename VecT<T>::V*>(p);
    if constexpr (VecT<T>::W == 2) { o[0] = v.x; o[1] = v.y; }
    else { o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w; }
}

template <class T>
__device__ __forceinline__ void vldg(const T* p, T (&o)[VecT<T>::W]) {
    typename VecT<T>::V v = __ldg(reinterpret_cast<const typename VecT<T>::V*>(p));
    if constexpr (VecT<T>::W == 2) { o[0] = v.x; o[1] = v.y; }
    else { o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w; }
}

template <class T>
__device__ __forceinline__ void vst(T* p, const T (&o)[VecT<T>::W]) {
    typename VecT<T>::V v;
    if constexpr (VecT<T>::W == 2) { v.x = o[0]; v.y = o[1]; }
    else { v.x = o[0]; v.y = o[1]; v.z = o[2]; v.w = o[3]; }
    *reinterpret_cast<typename VecT<T>::V*>(p) = v;
}

// Per-thread partial sums: FP64 for double data; for float data FP32 over at most 8 grid-stride
// steps, then folded into FP64.
template <class T>
struct Accum {
    static constexpr int W = VecT<T>::W;
    double tot[W];
    float part[W];
    int n;
    __device__ Accum() : n(0) {
        for (int v = 0; v < W; ++v) { tot[v] = 0.0; part[v] = 0.f; }
    }
    __device__ __forceinline__ void add(const T (&a)[W], const T (&b)[W]) {
        if constexpr (sizeof(T) == 8) {
            for (int v = 0; v < W; ++v) tot[v] = fma((double)a[v], (double)b[v], tot[v]);
        } else {
            for (int v = 0; v < W; ++v) part[v] = fmaf(a[v], b[v], part[v]);
            if (++n == 8) flush();
        }
    }
    __device__ __forceinline__ void flush() {
        if constexpr (sizeof(T) == 4) {
            for (int v = 0; v < W; ++v) { tot[v] += (double)part[v]; part[v] = 0.f; }
            n = 0;
        }
    }
};

// Coordinates of point P on a level.
struct Coord { int i, j, l; };
template <int DIM>
__device__ __forceinline__ Coord coord(const Lev& L, int P) {
    Coord c;
    const unsigned up = (unsigned)P, unx = (unsigned)L.nx;
    const unsigned rem = up / unx;
    c.i = (int)(up - rem * unx);
    if (DIM == 3) {
        const unsigned uny = (unsigned)L.ny;
        const unsigned r2 = rem / uny;
        c.j = (int)(rem - r2 * uny);
        c.l = (int)r2;
    } else {
        c.j = (int)rem;
        c.l = 0;
    }
    return c;
}

// Face weights of point P: m/p = lower/upper face along x, y, z.
template <class T>
struct Wts { T xm, xp, ym, yp, zm, zp; };

template <class T, int DIM, bool VAR>
__device__ __forceinline__ Wts<T> weights(const Lev& L, int P, const Coord& c) {
    Wts<T> w;
    if (VAR) {
        const T* fx = reinterpret_cast<const T*>(L.fx);
        const T* fy = reinterpret_cast<const T*>(L.fy);
        const size_t row = (size_t)c.l * L.ny + c.j;             // (l, j) row of x-faces: nx+1 each
        w.xm = __ldg(fx + row * (L.nx + 1) + c.i);
        w.xp = __ldg(fx + row * (L.nx + 1) + c.i + 1);
        const size_t ybase = ((size_t)c.l * (L.ny + 1) + c.j) * L.nx + c.i;
        w.ym = __ldg(fy + ybase);
        w.yp = __ldg(fy + ybase + L.nx);
        if (DIM == 3) {
            const T* fz = reinterpret_cast<const T*>(L.fz);
            w.zm = __ldg(fz + P);
            w.zp = __ldg(fz + P + L.plane);
        } else {
            w.zm = w.zp = T(0);
        }
    } else {
        w.xm = w.xp = (T)L.wx;
        w.ym = w.yp = (T)L.wy;
        w.zm = w.zp = (T)L.wz;
    }
    return w;
}

template <class T>
struct LoadPlain {
    const T* x;
    __device__ __forceinline__ void operator()(size_t idx, T (&o)[VecT<T>::W]) const { vld(x + idx, o); }
};

// p_new = z + beta * p_old evaluated on the fly (the p update fused into the operator apply).
template <class T>
struct LoadPUpd {
    const T* z;
    const T* p;
    T beta[VecT<T>::W];
    __device__ __forceinline__ void operator()(size_t idx, T (&o)[VecT<T>::W]) const {
        T a[VecT<T>::W], b[VecT<T>::W];
        vldg(z + idx, a);
        vldg(p + idx, b);
        for (int v = 0; v < VecT<T>::W; ++v) o[v] = fma(beta[v], b[v], a[v]);
    }
};

// A x at point P (no shift term) for the W systems of chunk `off`; xc = x(P), diag = A_PP.
template <class T, int DIM, bool VAR, class LD>
__device__ __forceinline__ void stencil(const Lev& L, int Kp, int P, int off, const LD& ld,
                                        T (&xc)[VecT<T>::W], T (&Ax)[VecT<T>::W], T& diag) {
    constexpr int W = VecT<T>::W;
    const Coord c = coord<DIM>(L, P);
    const Wts<T> w = weights<T, DIM, VAR>(L, P, c);
    diag = w.xm + w.xp + w.ym + w.yp;
    if (DIM == 3) diag += w.zm + w.zp;
    const size_t base = (size_t)P * Kp + off;
    ld(base, xc);
    T acc[W];
    for (int v = 0; v < W; ++v) acc[v] = diag * xc[v];
    T n[W];
    if (c.i > 0) { ld(base - Kp, n); for (int v = 0; v < W; ++v) acc[v] = fma(-w.xm, n[v], acc[v]); }
    if (c.i < L.nx - 1) { ld(base + Kp, n); for (int v = 0; v < W; ++v) acc[v] = fma(-w.xp, n[v], acc[v]); }
    const size_t sy = (size_t)L.nx * Kp;
    if (c.j > 0) { ld(base - sy, n); for (int v = 0; v < W; ++v) acc[v] = fma(-w.ym, n[v], acc[v]); }
    if (c.j < L.ny - 1) { ld(base + sy, n); for (int v = 0; v < W; ++v) acc[v] = fma(-w.yp, n[v], acc[v]); }
    if (DIM == 3) {
        const size_t sz = (size_t)L.plane * Kp;
        if (c.l > 0) { ld(base - sz, n); for (int v = 0; v < W; ++v) acc[v] = fma(-w.zm, n[v], acc[v]); }
        if (c.l < L.nz - 1) { ld(base + sz, n); for (int v = 0; v < W; ++v) acc[v] = fma(-w.zp, n[v], acc[v]); }
    }
    for (int v = 0; v < W; ++v) Ax[v] = acc[v];
}

// ------------------------------------------------------------------ reductions
__device__ __forceinline__ void finish_one(const Red& red, int s, double tot) {
    Scal* S = red.scal;
    switch (red.op) {
        case RED_ALPHA: {
            S->pq[s] = tot;
            double a = 0.0;
            if (S->active[s]) {
                if (!(tot > 0.0) || !isfinite(tot)) S->breakdown = 1;
                else a = S->rz[s] / tot;
            }
            S->alpha[s] = a;
            break;
        }
        case RED_CONV: {
            S->rr[s] = tot;
            if (S->active[s]) {
                S->iters[s] += 1;
                if (!isfinite(tot)) S->breakdown = 1;
                if (tot <= S->thr[s]) S->active[s] = 0;
            }
            break;
        }
        case RED_BETA: {
            double b = 0.0;
            if (S->active[s]) {
                if (!isfinite(tot)) S->breakdown = 1;
                b = tot / S->rz[s];
                S->rz[s] = tot;
            }
            S->beta[s] = b;
            break;
        }
        case RED_STORE:
            red.out[s] = tot;
            break;
        default:
            break;
    }
}

// Block reduction of per-thread partials (W systems per thread, chunk = threadIdx.x) followed by
// the grid reduction in the last block.  Every thread of the block must call this.
template <class T>
__device__ void reduce_finish(Accum<T>& acc, const Red& red, int Kp) {
    constexpr int W = VecT<T>::W;
    extern __shared__ double sm[];
    __shared__ int am_last;
    acc.flush();
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int nthr = blockDim.x * blockDim.y;
    for (int v = 0; v < W; ++v) sm[tid * W + v] = acc.tot[v];  // = sm[point * Kp + system]
    __syncthreads();
    const int G = nthr / Kp;
    double part = 0.0;
    if (tid < Kp * G) {
        const int s = tid % Kp, g = tid / Kp;
        for (int p = g; p < (int)blockDim.y; p += G) part += sm[p * Kp + s];
    }
    __syncthreads();
    if (tid < Kp * G) sm[tid] = part;
    __syncthreads();
    if (tid < Kp) {
        double tot = 0.0;
        for (int g = 0; g < G; ++g) tot += sm[g * Kp + tid];
        red.partial[(size_t)blockIdx.x * Kp + tid] = tot;
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) {
        const unsigned t = atomicAdd(&red.scal->ticket, 1u);
        am_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    part = 0.0;
    if (tid < Kp * G) {
        const int s = tid % Kp, g = tid / Kp;
        for (int b = g; b < (int)gridDim.x; b += G) part += __ldcg(red.partial + (size_t)b * Kp + s);
    }
    __syncthreads();
    if (tid < Kp * G) sm[tid] = part;
    __syncthreads();
    if (tid < Kp) {
        double tot = 0.0;
        for (int g = 0; g < G; ++g) tot += sm[g * Kp + tid];
        finish_one(red, tid, tot);
    }
    __syncthreads();
    if (tid == 0) {
        red.scal->ticket = 0u;
        if (red.op == RED_CONV) {
            int na = 0;
            for (int s = 0; s < Kp; ++s) na += red.scal->active[s] ? 1 : 0;
            red.scal->nactive = na;
        }
    }
}

// ------------------------------------------------------------------ kernels
template <class T>
__global__ void k_broadcast(const double* __restrict__ f, int N, int Kp, int K, T* r, T* x, T* p) {
    constexpr int W = VecT<T>::W;
    const int off = threadIdx.x * W;
    for (int tile = blockIdx.x; (long long)tile * blockDim.y < N; tile += gridDim.x) {
        const int P = tile * blockDim.y + threadIdx.y;
        if (P >= N) continue;
        const T fv = (T)f[P];
        T rv[W], zv[W];
        for (int v = 0; v < W; ++v) { rv[v] = (off + v < K) ? fv : T(0); zv[v] = T(0); }
        const size_t base = (size_t)P * Kp + off;
        vst(r + base, rv);
        vst(x + base, zv);
        vst(p + base, zv);
    }
}

template <class T, int DIM, bool VAR>
__global__ void k_spmv_p(Lev L, int Kp, const T* __restrict__ z, const T* __restrict__ pold, T* __restrict__ pnew,
                         T* __restrict__ q, Red red) {
    constexpr int W = VecT<T>::W;
    const int off = threadIdx.x * W;
    LoadPUpd<T> ld;
    ld.z = z;
    ld.p = pold;
    T dsh[W];
    for (int v = 0; v < W; ++v) { ld.beta[v] = (T)red.scal->beta[off + v]; dsh[v] = (T)red.scal->dsh[off + v]; }
    Accum<T> acc;
    for (int tile = blockIdx.x; (long long)tile * blockDim.y < L.N; tile += gridDim.x) {
        const int P = tile * blockDim.y + threadIdx.y;
        if (P >= L.N) continue;
        T pc[W], Ax[W], diag;
        stencil<T, DIM, VAR>(L, Kp, P, off, ld, pc, Ax, diag);
        T qv[W];
        for (int v = 0; v < W; ++v) qv[v] = fma(-dsh[v], pc[v], Ax[v]);
        const size_t base = (size_t)P * Kp + off;
        vst(pnew + base, pc);
        vst(q + base, qv);
        acc.add(pc, qv);
    }
    reduce_finish<T>(acc, red, Kp);
}

template <class T>
__global__ void k_cg_update(int N, int Kp, T* __restrict__ x, T* __restrict__ r, const T* __restrict__ p,
                            const T* __restrict__ q, Red red) {
    constexpr int W = VecT<T>::W;
    const int off = threadIdx.x * W;
    T a[W];
    for (int v = 0; v < W; ++v) a[v] = (T)red.scal->alpha[off + v];
    Accum<T> acc;
    for (int tile = blockIdx.x; (long long)tile * blockDim.y < N; tile += gridDim.x) {
        const int P = tile * blockDim.y + threadIdx.y;
        if (P >= N) continue;
        const size_t base = (size_t)P * Kp + off;
        T xv[W], rv[W], pv[W], qv[W];
        vld(x + base, xv);
        vld(r + base, rv);
        vldg(p + base, pv);
        vldg(q + base, qv);
        for (int v = 0; v < W; ++v) { xv[v] = fma(a[v], pv[v], xv[v]); rv[v] = fma(-a[v], qv[v], rv[v]); }
        vst(x + base, xv);
        vst(r + base, rv);
        acc.add(rv, rv);
    }
    reduce_finish<T>(acc, red, Kp);
}

// x = c2 Dinv b (first Chebyshev step from a zero initial guess; pointwise).
template <class T, int DIM, bool VAR>
__global__ void k_cheb_zero(Lev L, int Kp, const T* __restrict__ b, T* __restrict__ x, ChebStep cs,
                            const double* __restrict__ dsh) {
    constexpr int W = VecT<T>::W;
    const int off = threadIdx.x * W;
    T c2[W], d[W];
    for (int v = 0; v < W; ++v) { c2[v] = (T)cs.c2[off + v]; d[v] = (T)dsh[off + v]; }
    for (int tile = blockIdx.x; (long long)tile * blockDim.y < L.N; tile += gridDim.x) {
        const int P = tile * blockDim.y + threadIdx.y;
        if (P >= L.N) continue;
        const size_t base = (size_t)P * Kp + off;
        T bv[W], xv[W];
        vldg(b + base, bv);
        if (VAR) {
            const Coord c = coord<DIM>(L, P);
            const Wts<T> w = weights<T, DIM, VAR>(L, P, c);
            T diag = w.xm + w.xp + w.ym + w.yp;
            if (DIM == 3) diag += w.zm + w.zp;
            for (int v = 0; v < W; ++v) xv[v] = c2[v] * bv[v] / (diag - d[v]);
        } else {
            for (int v = 0; v < W; ++v) xv[v] = c2[v] * bv[v];
        }
        vst(x + base, xv);
    }
}

// One Chebyshev step: res = b - (A - dI) xin; dnew = c1 din + c2 Dinv res; xout = xin + dnew.
// din may be null (c1 = 0); dout may be null; red.op != RED_NONE accumulates b . xout.
template <class T, int DIM, bool VAR>
__global__ void k_cheb_step(Lev L, int Kp, const T* __restrict__ xin, const T* __restrict__ din,
                            const T* __restrict__ b, T* __restrict__ xout, T* __restrict__ dout, ChebStep cs,
                            const double* __restrict__ dsh, Red red) {
    constexpr int W = VecT<T>::W;
    const int off = threadIdx.x * W;
    T c1[W], c2[W], d[W];
    for (int v = 0; v < W; ++v) {
        c1[v] = cs.c1 ? (T)cs.c1[off + v] : T(0);
        c2[v] = (T)cs.c2[off + v];
        d[v] = (T)dsh[off + v];
    }
    LoadPlain<T> ld{xin};
    Accum<T> acc;
    const bool dot = red.op != RED_NONE;
    for (int tile = blockIdx.x; (long long)tile * blockDim.y < L.N; tile += gridDim.x) {
        const int P = tile * blockDim.y + threadIdx.y;
        if (P >= L.N) continue;
        T xc[W], Ax[W], diag;
        stencil<T, DIM, VAR>(L, Kp, P, off, ld, xc, Ax, diag);
        const size_t base = (size_t)P * Kp + off;
        T bv[W], dv[W], xo[W];
        vldg(b + base, bv);
        if (din) vld(din + base, dv);
        else for (int v = 0; v < W; ++v) dv[v] = T(0);
        for (int v = 0; v < W; ++v) {
            const T res = bv[v] - fma(-d[v], xc[v], Ax[v]);
            T g = c2[v] * res;
            if (VAR) g = g / (diag - d[v]);
            dv[v] = fma(c1[v], dv[v], g);
            xo[v] = xc[v] + dv[v];
        }
        vst(xout + base, xo);
        if (dout) vst(dout + base, dv);
        if (dot) acc.add(bv, xo);
    }
    if (dot) reduce_finish<T>(acc, red, Kp);
}

// bc = R (b - (A - dI) x): full weighting, R = P^T / 2^DIM with 1D weights (1/4, 1/2, 1/4).
template <class T, int DIM, bool VAR>
__global__ void k_restrict_res(Lev Lf, Lev Lc, int Kp, const T* __restrict__ x, const T* __restrict__ b,
                               T* __restrict__ bc, const double* __restrict__ dsh) {
    constexpr int W = VecT<T>::W;
    const int off = threadIdx.x * W;
    T d[W];
    for (int v = 0; v < W; ++v) d[v] = (T)dsh[off + v];
    const T w1[3] = {T(0.25), T(0.5), T(0.25)};
    LoadPlain<T> ld{x};
    for (int tile = blockIdx.x; (long long)tile * blockDim.y < Lc.N; tile += gridDim.x) {
        const int Pc = tile * blockDim.y + threadIdx.y;
        if (Pc >= Lc.N) continue;
        const Coord cc = coord<DIM>(Lc, Pc);
        const int fi = 2 * cc.i + 1, fj = 2 * cc.j + 1, fl = (DIM == 3) ? 2 * cc.l + 1 : 0;
        T sum[W];
        for (int v = 0; v < W; ++v) sum[v] = T(0);
        const int zlo = (DIM == 3) ? -1 : 0, zhi = (DIM == 3) ? 1 : 0;
        for (int dz = zlo; dz <= zhi; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const int P = ((fl + dz) * Lf.ny + (fj + dy)) * Lf.nx + (fi + dx);
                    T xc[W], Ax[W], diag;
                    stencil<T, DIM, VAR>(Lf, Kp, P, off, ld, xc, Ax, diag);
                    T bv[W];
                    vldg(b + (size_t)P * Kp + off, bv);
                    T wt = w1[dx + 1] * w1[dy + 1];
                    if (DIM == 3) wt *= w1[dz + 1];
                    for (int v = 0; v < W; ++v) sum[v] = fma(wt, bv[v] - fma(-d[v], xc[v], Ax[v]), sum[v]);
                }
        vst(bc + (size_t)Pc * Kp + off, sum);
    }
}

// x += P ec: bilinear / trilinear interpolation (coarse node I sits on fine node 2I+1).
template <class T, int DIM>
__global__ void k_prolong_add(Lev Lf, Lev Lc, int Kp, const T* __restrict__ ec, T* __restrict__ x) {
    constexpr int W = VecT<T>::W;
    const int off = threadIdx.x * W;
    for (int tile = blockIdx.x; (long long)tile * blockDim.y < Lf.N; tile += gridDim.x) {
        const int P = tile * blockDim.y + threadIdx.y;
        if (P >= Lf.N) continue;
        const Coord c = coord<DIM>(Lf, P);
        int ci[3][2], nc[3];
        T cw[3][2];
        const int fc[3] = {c.i, c.j, c.l};
        const int cn[3] = {Lc.nx, Lc.ny, Lc.nz};
        for (int a = 0; a < DIM; ++a) {
            const int f = fc[a];
            nc[a] = 0;
            if (f & 1) {
                ci[a][0] = (f - 1) >> 1; cw[a][0] = T(1); nc[a] = 1;
            } else {
                const int lo = (f >> 1) - 1, hi = f >> 1;
                if (lo >= 0) { ci[a][nc[a]] = lo; cw[a][nc[a]] = T(0.5); ++nc[a]; }
                if (hi < cn[a]) { ci[a][nc[a]] = hi; cw[a][nc[a]] = T(0.5); ++nc[a]; }
            }
        }
        if (DIM == 2) { nc[2] = 1; ci[2][0] = 0; cw[2][0] = T(1); }
        T sum[W];
        for (int v = 0; v < W; ++v) sum[v] = T(0);
        for (int a2 = 0; a2 < nc[2]; ++a2)
            for (int a1 = 0; a1 < nc[1]; ++a1)
                for (int a0 = 0; a0 < nc[0]; ++a0) {
                    const int Pc = (ci[2][a2] * Lc.ny + ci[1][a1]) * Lc.nx + ci[0][a0];
                    const T wt = cw[0][a0] * cw[1][a1] * cw[2][a2];
                    T e[W];
                    vldg(ec + (size_t)Pc * Kp + off, e);
                    for (int v = 0; v < W; ++v) sum[v] = fma(wt, e[v], sum[v]);
                }
        const size_t base = (size_t)P * Kp + off;
        T xv[W];
        vld(x + base, xv);
        for (int v = 0; v < W; ++v) xv[v] += sum[v];
        vst(x + base, xv);
    }
}

template <class T, int DIM, bool VAR>
__global__ void k_apply_shifted(Lev L, int Kp, const T* __restrict__ x, T* __restrict__ y,
                                const double* __restrict__ dsh) {
    constexpr int W = VecT<T>::W;
    const int off = threadIdx.x * W;
    T d[W];
    for (int v = 0; v < W; ++v) d[v] = (T)dsh[off + v];
    LoadPlain<T> ld{x};
    for (int tile = blockIdx.x; (long long)tile * blockDim.y < L.N; tile += gridDim.x) {
        const int P = tile * blockDim.y + threadIdx.y;
        if (P >= L.N) continue;
        T xc[W], Ax[W], diag;
        stencil<T, DIM, VAR>(L, Kp, P, off, ld, xc, Ax, diag);
        for (int v = 0; v < W; ++v) Ax[v] = fma(-d[v], xc[v], Ax[v]);
        vst(y + (size_t)P * Kp + off, Ax);
    }
}

template <class T>
__global__ void k_dot(int N, int Kp, const T* __restrict__ a, const T* __restrict__ b, Red red) {
    constexpr int W = VecT<T>::W;
    const int off = threadIdx.x * W;
    Accum<T> acc;
    for (int tile = blockIdx.x; (long long)tile * blockDim.y < N; tile += gridDim.x) {
        const int P = tile * blockDim.y + threadIdx.y;
        if (P >= N) continue;
        T av[W], bv[W];
        vldg(a + (size_t)P * Kp + off, av);
        vldg(b + (size_t)P * Kp + off, bv);
        acc.add(av, bv);
    }
    reduce_finish<T>(acc, red, Kp);
}

// ------------------------------------------------------------------ host launchers
inline dim3 blk(const Launch& g) { return dim3(g.C, g.PPB); }
inline size_t shm(const Launch& g, int W) { return (size_t)g.C * g.PPB * W * sizeof(double); }

#define BURA_DISPATCH(dim, var, KERNEL, ...)                                        \
    do {                                                                            \
        if (dim == 2 && !var) KERNEL<T, 2, false>__VA_ARGS__;                        \
        else if (dim == 2 && var) KERNEL<T, 2, true>__VA_ARGS__;                     \
        else if (dim == 3 && !var) KERNEL<T, 3, false>__VA_ARGS__;                   \
        else KERNEL<T, 3, true>__VA_ARGS__;                                          \
    } while (0)

template <class T>
void Ops<T>::broadcast(const Launch& g, const double* f, long long N, int K, T* r, T* x, T* p, cudaStream_t s) {
    k_broadcast<T><<<g.blocks, blk(g), 0, s>>>(f, (int)N, g.Kp, K, r, x, p);
}

template <class T>
void Ops<T>::spmv_p(const Launch& g, const Lev& L, int dim, bool var, const T* z, const T* pold, T* pnew, T* q,
                    const Red& red, cudaStream_t s) {
    const size_t sh = shm(g, VecT<T>::W);
    BURA_DISPATCH(dim, var, k_spmv_p, <<<g.blocks, blk(g), sh, s>>>(L, g.Kp, z, pold, pnew, q, red));
}

template <class T>
void Ops<T>::cg_update(const Launch& g, long long N, T* x, T* r, const T* p, const T* q, const Red& red,
                       cudaStream_t s) {
    k_cg_update<T><<<g.blocks, blk(g), shm(g, VecT<T>::W), s>>>((int)N, g.Kp, x, r, p, q, red);
}

template <class T>
void Ops<T>::cheb_zero(const Launch& g, const Lev& L, int dim, bool var, const T* b, T* x, ChebStep cs,
                       const double* dsh, cudaStream_t s) {
    BURA_DISPATCH(dim, var, k_cheb_zero, <<<g.blocks, blk(g), 0, s>>>(L, g.Kp, b, x, cs, dsh));
}

template <class T>
void Ops<T>::cheb_step(const Launch& g, const Lev& L, int dim, bool var, const T* xin, const T* din, const T* b,
                       T* xout, T* dout, ChebStep cs, const double* dsh, const Red& red, cudaStream_t s) {
    const size_t sh = red.op != RED_NONE ? shm(g, VecT<T>::W) : 0;
    BURA_DISPATCH(dim, var, k_cheb_step, <<<g.blocks, blk(g), sh, s>>>(L, g.Kp, xin, din, b, xout, dout, cs, dsh, red));
}

template <class T>
void Ops<T>::restrict_res(const Launch& gc, const Lev& Lf, const Lev& Lc, int dim, bool var, const T* x, const T* b,
                          T* bc, const double* dsh, cudaStream_t s) {
    BURA_DISPATCH(dim, var, k_restrict_res, <<<gc.blocks, blk(gc), 0, s>>>(Lf, Lc, gc.Kp, x, b, bc, dsh));
}

template <class T>
void Ops<T>::prolong_add(const Launch& gf, const Lev& Lf, const Lev& Lc, int dim, const T* ec, T* x, cudaStream_t s) {
    if (dim == 2) k_prolong_add<T, 2><<<gf.blocks, blk(gf), 0, s>>>(Lf, Lc, gf.Kp, ec, x);
    else k_prolong_add<T, 3><<<gf.blocks, blk(gf), 0, s>>>(Lf, Lc, gf.Kp, ec, x);
}

template <class T>
void Ops<T>::apply_shifted(const Launch& g, const Lev& L, int dim, bool var, const T* x, T* y, const double* dsh,
                           cudaStream_t s) {
    BURA_DISPATCH(dim, var, k_apply_shifted, <<<g.blocks, blk(g), 0, s>>>(L, g.Kp, x, y, dsh));
}

template <class T>
void Ops<T>::dot(const Launch& g, long long N, const T* a, const T* b, const Red& red, cudaStream_t s) {
    k_dot<T><<<g.blocks, blk(g), shm(g, VecT<T>::W), s>>>((int)N, g.Kp, a, b, red);
}

}  // namespace bura
