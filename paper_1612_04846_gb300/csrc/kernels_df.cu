// Refinement kernels of the mixed-precision path in double-float ("df") arithmetic.
//
// The accumulated solutions v_j of the iterative refinement are kept as unevaluated sums hi + lo of two
// FP32 values (|lo| <= ulp(hi)/2, about 48 significant bits) and every refinement operation -- adding
// the FP32 correction, the true residual f - (A - d_j I) v_j and the weighted sum sum_j c_j v_j -- is
// done with error-free FP32 transformations on the FP32 pipes.  GB300's FP64 rate (about 1.25
// TFLOP/s) would make the same work ALU-bound in FP64; in df it is bound by HBM.
//
// The building blocks are the classical exact transformations: TwoSum (Knuth) gives s + e = a + b
// exactly, FastTwoSum (Dekker) the same for |a| >= |b|, and TwoProd by a fused multiply-add gives
// p + e = a * b exactly.  A df sum or product built from them has a relative error of a few units of
// 2^-48 with respect to the magnitudes of its operands, like an FP64 operation at 2^-53.  Nothing here
// is compiled with fast-math, and the operations below are written so that no contraction into an
// FMA changes them (the only products are explicit fmaf/TwoProd).
#include <algorithm>

#include "kernels_impl.cuh"

namespace bura {

namespace {

struct dfv {
    float hi, lo;
};

__device__ __forceinline__ dfv two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return {s, e};
}

__device__ __forceinline__ dfv fast_two_sum(float a, float b) {
    const float s = a + b;
    return {s, b - (s - a)};
}

__device__ __forceinline__ dfv df_add(dfv x, dfv y) {
    const dfv s = two_sum(x.hi, y.hi);
    const float e = s.lo + (x.lo + y.lo);
    return fast_two_sum(s.hi, e);
}

__device__ __forceinline__ dfv df_neg(dfv x) { return {-x.hi, -x.lo}; }

__device__ __forceinline__ dfv df_add_f(dfv x, float b) {
    const dfv s = two_sum(x.hi, b);
    return fast_two_sum(s.hi, s.lo + x.lo);
}

__device__ __forceinline__ dfv df_mul(dfv x, dfv y) {
    const float p = x.hi * y.hi;
    float e = fmaf(x.hi, y.hi, -p);
    e = fmaf(x.hi, y.lo, e);
    e = fmaf(x.lo, y.hi, e);
    return fast_two_sum(p, e);
}

// v + x / sf for a power-of-two sf (the division is exact).
__device__ __forceinline__ dfv corrected(float vh, float vl, float x, float inv_sf) {
    return df_add_f(dfv{vh, vl}, x * inv_sf);
}

// Coefficients of the FP32 pair form of the level-0 operator.
struct DfOp {
    dfv wx, wy, wz;              // constant face weights (constant coefficients)
    const float* ch;             // diag - d_j, hi parts (constant coefficients), Kp entries
    const float* cl;             // ... lo parts
    const float* dh;             // d_j, hi parts (variable coefficients), Kp entries
    const float* dl;
    const float* fxh; const float* fxl;  // scaled face coefficients (variable coefficients)
    const float* fyh; const float* fyl;
    const float* fzh; const float* fzl;
};

// Update v <- v + x/sf (v read from vin, written to vout) and form the scaled FP32 right-hand side of
// the next inner solve, r32 = sf * (f - (A - d_j I) v), with sum_j-wise r32 . r32 (RED_STORE).  The
// neighbours' corrected values are recomputed from vin and x (never read back from vout), so the
// kernel has no read-after-write hazard between blocks.
template <int DIM, bool VAR>
__global__ void __launch_bounds__(kSweepThreads, 2)
    k_update_residual_df(Lev L, int Kp, DfOp op, const float* __restrict__ fh, const float* __restrict__ fl,
                         const float* __restrict__ vhin, const float* __restrict__ vlin, const float* __restrict__ x,
                         float* __restrict__ vhout, float* __restrict__ vlout, float* __restrict__ r32, float sf,
                         float inv_sf, Red red) {
    pdl_wait();
    constexpr int W = 4;
    const int off = threadIdx.x * W;
    dfv c0[W], dd[W];
    for (int q = 0; q < W; ++q) {
        c0[q] = VAR ? dfv{0.f, 0.f} : dfv{op.ch[off + q], op.cl[off + q]};
        dd[q] = VAR ? dfv{op.dh[off + q], op.dl[off + q]} : dfv{0.f, 0.f};
    }
    Accum<float> acc;
    const int b0 = blockIdx.x, nb = gridDim.x;
    BURA_SWEEP(L.N) {
        const Coord c = coord<DIM>(L, P);
        const size_t base = (size_t)P * Kp + off;
        // the corrected iterate at P and at its neighbours (zero outside the grid)
        auto vnew = [&](size_t idx, dfv (&o)[W]) {
            float a[W], b[W], e[W];
            vld(vhin + idx, a);
            vld(vlin + idx, b);
            vld(x + idx, e);
            for (int q = 0; q < W; ++q) o[q] = corrected(a[q], b[q], e[q], inv_sf);
        };
        dfv vc[W];
        vnew(base, vc);
        {
            float h[W], l[W];
            for (int q = 0; q < W; ++q) { h[q] = vc[q].hi; l[q] = vc[q].lo; }
            vst(vhout + base, h);
            vst(vlout + base, l);
        }
        const long long sx = Kp, sy = (long long)L.nx * Kp, sz = (long long)L.plane * Kp;
        const bool has[6] = {c.i > 0, c.i < L.nx - 1, c.j > 0, c.j < L.ny - 1, DIM == 3 && c.l > 0,
                             DIM == 3 && c.l < L.nz - 1};
        const long long step[6] = {-sx, sx, -sy, sy, -sz, sz};
        // the neighbour value of face f (zero outside the grid)
        auto neighbour = [&](int f, dfv (&o)[W]) {
            if (has[f]) vnew(base + step[f], o);
            else for (int q = 0; q < W; ++q) o[q] = dfv{0.f, 0.f};
        };
        dfv t[W];  // (A - d_j I) v at P, accumulated one face pair (constant) or face (variable) at a time
        if (!VAR) {
            for (int q = 0; q < W; ++q) t[q] = df_mul(c0[q], vc[q]);
            const dfv wts[3] = {op.wx, op.wy, op.wz};
            for (int a = 0; a < DIM; ++a) {
                dfv lo[W], hi[W];
                neighbour(2 * a, lo);
                neighbour(2 * a + 1, hi);
                for (int q = 0; q < W; ++q) t[q] = df_add(t[q], df_neg(df_mul(wts[a], df_add(lo[q], hi[q]))));
            }
        } else {
            // face coefficients of P: x faces (l, j, i) and (l, j, i+1); y faces; z faces
            const size_t row = (size_t)c.l * L.ny + c.j;
            const size_t xf = row * (L.nx + 1) + c.i;
            const size_t yf = ((size_t)c.l * (L.ny + 1) + c.j) * L.nx + c.i;
            const size_t fidx[6] = {xf, xf + 1, yf, yf + L.nx, (size_t)P, (size_t)P + L.plane};
            const float* wh[3] = {op.fxh, op.fyh, op.fzh};
            const float* wl[3] = {op.fxl, op.fyl, op.fzl};
            for (int q = 0; q < W; ++q) t[q] = df_neg(df_mul(dd[q], vc[q]));
            for (int f = 0; f < 2 * DIM; ++f) {
                const dfv w{wh[f / 2][fidx[f]], wl[f / 2][fidx[f]]};
                dfv o[W];
                neighbour(f, o);
                for (int q = 0; q < W; ++q) t[q] = df_add(t[q], df_mul(w, df_add(vc[q], df_neg(o[q]))));
            }
        }
        const dfv fv{fh[P], fl[P]};
        float rv[W];
        for (int q = 0; q < W; ++q) rv[q] = df_add(fv, df_neg(t[q])).hi * sf;
        vst(r32 + base, rv);
        acc.add(rv, rv);
    }
    pdl_trigger();
    reduce_finish<float>(acc, red, Kp);
}

// First inner right-hand side r32 = sf * f for every system (zero in the padding), the FP32 pair form
// of f, and zero iterate / direction.
__global__ void k_cast_f_df(int N, int Kp, int K, const double* __restrict__ f, double sf, float* __restrict__ r32,
                            float* __restrict__ x32, float* __restrict__ p32, float* __restrict__ fh,
                            float* __restrict__ fl) {
    const int off = threadIdx.x * 4;
    for (int tile = blockIdx.x; (long long)tile * blockDim.y < N; tile += gridDim.x) {
        const int P = tile * blockDim.y + threadIdx.y;
        if (P >= N) continue;
        const double fv = f[P];
        const float rf = (float)(fv * sf);
        float rv[4], zv[4];
        for (int q = 0; q < 4; ++q) { rv[q] = (off + q < K) ? rf : 0.f; zv[q] = 0.f; }
        const size_t base = (size_t)P * Kp + off;
        vst(r32 + base, rv);
        vst(x32 + base, zv);
        vst(p32 + base, zv);
        if (threadIdx.x == 0) {
            const float h = (float)fv;
            fh[P] = h;
            fl[P] = (float)(fv - (double)h);
        }
    }
}

// u = sum_j c_j v_j in df, converted to FP64 once per point.
__global__ void k_weighted_sum_df(int N, int Kp, int K, const float* __restrict__ vh, const float* __restrict__ vl,
                                  const float* __restrict__ ch, const float* __restrict__ cl, double* __restrict__ u,
                                  int accumulate) {
    __shared__ float sh[KMAXP], sl[KMAXP];
    if (threadIdx.x < KMAXP) {
        sh[threadIdx.x] = threadIdx.x < K ? ch[threadIdx.x] : 0.f;
        sl[threadIdx.x] = threadIdx.x < K ? cl[threadIdx.x] : 0.f;
    }
    __syncthreads();
    for (int P = blockIdx.x * blockDim.x + threadIdx.x; P < N; P += gridDim.x * blockDim.x) {
        const float4* hp = reinterpret_cast<const float4*>(vh + (size_t)P * Kp);
        const float4* lp = reinterpret_cast<const float4*>(vl + (size_t)P * Kp);
        dfv s{0.f, 0.f};
        for (int q = 0; q < Kp / 4; ++q) {
            const float4 a = hp[q], b = lp[q];
            const float ah[4] = {a.x, a.y, a.z, a.w}, bl[4] = {b.x, b.y, b.z, b.w};
            for (int v = 0; v < 4; ++v) {
                const int j = 4 * q + v;
                if (j >= K) break;
                s = df_add(s, df_mul(dfv{sh[j], sl[j]}, dfv{ah[v], bl[v]}));
            }
        }
        const double w = (double)s.hi + (double)s.lo;
        u[P] = accumulate ? u[P] + w : w;
    }
}

// V[j * N + P] = v_j(P) in FP64 (system-major output of bura_solve_systems).
__global__ void k_gather_df(int N, int Kp, int K, const float* __restrict__ vh, const float* __restrict__ vl,
                            double* __restrict__ V) {
    const long long total = (long long)N * K;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(i / N);
        const int P = (int)(i - (long long)j * N);
        const size_t idx = (size_t)P * Kp + j;
        V[i] = (double)vh[idx] + (double)vl[idx];
    }
}

}  // namespace

// Host side: the df operator coefficients live in a DfOp built by the solver.
void launch_update_residual_df(const Launch& g, const Lev& L, int dim, bool var, const DfOpHost& h, const float* fh,
                               const float* fl, const float* vhin, const float* vlin, const float* x, float* vhout,
                               float* vlout, float* r32, float sf, const Red& red, cudaStream_t s) {
    DfOp op;
    op.wx = {h.w[0][0], h.w[0][1]};
    op.wy = {h.w[1][0], h.w[1][1]};
    op.wz = {h.w[2][0], h.w[2][1]};
    op.ch = h.ch;
    op.cl = h.cl;
    op.dh = h.dh;
    op.dl = h.dl;
    op.fxh = h.fh[0]; op.fxl = h.fl[0];
    op.fyh = h.fh[1]; op.fyl = h.fl[1];
    op.fzh = h.fh[2]; op.fzl = h.fl[2];
    const float inv_sf = 1.0f / sf;
    const size_t sh = (size_t)g.C * g.PPB * 4 * sizeof(double);
    if (dim == 2 && !var)
        launch_pdl(k_update_residual_df<2, false>, dim3(g.blocks), dim3(g.C, g.PPB), sh, s, L, g.Kp, op, fh, fl, vhin,
                   vlin, x, vhout, vlout, r32, sf, inv_sf, red);
    else if (dim == 2)
        launch_pdl(k_update_residual_df<2, true>, dim3(g.blocks), dim3(g.C, g.PPB), sh, s, L, g.Kp, op, fh, fl, vhin,
                   vlin, x, vhout, vlout, r32, sf, inv_sf, red);
    else if (!var)
        launch_pdl(k_update_residual_df<3, false>, dim3(g.blocks), dim3(g.C, g.PPB), sh, s, L, g.Kp, op, fh, fl, vhin,
                   vlin, x, vhout, vlout, r32, sf, inv_sf, red);
    else
        launch_pdl(k_update_residual_df<3, true>, dim3(g.blocks), dim3(g.C, g.PPB), sh, s, L, g.Kp, op, fh, fl, vhin,
                   vlin, x, vhout, vlout, r32, sf, inv_sf, red);
}

void launch_cast_f_df(const Launch& g32, long long N, int K, const double* f, double sf, float* r32, float* x32,
                      float* p32, float* fh, float* fl, cudaStream_t s) {
    k_cast_f_df<<<g32.blocks, dim3(g32.C, g32.PPB), 0, s>>>((int)N, g32.Kp, K, f, sf, r32, x32, p32, fh, fl);
}

void launch_weighted_sum_df(long long N, int Kp, int K, const float* vh, const float* vl, const float* ch,
                            const float* cl, double* u, int accumulate, cudaStream_t s) {
    const int threads = 256;
    const int blocks = (int)std::min<long long>((N + threads - 1) / threads, 152LL * 16);
    k_weighted_sum_df<<<blocks, threads, 0, s>>>((int)N, Kp, K, vh, vl, ch, cl, u, accumulate);
}

void launch_gather_df(long long N, int Kp, int K, const float* vh, const float* vl, double* V, cudaStream_t s) {
    const int threads = 256;
    const long long total = N * K;
    const int blocks = (int)std::min<long long>((total + threads - 1) / threads, 152LL * 16);
    k_gather_df<<<blocks, threads, 0, s>>>((int)N, Kp, K, vh, vl, V);
}

}  // namespace bura
