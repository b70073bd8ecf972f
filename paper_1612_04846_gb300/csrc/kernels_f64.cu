// FP64 instantiation of the multi-shift MG-PCG kernels, plus the FP64 refinement, cast and output
// kernels shared by both precision paths.
#include <cstddef>

#include "kernels_impl.cuh"

namespace bura {
template struct Ops<double>;

// r = f - (A - d_j I) v (FP64 true residual of every system) and ||r_j||^2 -> red.out.
template <int DIM, bool VAR>
__global__ void k_residual64(Lev L, int Kp, const double* __restrict__ f_arg, const double* const* fp,
                             const double* __restrict__ v, double* __restrict__ r, const double* __restrict__ dsh, Red red) {
    constexpr int W = 2;
    const double* __restrict__ f = fp ? *fp : f_arg;  // a captured solve reads its right-hand side's address
    const int off = threadIdx.x * W;
    double d[W];
    for (int q = 0; q < W; ++q) d[q] = dsh[off + q];
    Accum<double> acc;
    if constexpr (!VAR) {
        // constant coefficients: r = f - (diag - d_j) v_c + wx (v_w + v_e) + wy (v_s + v_n) [+ wz (...)] as
        // three fused multiply-adds on f after the two pair sums: 5 (2-D) FP64 operations per value, plus
        // one for ||r_j||^2 (GB300's FP64 rate bounds this kernel)
        const double diag = 2.0 * (L.wx + L.wy + (DIM == 3 ? L.wz : 0.0));
        double c0[W];
        for (int q = 0; q < W; ++q) c0[q] = diag - d[q];
        struct St { double xc[W], sx[W], sy[W], sz[W], fv; };
        sweep_u<St>(
            L.N, blockIdx.x, gridDim.x,
            [&](int P, St& st) {
                const Coord c = coord<DIM>(L, P);
                const size_t base = (size_t)P * Kp + off;
                const size_t sy = (size_t)L.nx * Kp, sz = (size_t)L.plane * Kp;
                double a[W], b[W];
                vld(v + base, st.xc);
                auto pair = [&](bool lo_in, bool hi_in, size_t step, double (&out)[W]) {
                    for (int q = 0; q < W; ++q) { a[q] = 0.0; b[q] = 0.0; }
                    if (lo_in) vld(v + base - step, a);
                    if (hi_in) vld(v + base + step, b);
                    for (int q = 0; q < W; ++q) out[q] = a[q] + b[q];
                };
                pair(c.i > 0, c.i < L.nx - 1, (size_t)Kp, st.sx);
                pair(c.j > 0, c.j < L.ny - 1, sy, st.sy);
                if (DIM == 3) pair(c.l > 0, c.l < L.nz - 1, sz, st.sz);
                st.fv = __ldg(f + P);
            },
            [&](int P, St& st) {
                double rv[W];
                for (int q = 0; q < W; ++q) {
                    double t = fma(-c0[q], st.xc[q], st.fv);
                    t = fma(L.wx, st.sx[q], t);
                    t = fma(L.wy, st.sy[q], t);
                    if (DIM == 3) t = fma(L.wz, st.sz[q], t);
                    rv[q] = t;
                }
                vst(r + (size_t)P * Kp + off, rv);
                acc.add(rv, rv);
            });
    } else if constexpr (DIM == 3) {
        zmarch<double, VAR>(L, Kp, v, blockIdx.x, gridDim.x,
                            [&](int P, size_t base, const double(&xc)[W], const double(&Ax)[W], double) {
                                const double fv = __ldg(f + P);
                                double rv[W];
                                for (int q = 0; q < W; ++q) rv[q] = fv - fma(-d[q], xc[q], Ax[q]);
                                vst(r + base, rv);
                                acc.add(rv, rv);
                            });
    } else {
        LoadPlain<double> ld{v};
        sweep_u<StencilState<double>>(
            L.N, blockIdx.x, gridDim.x,
            [&](int P, StencilState<double>& st) {
                stencil<double, DIM, VAR>(L, Kp, P, off, ld, st.xc, st.Ax, st.diag);
                st.bv[0] = __ldg(f + P);
            },
            [&](int P, StencilState<double>& st) {
                double rv[W];
                for (int q = 0; q < W; ++q) rv[q] = st.bv[0] - fma(-d[q], st.xc[q], st.Ax[q]);
                vst(r + (size_t)P * Kp + off, rv);
                acc.add(rv, rv);
            });
    }
    pdl_trigger();
    reduce_finish<double>(acc, red, Kp);
}

void launch_residual64(const Launch& g, const Lev& L, int dim, bool var, const double* f, const double* v,
                       double* r, const Red& red, cudaStream_t s, const double* const* fp) {
    const size_t sh = (size_t)g.C * g.PPB * 2 * sizeof(double);
    // the shifts live in the device Scal record (address arithmetic only, no host dereference)
    const double* dsh = reinterpret_cast<const double*>(reinterpret_cast<const char*>(red.scal) + offsetof(Scal, dsh));
    if (dim == 0) k_residual64<0, true><<<g.blocks, dim3(g.C, g.PPB), sh, s>>>(L, g.Kp, f, fp, v, r, dsh, red);
    else if (dim == 2 && !var) k_residual64<2, false><<<g.blocks, dim3(g.C, g.PPB), sh, s>>>(L, g.Kp, f, fp, v, r, dsh, red);
    else if (dim == 2) k_residual64<2, true><<<g.blocks, dim3(g.C, g.PPB), sh, s>>>(L, g.Kp, f, fp, v, r, dsh, red);
    else if (!var) k_residual64<3, false><<<g.blocks, dim3(g.C, g.PPB), sh, s>>>(L, g.Kp, f, fp, v, r, dsh, red);
    else k_residual64<3, true><<<g.blocks, dim3(g.C, g.PPB), sh, s>>>(L, g.Kp, f, fp, v, r, dsh, red);
}

// r32 = r64 * invscale_j (systems j < K with invscale > 0, else 0); x32 = 0; p32 = 0.  FP32 layout.
__global__ void k_cast_scaled(int N, int Kp64, int Kp32, int K, const double* __restrict__ r64,
                              const double* __restrict__ invscale, float* __restrict__ r32, float* __restrict__ x32,
                              float* __restrict__ p32) {
    const int off = threadIdx.x * 4;
    double is[4];
    for (int q = 0; q < 4; ++q) is[q] = (off + q < K) ? invscale[off + q] : 0.0;
    for (int tile = blockIdx.x; (long long)tile * blockDim.y < N; tile += gridDim.x) {
        const int P = tile * blockDim.y + threadIdx.y;
        if (P >= N) continue;
        float rv[4], zv[4];
        for (int q = 0; q < 4; ++q) {
            rv[q] = (off + q < K) ? (float)(r64[(size_t)P * Kp64 + off + q] * is[q]) : 0.f;
            zv[q] = 0.f;
        }
        const size_t base = (size_t)P * Kp32 + off;
        vst(r32 + base, rv);
        vst(x32 + base, zv);
        vst(p32 + base, zv);
    }
}

void launch_cast_scaled(const Launch& g64, const Launch& g32, long long N, int K, const double* r64,
                        const double* invscale, float* r32, float* x32, float* p32, cudaStream_t s) {
    k_cast_scaled<<<g32.blocks, dim3(g32.C, g32.PPB), 0, s>>>((int)N, g64.Kp, g32.Kp, K, r64, invscale, r32, x32, p32);
}

// v += scale_j * e (FP32 correction promoted to FP64); one thread per (point, pair of systems).
__global__ void k_correct64(int N, int Kp64, int Kp32, int K, double* __restrict__ v, const float* __restrict__ e,
                            const double* __restrict__ scale) {
    const int off = threadIdx.x * 2;
    double sc[2];
    for (int q = 0; q < 2; ++q) sc[q] = (off + q < K) ? scale[off + q] : 0.0;
    for (int tile = blockIdx.x; (long long)tile * blockDim.y < N; tile += gridDim.x) {
        const int P = tile * blockDim.y + threadIdx.y;
        if (P >= N) continue;
        const size_t b64 = (size_t)P * Kp64 + off;
        const float2 ev = *reinterpret_cast<const float2*>(e + (size_t)P * Kp32 + off);
        double2 vv = *reinterpret_cast<double2*>(v + b64);
        vv.x = fma(sc[0], (double)ev.x, vv.x);
        vv.y = fma(sc[1], (double)ev.y, vv.y);
        *reinterpret_cast<double2*>(v + b64) = vv;
    }
}

void launch_correct64(const Launch& g64, const Launch& g32, long long N, int K, double* v, const float* e,
                      const double* scale, cudaStream_t s) {
    k_correct64<<<g64.blocks, dim3(g64.C, g64.PPB), 0, s>>>((int)N, g64.Kp, g32.Kp, K, v, e, scale);
}

// ||f||^2 of a plain FP64 vector (red.out[0]); threads laid out as (1, 256) with two lanes of which
// the second stays zero, so the shared reduction machinery applies unchanged.
__global__ void k_norm2(int N, const double* __restrict__ f_arg, const double* const* fp, Red red) {
    const double* __restrict__ f = fp ? *fp : f_arg;
    Accum<double> acc;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int nthr = blockDim.x * blockDim.y;
    for (int P = blockIdx.x * nthr + tid; P < N; P += gridDim.x * nthr) {
        const double a[2] = {f[P], 0.0};
        acc.add(a, a);
    }
    // launched as (8, 32) threads: the shared reduction sees 32 "points" of KMAXP = 8 x 2 "systems", so the
    // block tail sums 16 groups instead of 128; red.out[0..KMAXP-1] holds KMAXP partial sums that the host
    // adds in a fixed order
    reduce_finish<double>(acc, red, KMAXP);
}

void launch_norm2(long long N, const double* f, const Red& red, int nsm, cudaStream_t s, const double* const* fp) {
    long long b = (N + 255) / 256;
    const int blocks = (int)(b < nsm * 2 ? (b > 0 ? b : 1) : nsm * 2);
    static_assert(KMAXP == 8 * 2, "k_norm2's launch shape gives KMAXP lanes");
    k_norm2<<<blocks, dim3(8, 32), 256 * 2 * sizeof(double), s>>>((int)N, f, fp, red);
}

// Final step of a deferred grid reduction (Red::defer): the producer, the previous kernel on the
// stream, has completed when griddepcontrol.wait returns, so its partials are visible without fences.
// The CG state record is loaded into shared memory together with the partials (one L2 round trip for
// both), updated there and written back whole; no other kernel touches it meanwhile.
__global__ void __launch_bounds__(kRedFinishThreads) k_red_finish(Red red, int Kp) {
    __shared__ double sm[kRedFinishThreads];
    __shared__ Scal sc;
    constexpr int kWords = (int)(sizeof(Scal) / sizeof(unsigned));
    static_assert(sizeof(Scal) % sizeof(unsigned) == 0 && kWords <= 2 * kRedFinishThreads, "Scal copy");
    pdl_trigger();  // the next kernel may start its prologue; it waits for this grid to complete
    pdl_wait();
    const int tid = threadIdx.x;
    const unsigned* gs = reinterpret_cast<const unsigned*>(red.scal);
    const unsigned w0 = tid < kWords ? __ldcg(gs + tid) : 0u;
    const unsigned w1 = tid + kRedFinishThreads < kWords ? __ldcg(gs + tid + kRedFinishThreads) : 0u;
    const double part = red_thread_sum(red.partial, (int)__ldcg(red.nblk), Kp);
    unsigned* ss = reinterpret_cast<unsigned*>(&sc);
    if (tid < kWords) ss[tid] = w0;
    if (tid + kRedFinishThreads < kWords) ss[tid + kRedFinishThreads] = w1;
    red_apply(red, &sc, part, Kp, sm);  // its first barrier publishes the copy
    __syncthreads();
    unsigned* gd = reinterpret_cast<unsigned*>(red.scal);
    if (tid < kWords) gd[tid] = ss[tid];
    if (tid + kRedFinishThreads < kWords) gd[tid + kRedFinishThreads] = ss[tid + kRedFinishThreads];
}

void launch_red_finish(const Red& red, int Kp, cudaStream_t s) {
    launch_pdl(k_red_finish, dim3(1), dim3(kRedFinishThreads), 0, s, red, Kp);
}

// r32 = f * invscale_j for every active system (the residual of the zero initial guess); x32 = p32 = 0.
__global__ void k_cast_f(int N, int Kp32, int K, const double* __restrict__ f, const double* __restrict__ invscale,
                         float* __restrict__ r32, float* __restrict__ x32, float* __restrict__ p32) {
    const int off = threadIdx.x * 4;
    // in the first refinement step every active system has the same scale 1/||f|| (0 for the inactive
    // ones): one FP64 product and one conversion per point serve all of them
    double is = 0.0;
    bool on[4];
    for (int q = 0; q < K && q < KMAXP; ++q) is = fmax(is, invscale[q]);
    for (int q = 0; q < 4; ++q) on[q] = (off + q < K) && invscale[off + q] != 0.0;
    for (int tile = blockIdx.x; (long long)tile * blockDim.y < N; tile += gridDim.x) {
        const int P = tile * blockDim.y + threadIdx.y;
        if (P >= N) continue;
        const float rf = (float)(f[P] * is);
        float rv[4], zv[4];
        for (int q = 0; q < 4; ++q) { rv[q] = on[q] ? rf : 0.f; zv[q] = 0.f; }
        const size_t base = (size_t)P * Kp32 + off;
        vst(r32 + base, rv);
        vst(x32 + base, zv);
        vst(p32 + base, zv);
    }
}

void launch_cast_f(const Launch& g32, long long N, int K, const double* f, const double* invscale, float* r32,
                   float* x32, float* p32, cudaStream_t s) {
    k_cast_f<<<g32.blocks, dim3(g32.C, g32.PPB), 0, s>>>((int)N, g32.Kp, K, f, invscale, r32, x32, p32);
}

// u = sum_j c_j v_j (FP64, fixed order j = 0..K-1); one thread per point.
__global__ void k_weighted_sum(int N, int Kp, int K, const double* __restrict__ v, const double* __restrict__ c,
                               double* __restrict__ u, int accumulate) {
    __shared__ double cs[KMAXP];
    if (threadIdx.x < KMAXP) cs[threadIdx.x] = threadIdx.x < K ? c[threadIdx.x] : 0.0;
    __syncthreads();
    for (int P = blockIdx.x * blockDim.x + threadIdx.x; P < N; P += gridDim.x * blockDim.x) {
        const double2* vp = reinterpret_cast<const double2*>(v + (size_t)P * Kp);
        double s = 0.0;
        for (int q = 0; q < Kp / 2; ++q) {
            const double2 a = vp[q];
            s = fma(cs[2 * q], a.x, s);
            s = fma(cs[2 * q + 1], a.y, s);
        }
        u[P] = accumulate ? u[P] + s : s;
    }
}

static int grid1(long long N, int bs) {
    long long b = (N + bs - 1) / bs;
    return (int)(b < 152 * 16 ? (b > 0 ? b : 1) : 152 * 16);
}

void launch_weighted_sum(long long N, int Kp, int K, const double* v, const double* c, double* u, int accumulate,
                         cudaStream_t s) {
    k_weighted_sum<<<grid1(N, 256), 256, 0, s>>>((int)N, Kp, K, v, c, u, accumulate);
}

__global__ void k_gather(int N, int Kp, int K, const double* __restrict__ v, double* __restrict__ V) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)N * K;
         t += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(t / N), P = (int)(t - (long long)j * N);
        V[t] = v[(size_t)P * Kp + j];
    }
}

__global__ void k_gather_f(int N, int Kp, int K, const float* __restrict__ v, double* __restrict__ V) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)N * K;
         t += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(t / N), P = (int)(t - (long long)j * N);
        V[t] = (double)v[(size_t)P * Kp + j];
    }
}

__global__ void k_scatter(int N, int Kp, int K, const double* __restrict__ X, double* __restrict__ x) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)N * Kp;
         t += (long long)gridDim.x * blockDim.x) {
        const int P = (int)(t / Kp), j = (int)(t - (long long)P * Kp);
        x[t] = j < K ? X[(size_t)j * N + P] : 0.0;
    }
}

void launch_gather_systems(long long N, int Kp, int K, const double* v, double* V, cudaStream_t s) {
    k_gather<<<grid1(N * K, 256), 256, 0, s>>>((int)N, Kp, K, v, V);
}
void launch_gather_systems_f(long long N, int Kp, int K, const float* v, double* V, cudaStream_t s) {
    k_gather_f<<<grid1(N * K, 256), 256, 0, s>>>((int)N, Kp, K, v, V);
}
void launch_scatter_systems(long long N, int Kp, int K, const double* X, double* x, cudaStream_t s) {
    k_scatter<<<grid1(N * Kp, 256), 256, 0, s>>>((int)N, Kp, K, X, x);
}

}  // namespace bura
