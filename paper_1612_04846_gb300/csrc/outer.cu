// Device-side control of a whole solve, so that the FP64 path and the mixed path with FP64 refinement
// run as one captured graph with no host round trip: the controller kernels (one CTA, one thread per
// system) take the decisions the host otherwise takes between the inner solves: the FP64 thresholds of
// the stopping rule, the refinement plan, the per-system scales and inner thresholds, the convergence
// test and the outcome.  The arithmetic is that of the host driver, step for step.
#include <cmath>

#include "kernels_impl.cuh"

namespace bura {

namespace {

constexpr int kCtlThreads = 32;  // >= KMAXP

// Fill the inner CG state record for a new inner solve (the state the host's init writes).
__device__ void init_inner(const OuterCfg* cfg, Scal* sc, int j, int active, double thr) {
    sc->rz[j] = 1.0;
    sc->pq[j] = 0.0;
    sc->alpha[j] = 0.0;
    sc->beta[j] = 0.0;
    sc->rr[j] = 0.0;
    sc->thr[j] = j < cfg->K ? thr : 0.0;
    sc->dsh[j] = j < cfg->K ? cfg->d[j] : 0.0;
    sc->alphaf[j] = 0.f;
    sc->betaf[j] = 0.f;
    sc->dshf[j] = (float)sc->dsh[j];
    sc->active[j] = active;
    sc->iters[j] = 0;
}

__device__ void init_inner_scalars(const OuterCfg* cfg, Scal* sc, int nactive) {
    sc->nactive = nactive;
    sc->breakdown = 0;
    sc->ticket = 0u;
    sc->it = 0;
    sc->max_it = cfg->max_iters;
    sc->parity = 0;
    sc->fault = 0;
    sc->wait_cycles = cfg->wait_cycles;
}

// From the FP64 residuals st->rr: stop (converged, cap reached, non-finite) or plan the next FP32 inner
// solve of the systems still above their thresholds: scale_j = ||r_j||, the inner right-hand side
// r_j / ||r_j|| and the inner relative target max(step_j / 2, sqrt(thr64_j / rr_j) / 2).
__device__ void decide(const OuterCfg* cfg, OuterState* st, Scal* sc, double* scale, double* invscale,
                       unsigned long long cond_outer) {
    __shared__ int act[kCtlThreads];
    __shared__ int bad;
    __shared__ int go;
    const int j = threadIdx.x;
    const int K = cfg->K;
    const double rr = j < K ? st->rr[j] : 0.0;
    if (j == 0) bad = 0;
    __syncthreads();
    act[j] = 0;
    if (j < K) {
        if (!isfinite(rr)) atomicExch(&bad, 1);
        act[j] = rr > st->thr64[j] ? 1 : 0;
    }
    __syncthreads();
    if (j == 0) {
        int na = 0;
        for (int q = 0; q < K; ++q) na += act[q];
        go = 0;
        if (bad) st->status = -4;                         // BURA_ENOTSPD
        else if (na == 0) st->status = 0;                 // BURA_OK
        else if (st->outer >= cfg->max_outer) st->status = -5;  // BURA_ENOCONV
        else go = 1;
        if (go) init_inner_scalars(cfg, sc, na);
        else st->done = 1;
        cudaGraphSetConditional(cond_outer, go ? 1u : 0u);
    }
    __syncthreads();
    if (go && j < KMAXP) {
        const bool a = j < K && act[j];
        const double hs = a ? sqrt(rr) : 0.0;
        scale[j] = hs;
        invscale[j] = a ? 1.0 / hs : 0.0;
        double thr = 0.0;
        if (a) {
            const double need = 0.5 * sqrt(st->thr64[j] / rr);
            const double t = fmax(st->step[j] * 0.5, need);
            thr = t * t;
        }
        init_inner(cfg, sc, j, a ? 1 : 0, thr);
    }
}

// Thresholds of the stopping rule on ||r_j||^2 (sum_j c_j ||r_j|| / (lambda_lo - d_j) <= tol ||f||, or the
// relative residual rule without lambda_lo) and, for the refinement, the plan of each system: need_j =
// sqrt(thr64_j) / ||f|| is reached in n_j = ceil(log need_j / log inner_rtol) steps of reduction need_j^(1/n_j).
__device__ void thresholds(const OuterCfg* cfg, OuterState* st, int j) {
    const int K = cfg->K;
    if (j >= K) return;
    const double t = cfg->lambda_lo > 0 ? st->tol * (cfg->lambda_lo - cfg->d[j]) / (K * cfg->c[j]) : st->tol;
    st->thr64[j] = t * t * st->fnorm2;
    const double need = st->fnorm2 > 0 ? sqrt(st->thr64[j] / st->fnorm2) : 1.0;
    if (need >= 1.0) {
        st->step[j] = 1.0;
    } else {
        const int n = max(1, (int)ceil(log(need) / log(cfg->inner_rtol) - 1e-9));
        st->step[j] = pow(need, 1.0 / n);
    }
}

}  // namespace

__global__ void k_solve_params(OuterState* st, const double* f, double tol) {
    st->f = f;
    st->tol = tol;
    st->done = 0;
}

// After ||f||^2 (KMAXP partial sums in norm_partials, summed in order): thresholds and plan; fp64 = 1 sets
// up the single FP64 PCG (all systems active when f != 0), fp64 = 0 the first refinement step.
__global__ void __launch_bounds__(kCtlThreads) k_outer_begin(const OuterCfg* cfg, OuterState* st,
                                                             const double* norm_partials, Scal* sc, double* scale,
                                                             double* invscale, unsigned long long cond_outer,
                                                             unsigned long long cond_inner, int fp64) {
    __shared__ double fn2;
    const int j = threadIdx.x;
    if (j == 0) {
        double s = 0.0;
        for (int i = 0; i < KMAXP; ++i) s += norm_partials[i];
        fn2 = s;
        st->fnorm2 = s;
        st->outer = 0;
        st->total_it = 0;
        st->status = -5;
    }
    __syncthreads();
    thresholds(cfg, st, j);
    if (j < KMAXP) {
        st->siters[j] = 0;
        st->rr[j] = j < cfg->K ? fn2 : 0.0;
    }
    __syncthreads();
    if (fp64) {
        const int a = (j < cfg->K && fn2 > 0) ? 1 : 0;
        if (j < KMAXP) init_inner(cfg, sc, j, a, j < cfg->K ? st->thr64[j] : 0.0);
        if (j == 0) {
            init_inner_scalars(cfg, sc, fn2 > 0 ? cfg->K : 0);
            cudaGraphSetConditional(cond_inner, fn2 > 0 ? 1u : 0u);
        }
        return;
    }
    decide(cfg, st, sc, scale, invscale, cond_outer);
}

// After an inner solve, its correction and the FP64 residual (||r_j||^2 in rr_partials): the inner
// solve's counts, then the next decision.
__global__ void __launch_bounds__(kCtlThreads) k_outer_next(const OuterCfg* cfg, OuterState* st,
                                                            const double* rr_partials, Scal* sc, double* scale,
                                                            double* invscale, unsigned long long cond_outer) {
    __shared__ int stop;
    const int j = threadIdx.x;
    if (j < cfg->K) st->siters[j] += sc->iters[j];
    if (j == 0) {
        st->total_it += sc->it;
        stop = 0;
        if (sc->fault) { st->status = -6; stop = 1; }           // BURA_ETIMEOUT
        else if (sc->breakdown) { st->status = -4; stop = 1; }  // BURA_ENOTSPD
        st->outer += 1;
        if (stop) {
            st->done = 1;
            cudaGraphSetConditional(cond_outer, 0u);
        }
    }
    __syncthreads();
    if (stop) return;
    if (j < cfg->K) st->rr[j] = rr_partials[j];
    __syncthreads();
    decide(cfg, st, sc, scale, invscale, cond_outer);
}

// The FP64 path's outcome from its CG state.
__global__ void __launch_bounds__(kCtlThreads) k_outer_end_fp64(const OuterCfg* cfg, OuterState* st, const Scal* sc) {
    const int j = threadIdx.x;
    if (j < cfg->K) {
        st->siters[j] = st->fnorm2 > 0 ? sc->iters[j] : 0;
        st->rr[j] = st->fnorm2 > 0 ? sc->rr[j] : 0.0;
    }
    if (j == 0) {
        st->outer = 1;
        st->total_it = st->fnorm2 > 0 ? sc->it : 0;
        st->status = st->fnorm2 > 0 ? (sc->fault ? -6 : sc->breakdown ? -4 : sc->nactive > 0 ? -5 : 0) : 0;
        st->done = 1;
    }
}

// The inner right-hand side of the current refinement step in FP32 (x = p = 0): f / ||f|| in the first
// step, r64_j / ||r_j|| afterwards (invscale_j = 0 for systems that are done); also arms the inner loop.
__global__ void k_cast_outer(int N, int Kp64, int Kp32, int K, const OuterState* st, const double* __restrict__ r64,
                             const double* __restrict__ invscale, float* __restrict__ r32, float* __restrict__ x32,
                             float* __restrict__ p32, unsigned long long cond_inner) {
    if (blockIdx.x == 0 && threadIdx.x == 0 && threadIdx.y == 0) cudaGraphSetConditional(cond_inner, 1u);
    const int off = threadIdx.x * 4;
    const bool first = st->outer == 0;
    const double* __restrict__ f = st->f;
    double is[4];
    for (int q = 0; q < 4; ++q) is[q] = (off + q < K) ? invscale[off + q] : 0.0;
    for (int tile = blockIdx.x; (long long)tile * blockDim.y < N; tile += gridDim.x) {
        const int P = tile * blockDim.y + threadIdx.y;
        if (P >= N) continue;
        float rv[4], zv[4];
        if (first) {
            const double fv = f[P];
            for (int q = 0; q < 4; ++q) { rv[q] = (float)(fv * is[q]); zv[q] = 0.f; }
        } else {
            for (int q = 0; q < 4; ++q) {
                rv[q] = (off + q < K) ? (float)(r64[(size_t)P * Kp64 + off + q] * is[q]) : 0.f;
                zv[q] = 0.f;
            }
        }
        const size_t base = (size_t)P * Kp32 + off;
        vst(r32 + base, rv);
        vst(x32 + base, zv);
        vst(p32 + base, zv);
    }
}

void launch_solve_params(OuterState* st, const double* f, double tol, cudaStream_t s) {
    k_solve_params<<<1, 1, 0, s>>>(st, f, tol);
}
void launch_outer_begin(const OuterCfg* cfg, OuterState* st, const double* norm_partials, Scal* sc, double* scale,
                        double* invscale, unsigned long long cond_outer, unsigned long long cond_inner, int fp64,
                        cudaStream_t s) {
    k_outer_begin<<<1, kCtlThreads, 0, s>>>(cfg, st, norm_partials, sc, scale, invscale, cond_outer, cond_inner, fp64);
}
void launch_outer_next(const OuterCfg* cfg, OuterState* st, const double* rr_partials, Scal* sc, double* scale,
                       double* invscale, unsigned long long cond_outer, cudaStream_t s) {
    k_outer_next<<<1, kCtlThreads, 0, s>>>(cfg, st, rr_partials, sc, scale, invscale, cond_outer);
}
void launch_outer_end_fp64(const OuterCfg* cfg, OuterState* st, const Scal* sc, cudaStream_t s) {
    k_outer_end_fp64<<<1, kCtlThreads, 0, s>>>(cfg, st, sc);
}
void launch_cast_outer(const Launch& g64, const Launch& g32, long long N, int K, const OuterState* st,
                       const double* r64, const double* invscale, float* r32, float* x32, float* p32,
                       unsigned long long cond_inner, cudaStream_t s) {
    k_cast_outer<<<g32.blocks, dim3(g32.C, g32.PPB), 0, s>>>((int)N, g64.Kp, g32.Kp, K, st, r64, invscale, r32, x32,
                                                             p32, cond_inner);
}

}  // namespace bura
