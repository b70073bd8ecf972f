// Kernel templates of the multi-shift MG-PCG; instantiated for float and double in
// kernels_f32.cu / kernels_f64.cu.  See kernels.cuh for the data layout.
//
// Every per-level operation is a __device__ "sweep" over the points of one level, distributed over
// CTAs by (first tile, tile stride).  The grid kernels pass (blockIdx.x, gridDim.x); the single-CTA
// coarse kernel runs the whole small-level part of the V-cycle with (0, 1) and __syncthreads()
// between dependent sweeps.
#pragma once
#include <cooperative_groups.h>

#include <mutex>

#include "kernels.cuh"

namespace cg = cooperative_groups;

namespace bura {

// A CG scalar of the Scal record in the kernel's precision: the FP32 kernels read the FP32 copies.
template <class T>
__device__ __forceinline__ T scal_val(const double* d, const float* f, int i) {
    if constexpr (sizeof(T) == 4) return f[i];
    else return d[i];
}

template <class T>
__device__ __forceinline__ void vld(const T* p, T (&o)[VecT<T>::W]) {
    typename VecT<T>::V v = *reinterpret_cast<const typename VecT<T>::V*>(p);
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

struct Coord { int i, j, l; };

// CTAs per SM the grid sweeps are compiled for (the register budget is 65536 / (256 x this)): the
// 2-D constant-coefficient stencils fit 64 registers, the 3-D, variable-coefficient and sparse ones
// (face weights, diagonal, coordinates of three axes) need BURA_SWEEP_REG_MINB or they spill.
#ifndef BURA_SWEEP_REG_MINB
#define BURA_SWEEP_REG_MINB 3
#endif
template <int DIM, bool VAR>
constexpr int sweep_min_blocks() {
    return (DIM == 2 && !VAR) ? kSweepMinBlocks : BURA_SWEEP_REG_MINB;
}

// Division by a shifted diagonal inside the preconditioner (Jacobi scaling of the Chebyshev steps): the
// FP32 kernels use the fast reciprocal-based division (a deterministic function of its operands, so the
// smoother stays the same fixed operator in every pre- and post-smoothing step); FP64 divides exactly.
template <class T>
__device__ __forceinline__ T jdiv(T a, T b) {
    if constexpr (sizeof(T) == 4) return __fdividef(a, b);
    else return a / b;
}
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

// A face weight of a variable-coefficient level: element i of the array, stored as T or, for the FP32
// kernels of a level with cbf16, as bfloat16 (the upper 16 bits of an FP32 value).
template <class T>
__device__ __forceinline__ T coef(const Lev& L, const void* a, size_t i) {
    if constexpr (sizeof(T) == 4) {
        if (L.cbf16) return __uint_as_float((unsigned)__ldg(reinterpret_cast<const unsigned short*>(a) + i) << 16);
    }
    return __ldg(reinterpret_cast<const T*>(a) + i);
}

template <class T, int DIM, bool VAR>
__device__ __forceinline__ Wts<T> weights(const Lev& L, int P, const Coord& c) {
    Wts<T> w;
    if (VAR) {
        const size_t row = (size_t)c.l * L.ny + c.j;  // (l, j) row of x-faces: nx+1 each
        w.xm = coef<T>(L, L.fx, row * (L.nx + 1) + c.i);
        w.xp = coef<T>(L, L.fx, row * (L.nx + 1) + c.i + 1);
        const size_t ybase = ((size_t)c.l * (L.ny + 1) + c.j) * L.nx + c.i;
        w.ym = coef<T>(L, L.fy, ybase);
        w.yp = coef<T>(L, L.fy, ybase + L.nx);
        if (DIM == 3) {
            w.zm = coef<T>(L, L.fz, P);
            w.zp = coef<T>(L, L.fz, P + L.plane);
        } else {
            w.zm = w.zp = T(0);
        }
    } else {
        w.xm = w.xp = sizeof(T) == 4 ? (T)L.wxf : (T)L.wx;
        w.ym = w.yp = sizeof(T) == 4 ? (T)L.wyf : (T)L.wy;
        w.zm = w.zp = sizeof(T) == 4 ? (T)L.wzf : (T)L.wz;
    }
    return w;
}

template <class T, int DIM, bool VAR>
__device__ __forceinline__ T diag_at(const Lev& L, int P) {
    if (DIM == 0 || (VAR && L.dg)) return __ldg(reinterpret_cast<const T*>(L.dg) + P);
    const Coord c = coord<DIM>(L, P);
    const Wts<T> w = weights<T, DIM, VAR>(L, P, c);
    T dg = w.xm + w.xp + w.ym + w.yp;
    if (DIM == 3) dg += w.zm + w.zp;
    return dg;
}

// ------------------------------------------------------------------ value loaders
// A loader returns the W values of chunk `off` at point P (idx = P*Kp + off).
template <class T>
struct LoadPlain {
    const T* x;
    __device__ __forceinline__ void operator()(int, size_t idx, T (&o)[VecT<T>::W]) const { vld(x + idx, o); }
};

// p_new = z + beta p_old evaluated on the fly (the CG p update fused into the operator apply).
template <class T>
struct LoadPUpd {
    const T* z;
    const T* p;
    T beta[VecT<T>::W];
    __device__ __forceinline__ void operator()(int, size_t idx, T (&o)[VecT<T>::W]) const {
        T a[VecT<T>::W], b[VecT<T>::W];
        vld(z + idx, a);
        vld(p + idx, b);
        for (int v = 0; v < VecT<T>::W; ++v) o[v] = fma(beta[v], b[v], a[v]);
    }
};

// First Chebyshev iterate from a zero guess, x1 = c2_0 Dinv b, evaluated on the fly.
template <class T, int DIM, bool VAR>
struct LoadCheb0 {
    const T* dg;  // the level's diagonal (variable coefficients and sparse operators)
    const T* b;
    T c2[VecT<T>::W];
    T d[VecT<T>::W];
    __device__ __forceinline__ void operator()(int P, size_t idx, T (&o)[VecT<T>::W]) const {
        vld(b + idx, o);
        if (VAR) {
            const T dp = __ldg(dg + P);
            for (int v = 0; v < VecT<T>::W; ++v) o[v] = jdiv(c2[v] * o[v], dp - d[v]);
        } else {
            for (int v = 0; v < VecT<T>::W; ++v) o[v] *= c2[v];
        }
    }
};

// x + P ec (bilinear / trilinear prolongation of the coarse correction, added on the fly).
template <class T, int DIM>
__device__ __forceinline__ void prolong_at(const Lev& Lf, const Lev& Lc, int Kp, int off, int P, const T* ec,
                                           T (&sum)[VecT<T>::W]) {
    constexpr int W = VecT<T>::W;
    const Coord c = coord<DIM>(Lf, P);
    const int fc[3] = {c.i, c.j, c.l};
    const int cn[3] = {Lc.nx, Lc.ny, Lc.nz};
    int lo[3], hi[3];
    T wl[3], wh[3];
    for (int a = 0; a < 3; ++a) {
        if (a >= DIM) { lo[a] = hi[a] = 0; wl[a] = T(1); wh[a] = T(0); continue; }
        const int f = fc[a];
        if (f & 1) { lo[a] = hi[a] = (f - 1) >> 1; wl[a] = T(1); wh[a] = T(0); }
        else {
            lo[a] = (f >> 1) - 1; hi[a] = f >> 1;
            wl[a] = lo[a] >= 0 ? T(0.5) : T(0);
            wh[a] = hi[a] < cn[a] ? T(0.5) : T(0);
            if (lo[a] < 0) lo[a] = 0;
            if (hi[a] >= cn[a]) hi[a] = cn[a] - 1;
        }
    }
    for (int v = 0; v < W; ++v) sum[v] = T(0);
    const int nz = DIM == 3 ? 2 : 1;
    for (int dz = 0; dz < nz; ++dz) {
        const int zc = dz ? hi[2] : lo[2];
        const T wz = dz ? wh[2] : wl[2];
        if (wz == T(0)) continue;
        for (int dy = 0; dy < 2; ++dy) {
            const int yc = dy ? hi[1] : lo[1];
            const T wy = dy ? wh[1] : wl[1];
            if (wy == T(0)) continue;
            for (int dx = 0; dx < 2; ++dx) {
                const int xc = dx ? hi[0] : lo[0];
                const T wx = dx ? wh[0] : wl[0];
                if (wx == T(0)) continue;
                const int Pc = (zc * Lc.ny + yc) * Lc.nx + xc;
                T e[W];
                vld(ec + (size_t)Pc * Kp + off, e);
                const T wt = wx * wy * wz;
                for (int v = 0; v < W; ++v) sum[v] = fma(wt, e[v], sum[v]);
            }
        }
    }
}

template <class T, int DIM>
struct LoadProlong {
    Lev Lf, Lc;
    int Kp, off;
    const T* x;
    const T* ec;
    __device__ __forceinline__ void operator()(int P, size_t idx, T (&o)[VecT<T>::W]) const {
        T s[VecT<T>::W];
        prolong_at<T, DIM>(Lf, Lc, Kp, off, P, ec, s);
        vld(x + idx, o);
        for (int v = 0; v < VecT<T>::W; ++v) o[v] += s[v];
    }
};

// A x at point P (no shift term) for the W systems of chunk `off`; xc = x(P), diag = A_PP.
// DIM = 0: a sparse row of the operator (CSR): every entry's value and column are loaded once for the
// W systems of the chunk, and the values of x at the columns come from the loader.
template <class T, int DIM, bool VAR, class LD>
__device__ __forceinline__ void stencil(const Lev& L, int Kp, int P, int off, const LD& ld,
                                        T (&xc)[VecT<T>::W], T (&Ax)[VecT<T>::W], T& diag) {
    constexpr int W = VecT<T>::W;
    if constexpr (DIM == 0) {
        diag = __ldg(reinterpret_cast<const T*>(L.dg) + P);
        ld(P, (size_t)P * Kp + off, xc);
        T acc[W];
        for (int v = 0; v < W; ++v) acc[v] = T(0);
        const int e = __ldg(L.rowptr + P + 1);
        const T* __restrict__ val = reinterpret_cast<const T*>(L.val);
        for (int q = __ldg(L.rowptr + P); q < e; ++q) {
            const int cq = __ldg(L.col + q);
            const T a = __ldg(val + q);
            T n[W];
            ld(cq, (size_t)cq * Kp + off, n);
            for (int v = 0; v < W; ++v) acc[v] = fma(a, n[v], acc[v]);
        }
        for (int v = 0; v < W; ++v) Ax[v] = acc[v];
        return;
    } else {
    const Coord c = coord<DIM>(L, P);
    const Wts<T> w = weights<T, DIM, VAR>(L, P, c);
    if (VAR && L.dg) {
        diag = __ldg(reinterpret_cast<const T*>(L.dg) + P);
    } else {
        diag = w.xm + w.xp + w.ym + w.yp;
        if (DIM == 3) diag += w.zm + w.zp;
    }
    const size_t base = (size_t)P * Kp + off;
    ld(P, base, xc);
    T acc[W];
    for (int v = 0; v < W; ++v) acc[v] = diag * xc[v];
    T n[W];
    if (c.i > 0) { ld(P - 1, base - Kp, n); for (int v = 0; v < W; ++v) acc[v] = fma(-w.xm, n[v], acc[v]); }
    if (c.i < L.nx - 1) { ld(P + 1, base + Kp, n); for (int v = 0; v < W; ++v) acc[v] = fma(-w.xp, n[v], acc[v]); }
    const size_t sy = (size_t)L.nx * Kp;
    if (c.j > 0) { ld(P - L.nx, base - sy, n); for (int v = 0; v < W; ++v) acc[v] = fma(-w.ym, n[v], acc[v]); }
    if (c.j < L.ny - 1) { ld(P + L.nx, base + sy, n); for (int v = 0; v < W; ++v) acc[v] = fma(-w.yp, n[v], acc[v]); }
    if (DIM == 3) {
        const size_t sz = (size_t)L.plane * Kp;
        const int pz = (int)L.plane;
        if (c.l > 0) { ld(P - pz, base - sz, n); for (int v = 0; v < W; ++v) acc[v] = fma(-w.zm, n[v], acc[v]); }
        if (c.l < L.nz - 1) { ld(P + pz, base + sz, n); for (int v = 0; v < W; ++v) acc[v] = fma(-w.zp, n[v], acc[v]); }
    }
    for (int v = 0; v < W; ++v) Ax[v] = acc[v];
    }
}

// ------------------------------------------------------------------ 3-D column sweeps
// The 3-D grid sweeps march along z: a work item is a segment of blockDim.y consecutive points of one
// x-row over kZRun planes, a thread one point column of it (one 16-byte chunk).  The values of x on the
// plane below and on the current plane stay in registers, so a point costs five neighbour loads (the new
// plane above and the four in-plane neighbours) instead of seven, and the coordinates come from the item,
// not from divisions per point.  Items are taken in a fixed order per CTA (b0, b0 + nb, ...), so the
// per-thread partial sums are deterministic.
constexpr int kZRun = 16;

template <class T, bool VAR, class Body>
__device__ __forceinline__ void zmarch(const Lev& L, int Kp, const T* __restrict__ x, int b0, int nb, Body&& body) {
    constexpr int W = VecT<T>::W;
    const int off = threadIdx.x * W;
    const int PX = (int)blockDim.y;
    const int nxs = (L.nx + PX - 1) / PX;
    const int nzc = (L.nz + kZRun - 1) / kZRun;
    const int per_z = nxs * L.ny;
    const int items = per_z * nzc;
    const size_t sx = (size_t)Kp, sy = (size_t)L.nx * Kp, sz = (size_t)L.plane * Kp;
    const T wxc = sizeof(T) == 4 ? (T)L.wxf : (T)L.wx, wyc = sizeof(T) == 4 ? (T)L.wyf : (T)L.wy;
    const T wzc = sizeof(T) == 4 ? (T)L.wzf : (T)L.wz;
    for (int item = b0; item < items; item += nb) {
        const int zc = item / per_z;
        const int rem = item - zc * per_z;
        const int j = rem / nxs;
        const int i = (rem - j * nxs) * PX + (int)threadIdx.y;
        if (i >= L.nx) continue;
        const int l0 = zc * kZRun;
        const int l1 = min(L.nz, l0 + kZRun);
        int P = (l0 * L.ny + j) * L.nx + i;
        size_t base = (size_t)P * Kp + off;
        T xm1[W], x0[W], xp1[W];
        for (int v = 0; v < W; ++v) xm1[v] = T(0);
        if (l0 > 0) vld(x + base - sz, xm1);
        vld(x + base, x0);
        T zlo = T(0);  // the face weight between planes l - 1 and l
        if (VAR) zlo = coef<T>(L, L.fz, (size_t)P);
        for (int l = l0; l < l1; ++l, P += (int)L.plane, base += sz) {
            for (int v = 0; v < W; ++v) xp1[v] = T(0);
            if (l + 1 < L.nz) vld(x + base + sz, xp1);
            T xl[W], xr[W], xd[W], xu[W];
            for (int v = 0; v < W; ++v) xl[v] = xr[v] = xd[v] = xu[v] = T(0);
            if (i > 0) vld(x + base - sx, xl);
            if (i < L.nx - 1) vld(x + base + sx, xr);
            if (j > 0) vld(x + base - sy, xd);
            if (j < L.ny - 1) vld(x + base + sy, xu);
            T wxm, wxp, wym, wyp, wzm, wzp, diag;
            if (VAR) {
                const size_t row = (size_t)l * L.ny + j;
                wxm = coef<T>(L, L.fx, row * (L.nx + 1) + i);
                wxp = coef<T>(L, L.fx, row * (L.nx + 1) + i + 1);
                const size_t yb = ((size_t)l * (L.ny + 1) + j) * L.nx + i;
                wym = coef<T>(L, L.fy, yb);
                wyp = coef<T>(L, L.fy, yb + L.nx);
                wzm = zlo;
                wzp = coef<T>(L, L.fz, (size_t)P + L.plane);
                zlo = wzp;
                diag = __ldg(reinterpret_cast<const T*>(L.dg) + P);
            } else {
                wxm = wxp = wxc;
                wym = wyp = wyc;
                wzm = wzp = wzc;
                diag = wxm + wxp + wym + wyp;
                diag += wzm + wzp;  // the association of the point stencil's diagonal
            }
            T Ax[W];
            for (int v = 0; v < W; ++v) {
                T a = diag * x0[v];
                a = fma(-wxm, xl[v], a);
                a = fma(-wxp, xr[v], a);
                a = fma(-wym, xd[v], a);
                a = fma(-wyp, xu[v], a);
                a = fma(-wzm, xm1[v], a);
                a = fma(-wzp, xp1[v], a);
                Ax[v] = a;
            }
            body(P, base, x0, Ax, diag);
            for (int v = 0; v < W; ++v) {
                xm1[v] = x0[v];
                x0[v] = xp1[v];
            }
        }
    }
}

// ------------------------------------------------------------------ reductions
__device__ __forceinline__ void finish_one(const Red& red, Scal* S, int s, double tot) {
    switch (red.op) {
        case RED_ALPHA: {
            S->pq[s] = tot;
            double a = 0.0;
            if (S->active[s]) {
                if (!(tot > 0.0) || !isfinite(tot)) S->breakdown = 1;
                else a = S->rz[s] / tot;
            }
            S->alpha[s] = a;
            S->alphaf[s] = (float)a;
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
            S->betaf[s] = (float)b;
            break;
        }
        case RED_STORE:
            red.out[s] = tot;
            break;
        default:
            break;
    }
}

// Final step of a grid reduction, by every thread of one block.  red_thread_sum: thread (s, g) adds
// partials g, g + G, g + 2G, ... of system s in that order (G = threads / Kp), with up to kRedFinBatch
// loads in flight (one L2 round trip per batch, not per partial).  red_apply: the G sums of each system
// in order, op applied to the CG state S and, for RED_CONV, the PCG bookkeeping and loop control.  sm
// holds at least one double per thread.
__device__ __forceinline__ double red_thread_sum(const double* fin, int nfin, int Kp) {
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int G = (int)(blockDim.x * blockDim.y) / Kp;
    double part = 0.0;
    if (tid < Kp * G) {
        const int s = tid % Kp, g = tid / Kp;
        for (int b0 = g; b0 < nfin; b0 += kRedFinBatch * G) {
            double v[kRedFinBatch];
#pragma unroll
            for (int j = 0; j < kRedFinBatch; ++j) {
                const int b = b0 + j * G;
                v[j] = b < nfin ? __ldcg(fin + (size_t)b * Kp + s) : 0.0;
            }
#pragma unroll
            for (int j = 0; j < kRedFinBatch; ++j) part += v[j];
        }
    }
    return part;
}

__device__ __forceinline__ void red_apply(const Red& red, Scal* S, double part, int Kp, double* sm) {
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int G = (int)(blockDim.x * blockDim.y) / Kp;
    __syncthreads();
    if (tid < Kp * G) sm[tid] = part;
    __syncthreads();
    if (tid < Kp) {
        double tot = 0.0;
        for (int g = 0; g < G; ++g) tot += sm[g * Kp + tid];
        finish_one(red, S, tid, tot);
    }
    __syncthreads();
    if (tid == 0 && red.op == RED_CONV) {
        int na = 0;
        for (int s = 0; s < Kp; ++s) na += S->active[s] ? 1 : 0;
        S->nactive = na;
        S->it += 1;
        S->parity ^= 1;
        // device-side loop control of a captured PCG loop (conditional WHILE node)
        if (red.cond) {
            const bool go = na > 0 && !S->breakdown && !S->fault && S->it < S->max_it;
            cudaGraphSetConditional(red.cond, go ? 1u : 0u);
        }
    }
}

// Block reduction of per-thread partials (W systems per thread, chunk = threadIdx.x) followed by
// the grid reduction in the last block, or, for a deferred reduction, by k_red_finish.  Every thread
// of the block must call this.
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
    const int nblk = (int)gridDim.x;
    if (red.defer) {
        // visible to k_red_finish, which waits for this grid to complete
        if (tid < Kp) {
            double tot = 0.0;
            for (int g = 0; g < G; ++g) tot += sm[g * Kp + tid];
            red.partial[(size_t)blockIdx.x * Kp + tid] = tot;
        }
        if (tid == 0 && blockIdx.x == 0) *red.nblk = (unsigned)nblk;
        return;
    }
    // one level (the last block sums every block partial) for grids up to kRedOneLevel blocks, such as
    // the persistent TMA kernels; two levels (groups of kRedGroup blocks) for the grid-stride kernels
    const bool one_level = nblk <= kRedOneLevel;
    const int group = one_level ? 0 : (int)blockIdx.x / kRedGroup;
    const int ngroups = one_level ? 1 : (nblk + kRedGroup - 1) / kRedGroup;
    const int gsize = one_level ? nblk : min(kRedGroup, nblk - group * kRedGroup);
    double* part2 = red.partial + (size_t)nblk * Kp;
    if (tid < Kp) {
        double tot = 0.0;
        for (int g = 0; g < G; ++g) tot += sm[g * Kp + tid];
        red.partial[(size_t)blockIdx.x * Kp + tid] = tot;
        __threadfence();  // only the writers of the partials need their stores visible before the ticket
    }
    __syncthreads();
    // level 1: the last block of the group (of the grid, with one level) sums its block partials
    if (tid == 0) {
        const unsigned t = atomicAdd(&red.tickets[group], 1u);
        am_last = (t == (unsigned)gsize - 1);
    }
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    // the partials to sum in the final step, in a fixed order: the block partials (one level) or the
    // group partials (two levels)
    const double* fin = red.partial;
    int nfin = nblk;
    if (!one_level) {
        if (tid < Kp) {
            const double* src = red.partial + (size_t)group * kRedGroup * Kp + tid;
            double v[kRedGroup];
#pragma unroll
            for (int b = 0; b < kRedGroup; ++b) v[b] = b < gsize ? __ldcg(src + (size_t)b * Kp) : 0.0;
            double tot = 0.0;
#pragma unroll
            for (int b = 0; b < kRedGroup; ++b) tot += v[b];
            part2[(size_t)group * Kp + tid] = tot;
            __threadfence();
        }
        __syncthreads();
        if (tid == 0) {
            red.tickets[group] = 0u;
            const unsigned t = atomicAdd(&red.tickets[ngroups], 1u);
            am_last = (t == (unsigned)ngroups - 1);
        }
        __syncthreads();
        if (!am_last) return;
        __threadfence();
        fin = part2;
        nfin = ngroups;
    }
    if (tid == 0) red.tickets[one_level ? 0 : ngroups] = 0u;
    red_apply(red, red.scal, red_thread_sum(fin, nfin, Kp), Kp, sm);
}

// ------------------------------------------------------------------ sweeps (per level)
#define BURA_SWEEP(NPTS)                                                                  \
    for (int tile = b0; (long long)tile * blockDim.y < (NPTS); tile += nb)                \
        if (const int P = tile * blockDim.y + threadIdx.y; P < (NPTS))

// Two-phase sweep: every thread takes U tiles per grid-stride step, issues the loads of all U first
// (`load(P, state)`) and only then computes and stores (`finish(P, state)`), so U independent load
// chains are in flight per thread.  The per-thread order of points is fixed (deterministic sums).
constexpr int kUnroll = 2;
template <class State, class LoadF, class FinishF>
__device__ __forceinline__ void sweep_u(long long N, int b0, int nb, LoadF&& load, FinishF&& finish) {
    for (int t0 = b0 * kUnroll; (long long)t0 * blockDim.y < N; t0 += nb * kUnroll) {
        State st[kUnroll];
        int P[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            P[u] = (t0 + u) * (int)blockDim.y + (int)threadIdx.y;
            if (P[u] < N) load(P[u], st[u]);
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
            if (P[u] < N) finish(P[u], st[u]);
    }
}

template <class T>
struct StencilState {
    T xc[VecT<T>::W], Ax[VecT<T>::W], bv[VecT<T>::W], dv[VecT<T>::W];
    T diag;
};

// x = c2_0 Dinv b (first Chebyshev step from a zero initial guess; pointwise).
template <class T, int DIM, bool VAR>
__device__ __forceinline__ void sw_cheb_zero(const Lev& L, int Kp, const T* b, T* x, ChebStepT<T> cs, const T* dsh,
                                             int b0, int nb) {
    constexpr int W = VecT<T>::W;
    const int off = threadIdx.x * W;
    LoadCheb0<T, DIM, VAR> ld;
    ld.dg = reinterpret_cast<const T*>(L.dg);
    ld.b = b;
    for (int v = 0; v < W; ++v) { ld.c2[v] = (T)cs.c2[off + v]; ld.d[v] = (T)dsh[off + v]; }
    BURA_SWEEP(L.N) {
        T xv[W];
        const size_t base = (size_t)P * Kp + off;
        ld(P, base, xv);
        vst(x + base, xv);
    }
}

// One Chebyshev step: res = b - (A - dI) xin; dnew = c1 din + c2 Dinv res; xout = xin + dnew.
// The input iterate comes from a loader (plain, first-step-from-zero, or prolongation-corrected);
// din may be null (c1 = 0) and is the loader's own value when din_is_x; dout may be null.
template <class T, int DIM, bool VAR, class LD>
__device__ __forceinline__ void sw_cheb_step(const Lev& L, int Kp, const LD& ld, const T* din, bool din_is_x,
                                             const T* b, T* xout, T* dout, ChebStepT<T> cs, const T* dsh,
                                             Accum<T>* acc, int b0, int nb) {
    constexpr int W = VecT<T>::W;
    const int off = threadIdx.x * W;
    T c1[W], c2[W], d[W];
    for (int v = 0; v < W; ++v) {
        c1[v] = cs.c1 ? (T)cs.c1[off + v] : T(0);
        c2[v] = (T)cs.c2[off + v];
        d[v] = (T)dsh[off + v];
    }
    sweep_u<StencilState<T>>(
        L.N, b0, nb,
        [&](int P, StencilState<T>& st) {
            stencil<T, DIM, VAR>(L, Kp, P, off, ld, st.xc, st.Ax, st.diag);
            const size_t base = (size_t)P * Kp + off;
            vld(b + base, st.bv);
            if (din_is_x) { for (int v = 0; v < W; ++v) st.dv[v] = st.xc[v]; }
            else if (din) vld(din + base, st.dv);
            else for (int v = 0; v < W; ++v) st.dv[v] = T(0);
        },
        [&](int P, StencilState<T>& st) {
            const size_t base = (size_t)P * Kp + off;
            T xo[W];
            for (int v = 0; v < W; ++v) {
                const T res = st.bv[v] - fma(-d[v], st.xc[v], st.Ax[v]);
                T g = c2[v] * res;
                if (VAR) g = jdiv(g, st.diag - d[v]);
                st.dv[v] = fma(c1[v], st.dv[v], g);
                xo[v] = st.xc[v] + st.dv[v];
            }
            vst(xout + base, xo);
            if (dout) vst(dout + base, st.dv);
            if (acc) acc->add(st.bv, xo);
        });
}

// bc = R (b - (A - dI) x): full weighting, R = P^T / 2^DIM with 1D weights (1/4, 1/2, 1/4).
template <class T, int DIM, bool VAR>
__device__ __forceinline__ void sw_restrict(const Lev& Lf, const Lev& Lc, int Kp, const T* x, const T* b, T* bc,
                                            const T* dsh, int b0, int nb) {
    constexpr int W = VecT<T>::W;
    const int off = threadIdx.x * W;
    T d[W];
    for (int v = 0; v < W; ++v) d[v] = (T)dsh[off + v];
    const T w1[3] = {T(0.25), T(0.5), T(0.25)};
    LoadPlain<T> ld{x};
    struct St { T sum[VecT<T>::W]; };
    sweep_u<St>(
        Lc.N, b0, nb,
        [&](int P, St& st) {
            const Coord cc = coord<DIM>(Lc, P);
            const int fi = 2 * cc.i + 1, fj = 2 * cc.j + 1, fl = (DIM == 3) ? 2 * cc.l + 1 : 0;
            for (int v = 0; v < W; ++v) st.sum[v] = T(0);
            const int zlo = (DIM == 3) ? -1 : 0, zhi = (DIM == 3) ? 1 : 0;
            for (int dz = zlo; dz <= zhi; ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        const int Pf = ((fl + dz) * Lf.ny + (fj + dy)) * Lf.nx + (fi + dx);
                        T xc[W], Ax[W], diag;
                        stencil<T, DIM, VAR>(Lf, Kp, Pf, off, ld, xc, Ax, diag);
                        T bv[W];
                        vld(b + (size_t)Pf * Kp + off, bv);
                        T wt = w1[dx + 1] * w1[dy + 1];
                        if (DIM == 3) wt *= w1[dz + 1];
                        for (int v = 0; v < W; ++v) st.sum[v] = fma(wt, bv[v] - fma(-d[v], xc[v], Ax[v]), st.sum[v]);
                    }
        },
        [&](int P, St& st) { vst(bc + (size_t)P * Kp + off, st.sum); });
}

// r = b - (A - dI) x on one level (the residual that sw_restrict_r restricts).
template <class T, int DIM, bool VAR>
__device__ __forceinline__ void sw_residual(const Lev& L, int Kp, const T* x, const T* b, T* r, const T* dsh,
                                            int b0, int nb) {
    constexpr int W = VecT<T>::W;
    const int off = threadIdx.x * W;
    T d[W];
    for (int v = 0; v < W; ++v) d[v] = (T)dsh[off + v];
    LoadPlain<T> ld{x};
    sweep_u<StencilState<T>>(
        L.N, b0, nb,
        [&](int P, StencilState<T>& st) {
            stencil<T, DIM, VAR>(L, Kp, P, off, ld, st.xc, st.Ax, st.diag);
            vld(b + (size_t)P * Kp + off, st.bv);
        },
        [&](int P, StencilState<T>& st) {
            T rv[W];
            for (int v = 0; v < W; ++v) rv[v] = st.bv[v] - fma(-d[v], st.xc[v], st.Ax[v]);
            vst(r + (size_t)P * Kp + off, rv);
        });
}

// bc = R r: full weighting of a stored fine-level residual (weights 1/4, 1/2, 1/4 per axis).
template <class T, int DIM>
__device__ __forceinline__ void sw_restrict_r(const Lev& Lf, const Lev& Lc, int Kp, const T* r, T* bc, int b0, int nb) {
    constexpr int W = VecT<T>::W;
    const int off = threadIdx.x * W;
    const T w1[3] = {T(0.25), T(0.5), T(0.25)};
    struct St { T sum[VecT<T>::W]; };
    sweep_u<St>(
        Lc.N, b0, nb,
        [&](int P, St& st) {
            const Coord cc = coord<DIM>(Lc, P);
            const int fi = 2 * cc.i + 1, fj = 2 * cc.j + 1, fl = (DIM == 3) ? 2 * cc.l + 1 : 0;
            for (int v = 0; v < W; ++v) st.sum[v] = T(0);
            const int zlo = (DIM == 3) ? -1 : 0, zhi = (DIM == 3) ? 1 : 0;
            for (int dz = zlo; dz <= zhi; ++dz)
                for (int dy = -1; dy <= 1; ++dy) {
                    const size_t row = ((size_t)(fl + dz) * Lf.ny + (fj + dy)) * Lf.nx;
                    const T wyz = w1[dy + 1] * (DIM == 3 ? w1[dz + 1] : T(1));
                    for (int dx = -1; dx <= 1; ++dx) {
                        T rv[W];
                        vld(r + (row + fi + dx) * Kp + off, rv);
                        const T wt = w1[dx + 1] * wyz;
                        for (int v = 0; v < W; ++v) st.sum[v] = fma(wt, rv[v], st.sum[v]);
                    }
                }
        },
        [&](int P, St& st) { vst(bc + (size_t)P * Kp + off, st.sum); });
}

// x += P ec (prolongation of the coarse correction; pointwise on the fine level).
template <class T, int DIM>
__device__ __forceinline__ void sw_prolong_add(const Lev& Lf, const Lev& Lc, int Kp, const T* ec, T* x, int b0,
                                               int nb) {
    constexpr int W = VecT<T>::W;
    const int off = threadIdx.x * W;
    struct St { T sum[VecT<T>::W], xv[VecT<T>::W]; };
    sweep_u<St>(
        Lf.N, b0, nb,
        [&](int P, St& st) {
            prolong_at<T, DIM>(Lf, Lc, Kp, off, P, ec, st.sum);
            vld(x + (size_t)P * Kp + off, st.xv);
        },
        [&](int P, St& st) {
            for (int v = 0; v < W; ++v) st.xv[v] += st.sum[v];
            vst(x + (size_t)P * Kp + off, st.xv);
        });
}

// ------------------------------------------------------------------ grid kernels
template <class T>
__global__ void __launch_bounds__(kSweepThreads, kSweepMinBlocks) k_broadcast(const double* __restrict__ f_arg, const double* const* fp, int N, int Kp, int K, T* r, T* x, T* p) {
    pdl_wait();
    const double* __restrict__ f = fp ? *fp : f_arg;
    constexpr int W = VecT<T>::W;
    const int off = threadIdx.x * W;
    const int b0 = blockIdx.x, nb = gridDim.x;
    BURA_SWEEP(N) {
        const T fv = (T)f[P];
        T rv[W], zv[W];
        for (int v = 0; v < W; ++v) { rv[v] = (off + v < K) ? fv : T(0); zv[v] = T(0); }
        const size_t base = (size_t)P * Kp + off;
        vst(r + base, rv);
        vst(x + base, zv);
        vst(p + base, zv);
    }
}

// The two direction buffers pa/pb alternate roles each iteration; the parity lives in the Scal
// record (toggled by the last block of k_cg_update), so a captured loop body can stay fixed.
template <class T, int DIM, bool VAR>
__global__ void __launch_bounds__(kSweepThreads, sweep_min_blocks<DIM, VAR>()) k_spmv_p(Lev L, int Kp, const T* __restrict__ z, T* pa, T* pb, T* __restrict__ q, Red red) {
    pdl_wait();
    constexpr int W = VecT<T>::W;
    const int off = threadIdx.x * W;
    const int b0 = blockIdx.x, nb = gridDim.x;
    const int par = red.scal->parity;
    const T* __restrict__ pold = par ? pb : pa;
    T* __restrict__ pnew = par ? pa : pb;
    LoadPUpd<T> ld;
    ld.z = z;
    ld.p = pold;
    T dsh[W];
    for (int v = 0; v < W; ++v) {
        ld.beta[v] = scal_val<T>(red.scal->beta, red.scal->betaf, off + v);
        dsh[v] = scal_val<T>(red.scal->dsh, red.scal->dshf, off + v);
    }
    Accum<T> acc;
    sweep_u<StencilState<T>>(
        L.N, b0, nb, [&](int P, StencilState<T>& st) { stencil<T, DIM, VAR>(L, Kp, P, off, ld, st.xc, st.Ax, st.diag); },
        [&](int P, StencilState<T>& st) {
            T qv[W];
            for (int v = 0; v < W; ++v) qv[v] = fma(-dsh[v], st.xc[v], st.Ax[v]);
            const size_t base = (size_t)P * Kp + off;
            vst(pnew + base, st.xc);
            vst(q + base, qv);
            acc.add(st.xc, qv);
        });
    pdl_trigger();
    reduce_finish<T>(acc, red, Kp);
}

// p = z + beta p into the direction buffer the parity selects (the p update of k_spmv_p as its own
// pointwise sweep, for operators whose stencil is costly to evaluate twice per neighbour).
template <class T>
__global__ void __launch_bounds__(kSweepThreads, kSweepMinBlocks) k_pupdate(int N, int Kp, const T* __restrict__ z,
                                                                        T* pa, T* pb, Red red) {
    pdl_wait();
    constexpr int W = VecT<T>::W;
    const int off = threadIdx.x * W;
    const int par = red.scal->parity;
    const T* __restrict__ pold = par ? pb : pa;
    T* __restrict__ pnew = par ? pa : pb;
    T beta[W];
    for (int v = 0; v < W; ++v) beta[v] = scal_val<T>(red.scal->beta, red.scal->betaf, off + v);
    struct St { T zv[VecT<T>::W], pv[VecT<T>::W]; };
    sweep_u<St>(
        N, blockIdx.x, gridDim.x,
        [&](int P, St& st) {
            const size_t base = (size_t)P * Kp + off;
            vld(z + base, st.zv);
            vld(pold + base, st.pv);
        },
        [&](int P, St& st) {
            T o[W];
            for (int v = 0; v < W; ++v) o[v] = fma(beta[v], st.pv[v], st.zv[v]);
            vst(pnew + (size_t)P * Kp + off, o);
        });
    pdl_trigger();
}

// q = (A - dI) p and p.q for the direction k_pupdate wrote (pa or pb by the parity).
template <class T, int DIM, bool VAR>
__global__ void __launch_bounds__(kSweepThreads, sweep_min_blocks<DIM, VAR>()) k_spmv_q(Lev L, int Kp, const T* pa,
                                                                                     const T* pb, T* __restrict__ q,
                                                                                     Red red) {
    pdl_wait();
    constexpr int W = VecT<T>::W;
    const int off = threadIdx.x * W;
    const T* __restrict__ p = red.scal->parity ? pa : pb;
    LoadPlain<T> ld{p};
    T dsh[W];
    for (int v = 0; v < W; ++v) dsh[v] = scal_val<T>(red.scal->dsh, red.scal->dshf, off + v);
    Accum<T> acc;
    if constexpr (DIM == 3) {
        zmarch<T, VAR>(L, Kp, p, blockIdx.x, gridDim.x, [&](int, size_t base, const T(&xc)[W], const T(&Ax)[W], T) {
            T qv[W];
            for (int v = 0; v < W; ++v) qv[v] = fma(-dsh[v], xc[v], Ax[v]);
            vst(q + base, qv);
            acc.add(xc, qv);
        });
    } else {
        sweep_u<StencilState<T>>(
            L.N, blockIdx.x, gridDim.x,
            [&](int P, StencilState<T>& st) { stencil<T, DIM, VAR>(L, Kp, P, off, ld, st.xc, st.Ax, st.diag); },
            [&](int P, StencilState<T>& st) {
                T qv[W];
                for (int v = 0; v < W; ++v) qv[v] = fma(-dsh[v], st.xc[v], st.Ax[v]);
                vst(q + (size_t)P * Kp + off, qv);
                acc.add(st.xc, qv);
            });
    }
    pdl_trigger();
    reduce_finish<T>(acc, red, Kp);
}

template <class T>
__global__ void __launch_bounds__(kSweepThreads, kSweepMinBlocks) k_cg_update(int N, int Kp, T* __restrict__ x, T* __restrict__ r, const T* pa, const T* pb,
                            const T* __restrict__ q, Red red) {
    pdl_wait();
    constexpr int W = VecT<T>::W;
    const int off = threadIdx.x * W;
    const int b0 = blockIdx.x, nb = gridDim.x;
    const T* __restrict__ p = red.scal->parity ? pa : pb;  // the direction k_spmv_p just wrote
    T a[W];
    for (int v = 0; v < W; ++v) a[v] = scal_val<T>(red.scal->alpha, red.scal->alphaf, off + v);
    Accum<T> acc;
    struct St { T xv[VecT<T>::W], rv[VecT<T>::W], pv[VecT<T>::W], qv[VecT<T>::W]; };
    sweep_u<St>(
        N, b0, nb,
        [&](int P, St& st) {
            const size_t base = (size_t)P * Kp + off;
            vld(x + base, st.xv);
            vld(r + base, st.rv);
            vld(p + base, st.pv);
            vld(q + base, st.qv);
        },
        [&](int P, St& st) {
            const size_t base = (size_t)P * Kp + off;
            for (int v = 0; v < W; ++v) {
                st.xv[v] = fma(a[v], st.pv[v], st.xv[v]);
                st.rv[v] = fma(-a[v], st.qv[v], st.rv[v]);
            }
            vst(x + base, st.xv);
            vst(r + base, st.rv);
            acc.add(st.rv, st.rv);
        });
    pdl_trigger();
    reduce_finish<T>(acc, red, Kp);
}

template <class T, int DIM, bool VAR>
__global__ void __launch_bounds__(kSweepThreads, sweep_min_blocks<DIM, VAR>()) k_cheb_zero(Lev L, int Kp, const T* __restrict__ b, T* __restrict__ x, ChebStepT<T> cs,
                            const T* __restrict__ dsh) {
    pdl_wait();
    sw_cheb_zero<T, DIM, VAR>(L, Kp, b, x, cs, dsh, blockIdx.x, gridDim.x);
}

// Plain Chebyshev step (input iterate read from xin).
template <class T, int DIM, bool VAR>
__global__ void __launch_bounds__(kSweepThreads, sweep_min_blocks<DIM, VAR>()) k_cheb_step(Lev L, int Kp, const T* __restrict__ xin, const T* __restrict__ din,
                            const T* __restrict__ b, T* __restrict__ xout, T* __restrict__ dout, ChebStepT<T> cs,
                            const T* __restrict__ dsh, Red red) {
    pdl_wait();
    LoadPlain<T> ld{xin};
    Accum<T> acc;
    const bool dot = red.op != RED_NONE;
    if constexpr (DIM == 3) {
        constexpr int W = VecT<T>::W;
        const int off = threadIdx.x * W;
        T c1[W], c2[W], d[W];
        for (int v = 0; v < W; ++v) {
            c1[v] = cs.c1 ? (T)cs.c1[off + v] : T(0);
            c2[v] = (T)cs.c2[off + v];
            d[v] = (T)dsh[off + v];
        }
        zmarch<T, VAR>(L, Kp, xin, blockIdx.x, gridDim.x, [&](int, size_t base, const T(&xc)[W], const T(&Ax)[W], T diag) {
            T bv[W], dv[W], xo[W];
            vld(b + base, bv);
            if (din) vld(din + base, dv);
            else for (int v = 0; v < W; ++v) dv[v] = T(0);
            for (int v = 0; v < W; ++v) {
                const T res = bv[v] - fma(-d[v], xc[v], Ax[v]);
                T g = c2[v] * res;
                if (VAR) g = jdiv(g, diag - d[v]);
                dv[v] = fma(c1[v], dv[v], g);
                xo[v] = xc[v] + dv[v];
            }
            vst(xout + base, xo);
            if (dout) vst(dout + base, dv);
            if (dot) acc.add(bv, xo);
        });
    } else {
        sw_cheb_step<T, DIM, VAR>(L, Kp, ld, din, false, b, xout, dout, cs, dsh, dot ? &acc : nullptr, blockIdx.x,
                                  gridDim.x);
    }
    pdl_trigger();
    if (dot) reduce_finish<T>(acc, red, Kp);
}

// First two Chebyshev steps from a zero guess in one sweep: x1 = c2_0 Dinv b is evaluated at the
// stencil points on the fly (d_1 = x1), then the second step is applied.
template <class T, int DIM, bool VAR>
__global__ void __launch_bounds__(kSweepThreads, sweep_min_blocks<DIM, VAR>()) k_cheb_pre2(Lev L, int Kp, const T* __restrict__ b, T* __restrict__ xout, T* __restrict__ dout,
                            ChebStepT<T> cs0, ChebStepT<T> cs1, const T* __restrict__ dsh) {
    pdl_wait();
    constexpr int W = VecT<T>::W;
    const int off = threadIdx.x * W;
    LoadCheb0<T, DIM, VAR> ld;
    ld.dg = reinterpret_cast<const T*>(L.dg);
    ld.b = b;
    for (int v = 0; v < W; ++v) { ld.c2[v] = (T)cs0.c2[off + v]; ld.d[v] = (T)dsh[off + v]; }
    sw_cheb_step<T, DIM, VAR>(L, Kp, ld, nullptr, true, b, xout, dout, cs1, dsh, nullptr, blockIdx.x, gridDim.x);
}

// First post-smoothing step with the coarse-grid correction added on the fly: xin = x + P ec.
template <class T, int DIM, bool VAR>
__global__ void __launch_bounds__(kSweepThreads, sweep_min_blocks<DIM, VAR>()) k_post_prolong(Lev Lf, Lev Lc, int Kp, const T* __restrict__ x, const T* __restrict__ ec,
                               const T* __restrict__ b, T* __restrict__ xout, T* __restrict__ dout, ChebStepT<T> cs,
                               const T* __restrict__ dsh, Red red) {
    pdl_wait();
    constexpr int W = VecT<T>::W;
    LoadProlong<T, DIM> ld{Lf, Lc, Kp, (int)threadIdx.x * W, x, ec};
    Accum<T> acc;
    const bool dot = red.op != RED_NONE;
    sw_cheb_step<T, DIM, VAR>(Lf, Kp, ld, nullptr, false, b, xout, dout, cs, dsh, dot ? &acc : nullptr, blockIdx.x,
                              gridDim.x);
    pdl_trigger();
    if (dot) reduce_finish<T>(acc, red, Kp);
}

template <class T, int DIM>
__global__ void __launch_bounds__(kSweepThreads, kSweepMinBlocks) k_prolong_add(Lev Lf, Lev Lc, int Kp, const T* __restrict__ ec, T* __restrict__ x) {
    pdl_wait();
    sw_prolong_add<T, DIM>(Lf, Lc, Kp, ec, x, blockIdx.x, gridDim.x);
}

// 3-D x += P ec (trilinear) as z-marching columns, items as in zmarch: the bilinear (x, y) interpolation
// of the coarse correction on a coarse plane is formed once and serves the three fine planes that
// read it (2m, 2m + 1, 2m + 2); a fine plane takes it with weight 1 (odd) or the two neighbouring
// coarse planes with 1/2 each (even), zero outside the coarse grid.  The same operator as prolong_at,
// summed in another order (the (x, y) weights first).
template <class T>
__device__ __forceinline__ void prolong_axis(int f, int nc, int& lo, int& hi, T& wl, T& wh) {
    if (f & 1) { lo = hi = (f - 1) >> 1; wl = T(1); wh = T(0); }
    else {
        lo = (f >> 1) - 1; hi = f >> 1;
        wl = lo >= 0 ? T(0.5) : T(0);
        wh = hi < nc ? T(0.5) : T(0);
        if (lo < 0) lo = 0;
        if (hi >= nc) hi = nc - 1;
    }
}
template <class T>
__global__ void __launch_bounds__(kSweepThreads, sweep_min_blocks<3, true>()) k_prolong_add_z(Lev Lf, Lev Lc, int Kp, const T* __restrict__ ec, T* __restrict__ x) {
    pdl_wait();
    constexpr int W = VecT<T>::W;
    const int off = threadIdx.x * W;
    const int PX = (int)blockDim.y;
    const int nxs = (Lf.nx + PX - 1) / PX;
    const int nzc = (Lf.nz + kZRun - 1) / kZRun;
    const int per_z = nxs * Lf.ny;
    const int items = per_z * nzc;
    for (int item = blockIdx.x; item < items; item += gridDim.x) {
        const int zc = item / per_z;
        const int rem = item - zc * per_z;
        const int j = rem / nxs;
        const int i = (rem - j * nxs) * PX + (int)threadIdx.y;
        if (i >= Lf.nx) continue;
        int xl, xh, yl, yh;
        T wxl, wxh, wyl, wyh;
        prolong_axis<T>(i, Lc.nx, xl, xh, wxl, wxh);
        prolong_axis<T>(j, Lc.ny, yl, yh, wyl, wyh);
        const T w00 = wxl * wyl, w01 = wxh * wyl, w10 = wxl * wyh, w11 = wxh * wyh;
        // the footprint of coarse plane m (zero outside the coarse grid), and its (x, y) interpolation
        auto fetch = [&](int m, T (&e)[4][W]) {
            for (int q = 0; q < 4; ++q)
                for (int v = 0; v < W; ++v) e[q][v] = T(0);
            if (m < 0 || m >= Lc.nz) return;
            const size_t pb = (size_t)m * Lc.ny;
            if (w00 != T(0)) vld(ec + ((pb + yl) * Lc.nx + xl) * Kp + off, e[0]);
            if (w01 != T(0)) vld(ec + ((pb + yl) * Lc.nx + xh) * Kp + off, e[1]);
            if (w10 != T(0)) vld(ec + ((pb + yh) * Lc.nx + xl) * Kp + off, e[2]);
            if (w11 != T(0)) vld(ec + ((pb + yh) * Lc.nx + xh) * Kp + off, e[3]);
        };
        auto combine = [&](const T (&e)[4][W], T (&sv)[W]) {
            for (int v = 0; v < W; ++v) {
                T t = T(0);
                if (w00 != T(0)) t = fma(w00, e[0][v], t);
                if (w01 != T(0)) t = fma(w01, e[1][v], t);
                if (w10 != T(0)) t = fma(w10, e[2][v], t);
                if (w11 != T(0)) t = fma(w11, e[3][v], t);
                sv[v] = t;
            }
        };
        const int l0 = zc * kZRun;  // even
        const int l1 = min(Lf.nz, l0 + kZRun);
        T sp[W], sc[W];             // the interpolations on coarse planes l / 2 - 1 and l / 2 (l even)
        T en[4][W];                 // the footprint of the next coarse plane, fetched one fine plane early
        fetch((l0 >> 1) - 1, en);
        combine(en, sp);
        fetch(l0 >> 1, en);
        combine(en, sc);
        size_t base = ((size_t)l0 * Lf.plane + (size_t)j * Lf.nx + i) * Kp + off;
        const size_t sz = (size_t)Lf.plane * Kp;
        T xn[W];  // x on the next fine plane, loaded one plane early
        vld(x + base, xn);
        for (int l = l0; l < l1; ++l, base += sz) {
            T xv[W], val[W];
            for (int v = 0; v < W; ++v) xv[v] = xn[v];
            if (l + 1 < l1) vld(x + base + sz, xn);
            if (l & 1) {
                for (int v = 0; v < W; ++v) val[v] = sc[v];
                if (l + 1 < l1) fetch((l + 1) >> 1, en);  // the plane the next (even) fine plane adds
            } else {
                if (l > l0) {
                    for (int v = 0; v < W; ++v) sp[v] = sc[v];
                    combine(en, sc);
                }
                for (int v = 0; v < W; ++v) val[v] = fma(T(0.5), sc[v], T(0.5) * sp[v]);
            }
            for (int v = 0; v < W; ++v) xv[v] += val[v];
            vst(x + base, xv);
        }
    }
}

template <class T, int DIM, bool VAR>
__global__ void __launch_bounds__(kSweepThreads, sweep_min_blocks<DIM, VAR>()) k_restrict_res(Lev Lf, Lev Lc, int Kp, const T* __restrict__ x, const T* __restrict__ b,
                               T* __restrict__ bc, const T* __restrict__ dsh) {
    pdl_wait();
    sw_restrict<T, DIM, VAR>(Lf, Lc, Kp, x, b, bc, dsh, blockIdx.x, gridDim.x);
}

template <class T, int DIM, bool VAR>
__global__ void __launch_bounds__(kSweepThreads, sweep_min_blocks<DIM, VAR>()) k_residual(Lev L, int Kp, const T* __restrict__ x,
                                                                         const T* __restrict__ b, T* __restrict__ r,
                                                                         const T* __restrict__ dsh) {
    pdl_wait();
    if constexpr (DIM == 3) {
        constexpr int W = VecT<T>::W;
        const int off = threadIdx.x * W;
        T d[W];
        for (int v = 0; v < W; ++v) d[v] = (T)dsh[off + v];
        zmarch<T, VAR>(L, Kp, x, blockIdx.x, gridDim.x, [&](int, size_t base, const T(&xc)[W], const T(&Ax)[W], T) {
            T bv[W], rv[W];
            vld(b + base, bv);
            for (int v = 0; v < W; ++v) rv[v] = bv[v] - fma(-d[v], xc[v], Ax[v]);
            vst(r + base, rv);
        });
    } else {
        sw_residual<T, DIM, VAR>(L, Kp, x, b, r, dsh, blockIdx.x, gridDim.x);
    }
}

template <class T, int DIM>
__global__ void __launch_bounds__(kSweepThreads, kSweepMinBlocks) k_restrict_r(Lev Lf, Lev Lc, int Kp,
                                                                           const T* __restrict__ r, T* __restrict__ bc) {
    pdl_wait();
    sw_restrict_r<T, DIM>(Lf, Lc, Kp, r, bc, blockIdx.x, gridDim.x);
}

template <class T, int DIM, bool VAR>
__global__ void __launch_bounds__(kSweepThreads, sweep_min_blocks<DIM, VAR>()) k_apply_shifted(Lev L, int Kp, const T* __restrict__ x, T* __restrict__ y,
                                const T* __restrict__ dsh) {
    pdl_wait();
    constexpr int W = VecT<T>::W;
    const int off = threadIdx.x * W;
    const int b0 = blockIdx.x, nb = gridDim.x;
    T d[W];
    for (int v = 0; v < W; ++v) d[v] = (T)dsh[off + v];
    LoadPlain<T> ld{x};
    BURA_SWEEP(L.N) {
        T xc[W], Ax[W], diag;
        stencil<T, DIM, VAR>(L, Kp, P, off, ld, xc, Ax, diag);
        for (int v = 0; v < W; ++v) Ax[v] = fma(-d[v], xc[v], Ax[v]);
        vst(y + (size_t)P * Kp + off, Ax);
    }
}

template <class T>
__global__ void __launch_bounds__(kSweepThreads, kSweepMinBlocks) k_dot(int N, int Kp, const T* __restrict__ a, const T* __restrict__ b, Red red) {
    pdl_wait();
    constexpr int W = VecT<T>::W;
    const int off = threadIdx.x * W;
    const int b0 = blockIdx.x, nb = gridDim.x;
    Accum<T> acc;
    struct St { T av[VecT<T>::W], bv[VecT<T>::W]; };
    sweep_u<St>(
        N, b0, nb,
        [&](int P, St& st) {
            vld(a + (size_t)P * Kp + off, st.av);
            vld(b + (size_t)P * Kp + off, st.bv);
        },
        [&](int, St& st) { acc.add(st.av, st.bv); });
    pdl_trigger();
    reduce_finish<T>(acc, red, Kp);
}

// ------------------------------------------------------------------ single-CTA coarse V-cycle
// Runs levels l0..nlev-1 of the V-cycle (all with few points) with every vector in shared memory: the
// same sweeps as the grid kernels with (first tile, stride) = (0, 1) and __syncthreads() between
// dependent sweeps.  The V-cycle of one shifted system never touches another system's values, so CTA
// `blockIdx.x` runs the systems of one 16-byte chunk (W of them) on its own SM: the chunk's values are
// stored compactly (stride W) in shared memory and the global arrays are addressed at chunk offset
// blockIdx.x * W with their own stride Kp.  b of level l0 is read from and its result written to global.
template <class T, int DIM, bool VAR>
__global__ void __launch_bounds__(kCoarseThreads) k_coarse_cycle(CoarseArgs a) {
    pdl_wait();
    constexpr int W = VecT<T>::W;
    extern __shared__ __align__(16) unsigned char csm[];
    auto at = [&](unsigned int off) { return reinterpret_cast<T*>(csm + off); };
    const int nthr = blockDim.x * blockDim.y;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int ch = blockIdx.x * W;  // first system of this CTA's chunk
    const int Kp = a.Kp;            // stride of the global arrays
    constexpr int Ks = W;           // stride of the shared-memory vectors
    {
        const int n = (int)a.lev[0].L.N;
        const T* src = reinterpret_cast<const T*>(a.b_in) + ch;
        T* dst = at(a.lev[0].b);
        for (int i = tid; i < n; i += nthr) {
            T v[W];
            vld(src + (size_t)i * Kp, v);
            vst(dst + (size_t)i * Ks, v);
        }
        // the shifts and the small Chebyshev tables are read by every sweep: keep them on chip
        T* ds = at(a.dsh_ofs);
        for (int i = tid; i < W; i += nthr) ds[i] = reinterpret_cast<const T*>(a.dsh)[ch + i];
        for (int l = 0; l < a.nlev; ++l) {
            const CoarseLevel& c = a.lev[l];
            if (c.cofs == kNoCopy) continue;
            T* t = at(c.cofs);
            const int m = c.deg * W;
            for (int i = tid; i < m; i += nthr) {
                const int row = i / W, v = i - row * W;
                t[i] = reinterpret_cast<const T*>(c.c1)[row * Kp + ch + v];
                t[m + i] = reinterpret_cast<const T*>(c.c2)[row * Kp + ch + v];
            }
        }
        // this chunk's dense inverses (read once per V-cycle by the exact solve): independent 16-byte
        // loads by every thread now instead of a chain of dependent global loads per row later
        if (a.exact >= 0 && a.minv_ofs != kNoCopy) {
            const int n = (int)a.lev[a.exact].L.N;
            const T* src = reinterpret_cast<const T*>(a.minv) + ch;
            T* dst = at(a.minv_ofs);
            for (int i = tid; i < n * n; i += nthr) {
                T v[W];
                vld(src + (size_t)i * Kp, v);
                vst(dst + (size_t)i * W, v);
            }
        }
    }
    __syncthreads();
    const T* dsh = at(a.dsh_ofs);
    // step m of level c's Chebyshev tables: compact copies in shared memory or the global rows
    auto step = [&](const CoarseLevel& c, int m, bool with_c1) {
        if (c.cofs == kNoCopy)
            return ChebStepT<T>{with_c1 ? reinterpret_cast<const T*>(c.c1) + (size_t)m * Kp + ch : nullptr,
                                reinterpret_cast<const T*>(c.c2) + (size_t)m * Kp + ch};
        const T* t = at(c.cofs);
        return ChebStepT<T>{with_c1 ? t + m * W : nullptr, t + (c.deg + m) * W};
    };
    // down: pre-smoothing and restriction
    for (int l = 0; l < a.nlev; ++l) {
        const CoarseLevel& c = a.lev[l];
        const int deg = c.deg;
        T* A = at(c.xa);
        T* B = at(c.xb);
        T* D = at(c.dd);
        const T* b = at(c.b);
        if (l == a.exact) {  // dense exact solve of every shifted system: A = M_j b
            const int n = (int)c.L.N;
            const bool staged = a.minv_ofs != kNoCopy;
            const T* M = staged ? at(a.minv_ofs) : reinterpret_cast<const T*>(a.minv) + ch;
            const int ms = staged ? W : Kp;  // stride between the entries of M
            for (int i = threadIdx.y; i < n; i += blockDim.y) {
                T acc[W];
                for (int v = 0; v < W; ++v) acc[v] = T(0);
                const T* row = M + (size_t)i * n * ms;
#pragma unroll 4
                for (int jj = 0; jj < n; ++jj) {
                    T m[W], bv[W];
                    vld(row + (size_t)jj * ms, m);
                    vld(b + (size_t)jj * Ks, bv);
                    for (int v = 0; v < W; ++v) acc[v] = fma(m[v], bv[v], acc[v]);
                }
                vst(A + (size_t)i * Ks, acc);
            }
            __syncthreads();
            break;
        }
        sw_cheb_zero<T, DIM, VAR>(c.L, Ks, b, A, step(c, 0, true), dsh, 0, 1);
        __syncthreads();
        T* cur = A;
        T* oth = B;
        for (int m = 1; m < deg; ++m) {
            LoadPlain<T> ld{cur};
            // after the step from zero the previous Chebyshev direction is the iterate itself
            sw_cheb_step<T, DIM, VAR>(c.L, Ks, ld, m == 1 ? nullptr : D, m == 1, b, oth, m < deg - 1 ? D : nullptr,
                                      step(c, m, true), dsh, nullptr, 0, 1);
            __syncthreads();
            T* t = cur; cur = oth; oth = t;
        }
        if (l + 1 < a.nlev) {
            sw_restrict<T, DIM, VAR>(c.L, a.lev[l + 1].L, Ks, cur, b, at(a.lev[l + 1].b), dsh, 0, 1);
            __syncthreads();
        }
    }
    // up: correction and post-smoothing (the coarsest level has no post-smoothing)
    for (int l = a.nlev - 2; l >= 0; --l) {
        const CoarseLevel& c = a.lev[l];
        const int deg = c.deg;
        T* A = at(c.xa);
        T* B = at(c.xb);
        T* D = at(c.dd);
        const T* b = at(c.b);
        T* cur = ((deg - 1) % 2 == 0) ? A : B;  // where the pre-smoothing ended
        T* oth = cur == A ? B : A;
        sw_prolong_add<T, DIM>(c.L, a.lev[l + 1].L, Ks, at(a.lev[l + 1].result), cur, 0, 1);
        __syncthreads();
        for (int m = 0; m < deg; ++m) {
            LoadPlain<T> ld{cur};
            sw_cheb_step<T, DIM, VAR>(c.L, Ks, ld, m == 0 ? nullptr : D, false, b, oth, m < deg - 1 ? D : nullptr,
                                      step(c, m, m != 0), dsh, nullptr, 0, 1);
            __syncthreads();
            T* t = cur; cur = oth; oth = t;
        }
    }
    {
        const int n = (int)a.lev[0].L.N;
        const T* src = at(a.lev[0].result);
        T* dst = reinterpret_cast<T*>(a.x_out) + ch;
        for (int i = tid; i < n; i += nthr) {
            T v[W];
            vld(src + (size_t)i * Ks, v);
            vst(dst + (size_t)i * Kp, v);
        }
    }
}

// ------------------------------------------------------------------ clustered coarse V-cycle
// The small levels (levels 0..nlev-1 of the argument, all L2 resident) run in one thread-block
// cluster: every sweep is spread over the cluster's CTAs (tile stride = cluster size) and the
// hardware cluster barrier (release/acquire) separates dependent sweeps.  The first level's right-hand
// side is its b buffer; each level's result ends in the buffer the host predicts (lev[].result).
template <class T, int DIM, bool VAR>
__global__ void __launch_bounds__(kClusterThreads, 1) k_coarse_cluster(ClusterArgs a) {
    pdl_wait();
    cg::cluster_group cl = cg::this_cluster();
    const T* dshT = reinterpret_cast<const T*>(a.dsh);
    const int rank = (int)cl.block_rank();
    const int ncta = (int)cl.num_blocks();
    for (int l = 0; l < a.nlev; ++l) {
        const ClusterLevel& c = a.lev[l];
        const int deg = c.deg;
        T* A = reinterpret_cast<T*>(c.xa);
        T* B = reinterpret_cast<T*>(c.xb);
        T* D = reinterpret_cast<T*>(c.dd);
        const T* b = reinterpret_cast<const T*>(c.b);
        if (l == a.exact) {  // dense exact solve of every shifted system: A = M_j b
            constexpr int W = VecT<T>::W;
            const int n = (int)c.L.N;
            const int off = threadIdx.x * W;
            const T* M = reinterpret_cast<const T*>(a.minv);
            for (int i = rank * blockDim.y + threadIdx.y; i < n; i += ncta * blockDim.y) {
                T acc[W];
                for (int v = 0; v < W; ++v) acc[v] = T(0);
                const T* row = M + (size_t)i * n * a.Kp + off;
#pragma unroll 4
                for (int jj = 0; jj < n; ++jj) {
                    T m[W], bv[W];
                    vld(row + (size_t)jj * a.Kp, m);
                    vld(b + (size_t)jj * a.Kp + off, bv);
                    for (int v = 0; v < W; ++v) acc[v] = fma(m[v], bv[v], acc[v]);
                }
                vst(A + (size_t)i * a.Kp + off, acc);
            }
            cl.sync();
            break;
        }
        sw_cheb_zero<T, DIM, VAR>(c.L, a.Kp, b, A, ChebStepT<T>{reinterpret_cast<const T*>(c.c1), reinterpret_cast<const T*>(c.c2)}, dshT, rank, ncta);
        cl.sync();
        T* cur = A;
        T* oth = B;
        for (int m = 1; m < deg; ++m) {
            LoadPlain<T> ld{cur};
            // after the step from zero the previous Chebyshev direction is the iterate itself
            sw_cheb_step<T, DIM, VAR>(c.L, a.Kp, ld, m == 1 ? nullptr : D, m == 1, b, oth, m < deg - 1 ? D : nullptr,
                                      ChebStepT<T>{reinterpret_cast<const T*>(c.c1) + m * a.Kp, reinterpret_cast<const T*>(c.c2) + m * a.Kp},
                                      dshT, nullptr, rank, ncta);
            cl.sync();
            T* t = cur; cur = oth; oth = t;
        }
        if (l + 1 < a.nlev) {
            sw_restrict<T, DIM, VAR>(c.L, a.lev[l + 1].L, a.Kp, cur, b, reinterpret_cast<T*>(a.lev[l + 1].b), dshT,
                                     rank, ncta);
            cl.sync();
        }
    }
    for (int l = a.nlev - 2; l >= 0; --l) {
        const ClusterLevel& c = a.lev[l];
        const int deg = c.deg;
        T* A = reinterpret_cast<T*>(c.xa);
        T* B = reinterpret_cast<T*>(c.xb);
        T* D = reinterpret_cast<T*>(c.dd);
        const T* b = reinterpret_cast<const T*>(c.b);
        T* cur = ((deg - 1) % 2 == 0) ? A : B;  // where the pre-smoothing ended
        T* oth = cur == A ? B : A;
        sw_prolong_add<T, DIM>(c.L, a.lev[l + 1].L, a.Kp, reinterpret_cast<const T*>(a.lev[l + 1].result), cur, rank,
                               ncta);
        cl.sync();
        for (int m = 0; m < deg; ++m) {
            LoadPlain<T> ld{cur};
            sw_cheb_step<T, DIM, VAR>(c.L, a.Kp, ld, m == 0 ? nullptr : D, false, b, oth, m < deg - 1 ? D : nullptr,
                                      ChebStepT<T>{m == 0 ? nullptr : reinterpret_cast<const T*>(c.c1) + m * a.Kp,
                                                   reinterpret_cast<const T*>(c.c2) + m * a.Kp},
                                      dshT, nullptr,
                                      rank, ncta);
            cl.sync();
            T* t = cur; cur = oth; oth = t;
        }
    }
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

// dim 0: the sparse (CSR) operator, for the kernels a one-level operator uses (no grid transfers)
#define BURA_DISPATCH_PDL0(dim, var, KERNEL, GRID, BLOCK, SMEM, S, ...)                                \
    do {                                                                                             \
        if (dim == 0) launch_pdl(KERNEL<T, 0, true>, GRID, BLOCK, SMEM, S, __VA_ARGS__);             \
        else BURA_DISPATCH_PDL(dim, var, KERNEL, GRID, BLOCK, SMEM, S, __VA_ARGS__);                  \
    } while (0)

#define BURA_DISPATCH_PDL(dim, var, KERNEL, GRID, BLOCK, SMEM, S, ...)                                 \
    do {                                                                                             \
        if (dim == 2 && !var) launch_pdl(KERNEL<T, 2, false>, GRID, BLOCK, SMEM, S, __VA_ARGS__);    \
        else if (dim == 2 && var) launch_pdl(KERNEL<T, 2, true>, GRID, BLOCK, SMEM, S, __VA_ARGS__); \
        else if (dim == 3 && !var) launch_pdl(KERNEL<T, 3, false>, GRID, BLOCK, SMEM, S, __VA_ARGS__); \
        else launch_pdl(KERNEL<T, 3, true>, GRID, BLOCK, SMEM, S, __VA_ARGS__);                      \
    } while (0)

template <class T>
void Ops<T>::broadcast(const Launch& g, const double* f, long long N, int K, T* r, T* x, T* p, cudaStream_t s,
                       const double* const* fp) {
    launch_pdl(k_broadcast<T>, dim3(g.blocks), blk(g), 0, s, f, fp, (int)N, g.Kp, K, r, x, p);
}

template <class T>
void Ops<T>::spmv_p(const Launch& g, const Lev& L, int dim, bool var, const T* z, T* pa, T* pb, T* q,
                    const Red& red, cudaStream_t s) {
    BURA_DISPATCH_PDL0(dim, var, k_spmv_p, dim3(g.blocks), blk(g), shm(g, VecT<T>::W), s, L, g.Kp, z, pa, pb, q, red);
}

template <class T>
void Ops<T>::pupdate(const Launch& g, long long N, const T* z, T* pa, T* pb, const Red& red, cudaStream_t s) {
    launch_pdl(k_pupdate<T>, dim3(g.blocks), blk(g), 0, s, (int)N, g.Kp, z, pa, pb, red);
}

template <class T>
void Ops<T>::spmv_q(const Launch& g, const Lev& L, int dim, bool var, const T* pa, const T* pb, T* q, const Red& red,
                    cudaStream_t s) {
    BURA_DISPATCH_PDL0(dim, var, k_spmv_q, dim3(g.blocks), blk(g), shm(g, VecT<T>::W), s, L, g.Kp, pa, pb, q, red);
}

template <class T>
void Ops<T>::cg_update(const Launch& g, long long N, T* x, T* r, const T* pa, const T* pb, const T* q,
                       const Red& red, cudaStream_t s) {
    launch_pdl(k_cg_update<T>, dim3(g.blocks), blk(g), shm(g, VecT<T>::W), s, (int)N, g.Kp, x, r, pa, pb, q, red);
}

template <class T>
void Ops<T>::cheb_zero(const Launch& g, const Lev& L, int dim, bool var, const T* b, T* x, ChebStepT<T> cs,
                       const T* dsh, cudaStream_t s) {
    BURA_DISPATCH_PDL0(dim, var, k_cheb_zero, dim3(g.blocks), blk(g), 0, s, L, g.Kp, b, x, cs, dsh);
}

template <class T>
void Ops<T>::cheb_step(const Launch& g, const Lev& L, int dim, bool var, const T* xin, const T* din, const T* b,
                       T* xout, T* dout, ChebStepT<T> cs, const T* dsh, const Red& red, cudaStream_t s) {
    const size_t sh = red.op != RED_NONE ? shm(g, VecT<T>::W) : 0;
    BURA_DISPATCH_PDL0(dim, var, k_cheb_step, dim3(g.blocks), blk(g), sh, s, L, g.Kp, xin, din, b, xout, dout, cs, dsh,
                      red);
}

template <class T>
void Ops<T>::cheb_pre2(const Launch& g, const Lev& L, int dim, bool var, const T* b, T* xout, T* dout, ChebStepT<T> cs0,
                       ChebStepT<T> cs1, const T* dsh, cudaStream_t s) {
    BURA_DISPATCH_PDL0(dim, var, k_cheb_pre2, dim3(g.blocks), blk(g), 0, s, L, g.Kp, b, xout, dout, cs0, cs1, dsh);
}

template <class T>
void Ops<T>::post_prolong(const Launch& g, const Lev& Lf, const Lev& Lc, int dim, bool var, const T* x, const T* ec,
                          const T* b, T* xout, T* dout, ChebStepT<T> cs, const T* dsh, const Red& red,
                          cudaStream_t s) {
    const size_t sh = red.op != RED_NONE ? shm(g, VecT<T>::W) : 0;
    BURA_DISPATCH_PDL(dim, var, k_post_prolong, dim3(g.blocks), blk(g), sh, s, Lf, Lc, g.Kp, x, ec, b, xout, dout, cs,
                      dsh, red);
}

template <class T>
void Ops<T>::restrict_res(const Launch& gc, const Lev& Lf, const Lev& Lc, int dim, bool var, const T* x, const T* b,
                          T* bc, const T* dsh, cudaStream_t s) {
    BURA_DISPATCH_PDL(dim, var, k_restrict_res, dim3(gc.blocks), blk(gc), 0, s, Lf, Lc, gc.Kp, x, b, bc, dsh);
}

template <class T>
void Ops<T>::residual(const Launch& g, const Lev& L, int dim, bool var, const T* x, const T* b, T* r, const T* dsh,
                      cudaStream_t s) {
    BURA_DISPATCH_PDL0(dim, var, k_residual, dim3(g.blocks), blk(g), 0, s, L, g.Kp, x, b, r, dsh);
}

template <class T>
void Ops<T>::restrict_r(const Launch& gc, const Lev& Lf, const Lev& Lc, int dim, const T* r, T* bc, cudaStream_t s) {
    if (dim == 2) launch_pdl(k_restrict_r<T, 2>, dim3(gc.blocks), blk(gc), 0, s, Lf, Lc, gc.Kp, r, bc);
    else launch_pdl(k_restrict_r<T, 3>, dim3(gc.blocks), blk(gc), 0, s, Lf, Lc, gc.Kp, r, bc);
}

template <class T>
void Ops<T>::prolong_add(const Launch& gf, const Lev& Lf, const Lev& Lc, int dim, const T* ec, T* x, cudaStream_t s) {
    if (dim == 2) launch_pdl(k_prolong_add<T, 2>, dim3(gf.blocks), blk(gf), 0, s, Lf, Lc, gf.Kp, ec, x);
    else launch_pdl(k_prolong_add_z<T>, dim3(gf.blocks), blk(gf), 0, s, Lf, Lc, gf.Kp, ec, x);
}

// The dynamic shared memory limit is a property of the kernel function (per device), not of a launch, so
// it is only ever raised: a plan set up later with a smaller coarse CTA must not lower the limit under a
// plan whose graph launches more.
template <class T, int DIM, bool VAR>
cudaError_t prepare_coarse_t(int bytes) {
    static std::mutex m;
    static int limit[kMaxDevices] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(m);
    if (bytes <= limit[dev]) return cudaSuccess;
    e = cudaFuncSetAttribute(k_coarse_cycle<T, DIM, VAR>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) limit[dev] = bytes;
    return e;
}

template <class T>
cudaError_t Ops<T>::prepare_coarse(int dim, bool var, size_t smem_bytes) {
    const int b = (int)smem_bytes;
    if (dim == 2 && !var) return prepare_coarse_t<T, 2, false>(b);
    if (dim == 2 && var) return prepare_coarse_t<T, 2, true>(b);
    if (dim == 3 && !var) return prepare_coarse_t<T, 3, false>(b);
    return prepare_coarse_t<T, 3, true>(b);
}

template <class T>
void Ops<T>::coarse_cycle(const Launch& g1, int dim, bool var, const CoarseArgs& a, cudaStream_t s) {
    // one CTA per 16-byte chunk of systems, each with its whole thread block on that chunk
    BURA_DISPATCH_PDL(dim, var, k_coarse_cycle, dim3(g1.C), dim3(1, kCoarseThreads), (size_t)a.smem_bytes, s, a);
}

template <class T>
cudaError_t Ops<T>::coarse_cluster(const Launch& g1, int csize, int dim, bool var, const ClusterArgs& a,
                                   cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(csize);
    cfg.blockDim = blk(g1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = csize;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (dim == 2 && !var) return cudaLaunchKernelEx(&cfg, k_coarse_cluster<T, 2, false>, a);
    if (dim == 2 && var) return cudaLaunchKernelEx(&cfg, k_coarse_cluster<T, 2, true>, a);
    if (dim == 3 && !var) return cudaLaunchKernelEx(&cfg, k_coarse_cluster<T, 3, false>, a);
    return cudaLaunchKernelEx(&cfg, k_coarse_cluster<T, 3, true>, a);
}

template <class T, int DIM, bool VAR>
cudaError_t cluster_prepare_t(int threads, int want, int* csize) {
    auto fn = k_coarse_cluster<T, DIM, VAR>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    *csize = 1;
    for (int c = 16; c >= 2; c /= 2) {
        if (c > want) continue;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(c);
        cfg.blockDim = dim3(threads);
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = c;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int n = 0;
        e = cudaOccupancyMaxActiveClusters(&n, fn, &cfg);
        if (e != cudaSuccess) { cudaGetLastError(); continue; }
        if (n >= 1) { *csize = c; return cudaSuccess; }
    }
    return cudaSuccess;
}

template <class T>
cudaError_t Ops<T>::cluster_prepare(int dim, bool var, int threads, int want, int* csize) {
    if (dim == 2 && !var) return cluster_prepare_t<T, 2, false>(threads, want, csize);
    if (dim == 2 && var) return cluster_prepare_t<T, 2, true>(threads, want, csize);
    if (dim == 3 && !var) return cluster_prepare_t<T, 3, false>(threads, want, csize);
    return cluster_prepare_t<T, 3, true>(threads, want, csize);
}

template <class T>
void Ops<T>::apply_shifted(const Launch& g, const Lev& L, int dim, bool var, const T* x, T* y, const T* dsh,
                           cudaStream_t s) {
    BURA_DISPATCH_PDL0(dim, var, k_apply_shifted, dim3(g.blocks), blk(g), 0, s, L, g.Kp, x, y, dsh);
}

template <class T>
void Ops<T>::dot(const Launch& g, long long N, const T* a, const T* b, const Red& red, cudaStream_t s) {
    launch_pdl(k_dot<T>, dim3(g.blocks), blk(g), shm(g, VecT<T>::W), s, (int)N, g.Kp, a, b, red);
}

}  // namespace bura
