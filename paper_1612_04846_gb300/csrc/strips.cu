// Prolongation and both post-smoothing steps of a 2-D constant-coefficient level (FP32) as y-marching
// strips.
//
// A work item is a strip of kSW columns [X0, X0 + kSW) over the rows [Y0, Y0 + SH) of the level.  Thread
// (chunk c, column col) owns grid column X0 - 2 + col (col = 0 .. kSW + 3) and walks down the rows; at
// step t (row y = Y0 + t) it forms
//   (1) xin = x + P e_c at row y + 2 (the strip's columns and two more on each side),
//   (2) the first Chebyshev step, x1 = xin + d1, at row y + 1 (one more column on each side), and
//   (3) the second step at row y (the strip's columns), stored to global memory, with b . xout.
// The values of its own column that the stencils need (xin on three rows, x1 on three, d1 and b on two)
// stay in registers; the left and right neighbours come from two-row rings of xin and x1 in shared
// memory, and the coarse correction from a three-row ring of coarse rows.  Each thread streams its own
// column of x and b through a kSRing-row ring in shared memory with asynchronous 16-byte copies
// (cp.async, zero-filled outside the grid) issued kSRing steps ahead, so the HBM latency overlaps the
// steps in between.  A step reads only what the
// previous step wrote, so it ends with one CTA barrier, and no row is computed twice inside an item (an
// item recomputes the two rows above and the two below it, a strip two columns on each side).
// Per point the arithmetic is k_post2_tma's, operation for operation, with points outside the grid
// holding zero (the homogeneous Dirichlet boundary).
// Measured on GB300 (1023^2, Kp = 8): 47 us per launch against 43 us for k_post2_tma.  Both are bound by
// instruction issue rather than by HBM or shared memory: the halo rows the tiles recompute cost less
// than a barrier per row and the per-row ring and address arithmetic here, so the tiles are the default
// (bura_options.post_smooth_split = 2 selects this kernel).
#include "kernels_impl.cuh"
#include "tma.cuh"

namespace bura {

namespace {

constexpr int kSW = 124;             // columns a strip stores
constexpr int kSCols = kSW + 4;      // columns of the two-point halo (threads per chunk): 128
constexpr int kSCc = kSW / 2 + 3;    // coarse columns the strip's correction reads
constexpr int kSRing = 8;            // rows of x and b in flight per thread

// 16-byte asynchronous copy global -> shared; nbytes = 0 zero-fills the destination (src is not read)
__device__ __forceinline__ void cp_async16(void* dst, const void* src, int nbytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(nbytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ void ld4s(const float* p, float (&o)[4]) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
__device__ __forceinline__ void st4s(float* p, const float (&o)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
}
__device__ __forceinline__ int ring3(int m) { return ((m % 3) + 3) % 3; }

// two CTAs per SM up to Kp = 8 (128 registers a thread), one above
template <int C>
__global__ void __launch_bounds__(C * kSCols, C <= 2 ? 2 : 1)
    k_post2_strip(StripGeo g, const float* __restrict__ x, const float* __restrict__ ec, const float* __restrict__ b,
                  float* __restrict__ xout, ChebStepT<float> cs0, ChebStepT<float> cs1, const float* __restrict__ dsh,
                  Red red) {
    pdl_wait();
    constexpr int Kp = 4 * C;
    extern __shared__ __align__(16) unsigned char smraw[];
    float* XIN = reinterpret_cast<float*>(smraw);  // [2][kSCols][Kp], by row parity
    float* X1 = XIN + 2 * kSCols * Kp;             // [2][kSCols][Kp], by row parity
    float* ECR = X1 + 2 * kSCols * Kp;             // [3][kSCc][Kp], coarse row m in slot m mod 3
    float* CST = ECR + 3 * kSCc * Kp;              // [4][Kp]: c2 of step 1, c1 and c2 of step 2, the shifts
    float* XR = CST + 4 * Kp;                      // [kSRing][kSCols][Kp]: x, row of phase (1) of step t in slot t
    float* BR = XR + kSRing * kSCols * Kp;         // [kSRing][kSCols][Kp]: b, row of phase (2)
    const int col = threadIdx.y;
    const int off = threadIdx.x * 4;
    // the step coefficients are read from shared memory where they are used (not held in registers)
    if (col == 0)
        for (int v = 0; v < 4; ++v) {
            CST[off + v] = cs0.c2[off + v];
            CST[Kp + off + v] = cs1.c1 ? cs1.c1[off + v] : 0.f;
            CST[2 * Kp + off + v] = cs1.c2[off + v];
            CST[3 * Kp + off + v] = dsh[off + v];
        }
    const float wx = g.wx, wy = g.wy;
    const float diag = wx + wx + wy + wy;
    const bool dot = red.op != RED_NONE;
    Accum<float> acc;
    for (int item = blockIdx.x; item < g.items; item += gridDim.x) {
        const int X0 = (item % g.nstrips) * kSW, Y0 = (item / g.nstrips) * g.SH;
        const int gx = X0 - 2 + col;
        const bool colin = gx >= 0 && gx < g.nx;
        const bool godd = (gx & 1) != 0;
        const int ci0 = X0 / 2 - 2;  // coarse column of ring column 0
        const int ccl = col >> 1;    // ring columns of the coarse neighbours: even column (ccl, ccl + 1),
        const int cco = (col + 1) >> 1;  // odd column cco
        const int nrows = min(g.SH, g.ny - Y0);
        const int T = nrows + (nrows & 1);
        // coarse row m, this thread's share (ring column col < kSCc, chunk off); zero outside the coarse grid
        auto coarse_row = [&](int m, float (&cv)[4]) {
            const int qi = ci0 + col;
            for (int v = 0; v < 4; ++v) cv[v] = 0.f;
            if (col < kSCc && qi >= 0 && qi < g.nxc && m >= 0 && m < g.nyc)
                ld4s(ec + ((size_t)m * g.nxc + qi) * Kp + off, cv);
        };
        auto put_coarse = [&](int m, const float (&cv)[4]) {
            if (col < kSCc) st4s(ECR + ((size_t)ring3(m) * kSCc + col) * Kp + off, cv);
        };
        // this thread's chunk of x at the phase-(1) row and of b at the phase-(2) row of step t, into slot t
        auto fetch = [&](int t) {
            const int sl = (t + 4) & (kSRing - 1);
            float* dx = XR + ((size_t)sl * kSCols + col) * Kp + off;
            float* db = BR + ((size_t)sl * kSCols + col) * Kp + off;
            const int rx = Y0 + t + 2, rb = Y0 + t + 1;
            const bool okx = colin && rx >= 0 && rx < g.ny, okb = colin && rb >= 0 && rb < g.ny;
            cp_async16(dx, okx ? x + ((size_t)rx * g.nx + gx) * Kp + off : x, okx ? 16 : 0);
            cp_async16(db, okb ? b + ((size_t)rb * g.nx + gx) * Kp + off : b, okb ? 16 : 0);
            cp_async_commit();
        };
        // the two coarse rows the first fine row (Y0 - 2, even) interpolates from
        {
            float cv[4];
            coarse_row(Y0 / 2 - 2, cv);
            put_coarse(Y0 / 2 - 2, cv);
            coarse_row(Y0 / 2 - 1, cv);
            put_coarse(Y0 / 2 - 1, cv);
        }
        float xin_m1[4], xin_0[4], xin_p1[4], x1_m1[4], x1_0[4], x1_p1[4], d1_0[4], d1_p1[4], b_0[4], b_p1[4];
        float creg[4];
        for (int v = 0; v < 4; ++v) {
            xin_m1[v] = xin_0[v] = xin_p1[v] = 0.f;
            x1_m1[v] = x1_0[v] = x1_p1[v] = 0.f;
            d1_0[v] = d1_p1[v] = b_0[v] = b_p1[v] = creg[v] = 0.f;
        }
        for (int t = -4; t < -4 + kSRing; ++t) fetch(t);
        __syncthreads();  // the primed coarse rows
        for (int t = -4; t < T; ++t) {
            const int y = Y0 + t;
            float xv[4], bv2[4];
            cp_async_wait<kSRing - 1>();  // this thread's copies of step t have landed
            {
                const int sl = (t + 4) & (kSRing - 1);
                ld4s(XR + ((size_t)sl * kSCols + col) * Kp + off, xv);
                ld4s(BR + ((size_t)sl * kSCols + col) * Kp + off, bv2);
            }
            // (1) xin at row fy = y + 2
            const int fy = y + 2;
            {
                float s[4];
                const bool rodd = (fy & 1) != 0;
                if (rodd) {
                    const float* er = ECR + (size_t)ring3((fy - 1) >> 1) * kSCc * Kp + off;
                    if (godd) {
                        float e11[4];
                        ld4s(er + cco * Kp, e11);
                        for (int v = 0; v < 4; ++v) s[v] = fmaf(1.f, e11[v], 0.f);
                    } else {
                        float e10[4], e11[4];
                        ld4s(er + ccl * Kp, e10);
                        ld4s(er + (ccl + 1) * Kp, e11);
                        for (int v = 0; v < 4; ++v) s[v] = fmaf(0.5f, e11[v], fmaf(0.5f, e10[v], 0.f));
                    }
                } else {
                    const float* elo = ECR + (size_t)ring3((fy >> 1) - 1) * kSCc * Kp + off;
                    const float* ehi = ECR + (size_t)ring3(fy >> 1) * kSCc * Kp + off;
                    if (godd) {
                        float e01[4], e11[4];
                        ld4s(elo + cco * Kp, e01);
                        ld4s(ehi + cco * Kp, e11);
                        for (int v = 0; v < 4; ++v) s[v] = fmaf(0.5f, e11[v], fmaf(0.5f, e01[v], 0.f));
                    } else {
                        float e00[4], e01[4], e10[4], e11[4];
                        ld4s(elo + ccl * Kp, e00);
                        ld4s(elo + (ccl + 1) * Kp, e01);
                        ld4s(ehi + ccl * Kp, e10);
                        ld4s(ehi + (ccl + 1) * Kp, e11);
                        for (int v = 0; v < 4; ++v) {
                            float tt = fmaf(0.25f, e00[v], 0.f);
                            tt = fmaf(0.25f, e01[v], tt);
                            tt = fmaf(0.25f, e10[v], tt);
                            s[v] = fmaf(0.25f, e11[v], tt);
                        }
                    }
                }
                float xn[4] = {0.f, 0.f, 0.f, 0.f};
                if (colin && fy >= 0 && fy < g.ny)
                    for (int v = 0; v < 4; ++v) xn[v] = xv[v] + s[v];
                st4s(XIN + ((size_t)(fy & 1) * kSCols + col) * Kp + off, xn);
                for (int v = 0; v < 4; ++v) {
                    xin_m1[v] = xin_0[v];
                    xin_0[v] = xin_p1[v];
                    xin_p1[v] = xn[v];
                }
                // the coarse ring: row fy / 2 + 1 is read at an even row and stored at the next (odd) one
                if (rodd) put_coarse((fy + 1) >> 1, creg);
                else coarse_row((fy >> 1) + 1, creg);
            }
            // (2) the first step at row py = y + 1 (rows from Y0 - 1 on)
            if (t >= -2) {
                const int py = y + 1;
                float x1n[4] = {0.f, 0.f, 0.f, 0.f}, d1n[4] = {0.f, 0.f, 0.f, 0.f};
                if (col >= 1 && col <= kSW + 2) {
                    if (colin && py >= 0 && py < g.ny) {
                        float xl[4], xr[4], c20[4], d[4];
                        ld4s(CST + off, c20);
                        ld4s(CST + 3 * Kp + off, d);
                        const float* rowp = XIN + (size_t)(py & 1) * kSCols * Kp + off;
                        ld4s(rowp + (col - 1) * Kp, xl);
                        ld4s(rowp + (col + 1) * Kp, xr);
                        for (int v = 0; v < 4; ++v) {
                            const float xc = xin_0[v];
                            float a = diag * xc;
                            a = fmaf(-wx, xl[v], a);
                            a = fmaf(-wx, xr[v], a);
                            a = fmaf(-wy, xin_m1[v], a);
                            a = fmaf(-wy, xin_p1[v], a);
                            const float res = bv2[v] - fmaf(-d[v], xc, a);
                            const float gg = c20[v] * res;
                            d1n[v] = fmaf(0.f, 0.f, gg);
                            x1n[v] = xc + d1n[v];
                        }
                    }
                    st4s(X1 + ((size_t)(py & 1) * kSCols + col) * Kp + off, x1n);
                }
                for (int v = 0; v < 4; ++v) {
                    x1_m1[v] = x1_0[v];
                    x1_0[v] = x1_p1[v];
                    x1_p1[v] = x1n[v];
                    d1_0[v] = d1_p1[v];
                    d1_p1[v] = d1n[v];
                    b_0[v] = b_p1[v];
                    b_p1[v] = bv2[v];
                }
            }
            // (3) the second step at row y, stored
            if (t >= 0 && t < nrows && col >= 2 && col <= kSW + 1 && colin) {
                float xl[4], xr[4], xo[4], c11[4], c21[4], d[4];
                ld4s(CST + Kp + off, c11);
                ld4s(CST + 2 * Kp + off, c21);
                ld4s(CST + 3 * Kp + off, d);
                const float* rowp = X1 + (size_t)(y & 1) * kSCols * Kp + off;
                ld4s(rowp + (col - 1) * Kp, xl);
                ld4s(rowp + (col + 1) * Kp, xr);
                for (int v = 0; v < 4; ++v) {
                    const float xc = x1_0[v];
                    float a = diag * xc;
                    a = fmaf(-wx, xl[v], a);
                    a = fmaf(-wx, xr[v], a);
                    a = fmaf(-wy, x1_m1[v], a);
                    a = fmaf(-wy, x1_p1[v], a);
                    const float res = b_0[v] - fmaf(-d[v], xc, a);
                    const float gg = c21[v] * res;
                    const float dv = fmaf(c11[v], d1_0[v], gg);
                    xo[v] = xc + dv;
                }
                st4s(xout + ((size_t)y * g.nx + gx) * Kp + off, xo);
                if (dot) acc.add(b_0, xo);
            }
            // slot t is free again (its values were used above): refill it for step t + kSRing
            fetch(t + kSRing);
            __syncthreads();
        }
        cp_async_wait<0>();  // no copy into this CTA's ring outlives the item
    }
    pdl_trigger();
    if (dot) reduce_finish<float>(acc, red, Kp);
}

}  // namespace

StripGeo strip_geo(int nx, int ny, int nxc, int nyc, int Kp, float wx, float wy, int nsm) {
    StripGeo g;
    g.nx = nx;
    g.ny = ny;
    g.nxc = nxc;
    g.nyc = nyc;
    g.Kp = Kp;
    g.wx = wx;
    g.wy = wy;
    g.nstrips = (nx + kSW - 1) / kSW;
    // rows per item: about two items per SM (two CTAs of the strip kernel fit an SM up to Kp = 8), an
    // even count
    int sh = (int)(((long long)ny * g.nstrips + 2LL * nsm - 1) / (2LL * nsm));
    sh = std::max(8, sh + (sh & 1));
    g.SH = sh;
    g.items = g.nstrips * ((ny + sh - 1) / sh);
    return g;
}

cudaError_t strip_prepare(int Kp) {
    // one fixed size per instantiation, set on the current device before any capture launches it
    const int bytes = (int)strip_smem_bytes(Kp);
    switch (Kp / 4) {
        case 1: return cudaFuncSetAttribute(k_post2_strip<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        case 2: return cudaFuncSetAttribute(k_post2_strip<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        case 3: return cudaFuncSetAttribute(k_post2_strip<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        case 4: return cudaFuncSetAttribute(k_post2_strip<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        default: return cudaErrorInvalidValue;
    }
}

size_t strip_smem_bytes(int Kp) {
    return (size_t)(4 * kSCols + 3 * kSCc + 4 + 2 * kSRing * kSCols) * Kp * sizeof(float);
}

cudaError_t launch_post2_strip(const StripGeo& g, int nsm, const float* x, const float* ec, const float* b, float* xout,
                               ChebStepT<float> cs0, ChebStepT<float> cs1, const float* dsh, const Red& red,
                               cudaStream_t s) {
    const int C = g.Kp / 4;
    const int grid = std::min(g.items, 2 * nsm);
    const size_t smem = strip_smem_bytes(g.Kp);
    switch (C) {
        case 1: launch_pdl(k_post2_strip<1>, dim3(grid), dim3(1, kSCols), smem, s, g, x, ec, b, xout, cs0, cs1, dsh, red); break;
        case 2: launch_pdl(k_post2_strip<2>, dim3(grid), dim3(2, kSCols), smem, s, g, x, ec, b, xout, cs0, cs1, dsh, red); break;
        case 3: launch_pdl(k_post2_strip<3>, dim3(grid), dim3(3, kSCols), smem, s, g, x, ec, b, xout, cs0, cs1, dsh, red); break;
        case 4: launch_pdl(k_post2_strip<4>, dim3(grid), dim3(4, kSCols), smem, s, g, x, ec, b, xout, cs0, cs1, dsh, red); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace bura
