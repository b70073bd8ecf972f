// TMA (cp.async.bulk.tensor) and mbarrier helpers in inline PTX, and the host-side declarations of
// the TMA-staged fine-level sweeps (kernels_tma.cu).
//
// Every wait on an mbarrier is bounded in time: after a budget of SM clocks without the phase completing
// (kTmaWaitCycles unless the plan sets another, Scal::wait_cycles), the wait gives up and the kernel
// records a fault in its Scal record (the host returns BURA_ETIMEOUT) instead of spinning forever.  The
// copies still in flight are then drained under the full kTmaWaitCycles budget before the CTA exits.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.cuh"

namespace bura {

// Tile of grid points staged per TMA load (x extent, y extent); the stencil input is loaded with a
// one-point halo on every side, (kTX + 2) x (kTY + 2) points.
#ifndef BURA_TMA_TX
#define BURA_TMA_TX 32
#endif
#ifndef BURA_TMA_TY
#define BURA_TMA_TY 8
#endif
constexpr int kTX = BURA_TMA_TX;
constexpr int kTY = BURA_TMA_TY;
// Coarse tile of the fused smoothing + restriction kernel: kTXc x kTYc coarse points, i.e. the fine
// region of one fine tile; its right-hand side is loaded with a two-point halo (2 kTXc + 5 points).
constexpr int kTXc = kTX / 2;
constexpr int kTYc = kTY / 2;

// Box shapes of the tensor maps (x extent, y extent in grid points; the innermost box extent is Kp).
enum TmaBox {
    TB_HALO = 0,   // (kTX + 2, kTY + 2): stencil input of a fine tile
    TB_PLAIN = 1,  // (kTX, kTY): pointwise input of a fine tile
    TB_RSRC = 2,   // (2 kTXc + 5, 2 kTYc + 5): right-hand side of the fused smoothing + restriction
    TB_CPRO = 3,   // (kTX / 2 + 2, kTY / 2 + 2): coarse correction prolongated onto a fine tile + halo
    TB_HALO2 = 4,  // (kTX + 4, kTY + 4): input of two stencil steps on a fine tile (two-point halo)
    TB_CPRO2 = 5,  // (kTX / 2 + 3, kTY / 2 + 3): coarse correction prolongated onto a fine tile + 2 halo
    TB_N = 6
};
inline void tma_box_dims(int kind, int* bx, int* by) {
    switch (kind) {
        case TB_HALO: *bx = kTX + 2; *by = kTY + 2; break;
        case TB_PLAIN: *bx = kTX; *by = kTY; break;
        case TB_RSRC: *bx = 2 * kTXc + 5; *by = 2 * kTYc + 5; break;
        case TB_HALO2: *bx = kTX + 4; *by = kTY + 4; break;
        case TB_CPRO2: *bx = kTX / 2 + 3; *by = kTY / 2 + 3; break;
        default: *bx = kTX / 2 + 2; *by = kTY / 2 + 2; break;
    }
}
constexpr int kTmaThreads = 256;     // threads per CTA
constexpr int kTmaMaxCtasPerSM = 3;  // CTAs per SM when their rings fit shared memory
constexpr int kTmaStages = 2;     // default depth of the shared-memory ring of a CTA
constexpr int kTmaMaxStages = 4;  // deepest ring (bura_options.tma_stages)
constexpr long long kTmaWaitCycles = 4000000000LL;  // about 2 s at the maximum SM clock

#ifdef __CUDACC__
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Make the initialised barriers visible to the async (TMA) proxy.
__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Order this thread's generic-proxy writes to shared memory before later async-proxy (TMA) writes to
// the same bytes; executed by the writers, before the barrier after which the TMA load is issued.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Non-blocking test of phase `parity`.
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Budgets below this many SM clocks poll with the non-blocking test (a blocking try_wait may suspend
// the thread for longer than such a budget).
constexpr long long kTmaShortWait = 100000;

// Wait for phase `parity` of the barrier; false if it did not complete within `budget` SM clocks.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity, long long budget) {
    const long long t0 = clock64();
    if (budget < kTmaShortWait) {
        while (!mbar_test_wait(bar, parity))
            if (clock64() - t0 > budget) return false;
        return true;
    }
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > budget) return false;
    return true;
}

// 2-D tiled TMA load of the box at coordinates (c0, c1) (innermost first) into shared memory;
// completion is signalled on `bar` (transaction bytes).
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int c0, int c1, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(smem_u32(dst)),
        "l"((unsigned long long)map), "r"(c0), "r"(c1), "r"(smem_u32(bar))
        : "memory");
}

// 3-D tiled TMA load of the box at coordinates (c0, c1, c2) (innermost first) into shared memory;
// completion is signalled on `bar` (transaction bytes).  c0 is always 0 here (16-byte aligned).
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_u32(dst)),
        "l"((unsigned long long)map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}
#endif

// Geometry of one 2-D level for the tiled sweeps (and of its coarse level, for the transfers).
struct TmaGeo {
    int nx, ny;        // grid points
    int ntx, nty;      // tiles along x and y
    int ntiles;
    int Kp;            // floats per point
    float wx, wy;      // constant face weights of the scaled operator
    int nxc, nyc;      // the next coarser level (0 if none)
    int ncx, ncy;      // coarse tiles (kTXc x kTYc) of the fused smoothing + restriction
    int nctiles;
    int flat;          // 1: 2-D maps over 8-byte elements (a tile row is one contiguous box row),
                       // 0: 3-D maps (Kp floats innermost), used when a box row would exceed 256 elements
    int stages;        // requested depth of the shared-memory ring (2..kTmaMaxStages); each launch uses the
                       // deepest ring up to this that fits its kind's shared memory
};

#ifdef __CUDACC__
// Load the box whose first grid point is (x, y) (may be negative: zero fill); the shared-memory layout
// is [rows][points][Kp floats] for both map kinds.
__device__ __forceinline__ void tma_load_pt(void* dst, const CUtensorMap* map, const TmaGeo& g, int x, int y,
                                            uint64_t* bar) {
    if (g.flat) tma_load_2d(dst, map, x * (g.Kp / 2), y, bar);
    else tma_load_3d(dst, map, 0, x, y, bar);
}
#endif

struct TmaMaps3 {
    CUtensorMap m[3];
};

struct TmaMaps5 {
    CUtensorMap m[5];
};

// Host side.  Every launcher returns the launch status; the kernels take the fault flag from red.scal.
bool tma_supported(int Kp);
TmaGeo tma_geo(const Lev& L, const Lev* Lc, int Kp);
// Whether the maps of a level with Kp floats per point are flat (2-D over 8-byte elements).
bool tma_flat(int Kp);
// Tensor map of an [ny][nx][Kp] float vector with a box of kind TmaBox.
cudaError_t tma_encode(CUtensorMap* m, const float* base, int Kp, int nx, int ny, int box);
cudaError_t tma_prepare(int Kp);
cudaError_t tma_cheb_step(const TmaGeo& g, int nsm, const CUtensorMap& mx, const CUtensorMap* md, const CUtensorMap& mb,
                          float* xout, float* dout, ChebStepT<float> cs, const float* dsh, const Red& red, cudaStream_t s);
cudaError_t tma_pre2(const TmaGeo& g, int nsm, const CUtensorMap& mb_halo, float* xout, float* dout, ChebStepT<float> cs0,
                     ChebStepT<float> cs1, const float* dsh, const Red& none, cudaStream_t s);
// pre2 fused with the residual restriction: x2 = two Chebyshev steps from zero (written to x2out) and
// bc = R (b - (A - dI) x2) on the coarse level; one tile = kTXc x kTYc coarse points.
cudaError_t tma_pre2_restrict(const TmaGeo& g, int nsm, const CUtensorMap& mb_rsrc, float* x2out, float* bc,
                              ChebStepT<float> cs0, ChebStepT<float> cs1, const float* dsh, const Red& none, cudaStream_t s);
// First post-smoothing step on x + P ec (prolongation fused): xout = xin + dnew, dout = dnew with
// dnew = c2 Dinv (b - (A - dI) xin), xin = x + P ec never stored.
cudaError_t tma_prolong_cheb(const TmaGeo& g, int nsm, const CUtensorMap& mx_halo, const CUtensorMap& mec_cpro,
                             const CUtensorMap& mb, float* xout, float* dout, ChebStepT<float> cs, const float* dsh,
                             const Red& none, cudaStream_t s);
// Both post-smoothing steps with the prolongation fused: xin = x + P ec on the tile and a two-point halo,
// x1 = xin + d1 (first step, d1 = c2 Dinv (b - (A - dI) xin)) on a one-point halo, and on the tile the
// second step xout = x1 + c1 d1 + c2 Dinv (b - (A - dI) x1), with b . xout when red asks for it.  Only
// xout is stored.  x is read through a TB_HALO2 map, ec through a TB_CPRO2 map of the coarse level, b
// through a TB_HALO map.
cudaError_t tma_post2(const TmaGeo& g, int nsm, const CUtensorMap& mx_halo2, const CUtensorMap& mec_cpro2,
                      const CUtensorMap& mb_halo, float* xout, ChebStepT<float> cs0, ChebStepT<float> cs1,
                      const float* dsh, const Red& red, cudaStream_t s);
// CG update x += alpha p, r -= alpha q with r.r (RED_CONV) from TMA-staged tiles of x, r, p, q (pointwise);
// the direction is pa or pb by the Scal parity, as in the grid kernel.  False from tma_cg_fits when the
// ring of at least two stages does not fit.
bool tma_cg_fits(int Kp);
cudaError_t tma_cg_update(const TmaGeo& g, int nsm, const CUtensorMap& mx, const CUtensorMap& mr,
                          const CUtensorMap& mpa, const CUtensorMap& mpb, const CUtensorMap& mq, float* x, float* r,
                          const Red& red, cudaStream_t s);
cudaError_t tma_spmv_p(const TmaGeo& g, int nsm, const CUtensorMap& mz, const CUtensorMap& mpa,
                       const CUtensorMap& mpb, float* pa, float* pb, float* q, const Red& red, cudaStream_t s);

}  // namespace bura
