// TMA-staged sweeps of the large 2-D levels (FP32, constant coefficients).
//
// A persistent grid walks tiles of kTX x kTY grid points (tile t = blockIdx.x + k * gridDim.x, a fixed
// order, so the per-thread partial sums and hence the reductions are deterministic).  For each tile one
// thread issues tiled TMA loads of the vectors the sweep reads into a ring of 2 to kTmaMaxStages
// shared-memory stages, each completed on its own mbarrier; the vectors a stencil reads are loaded with
// a one-point halo, and TMA's zero fill outside the grid is the homogeneous Dirichlet boundary.  All
// threads then compute the tile from shared memory and store their results straight to global memory
// (16-byte stores, contiguous along each tile row).  The loads of the next stage are in flight while a
// tile is computed, so the bytes in flight no longer depend on registers and occupancy.
//
// The arithmetic is the grid kernels' (kernels_impl.cuh), operation for operation: the stencil sums
// diag*x and the four neighbours in the same order with the same fused multiply-adds, and a missing
// neighbour contributes fma(-w, 0, acc) = acc.
#include <cudaTypedefs.h>

#include "kernels_impl.cuh"
#include "tma.cuh"

namespace bura {

namespace {

constexpr int kHaloPts = (kTX + 2) * (kTY + 2);
constexpr int kTilePts = kTX * kTY;

__host__ __device__ constexpr size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }
__host__ __device__ constexpr size_t halo_bytes(int Kp) { return align_up((size_t)kHaloPts * Kp * sizeof(float), 1024); }
__host__ __device__ constexpr size_t plain_bytes(int Kp) { return align_up((size_t)kTilePts * Kp * sizeof(float), 1024); }

// Fused smoothing + restriction: b with a two-point halo (kRsX x kRsY), x2 on the one-point halo
// region (kE1X x kE1Y) and the fine residual on the region the coarse tile restricts (kRX x kRY).
constexpr int kRsX = 2 * kTXc + 5, kRsY = 2 * kTYc + 5;
constexpr int kE1X = 2 * kTXc + 3, kE1Y = 2 * kTYc + 3;
constexpr int kRX = 2 * kTXc + 1, kRY = 2 * kTYc + 1;
// Fused prolongation + smoothing: coarse correction box (kCpX x kCpY) of one fine tile + halo.
constexpr int kCpX = kTX / 2 + 2, kCpY = kTY / 2 + 2;
// Fused prolongation + both post-smoothing steps: x on a two-point halo (kH2X x kH2Y) and its coarse
// correction box (kCp2X x kCp2Y).
constexpr int kH2X = kTX + 4, kH2Y = kTY + 4;
constexpr int kCp2X = kTX / 2 + 3, kCp2Y = kTY / 2 + 3;
static_assert(kTX % 2 == 0 && kTY % 2 == 0, "fine tiles start on even grid coordinates");

__host__ __device__ constexpr size_t vec_bytes(int pts, int Kp) { return align_up((size_t)pts * Kp * sizeof(float), 1024); }

// Shared-memory bytes of one stage of each kernel kind, and of its unstaged scratch.
enum TmaKind { TK_CHEB = 0, TK_CHEB_D = 1, TK_PRE2 = 2, TK_SPMV = 3, TK_PRE2R = 4, TK_PROCHEB = 5, TK_CG = 6,
               TK_POST2 = 7, TK_NKIND = 8 };
__host__ __device__ constexpr size_t stage_bytes(int kind, int Kp) {
    return kind == TK_CHEB ? halo_bytes(Kp) + plain_bytes(Kp)
         : kind == TK_CHEB_D ? halo_bytes(Kp) + 2 * plain_bytes(Kp)
         : kind == TK_PRE2 ? halo_bytes(Kp)
         : kind == TK_SPMV ? 2 * halo_bytes(Kp)
         : kind == TK_PRE2R ? vec_bytes(kRsX * kRsY, Kp)
         : kind == TK_CG ? 4 * plain_bytes(Kp)
         : kind == TK_POST2 ? vec_bytes(kH2X * kH2Y, Kp) + vec_bytes(kCp2X * kCp2Y, Kp) + halo_bytes(Kp)
         : halo_bytes(Kp) + vec_bytes(kCpX * kCpY, Kp) + plain_bytes(Kp);
}
__host__ __device__ constexpr size_t scratch_bytes(int kind, int Kp) {
    return kind == TK_PRE2R ? vec_bytes(kE1X * kE1Y, Kp) + vec_bytes(kRX * kRY, Kp)
         : kind == TK_PROCHEB ? halo_bytes(Kp)
         : kind == TK_POST2 ? halo_bytes(Kp) + plain_bytes(Kp)
         : 0;
}
__host__ __device__ constexpr size_t dyn_smem(int kind, int Kp, int S) {
    return S * stage_bytes(kind, Kp) + scratch_bytes(kind, Kp);
}
constexpr size_t kSmemPerSM = 228 * 1024;    // shared memory of an SM
constexpr size_t kSmemPerCTA = 226 * 1024;   // largest dynamic allocation of one CTA (the 227 KB opt-in limit
                                             // covers static shared memory too: keep 1 KB for it)
constexpr size_t kSmemReserved = 1024;       // per CTA, by the system
#ifndef BURA_POST2_CTAS
#define BURA_POST2_CTAS 2
#endif
#ifndef BURA_POST2_STAGES
#define BURA_POST2_STAGES 0
#endif
constexpr int kPost2CtasPerSM = BURA_POST2_CTAS;  // the fused post-smoothing ring + scratch: 2 CTAs per SM (FP32,
                                                  // 8 values per point), so its registers may be more
constexpr int kPost2Stages = BURA_POST2_STAGES;   // ring depth of the fused post-smoothing (0: the plan's)

// The tile pipeline.  issue(stage, tile, bar) is called by thread 0 only; compute(stage, tile) by
// every thread.  Returns false (after draining the copies in flight and flagging the fault) when a
// stage did not arrive in time; the caller still runs its epilogue, so every block joins the grid
// reduction and the reduction tickets stay consistent.
// SYNC_COMPUTE: compute() has CTA barriers of its own, so every thread must call it for every tile and
// the threads agree on a timed-out wait before it (one more barrier per tile).  Without, a thread whose
// wait timed out skips compute() and the agreement rides on the barrier that frees the stage.
template <bool SYNC_COMPUTE, class Issue, class Compute>
__device__ __forceinline__ bool tile_loop(int ntiles, int S, unsigned char* smem, size_t sbytes, Scal* scal,
                                          Issue&& issue, Compute&& compute) {
    __shared__ __align__(8) uint64_t bars[kTmaMaxStages];
    __shared__ int timed_out;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int nmine = ntiles > (int)blockIdx.x ? (ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x : 0;
    if (tid == 0) {
        for (int s = 0; s < S; ++s) mbar_init(&bars[s], 1);
        mbar_fence_init();
        timed_out = 0;
    }
    __syncthreads();
    if (tid == 0)
        for (int s = 0; s < S && s < nmine; ++s)
            issue(smem + s * sbytes, (int)blockIdx.x + s * (int)gridDim.x, &bars[s]);
    int k = 0;
    bool ok = true;
    const long long budget = scal->wait_cycles > 0 ? scal->wait_cycles : kTmaWaitCycles;
    for (; k < nmine; ++k) {
        const int s = k % S;
        const bool got = mbar_wait_bounded(&bars[s], (unsigned)(k / S) & 1u, budget);
        if constexpr (SYNC_COMPUTE) {
            if (__syncthreads_or(!got)) { ok = false; break; }
            compute(smem + s * sbytes, (int)blockIdx.x + k * (int)gridDim.x);
            __syncthreads();  // stage s is free again
        } else {
            if (got) compute(smem + s * sbytes, (int)blockIdx.x + k * (int)gridDim.x);
            else timed_out = 1;
            __syncthreads();  // stage s is free again; timed_out is the same for every thread now
            if (timed_out) { ok = false; break; }
        }
        if (tid == 0 && k + S < nmine)
            issue(smem + s * sbytes, (int)blockIdx.x + (k + S) * (int)gridDim.x, &bars[s]);
    }
    if (!ok) {
        // tiles k .. k+S-1 may still have copies in flight into this CTA's shared memory: drained under
        // the full budget, so no CTA exits while a copy can still write its shared memory
        for (int j = k; j < nmine && j < k + S; ++j)
            (void)mbar_wait_bounded(&bars[j % S], (unsigned)(j / S) & 1u, kTmaWaitCycles);
        if (tid == 0) atomicExch(&scal->fault, 1);
        __syncthreads();
    }
    return ok;
}

// The stage ring starts at the first 1024-byte boundary of the dynamic shared memory (TMA destinations
// are kept 1024-byte aligned); kRingSlack extra bytes are requested for this.
constexpr size_t kRingSlack = 1024;
__device__ __forceinline__ unsigned char* aligned_ring(unsigned char* raw) {
    return raw + ((1024u - (smem_u32(raw) & 1023u)) & 1023u);
}

__device__ __forceinline__ void tile_origin(const TmaGeo& g, int t, int& x0, int& y0) {
    const int ty = t / g.ntx;
    x0 = (t - ty * g.ntx) * kTX;
    y0 = ty * kTY;
}

__device__ __forceinline__ void ld4(const float* p, float (&o)[4]) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}

__device__ __forceinline__ void st4(float* p, const float (&o)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
}

// A x at a tile point (no shift term) from a halo tile H ([kTY+2][kTX+2][Kp] floats) whose values are
// x(point) = val(h) for a loader `val` of the halo index; diag = 2 wx + 2 wy.
template <int ROW = kTX + 2, class Val>
__device__ __forceinline__ void stencil_tile(const TmaGeo& g, int hidx, const Val& val, float (&xc)[4],
                                             float (&Ax)[4]) {
    const float diag = g.wx + g.wx + g.wy + g.wy;
    const int sy = ROW * g.Kp;
    float n[4];
    val(hidx, xc);
    float acc[4];
    for (int v = 0; v < 4; ++v) acc[v] = diag * xc[v];
    val(hidx - g.Kp, n);
    for (int v = 0; v < 4; ++v) acc[v] = fmaf(-g.wx, n[v], acc[v]);
    val(hidx + g.Kp, n);
    for (int v = 0; v < 4; ++v) acc[v] = fmaf(-g.wx, n[v], acc[v]);
    val(hidx - sy, n);
    for (int v = 0; v < 4; ++v) acc[v] = fmaf(-g.wy, n[v], acc[v]);
    val(hidx + sy, n);
    for (int v = 0; v < 4; ++v) acc[v] = fmaf(-g.wy, n[v], acc[v]);
    for (int v = 0; v < 4; ++v) Ax[v] = acc[v];
}

// One Chebyshev step, xout = xin + dnew with dnew = c1 din + c2 Dinv (b - (A - dI) xin); stages hold
// xin (halo), [din,] b.  With a reduction, also sum b . xout per system (the CG r.z).
template <int C, bool HAS_DIN>
__global__ void __launch_bounds__(kTmaThreads, kTmaMaxCtasPerSM)
    k_cheb_tma(const __grid_constant__ TmaMaps3 mp, TmaGeo g, float* __restrict__ xout, float* __restrict__ dout,
               ChebStepT<float> cs, const float* __restrict__ dsh, Red red) {
    pdl_wait();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char* smem = aligned_ring(smem_raw);
    constexpr int kind = HAS_DIN ? TK_CHEB_D : TK_CHEB;
    const int Kp = C * 4;
    const size_t sb = stage_bytes(kind, Kp);
    const int off = threadIdx.x * 4;
    float c1[4], c2[4], d[4];
    for (int v = 0; v < 4; ++v) {
        c1[v] = cs.c1 ? (float)cs.c1[off + v] : 0.f;
        c2[v] = (float)cs.c2[off + v];
        d[v] = (float)dsh[off + v];
    }
    const unsigned tx_bytes = (unsigned)(kHaloPts * Kp * 4 + (HAS_DIN ? 2 : 1) * kTilePts * Kp * 4);
    Accum<float> acc;
    const bool dot = red.op != RED_NONE;
    tile_loop<false>(
        g.ntiles, g.stages, smem, sb, red.scal,
        [&](unsigned char* st, int t, uint64_t* bar) {
            int x0, y0;
            tile_origin(g, t, x0, y0);
            mbar_expect_tx(bar, tx_bytes);
            tma_load_pt(st, &mp.m[0], g, x0 - 1, y0 - 1, bar);
            unsigned char* q = st + halo_bytes(Kp);
            if (HAS_DIN) {
                tma_load_pt(q, &mp.m[1], g, x0, y0, bar);
                q += plain_bytes(Kp);
            }
            tma_load_pt(q, &mp.m[2], g, x0, y0, bar);
        },
        [&](unsigned char* st, int t) {
            int x0, y0;
            tile_origin(g, t, x0, y0);
            const float* X = reinterpret_cast<const float*>(st);
            const float* D = reinterpret_cast<const float*>(st + halo_bytes(Kp));
            const float* B = reinterpret_cast<const float*>(st + halo_bytes(Kp) + (HAS_DIN ? plain_bytes(Kp) : 0));
            for (int p = threadIdx.y; p < kTilePts; p += blockDim.y) {
                const int ly = p / kTX, lx = p - ly * kTX;
                const int gx = x0 + lx, gy = y0 + ly;
                if (gx >= g.nx || gy >= g.ny) continue;
                const int hidx = ((ly + 1) * (kTX + 2) + lx + 1) * Kp + off;
                float xc[4], Ax[4], bv[4], dv[4];
                stencil_tile(g, hidx, [&](int h, float (&o)[4]) { ld4(X + h, o); }, xc, Ax);
                const int pidx = p * Kp + off;
                ld4(B + pidx, bv);
                if (HAS_DIN) ld4(D + pidx, dv);
                else for (int v = 0; v < 4; ++v) dv[v] = 0.f;
                float xo[4];
                for (int v = 0; v < 4; ++v) {
                    const float res = bv[v] - fmaf(-d[v], xc[v], Ax[v]);
                    const float gg = c2[v] * res;
                    dv[v] = fmaf(c1[v], dv[v], gg);
                    xo[v] = xc[v] + dv[v];
                }
                const size_t gidx = ((size_t)gy * g.nx + gx) * Kp + off;
                st4(xout + gidx, xo);
                if (dout) st4(dout + gidx, dv);
                if (dot) acc.add(bv, xo);
            }
        });
    pdl_trigger();
    if (dot) reduce_finish<float>(acc, red, Kp);
}

// The first two Chebyshev steps from a zero guess: x1 = c2_0 Dinv b at the stencil points (d_1 = x1),
// then the second step; the stage holds b with its halo.
template <int C>
__global__ void __launch_bounds__(kTmaThreads, kTmaMaxCtasPerSM)
    k_pre2_tma(const __grid_constant__ TmaMaps3 mp, TmaGeo g, float* __restrict__ xout, float* __restrict__ dout,
               ChebStepT<float> cs0, ChebStepT<float> cs1, const float* __restrict__ dsh, Red none) {
    pdl_wait();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char* smem = aligned_ring(smem_raw);
    const int Kp = C * 4;
    const size_t sb = stage_bytes(TK_PRE2, Kp);
    const int off = threadIdx.x * 4;
    float c20[4], c1[4], c2[4], d[4];
    for (int v = 0; v < 4; ++v) {
        c20[v] = (float)cs0.c2[off + v];
        c1[v] = (float)cs1.c1[off + v];
        c2[v] = (float)cs1.c2[off + v];
        d[v] = (float)dsh[off + v];
    }
    const unsigned tx_bytes = (unsigned)(kHaloPts * Kp * 4);
    tile_loop<false>(
        g.ntiles, g.stages, smem, sb, none.scal,
        [&](unsigned char* st, int t, uint64_t* bar) {
            int x0, y0;
            tile_origin(g, t, x0, y0);
            mbar_expect_tx(bar, tx_bytes);
            tma_load_pt(st, &mp.m[0], g, x0 - 1, y0 - 1, bar);
        },
        [&](unsigned char* st, int t) {
            int x0, y0;
            tile_origin(g, t, x0, y0);
            const float* Bh = reinterpret_cast<const float*>(st);
            for (int p = threadIdx.y; p < kTilePts; p += blockDim.y) {
                const int ly = p / kTX, lx = p - ly * kTX;
                const int gx = x0 + lx, gy = y0 + ly;
                if (gx >= g.nx || gy >= g.ny) continue;
                const int hidx = ((ly + 1) * (kTX + 2) + lx + 1) * Kp + off;
                float xc[4], Ax[4], bv[4];
                stencil_tile(g, hidx,
                             [&](int h, float (&o)[4]) {
                                 ld4(Bh + h, o);
                                 for (int v = 0; v < 4; ++v) o[v] *= c20[v];
                             },
                             xc, Ax);
                ld4(Bh + hidx, bv);
                float xo[4], dv[4];
                for (int v = 0; v < 4; ++v) {
                    const float res = bv[v] - fmaf(-d[v], xc[v], Ax[v]);
                    const float gg = c2[v] * res;
                    dv[v] = fmaf(c1[v], xc[v], gg);
                    xo[v] = xc[v] + dv[v];
                }
                const size_t gidx = ((size_t)gy * g.nx + gx) * Kp + off;
                st4(xout + gidx, xo);
                if (dout) st4(dout + gidx, dv);
            }
        });
    pdl_trigger();
}

// CG direction update and operator apply: p_new = z + beta p_old at the stencil points, q = (A - dI)
// p_new, and p_new . q per system; the stages hold z and p_old with their halos.  p_new is formed once
// per halo point, in place over z in the stage, and the stencil then reads it from there.  The
// direction buffers alternate by the parity in the Scal record, as in the grid kernel.
template <int C>
__global__ void __launch_bounds__(kTmaThreads, kTmaMaxCtasPerSM)
    k_spmv_tma(const __grid_constant__ TmaMaps3 mp, TmaGeo g, float* pa, float* pb, float* __restrict__ q, Red red) {
    pdl_wait();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char* smem = aligned_ring(smem_raw);
    const int Kp = C * 4;
    const size_t sb = stage_bytes(TK_SPMV, Kp);
    const int off = threadIdx.x * 4;
    const int par = red.scal->parity;
    const CUtensorMap* mold = par ? &mp.m[2] : &mp.m[1];
    float* __restrict__ pnew = par ? pa : pb;
    float beta[4], dsh[4];
    for (int v = 0; v < 4; ++v) {
        beta[v] = red.scal->betaf[off + v];
        dsh[v] = red.scal->dshf[off + v];
    }
    const unsigned tx_bytes = (unsigned)(2 * kHaloPts * Kp * 4);
    Accum<float> acc;
    tile_loop<true>(
        g.ntiles, g.stages, smem, sb, red.scal,
        [&](unsigned char* st, int t, uint64_t* bar) {
            int x0, y0;
            tile_origin(g, t, x0, y0);
            mbar_expect_tx(bar, tx_bytes);
            tma_load_pt(st, &mp.m[0], g, x0 - 1, y0 - 1, bar);
            tma_load_pt(st + halo_bytes(Kp), mold, g, x0 - 1, y0 - 1, bar);
        },
        [&](unsigned char* st, int t) {
            int x0, y0;
            tile_origin(g, t, x0, y0);
            float* Z = reinterpret_cast<float*>(st);
            const float* Po = reinterpret_cast<const float*>(st + halo_bytes(Kp));
            // p_new on the tile and its halo (zero outside the grid, where z and p_old are zero-filled)
            for (int p = threadIdx.y; p < kHaloPts; p += blockDim.y) {
                const int h = p * Kp + off;
                float a[4], b[4];
                ld4(Z + h, a);
                ld4(Po + h, b);
                for (int v = 0; v < 4; ++v) a[v] = fmaf(beta[v], b[v], a[v]);
                st4(Z + h, a);
            }
            fence_proxy_async_smem();  // the stage is refilled by TMA after the tile
            __syncthreads();
            for (int p = threadIdx.y; p < kTilePts; p += blockDim.y) {
                const int ly = p / kTX, lx = p - ly * kTX;
                const int gx = x0 + lx, gy = y0 + ly;
                if (gx >= g.nx || gy >= g.ny) continue;
                const int hidx = ((ly + 1) * (kTX + 2) + lx + 1) * Kp + off;
                float pc[4], Ax[4];
                stencil_tile(g, hidx, [&](int h, float (&o)[4]) { ld4(Z + h, o); }, pc, Ax);
                float qv[4];
                for (int v = 0; v < 4; ++v) qv[v] = fmaf(-dsh[v], pc[v], Ax[v]);
                const size_t gidx = ((size_t)gy * g.nx + gx) * Kp + off;
                st4(pnew + gidx, pc);
                st4(q + gidx, qv);
                acc.add(pc, qv);
            }
        });
    pdl_trigger();
    reduce_finish<float>(acc, red, Kp);
}

// pre2 fused with the restriction of its residual.  One tile = kTXc x kTYc coarse points starting at
// (X0, Y0); it owns the fine points [2 X0, 2 X0 + 2 kTXc) x [2 Y0, 2 Y0 + 2 kTYc) (the last tile along
// an axis also the last fine point).  x2 is computed, as k_pre2_tma does, on those points plus a
// one-point halo (recomputed by neighbouring tiles, bit for bit the same), the residual on the fine
// points the coarse tile's full weighting reads, and the weighted sums in the grid kernel's order.
template <int C>
__global__ void __launch_bounds__(kTmaThreads, kTmaMaxCtasPerSM)
    k_pre2_restrict_tma(const __grid_constant__ TmaMaps3 mp, TmaGeo g, float* __restrict__ x2out,
                        float* __restrict__ bc, ChebStepT<float> cs0, ChebStepT<float> cs1, const float* __restrict__ dsh, Red none) {
    pdl_wait();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char* smem = aligned_ring(smem_raw);
    const int Kp = C * 4;
    const size_t sb = stage_bytes(TK_PRE2R, Kp);
    float* X2s = reinterpret_cast<float*>(smem + g.stages * sb);
    float* Rs = reinterpret_cast<float*>(smem + g.stages * sb + vec_bytes(kE1X * kE1Y, Kp));
    const int off = threadIdx.x * 4;
    float c20[4], c1[4], c2[4], d[4];
    for (int v = 0; v < 4; ++v) {
        c20[v] = (float)cs0.c2[off + v];
        c1[v] = (float)cs1.c1[off + v];
        c2[v] = (float)cs1.c2[off + v];
        d[v] = (float)dsh[off + v];
    }
    const float w1[3] = {0.25f, 0.5f, 0.25f};
    const float diag = g.wx + g.wx + g.wy + g.wy;
    const unsigned tx_bytes = (unsigned)(kRsX * kRsY * Kp * 4);
    tile_loop<true>(
        g.nctiles, g.stages, smem, sb, none.scal,
        [&](unsigned char* st, int t, uint64_t* bar) {
            const int cy = t / g.ncx, cx = t - cy * g.ncx;
            mbar_expect_tx(bar, tx_bytes);
            tma_load_pt(st, &mp.m[0], g, 2 * cx * kTXc - 2, 2 * cy * kTYc - 2, bar);
        },
        [&](unsigned char* st, int t) {
            const int cy = t / g.ncx, cx = t - cy * g.ncx;
            const int X0 = cx * kTXc, Y0 = cy * kTYc;
            const int ihi = X0 + kTXc >= g.nxc ? g.nx : 2 * X0 + 2 * kTXc;
            const int jhi = Y0 + kTYc >= g.nyc ? g.ny : 2 * Y0 + 2 * kTYc;
            const float* Bs = reinterpret_cast<const float*>(st);
            // x2 on the owned fine points plus a one-point halo (zero outside the grid)
            for (int p = threadIdx.y; p < kE1X * kE1Y; p += blockDim.y) {
                const int ey = p / kE1X, ex = p - ey * kE1X;
                const int fi = 2 * X0 - 1 + ex, fj = 2 * Y0 - 1 + ey;
                float x2[4] = {0.f, 0.f, 0.f, 0.f};
                if (fi >= 0 && fi < g.nx && fj >= 0 && fj < g.ny) {
                    const int bidx = ((ey + 1) * kRsX + ex + 1) * Kp + off;
                    const int sy = kRsX * Kp;
                    float xc[4], acc[4], n[4], bv[4];
                    auto x1 = [&](int h, float (&o)[4]) {
                        ld4(Bs + h, o);
                        for (int v = 0; v < 4; ++v) o[v] *= c20[v];
                    };
                    x1(bidx, xc);
                    for (int v = 0; v < 4; ++v) acc[v] = diag * xc[v];
                    x1(bidx - Kp, n);
                    for (int v = 0; v < 4; ++v) acc[v] = fmaf(-g.wx, n[v], acc[v]);
                    x1(bidx + Kp, n);
                    for (int v = 0; v < 4; ++v) acc[v] = fmaf(-g.wx, n[v], acc[v]);
                    x1(bidx - sy, n);
                    for (int v = 0; v < 4; ++v) acc[v] = fmaf(-g.wy, n[v], acc[v]);
                    x1(bidx + sy, n);
                    for (int v = 0; v < 4; ++v) acc[v] = fmaf(-g.wy, n[v], acc[v]);
                    ld4(Bs + bidx, bv);
                    for (int v = 0; v < 4; ++v) {
                        const float res = bv[v] - fmaf(-d[v], xc[v], acc[v]);
                        const float gg = c2[v] * res;
                        const float dv = fmaf(c1[v], xc[v], gg);
                        x2[v] = xc[v] + dv;
                    }
                    if (fi >= 2 * X0 && fi < ihi && fj >= 2 * Y0 && fj < jhi)
                        st4(x2out + ((size_t)fj * g.nx + fi) * Kp + off, x2);
                }
                st4(X2s + p * Kp + off, x2);
            }
            __syncthreads();
            // fine residual b - (A - dI) x2 on the (2 kTXc + 1) x (2 kTYc + 1) points the tile restricts
            for (int p = threadIdx.y; p < kRX * kRY; p += blockDim.y) {
                const int ry = p / kRX, rx = p - ry * kRX;
                const int eidx = ((ry + 1) * kE1X + rx + 1) * Kp + off;
                const int sy = kE1X * Kp;
                float xc[4], acc[4], n[4], bv[4], r[4];
                ld4(X2s + eidx, xc);
                for (int v = 0; v < 4; ++v) acc[v] = diag * xc[v];
                ld4(X2s + eidx - Kp, n);
                for (int v = 0; v < 4; ++v) acc[v] = fmaf(-g.wx, n[v], acc[v]);
                ld4(X2s + eidx + Kp, n);
                for (int v = 0; v < 4; ++v) acc[v] = fmaf(-g.wx, n[v], acc[v]);
                ld4(X2s + eidx - sy, n);
                for (int v = 0; v < 4; ++v) acc[v] = fmaf(-g.wy, n[v], acc[v]);
                ld4(X2s + eidx + sy, n);
                for (int v = 0; v < 4; ++v) acc[v] = fmaf(-g.wy, n[v], acc[v]);
                ld4(Bs + ((ry + 2) * kRsX + rx + 2) * Kp + off, bv);
                for (int v = 0; v < 4; ++v) r[v] = bv[v] - fmaf(-d[v], xc[v], acc[v]);
                st4(Rs + p * Kp + off, r);
            }
            __syncthreads();
            // full weighting onto the coarse points of the tile
            for (int p = threadIdx.y; p < kTXc * kTYc; p += blockDim.y) {
                const int ly = p / kTXc, lx = p - ly * kTXc;
                const int I = X0 + lx, J = Y0 + ly;
                if (I >= g.nxc || J >= g.nyc) continue;
                float sum[4] = {0.f, 0.f, 0.f, 0.f};
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        float r[4];
                        ld4(Rs + ((2 * ly + 1 + dy) * kRX + 2 * lx + 1 + dx) * Kp + off, r);
                        const float wt = w1[dx + 1] * w1[dy + 1];
                        for (int v = 0; v < 4; ++v) sum[v] = fmaf(wt, r[v], sum[v]);
                    }
                st4(bc + ((size_t)J * g.nxc + I) * Kp + off, sum);
            }
        });
    pdl_trigger();
}

// The first post-smoothing step with the coarse correction added on the fly: xin = x + P ec on the
// tile and its halo (P = bilinear interpolation; the coarse box is zero outside the coarse grid, which
// adds +0 where the grid kernel skips a zero weight), then the Chebyshev step without a previous
// direction.  xin itself is never stored: only xout and dout are.
template <int C>
__global__ void __launch_bounds__(kTmaThreads, kTmaMaxCtasPerSM)
    k_prolong_cheb_tma(const __grid_constant__ TmaMaps3 mp, TmaGeo g, float* __restrict__ xout,
                       float* __restrict__ dout, ChebStepT<float> cs, const float* __restrict__ dsh, Red none) {
    pdl_wait();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char* smem = aligned_ring(smem_raw);
    const int Kp = C * 4;
    const size_t sb = stage_bytes(TK_PROCHEB, Kp);
    float* Xn = reinterpret_cast<float*>(smem + g.stages * sb);
    const int off = threadIdx.x * 4;
    float c2[4], d[4];
    for (int v = 0; v < 4; ++v) {
        c2[v] = (float)cs.c2[off + v];
        d[v] = (float)dsh[off + v];
    }
    const unsigned tx_bytes = (unsigned)((kHaloPts + kCpX * kCpY + kTilePts) * Kp * 4);
    tile_loop<true>(
        g.ntiles, g.stages, smem, sb, none.scal,
        [&](unsigned char* st, int t, uint64_t* bar) {
            int x0, y0;
            tile_origin(g, t, x0, y0);
            mbar_expect_tx(bar, tx_bytes);
            tma_load_pt(st, &mp.m[0], g, x0 - 1, y0 - 1, bar);
            tma_load_pt(st + halo_bytes(Kp), &mp.m[1], g, x0 / 2 - 1, y0 / 2 - 1, bar);
            tma_load_pt(st + halo_bytes(Kp) + vec_bytes(kCpX * kCpY, Kp), &mp.m[2], g, x0, y0, bar);
        },
        [&](unsigned char* st, int t) {
            int x0, y0;
            tile_origin(g, t, x0, y0);
            const float* X = reinterpret_cast<const float*>(st);
            const float* E = reinterpret_cast<const float*>(st + halo_bytes(Kp));
            const float* B = reinterpret_cast<const float*>(st + halo_bytes(Kp) + vec_bytes(kCpX * kCpY, Kp));
            const int cx0 = x0 / 2 - 1, cy0 = y0 / 2 - 1;
            for (int p = threadIdx.y; p < kHaloPts; p += blockDim.y) {
                const int hy = p / (kTX + 2), hx = p - hy * (kTX + 2);
                const int fi = x0 - 1 + hx, fj = y0 - 1 + hy;
                float xn[4] = {0.f, 0.f, 0.f, 0.f};
                if (fi >= 0 && fi < g.nx && fj >= 0 && fj < g.ny) {
                    int yl[2], xl[2];
                    float wy[2], wx[2];
                    if (fj & 1) { yl[0] = yl[1] = (fj - 1) >> 1; wy[0] = 1.f; wy[1] = 0.f; }
                    else { yl[0] = (fj >> 1) - 1; yl[1] = fj >> 1; wy[0] = wy[1] = 0.5f; }
                    if (fi & 1) { xl[0] = xl[1] = (fi - 1) >> 1; wx[0] = 1.f; wx[1] = 0.f; }
                    else { xl[0] = (fi >> 1) - 1; xl[1] = fi >> 1; wx[0] = wx[1] = 0.5f; }
                    float sum[4] = {0.f, 0.f, 0.f, 0.f};
                    for (int a = 0; a < 2; ++a) {
                        if (wy[a] == 0.f) continue;
                        for (int b2 = 0; b2 < 2; ++b2) {
                            if (wx[b2] == 0.f) continue;
                            float e[4];
                            ld4(E + ((yl[a] - cy0) * kCpX + (xl[b2] - cx0)) * Kp + off, e);
                            const float wt = wx[b2] * wy[a];
                            for (int v = 0; v < 4; ++v) sum[v] = fmaf(wt, e[v], sum[v]);
                        }
                    }
                    ld4(X + p * Kp + off, xn);
                    for (int v = 0; v < 4; ++v) xn[v] += sum[v];
                }
                st4(Xn + p * Kp + off, xn);
            }
            __syncthreads();
            for (int p = threadIdx.y; p < kTilePts; p += blockDim.y) {
                const int ly = p / kTX, lx = p - ly * kTX;
                const int gx = x0 + lx, gy = y0 + ly;
                if (gx >= g.nx || gy >= g.ny) continue;
                const int hidx = ((ly + 1) * (kTX + 2) + lx + 1) * Kp + off;
                float xc[4], Ax[4], bv[4];
                stencil_tile(g, hidx, [&](int h, float (&o)[4]) { ld4(Xn + h, o); }, xc, Ax);
                ld4(B + p * Kp + off, bv);
                float xo[4], dv[4];
                for (int v = 0; v < 4; ++v) {
                    const float res = bv[v] - fmaf(-d[v], xc[v], Ax[v]);
                    const float gg = c2[v] * res;
                    dv[v] = fmaf(0.f, 0.f, gg);
                    xo[v] = xc[v] + dv[v];
                }
                const size_t gidx = ((size_t)gy * g.nx + gx) * Kp + off;
                st4(xout + gidx, xo);
                st4(dout + gidx, dv);
            }
        });
    pdl_trigger();
}

// Prolongation and both post-smoothing steps in one sweep.  Per tile: (1) xin = x + P ec on the tile and
// a two-point halo, in place over the x stage; (2) the first step on the tile and a one-point halo,
// x1 = xin + d1 (recomputed by neighbouring tiles, bit for bit the same) into scratch, d1 kept for the
// tile points; (3) the second step on the tile, stored, with b . xout when red asks for it.  Each step
// is k_prolong_cheb_tma's and k_cheb_tma's arithmetic, operation for operation; points outside the grid
// hold zero (Dirichlet).  Traffic per tile: x, ec, b in, xout out, against x, ec, b in and x1, d1 out,
// then x1, d1, b in and xout out for the two-kernel form.
template <int C>
__global__ void __launch_bounds__(kTmaThreads, kPost2CtasPerSM)
    k_post2_tma(const __grid_constant__ TmaMaps3 mp, TmaGeo g, float* __restrict__ xout, ChebStepT<float> cs0,
                ChebStepT<float> cs1, const float* __restrict__ dsh, Red red) {
    pdl_wait();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char* smem = aligned_ring(smem_raw);
    const int Kp = C * 4;
    const size_t sb = stage_bytes(TK_POST2, Kp);
    float* X1 = reinterpret_cast<float*>(smem + g.stages * sb);
    float* D1 = reinterpret_cast<float*>(smem + g.stages * sb + halo_bytes(Kp));
    const int off = threadIdx.x * 4;
    float c20[4], c11[4], c21[4], d[4];
    for (int v = 0; v < 4; ++v) {
        c20[v] = (float)cs0.c2[off + v];
        c11[v] = cs1.c1 ? (float)cs1.c1[off + v] : 0.f;
        c21[v] = (float)cs1.c2[off + v];
        d[v] = (float)dsh[off + v];
    }
    const size_t e_ofs = vec_bytes(kH2X * kH2Y, Kp);
    const size_t b_ofs = e_ofs + vec_bytes(kCp2X * kCp2Y, Kp);
    const unsigned tx_bytes = (unsigned)((kH2X * kH2Y + kCp2X * kCp2Y + kHaloPts) * Kp * 4);
    const bool dot = red.op != RED_NONE;
    Accum<float> acc;
    tile_loop<true>(
        g.ntiles, g.stages, smem, sb, red.scal,
        [&](unsigned char* st, int t, uint64_t* bar) {
            int x0, y0;
            tile_origin(g, t, x0, y0);
            mbar_expect_tx(bar, tx_bytes);
            tma_load_pt(st, &mp.m[0], g, x0 - 2, y0 - 2, bar);
            tma_load_pt(st + e_ofs, &mp.m[1], g, x0 / 2 - 2, y0 / 2 - 2, bar);
            tma_load_pt(st + b_ofs, &mp.m[2], g, x0 - 1, y0 - 1, bar);
        },
        [&](unsigned char* st, int t) {
            int x0, y0;
            tile_origin(g, t, x0, y0);
            float* X = reinterpret_cast<float*>(st);
            const float* E = reinterpret_cast<const float*>(st + e_ofs);
            const float* B = reinterpret_cast<const float*>(st + b_ofs);
            // (1) xin = x + P ec on the two-point halo region, by 2 x 2 blocks of fine points: the block
            // at even (fi, fj) interpolates from coarse points (fi/2 - 1 .. fi/2) x (fj/2 - 1 .. fj/2),
            // at box offsets (bx, by); the weighted sums are k_prolong_cheb_tma's, term for term.  Item q
            // is the column hx = 2 bx + (q & 1) of block q >> 1 (its two points): consecutive threads
            // touch consecutive points of the x stage, so its loads and stores are free of bank conflicts.
            for (int q = threadIdx.y; q < kH2X * (kH2Y / 2); q += blockDim.y) {
                const int blk = q >> 1, px = q & 1;
                const int by = blk / (kH2X / 2), bx = blk - by * (kH2X / 2);
                float e01[4], e11[4], sa[4], sb[4];  // sa: point (px, 0), sb: point (px, 1) of the block
                ld4(E + (by * kCp2X + bx + 1) * Kp + off, e01);
                ld4(E + ((by + 1) * kCp2X + bx + 1) * Kp + off, e11);
                if (px == 0) {
                    float e00[4], e10[4];
                    ld4(E + (by * kCp2X + bx) * Kp + off, e00);
                    ld4(E + ((by + 1) * kCp2X + bx) * Kp + off, e10);
                    for (int v = 0; v < 4; ++v) {
                        float t = fmaf(0.25f, e00[v], 0.f);
                        t = fmaf(0.25f, e01[v], t);
                        t = fmaf(0.25f, e10[v], t);
                        sa[v] = fmaf(0.25f, e11[v], t);
                        sb[v] = fmaf(0.5f, e11[v], fmaf(0.5f, e10[v], 0.f));
                    }
                } else {
                    for (int v = 0; v < 4; ++v) {
                        sa[v] = fmaf(0.5f, e11[v], fmaf(0.5f, e01[v], 0.f));
                        sb[v] = fmaf(1.f, e11[v], 0.f);
                    }
                }
                const int hx = 2 * bx + px;
                const int fi = x0 - 2 + hx;
                for (int r = 0; r < 2; ++r) {
                    const int hy = 2 * by + r, fj = y0 - 2 + hy;
                    const int h = (hy * kH2X + hx) * Kp + off;
                    float xn[4] = {0.f, 0.f, 0.f, 0.f};
                    if (fi >= 0 && fi < g.nx && fj >= 0 && fj < g.ny) {
                        ld4(X + h, xn);
                        for (int v = 0; v < 4; ++v) xn[v] += r ? sb[v] : sa[v];
                    }
                    st4(X + h, xn);
                }
            }
            fence_proxy_async_smem();  // the x stage is refilled by TMA after the tile
            __syncthreads();
            // (2) first step on the one-point halo region, by vertical pairs of points (rows 2m, 2m + 1 of
            // the region): the pair shares its column of four values and its index arithmetic
            for (int q = threadIdx.y; q < (kTX + 2) * ((kTY + 2) / 2); q += blockDim.y) {
                const int pr = q / (kTX + 2), hx = q - pr * (kTX + 2);
                const int hy0 = 2 * pr;
                const int fi = x0 - 1 + hx, fj0 = y0 - 1 + hy0;
                // x at 2-halo rows hy0 .. hy0 + 3 of column hx + 1, and the left / right neighbours of the pair
                const int c0 = (hy0 * kH2X + hx + 1) * Kp + off;
                float up[4], m0[4], m1[4], dn[4], l0[4], r0[4], l1[4], r1[4];
                ld4(X + c0, up);
                ld4(X + c0 + kH2X * Kp, m0);
                ld4(X + c0 + 2 * kH2X * Kp, m1);
                ld4(X + c0 + 3 * kH2X * Kp, dn);
                ld4(X + c0 + kH2X * Kp - Kp, l0);
                ld4(X + c0 + kH2X * Kp + Kp, r0);
                ld4(X + c0 + 2 * kH2X * Kp - Kp, l1);
                ld4(X + c0 + 2 * kH2X * Kp + Kp, r1);
                const bool in_x = fi >= 0 && fi < g.nx;
                for (int j = 0; j < 2; ++j) {
                    const int hy = hy0 + j, fj = fj0 + j;
                    const float(&xc)[4] = j ? m1 : m0;
                    const float(&xl)[4] = j ? l1 : l0;
                    const float(&xr)[4] = j ? r1 : r0;
                    const float(&xu)[4] = j ? m0 : up;
                    const float(&xd)[4] = j ? dn : m1;
                    float xo[4] = {0.f, 0.f, 0.f, 0.f};
                    if (in_x && fj >= 0 && fj < g.ny) {
                        const float diag = g.wx + g.wx + g.wy + g.wy;
                        float bv[4], dv[4];
                        ld4(B + (hy * (kTX + 2) + hx) * Kp + off, bv);
                        for (int v = 0; v < 4; ++v) {
                            float a = diag * xc[v];
                            a = fmaf(-g.wx, xl[v], a);
                            a = fmaf(-g.wx, xr[v], a);
                            a = fmaf(-g.wy, xu[v], a);
                            a = fmaf(-g.wy, xd[v], a);
                            const float res = bv[v] - fmaf(-d[v], xc[v], a);
                            const float gg = c20[v] * res;
                            dv[v] = fmaf(0.f, 0.f, gg);
                            xo[v] = xc[v] + dv[v];
                        }
                        if (hx >= 1 && hx <= kTX && hy >= 1 && hy <= kTY)
                            st4(D1 + ((hy - 1) * kTX + hx - 1) * Kp + off, dv);
                    }
                    st4(X1 + (hy * (kTX + 2) + hx) * Kp + off, xo);
                }
            }
            __syncthreads();
            // (3) second step on the tile, by vertical pairs of points
            for (int q = threadIdx.y; q < kTX * (kTY / 2); q += blockDim.y) {
                const int pr = q / kTX, lx = q - pr * kTX;
                const int ly0 = 2 * pr;
                const int gx = x0 + lx, gy0 = y0 + ly0;
                if (gx >= g.nx || gy0 >= g.ny) continue;
                // x1 at 1-halo rows ly0 .. ly0 + 3 of column lx + 1, and the neighbours of the pair
                const int c0 = (ly0 * (kTX + 2) + lx + 1) * Kp + off;
                const int sy = (kTX + 2) * Kp;
                float up[4], m0[4], m1[4], dn[4], l0[4], r0[4], l1[4], r1[4];
                ld4(X1 + c0, up);
                ld4(X1 + c0 + sy, m0);
                ld4(X1 + c0 + 2 * sy, m1);
                ld4(X1 + c0 + 3 * sy, dn);
                ld4(X1 + c0 + sy - Kp, l0);
                ld4(X1 + c0 + sy + Kp, r0);
                ld4(X1 + c0 + 2 * sy - Kp, l1);
                ld4(X1 + c0 + 2 * sy + Kp, r1);
                for (int j = 0; j < 2; ++j) {
                    const int gy = gy0 + j;
                    if (gy >= g.ny) break;
                    const float(&xc)[4] = j ? m1 : m0;
                    const float(&xl)[4] = j ? l1 : l0;
                    const float(&xr)[4] = j ? r1 : r0;
                    const float(&xu)[4] = j ? m0 : up;
                    const float(&xd)[4] = j ? dn : m1;
                    const float diag = g.wx + g.wx + g.wy + g.wy;
                    float bv[4], dv[4], xo[4];
                    ld4(B + c0 + (1 + j) * sy, bv);
                    ld4(D1 + ((ly0 + j) * kTX + lx) * Kp + off, dv);
                    for (int v = 0; v < 4; ++v) {
                        float a = diag * xc[v];
                        a = fmaf(-g.wx, xl[v], a);
                        a = fmaf(-g.wx, xr[v], a);
                        a = fmaf(-g.wy, xu[v], a);
                        a = fmaf(-g.wy, xd[v], a);
                        const float res = bv[v] - fmaf(-d[v], xc[v], a);
                        const float gg = c21[v] * res;
                        dv[v] = fmaf(c11[v], dv[v], gg);
                        xo[v] = xc[v] + dv[v];
                    }
                    st4(xout + ((size_t)gy * g.nx + gx) * Kp + off, xo);
                    if (dot) acc.add(bv, xo);
                }
            }
        });
    pdl_trigger();
    if (dot) reduce_finish<float>(acc, red, Kp);
}

// CG vector update from TMA-staged tiles: x += alpha p, r -= alpha q and r.r per system (pointwise, no
// halo).  The grid-stride kernel is limited to 8 CTAs of 4 warps per SM by its registers; here the bytes
// in flight are the ring's stages, whatever the occupancy.
template <int C>
__global__ void __launch_bounds__(kTmaThreads, kTmaMaxCtasPerSM)
    k_cg_update_tma(const __grid_constant__ TmaMaps5 mp, TmaGeo g, float* __restrict__ x, float* __restrict__ r,
                    Red red) {
    pdl_wait();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char* smem = aligned_ring(smem_raw);
    const int Kp = C * 4;
    const size_t sb = stage_bytes(TK_CG, Kp);
    const size_t pb = plain_bytes(Kp);
    const int off = threadIdx.x * 4;
    // the direction k_spmv_tma just wrote (its pnew), selected by the same parity
    const CUtensorMap* mp_dir = red.scal->parity ? &mp.m[2] : &mp.m[3];
    float a[4];
    for (int v = 0; v < 4; ++v) a[v] = red.scal->alphaf[off + v];
    const unsigned tx_bytes = (unsigned)(4 * kTilePts * Kp * 4);
    Accum<float> acc;
    tile_loop<false>(
        g.ntiles, g.stages, smem, sb, red.scal,
        [&](unsigned char* st, int t, uint64_t* bar) {
            int x0, y0;
            tile_origin(g, t, x0, y0);
            mbar_expect_tx(bar, tx_bytes);
            tma_load_pt(st, &mp.m[0], g, x0, y0, bar);
            tma_load_pt(st + pb, &mp.m[1], g, x0, y0, bar);
            tma_load_pt(st + 2 * pb, mp_dir, g, x0, y0, bar);
            tma_load_pt(st + 3 * pb, &mp.m[4], g, x0, y0, bar);
        },
        [&](unsigned char* st, int t) {
            int x0, y0;
            tile_origin(g, t, x0, y0);
            const float* X = reinterpret_cast<const float*>(st);
            const float* R = reinterpret_cast<const float*>(st + pb);
            const float* P = reinterpret_cast<const float*>(st + 2 * pb);
            const float* Q = reinterpret_cast<const float*>(st + 3 * pb);
            for (int p = threadIdx.y; p < kTilePts; p += blockDim.y) {
                const int ly = p / kTX, lx = p - ly * kTX;
                const int gx = x0 + lx, gy = y0 + ly;
                if (gx >= g.nx || gy >= g.ny) continue;
                const int i = p * Kp + off;
                float xv[4], rv[4], pv[4], qv[4];
                ld4(X + i, xv);
                ld4(R + i, rv);
                ld4(P + i, pv);
                ld4(Q + i, qv);
                for (int v = 0; v < 4; ++v) {
                    xv[v] = fmaf(a[v], pv[v], xv[v]);
                    rv[v] = fmaf(-a[v], qv[v], rv[v]);
                }
                const size_t gidx = ((size_t)gy * g.nx + gx) * Kp + off;
                st4(x + gidx, xv);
                st4(r + gidx, rv);
                acc.add(rv, rv);
            }
        });
    pdl_trigger();
    reduce_finish<float>(acc, red, Kp);
}

template <int C>
cudaError_t prepare_c() {
    // every TMA kernel may take up to a whole SM's worth of ring (the launch asks for what it uses)
    const int mx = (int)kSmemPerCTA;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_cheb_tma<C, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_cheb_tma<C, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_pre2_tma<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_pre2_restrict_tma<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx)) !=
        cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_prolong_cheb_tma<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx)) !=
        cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_post2_tma<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_cg_update_tma<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx)) != cudaSuccess)
        return e;
    return cudaFuncSetAttribute(k_spmv_tma<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
}

template <class K, class... Args>
cudaError_t launch_tile(K kernel, int blocks, int threads, int C, size_t smem, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(C, threads / C);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

}  // namespace

bool tma_supported(int Kp) { return Kp == 4 || Kp == 8 || Kp == 12 || Kp == 16; }

// The widest box row is the fused restriction's, (2 kTXc + 5) points of Kp / 2 eight-byte elements.
bool tma_flat(int Kp) { return (2 * kTXc + 5) * (Kp / 2) <= 256; }

TmaGeo tma_geo(const Lev& L, const Lev* Lc, int Kp) {
    TmaGeo g;
    g.nxc = Lc ? Lc->nx : 0;
    g.nyc = Lc ? Lc->ny : 0;
    g.ncx = (g.nxc + kTXc - 1) / kTXc;
    g.ncy = (g.nyc + kTYc - 1) / kTYc;
    g.nctiles = g.ncx * g.ncy;
    g.nx = L.nx;
    g.ny = L.ny;
    g.ntx = (L.nx + kTX - 1) / kTX;
    g.nty = (L.ny + kTY - 1) / kTY;
    g.ntiles = g.ntx * g.nty;
    g.Kp = Kp;
    g.wx = (float)L.wx;
    g.wy = (float)L.wy;
    g.flat = tma_flat(Kp) ? 1 : 0;
    g.stages = kTmaStages;
    return g;
}

cudaError_t tma_encode(CUtensorMap* m, const float* base, int Kp, int nx, int ny, int boxkind) {
    // resolved once per process (a thread-safe static initialisation: plans may be set up concurrently)
    static const PFN_cuTensorMapEncodeTiled_v12000 encode = [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        return (e == cudaSuccess && q == cudaDriverEntryPointSuccess) ? reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn)
                                                                        : nullptr;
    }();
    if (!encode) return cudaErrorNotSupported;
    int bx = 0, by = 0;
    tma_box_dims(boxkind, &bx, &by);
    const cuuint32_t estr[3] = {1, 1, 1};
    CUresult r;
    if (tma_flat(Kp)) {
        // rows of nx * Kp / 2 eight-byte elements: a box row is (bx points) contiguous bytes; zero fill
        // outside the row is the Dirichlet boundary exactly as in the 3-D form (all-zero bits = 0.0f)
        const cuuint64_t dims[2] = {(cuuint64_t)nx * (Kp / 2), (cuuint64_t)ny};
        const cuuint64_t strides[1] = {(cuuint64_t)nx * Kp * sizeof(float)};
        const cuuint32_t box[2] = {(cuuint32_t)(bx * (Kp / 2)), (cuuint32_t)by};
        r = encode(m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, const_cast<float*>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    } else {
        const cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)nx, (cuuint64_t)ny};
        const cuuint64_t strides[2] = {(cuuint64_t)Kp * sizeof(float), (cuuint64_t)nx * Kp * sizeof(float)};
        const cuuint32_t box[3] = {(cuuint32_t)Kp, (cuuint32_t)bx, (cuuint32_t)by};
        r = encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    }
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t tma_prepare(int Kp) {
    switch (Kp) {
        case 4: return prepare_c<1>();
        case 8: return prepare_c<2>();
        case 12: return prepare_c<3>();
        case 16: return prepare_c<4>();
        default: return cudaErrorInvalidValue;
    }
}

// Ring depth of a launch: the requested depth, reduced until the ring fits one CTA (at least 1).
int ring_stages(const TmaGeo& g, int kind) {
    int S = g.stages < 1 ? kTmaStages : (g.stages > kTmaMaxStages ? kTmaMaxStages : g.stages);
    if (kind == TK_POST2 && kPost2Stages > 0) S = kPost2Stages;
    while (S > 1 && dyn_smem(kind, g.Kp, S) + kRingSlack > kSmemPerCTA) --S;
    return S;
}

// Persistent grid: as many CTAs per SM as their rings fit in shared memory (at most kTmaMaxCtasPerSM, or
// kPost2CtasPerSM for the fused post-smoothing, whose launch bounds allow more registers).
int tma_blocks(const TmaGeo& g, int Kp, int nsm, int kind, int S) {
    const size_t smem = dyn_smem(kind, Kp, S) + kRingSlack + kSmemReserved + 64;  // + static
    int per_sm = (int)(kSmemPerSM / smem);
    const int cap = kind == TK_POST2 ? kPost2CtasPerSM : kTmaMaxCtasPerSM;  // the launch bounds' registers
    per_sm = per_sm < 1 ? 1 : (per_sm > cap ? cap : per_sm);
    const int nt = kind == TK_PRE2R ? g.nctiles : g.ntiles;
    return nt < nsm * per_sm ? nt : nsm * per_sm;
}

// Launch geometry of one kind: g with its ring depth, CTAs, dynamic shared memory.
struct Shape {
    TmaGeo g;
    int blocks;
    int threads;
    size_t smem;
};
Shape shape_of(const TmaGeo& g0, int nsm, int kind) {
    Shape sh;
    sh.g = g0;
    sh.g.stages = ring_stages(g0, kind);
    sh.blocks = tma_blocks(sh.g, g0.Kp, nsm, kind, sh.g.stages);
    sh.threads = kTmaThreads;
    sh.smem = dyn_smem(kind, g0.Kp, sh.g.stages) + kRingSlack;
    return sh;
}

#define BURA_TMA_C(Kp, CALL)            \
    switch (Kp) {                       \
        case 4: { constexpr int C = 1; CALL; } \
        case 8: { constexpr int C = 2; CALL; } \
        case 12: { constexpr int C = 3; CALL; } \
        case 16: { constexpr int C = 4; CALL; } \
        default: return cudaErrorInvalidValue; \
    }

cudaError_t tma_cheb_step(const TmaGeo& g, int nsm, const CUtensorMap& mx, const CUtensorMap* md, const CUtensorMap& mb,
                          float* xout, float* dout, ChebStepT<float> cs, const float* dsh, const Red& red, cudaStream_t s) {
    TmaMaps3 mp;
    mp.m[0] = mx;
    mp.m[1] = md ? *md : mx;
    mp.m[2] = mb;
    const Shape sh = shape_of(g, nsm, md ? TK_CHEB_D : TK_CHEB);
    if (md)
        BURA_TMA_C(g.Kp, return launch_tile(k_cheb_tma<C, true>, sh.blocks, sh.threads, C, sh.smem, s, mp, sh.g, xout, dout, cs, dsh,
                                            red))
    BURA_TMA_C(g.Kp, return launch_tile(k_cheb_tma<C, false>, sh.blocks, sh.threads, C, sh.smem, s, mp, sh.g, xout, dout, cs, dsh,
                                        red))
}

cudaError_t tma_pre2(const TmaGeo& g, int nsm, const CUtensorMap& mb_halo, float* xout, float* dout, ChebStepT<float> cs0,
                     ChebStepT<float> cs1, const float* dsh, const Red& none, cudaStream_t s) {
    TmaMaps3 mp;
    mp.m[0] = mp.m[1] = mp.m[2] = mb_halo;
    const Shape sh = shape_of(g, nsm, TK_PRE2);
    BURA_TMA_C(g.Kp, return launch_tile(k_pre2_tma<C>, sh.blocks, sh.threads, C, sh.smem, s, mp, sh.g, xout, dout, cs0, cs1, dsh,
                                        none))
}

cudaError_t tma_pre2_restrict(const TmaGeo& g, int nsm, const CUtensorMap& mb_rsrc, float* x2out, float* bc,
                              ChebStepT<float> cs0, ChebStepT<float> cs1, const float* dsh, const Red& none, cudaStream_t s) {
    TmaMaps3 mp;
    mp.m[0] = mp.m[1] = mp.m[2] = mb_rsrc;
    const Shape sh = shape_of(g, nsm, TK_PRE2R);
    BURA_TMA_C(g.Kp, return launch_tile(k_pre2_restrict_tma<C>, sh.blocks, sh.threads, C, sh.smem, s, mp, sh.g, x2out, bc, cs0,
                                        cs1, dsh, none))
}

cudaError_t tma_prolong_cheb(const TmaGeo& g, int nsm, const CUtensorMap& mx_halo, const CUtensorMap& mec_cpro,
                             const CUtensorMap& mb, float* xout, float* dout, ChebStepT<float> cs, const float* dsh,
                             const Red& none, cudaStream_t s) {
    TmaMaps3 mp;
    mp.m[0] = mx_halo;
    mp.m[1] = mec_cpro;
    mp.m[2] = mb;
    const Shape sh = shape_of(g, nsm, TK_PROCHEB);
    BURA_TMA_C(g.Kp, return launch_tile(k_prolong_cheb_tma<C>, sh.blocks, sh.threads, C, sh.smem, s, mp, sh.g, xout, dout, cs, dsh,
                                        none))
}

cudaError_t tma_post2(const TmaGeo& g, int nsm, const CUtensorMap& mx_halo2, const CUtensorMap& mec_cpro2,
                      const CUtensorMap& mb_halo, float* xout, ChebStepT<float> cs0, ChebStepT<float> cs1,
                      const float* dsh, const Red& red, cudaStream_t s) {
    TmaMaps3 mp;
    mp.m[0] = mx_halo2;
    mp.m[1] = mec_cpro2;
    mp.m[2] = mb_halo;
    const Shape sh = shape_of(g, nsm, TK_POST2);
    BURA_TMA_C(g.Kp, return launch_tile(k_post2_tma<C>, sh.blocks, sh.threads, C, sh.smem, s, mp, sh.g, xout, cs0, cs1,
                                        dsh, red))
}

cudaError_t tma_spmv_p(const TmaGeo& g, int nsm, const CUtensorMap& mz, const CUtensorMap& mpa,
                       const CUtensorMap& mpb, float* pa, float* pb, float* q, const Red& red, cudaStream_t s) {
    TmaMaps3 mp;
    mp.m[0] = mz;
    mp.m[1] = mpa;
    mp.m[2] = mpb;
    const Shape sh = shape_of(g, nsm, TK_SPMV);
    BURA_TMA_C(g.Kp, return launch_tile(k_spmv_tma<C>, sh.blocks, sh.threads, C, sh.smem, s, mp, sh.g, pa, pb, q, red))
}

bool tma_cg_fits(int Kp) { return dyn_smem(TK_CG, Kp, 2) + kRingSlack <= kSmemPerCTA; }

cudaError_t tma_cg_update(const TmaGeo& g, int nsm, const CUtensorMap& mx, const CUtensorMap& mr,
                          const CUtensorMap& mpa, const CUtensorMap& mpb, const CUtensorMap& mq, float* x, float* r,
                          const Red& red, cudaStream_t s) {
    TmaMaps5 mp;
    mp.m[0] = mx;
    mp.m[1] = mr;
    mp.m[2] = mpa;
    mp.m[3] = mpb;
    mp.m[4] = mq;
    TmaGeo g1 = g;
    if (g1.stages < 3) g1.stages = 3;  // pointwise: the deepest ring that fits (1 CTA per SM)
    const Shape sh = shape_of(g1, nsm, TK_CG);
    BURA_TMA_C(g.Kp, return launch_tile(k_cg_update_tma<C>, sh.blocks, sh.threads, C, sh.smem, s, mp, sh.g, x, r, red))
}

}  // namespace bura
