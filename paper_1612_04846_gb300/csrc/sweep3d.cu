// The 3-D Chebyshev step and the 3-D residual r = b - (A - d_j I) x (FP32) with their inputs staged in
// shared memory.
//
// A work item is a tile of kPX x kPY points of the (x, y) plane over pz consecutive planes (kPZ where the
// items of a level fill the grid's CTA slots, kPZ / 2 on levels where they do not).  A CTA of
// Kp/4 x kPX x kPY threads (one 16-byte chunk of one point each) marches the item along z: a ring of
// kPRing plane slots in shared memory holds, per plane, x on the tile with a one-point halo, b, the
// previous direction d, and for variable coefficients the face weights and the diagonal of the tile's
// points.  Every thread fills its share of a slot with asynchronous copies (cp.async; zero-filled
// outside the grid, which is the homogeneous Dirichlet boundary) kPRing - 1 planes ahead of the plane
// it computes, so the bytes in flight no longer depend on registers.  One CTA barrier per plane makes
// the landed slots visible to all threads and frees the oldest slot for refilling.
// x on the plane below stays in registers; per point the arithmetic is the z-marching sweep's
// (zmarch in kernels_impl.cuh), operation for operation.
#include "kernels_impl.cuh"

namespace bura {

namespace {

constexpr int kPX = 16, kPY = 8;      // tile points along x and y
#ifndef BURA_3S_PZ
#define BURA_3S_PZ 128
#endif
constexpr int kPZ = BURA_3S_PZ;       // planes per work item on levels whose items fill the grid
constexpr int kPRing = 4;             // plane slots of the ring
constexpr int kPHx = kPX + 2, kPHy = kPY + 2;  // the tile with its one-point halo
constexpr int kPPts = kPX * kPY;
constexpr int kPHalo = kPHx * kPHy;
// face weights of a tile plane: fx (kPX + 1) x kPY, fy kPX x (kPY + 1), fz (the face below each point)
// kPX x kPY, the diagonal kPX x kPY
constexpr int kPFx = (kPX + 1) * kPY, kPFy = kPX * (kPY + 1), kPFz = kPPts, kPDg = kPPts;
constexpr int kPFaces = kPFx + kPFy + kPFz + kPDg;

__device__ __forceinline__ void cpa16(void* dst, const void* src, bool ok) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(ok ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cpa4(void* dst, const void* src, bool ok) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(ok ? 4 : 0)
                 : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cpa_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Floats of one slot: x halo, b, d (Kp each per point) and, with VAR, the faces and the diagonal.
template <bool VAR>
__host__ __device__ constexpr int slot_floats(int Kp) {
    return (kPHalo + 2 * kPPts) * Kp + (VAR ? kPFaces : 0);
}

// RES: store the residual b - (A - d_j I) x instead of the Chebyshev step (no d, no coefficients, no sum)
template <int C, bool VAR, bool RES>
__global__ void __launch_bounds__(C * kPPts, C <= 3 ? 2 : 1)
    k_cheb_step3s(Lev L, const float* __restrict__ xin, const float* __restrict__ din, const float* __restrict__ b,
                  float* __restrict__ xout, float* __restrict__ dout, ChebStepT<float> cs,
                  const float* __restrict__ dsh, Red red, int pz) {
    pdl_wait();
    constexpr int Kp = 4 * C;
    constexpr int SF = slot_floats<VAR>(Kp);
    extern __shared__ __align__(16) float ring[];
    const int nx = L.nx, ny = L.ny, nz = L.nz;
    const int c = threadIdx.x, p = threadIdx.y;
    const int off = c * 4;
    const int px = p % kPX, py = p / kPX;
    const int tid = p * C + c, nthr = C * kPPts;
    float c1[4], c2[4], d[4];
    for (int v = 0; v < 4; ++v) {
        c1[v] = !RES && cs.c1 ? cs.c1[off + v] : 0.f;
        c2[v] = RES ? 0.f : cs.c2[off + v];
        d[v] = dsh[off + v];
    }
    const float* fx = reinterpret_cast<const float*>(L.fx);
    const float* fy = reinterpret_cast<const float*>(L.fy);
    const float* fz = reinterpret_cast<const float*>(L.fz);
    const float* dg = reinterpret_cast<const float*>(L.dg);
    const bool dot = !RES && red.op != RED_NONE;
    Accum<float> acc;
    const int ntx = (nx + kPX - 1) / kPX, nty = (ny + kPY - 1) / kPY, nzs = (nz + pz - 1) / pz;
    const int items = ntx * nty * nzs;
    for (int item = blockIdx.x; item < items; item += gridDim.x) {
        const int tz = item / (ntx * nty);
        const int rem = item - tz * ntx * nty;
        const int ty = rem / ntx, tx = rem - ty * ntx;
        const int X0 = tx * kPX, Y0 = ty * kPY, l0 = tz * pz, l1 = min(nz, l0 + pz);
        // this thread's copies of a plane, fixed per item (slot offset, offset within the plane, in range):
        // halo chunks tid and tid + nthr of the (kPX + 2) x (kPY + 2) x C, the b (and d) chunk tid, and face
        // weights tid + u nthr (u < kFc)
        constexpr int kFc = (kPFaces + C * kPPts - 1) / (C * kPPts);
        int hs[2], hg[2];
        bool hok[2], hin[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int i = tid + u * nthr;
            hin[u] = i < kPHalo * C;
            const int h = hin[u] ? i / C : 0, cc = i - (i / C) * C;
            const int gx = X0 - 1 + h % kPHx, gy = Y0 - 1 + h / kPHx;
            hs[u] = h * Kp + cc * 4;
            hok[u] = hin[u] && gx >= 0 && gx < nx && gy >= 0 && gy < ny;
            hg[u] = hok[u] ? (gy * nx + gx) * Kp + cc * 4 : 0;
        }
        int bs, bg;
        bool bok;
        {
            const int q = tid / C, cc = tid - q * C;
            const int gx = X0 + q % kPX, gy = Y0 + q / kPX;
            bs = (kPHalo + q) * Kp + cc * 4;
            bok = gx < nx && gy < ny;
            bg = bok ? (gy * nx + gx) * Kp + cc * 4 : 0;
        }
        int fgo[kFc], ft[kFc];
        bool fok[kFc];
#pragma unroll
        for (int u = 0; u < kFc; ++u) {
            const int i = tid + u * nthr;
            int k = i, t = 0, qx = 0, qy = 0;
            if (k >= kPFx) { k -= kPFx; t = 1; }
            if (t == 1 && k >= kPFy) { k -= kPFy; t = 2; }
            if (t == 2 && k >= kPFz) { k -= kPFz; t = 3; }
            if (t == 0) {
                qx = k % (kPX + 1); qy = k / (kPX + 1);
                fok[u] = X0 + qx <= nx && Y0 + qy < ny;
                fgo[u] = (Y0 + qy) * (nx + 1) + X0 + qx;
            } else if (t == 1) {
                qx = k % kPX; qy = k / kPX;
                fok[u] = X0 + qx < nx && Y0 + qy <= ny;
                fgo[u] = (Y0 + qy) * nx + X0 + qx;
            } else {
                qx = k % kPX; qy = k / kPX;
                fok[u] = X0 + qx < nx && Y0 + qy < ny;
                fgo[u] = (Y0 + qy) * nx + X0 + qx;
            }
            fok[u] = fok[u] && i < kPFaces;
            if (!fok[u]) fgo[u] = 0;
            ft[u] = t;
        }
        const size_t pv = (size_t)nx * ny * Kp;  // floats per plane of a vector
        auto fetch = [&](int l) {
            if (l <= l1) {
                float* S = ring + (size_t)((l - l0) % kPRing) * SF;
                const bool lin = l < nz;
                const size_t lo = lin ? (size_t)l * pv : 0;
#pragma unroll
                for (int u = 0; u < 2; ++u)
                    if (hin[u]) cpa16(S + hs[u], xin + lo + hg[u], lin && hok[u]);
                cpa16(S + bs, b + lo + bg, lin && bok);
                if (din) cpa16(S + kPPts * Kp + bs, din + lo + bg, lin && bok);
                if (VAR) {
                    float* F = S + (kPHalo + 2 * kPPts) * Kp;
#pragma unroll
                    for (int u = 0; u < kFc; ++u) {
                        const int i = tid + u * nthr;
                        if (i < kPFaces) {
                            const int t = ft[u];
                            const float* base = t == 0 ? fx + (size_t)l * ny * (nx + 1)
                                              : t == 1 ? fy + (size_t)l * (ny + 1) * nx
                                              : t == 2 ? fz + (size_t)l * ny * nx
                                                       : dg + (size_t)l * ny * nx;
                            const bool ok = fok[u] && (t == 2 ? l <= nz : lin);
                            cpa4(F + i, ok ? base + fgo[u] : fx, ok);
                        }
                    }
                }
            }
            cpa_commit();
        };
        const int gx = X0 + px, gy = Y0 + py;
        const bool mine = gx < nx && gy < ny;
        float xm1[4] = {0.f, 0.f, 0.f, 0.f};  // x on the plane below
        if (mine && l0 > 0) {
            const float4 q = *reinterpret_cast<const float4*>(xin + (((size_t)(l0 - 1) * ny + gy) * nx + gx) * Kp + off);
            xm1[0] = q.x; xm1[1] = q.y; xm1[2] = q.z; xm1[3] = q.w;
        }
        for (int l = l0; l < l0 + kPRing - 1; ++l) fetch(l);
        const int hc = ((py + 1) * kPHx + px + 1) * Kp + off;  // the point in the halo tile
        for (int l = l0; l < l1; ++l) {
            cpa_wait<kPRing - 3>();  // planes l and l + 1 have landed (this thread's copies)
            __syncthreads();         // ... everyone's; and the slot of plane l - 1 is free
            fetch(l + kPRing - 1);
            const float* S = ring + (size_t)((l - l0) % kPRing) * SF;
            const float* Sn = ring + (size_t)((l + 1 - l0) % kPRing) * SF;
            if (!mine) continue;
            float x0[4], xl[4], xr[4], xd[4], xu[4], xp1[4];
            auto ld = [](const float* q, float (&o)[4]) {
                const float4 v = *reinterpret_cast<const float4*>(q);
                o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
            };
            ld(S + hc, x0);
            ld(S + hc - Kp, xl);
            ld(S + hc + Kp, xr);
            ld(S + hc - kPHx * Kp, xd);
            ld(S + hc + kPHx * Kp, xu);
            ld(Sn + hc, xp1);
            float wxm, wxp, wym, wyp, wzm, wzp, diag;
            if (VAR) {
                const float* F = S + (kPHalo + 2 * kPPts) * Kp;
                const float* Fn = Sn + (kPHalo + 2 * kPPts) * Kp;
                wxm = F[py * (kPX + 1) + px];
                wxp = F[py * (kPX + 1) + px + 1];
                wym = F[kPFx + py * kPX + px];
                wyp = F[kPFx + (py + 1) * kPX + px];
                wzm = F[kPFx + kPFy + py * kPX + px];
                wzp = Fn[kPFx + kPFy + py * kPX + px];
                diag = F[kPFx + kPFy + kPFz + py * kPX + px];
            } else {
                wxm = wxp = L.wxf;
                wym = wyp = L.wyf;
                wzm = wzp = L.wzf;
                diag = wxm + wxp + wym + wyp;
                diag += wzm + wzp;
            }
            const int q = (py * kPX + px) * Kp + off;
            float bv[4], dv[4] = {0.f, 0.f, 0.f, 0.f}, xo[4];
            ld(S + kPHalo * Kp + q, bv);
            if (din) ld(S + (kPHalo + kPPts) * Kp + q, dv);
            for (int v = 0; v < 4; ++v) {
                float a = diag * x0[v];
                a = fmaf(-wxm, xl[v], a);
                a = fmaf(-wxp, xr[v], a);
                a = fmaf(-wym, xd[v], a);
                a = fmaf(-wyp, xu[v], a);
                a = fmaf(-wzm, xm1[v], a);
                a = fmaf(-wzp, xp1[v], a);
                const float res = bv[v] - fmaf(-d[v], x0[v], a);
                if (RES) {
                    xo[v] = res;
                    xm1[v] = x0[v];
                    continue;
                }
                float g = c2[v] * res;
                if (VAR) g = jdiv(g, diag - d[v]);
                dv[v] = fmaf(c1[v], dv[v], g);
                xo[v] = x0[v] + dv[v];
                xm1[v] = x0[v];
            }
            const size_t go = (((size_t)l * ny + gy) * nx + gx) * Kp + off;
            *reinterpret_cast<float4*>(xout + go) = make_float4(xo[0], xo[1], xo[2], xo[3]);
            if (dout) *reinterpret_cast<float4*>(dout + go) = make_float4(dv[0], dv[1], dv[2], dv[3]);
            if (dot) acc.add(bv, xo);
        }
        cpa_wait<0>();
        __syncthreads();  // no copy of this item lands after the next item starts refilling the ring
    }
    pdl_trigger();
    if (dot) reduce_finish<float>(acc, red, Kp);
}

// Planes per work item for a level and the grid: kPZ planes where the level's items fill the CTA slots,
// else kPZ / 2 (a 127^3 level has 128 items of 128 planes for 304 slots of 152 SMs).
int item_grid(const Lev& L, long long slots, int& pz) {
    const long long cols = (long long)((L.nx + kPX - 1) / kPX) * ((L.ny + kPY - 1) / kPY);
    pz = cols * ((L.nz + kPZ - 1) / kPZ) >= slots ? kPZ : kPZ / 2;
    return (int)std::min<long long>(cols * ((L.nz + pz - 1) / pz), slots);
}

}  // namespace

size_t cheb3s_smem_bytes(int Kp, bool var) {
    return (size_t)kPRing * (var ? slot_floats<true>(Kp) : slot_floats<false>(Kp)) * sizeof(float);
}

#define BURA_3S_SWITCH(Kp, var, CALL)                                         \
    switch (Kp) {                                                             \
        case 4: if (var) { constexpr int C = 1; constexpr bool V = true; CALL; } else { constexpr int C = 1; constexpr bool V = false; CALL; } break; \
        case 8: if (var) { constexpr int C = 2; constexpr bool V = true; CALL; } else { constexpr int C = 2; constexpr bool V = false; CALL; } break; \
        case 12: if (var) { constexpr int C = 3; constexpr bool V = true; CALL; } else { constexpr int C = 3; constexpr bool V = false; CALL; } break; \
        case 16: if (var) { constexpr int C = 4; constexpr bool V = true; CALL; } else { constexpr int C = 4; constexpr bool V = false; CALL; } break; \
        default: return cudaErrorInvalidValue;                                \
    }

cudaError_t cheb3s_prepare(int Kp, bool var) {
    const int bytes = (int)cheb3s_smem_bytes(Kp, var);
    cudaError_t e = cudaSuccess;
    BURA_3S_SWITCH(Kp, var, e = cudaFuncSetAttribute(k_cheb_step3s<C, V, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes))
    if (e != cudaSuccess) return e;
    BURA_3S_SWITCH(Kp, var, e = cudaFuncSetAttribute(k_cheb_step3s<C, V, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes))
    return e;
}

cudaError_t launch_cheb_step3s(const Lev& L, int Kp, bool var, int nsm, const float* xin, const float* din,
                               const float* b, float* xout, float* dout, ChebStepT<float> cs, const float* dsh,
                               const Red& red, cudaStream_t s) {
    const int per_sm = Kp <= 12 ? 2 : 1;
    int pz = 0;
    const int grid = item_grid(L, (long long)per_sm * nsm, pz);
    const size_t smem = cheb3s_smem_bytes(Kp, var);
    BURA_3S_SWITCH(Kp, var, launch_pdl(k_cheb_step3s<C, V, false>, dim3(grid), dim3(C, kPPts), smem, s, L, xin, din, b,
                                       xout, dout, cs, dsh, red, pz))
    return cudaGetLastError();
}

cudaError_t launch_residual3s(const Lev& L, int Kp, bool var, int nsm, const float* x, const float* b, float* r,
                              const float* dsh, cudaStream_t s) {
    const int per_sm = Kp <= 12 ? 2 : 1;
    int pz = 0;
    const int grid = item_grid(L, (long long)per_sm * nsm, pz);
    const size_t smem = cheb3s_smem_bytes(Kp, var);
    const ChebStepT<float> none_cs{nullptr, nullptr};
    const Red none{};
    BURA_3S_SWITCH(Kp, var, launch_pdl(k_cheb_step3s<C, V, true>, dim3(grid), dim3(C, kPPts), smem, s, L, x,
                                       (const float*)nullptr, b, r, (float*)nullptr, none_cs, dsh, none, pz))
    return cudaGetLastError();
}

}  // namespace bura
