// Exact solve of the coarsest multigrid level of a 2-D constant-coefficient operator by fast
// diagonalization.
//
// On an nx x ny grid with homogeneous Dirichlet boundaries the scaled level operator is the Kronecker
// sum A = T_x (+) T_y, T = w tridiag(-1, 2, -1) along each axis.  The orthonormal sine basis
// S_ik = sqrt(2/(n+1)) sin(pi (i+1)(k+1)/(n+1)) (symmetric, its own inverse) diagonalizes T with the
// eigenvalues w (2 - 2 cos(pi (k+1)/(n+1))), so with B the ny x nx array of b (row y = grid line y)
//     (A - d_j I)^{-1} b = S_y [ (S_y B S_x) ./ (lam_x[kx] + lam_y[ky] - d_j) ] S_x.
// That is the direct coarse-grid solve of the V-cycle, exact up to rounding, for every shifted system.
//
// One thread-block cluster per system j (the grid holds Kp clusters of G CTAs; padding systems have
// d = 0 and give finite values).  CTA g owns the rows [g ry, (g+1) ry) and the columns [g cx, (g+1) cx):
//   (A) its rows of B, read from global, times S_x -> R (its rows of B S_x);
//   (B) its columns of B S_x, gathered from the CTAs' R through distributed shared memory, times S_y
//       from the left, divided by the eigenvalue sums, times S_y again -> C (its columns of the result
//       before the last transform);
//   (C) its rows of that, gathered from the CTAs' C, times S_x -> the solution rows, stored to global.
// Each product runs from shared memory in register blocks of RM x RN outputs, summing over k in
// increasing order: 1 x 2 blocks for levels of up to 63 points per axis (enough blocks to keep every
// thread busy), 2 x 4 above (fewer shared-memory loads per multiply-add).  S_x and S_y reach shared memory as one bulk asynchronous copy of an image laid out
// on the host exactly as the CTA keeps them (issued before the wait for the previous kernel).
#include <cooperative_groups.h>

#include <mutex>

#include "kernels_impl.cuh"
#include "tma.cuh"

namespace cg = cooperative_groups;

namespace bura {

namespace {

constexpr int kFdThreads = 256;
constexpr int kFdSmallN = 63;  // most points per axis of the small block shape

__host__ __device__ constexpr int rup(int v, int m) { return (v + m - 1) / m * m; }

// Shared-memory layout of one CTA (element offsets).  The A operands of the products (rows read one
// element at a time, several rows per warp) have an odd leading dimension, which spreads the rows over
// the banks; the B operands (rows read as 16-byte vectors) have a leading dimension that is a multiple
// of 4.
template <int kRM>
struct FdLayout {
    int ry, cx;                     // rows and columns per CTA
    int ldsx, ldsy, ldr, ldc, ldb;  // leading dimensions of S_x, S_y, R, C / D, and the row slabs
    int osx, osy, obs, orr, occ, ocd, total;
    __host__ __device__ FdLayout(int nx, int ny, int G) {
        ry = (ny + G - 1) / G;
        cx = (nx + G - 1) / G;
        ldsx = rup(nx, 4);
        ldsy = rup(ny, 4) + 1;
        ldb = rup(nx, 4) + 1;
        ldr = nx;
        ldc = rup(cx, 4);
        // every array starts on a 4-element boundary (16-byte vectors of the B operands)
        osx = 0;
        osy = rup(osx + nx * ldsx, 4);
        obs = rup(osy + rup(ny, kRM) * ldsy, 4);
        orr = rup(obs + rup(ry, kRM) * ldb, 4);
        occ = rup(orr + ry * ldr, 4);
        ocd = rup(occ + ny * ldc, 4);
        total = ocd + ny * ldc;
    }
    // bytes of the S_x, S_y image (elements [osx, obs)), of all arrays, and the mbarrier's byte offset
    __host__ __device__ size_t image_bytes(size_t es) const { return (size_t)obs * es; }
    __host__ __device__ size_t bar_offset(size_t es) const { return ((size_t)total * es + 15) / 16 * 16; }
    __host__ __device__ size_t bytes(size_t es) const { return bar_offset(es) + 16; }
};

// One bulk asynchronous copy of `bytes` (a multiple of 16; both addresses 16-byte aligned) from global
// memory into this CTA's shared memory, completed on `bar`.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// Gather n elements: dst(i) = src(i) for i = tid, tid + nthr, ...; kGather loads are issued before
// their stores, so the latencies of global or distributed-shared-memory loads overlap.
constexpr int kGather = 8;
template <class T, class Src, class Dst>
__device__ __forceinline__ void gather(int n, Src&& src, Dst&& dst) {
    for (int i0 = threadIdx.x; i0 < n; i0 += kGather * blockDim.x) {
        T v[kGather];
#pragma unroll
        for (int u = 0; u < kGather; ++u) {
            const int i = i0 + u * blockDim.x;
            if (i < n) v[u] = src(i);
        }
#pragma unroll
        for (int u = 0; u < kGather; ++u) {
            const int i = i0 + u * blockDim.x;
            if (i < n) dst(i, v[u]);
        }
    }
}

// RN consecutive elements (RN = 2 or 4, the address aligned to RN elements).
template <class T, int RN>
__device__ __forceinline__ void ld_row(const T* p, T (&v)[RN]) {
    if constexpr (sizeof(T) == 4 && RN == 4) {
        const float4 q = *reinterpret_cast<const float4*>(p);
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    } else if constexpr (sizeof(T) == 4) {
        const float2 q = *reinterpret_cast<const float2*>(p);
        v[0] = q.x; v[1] = q.y;
    } else {
        for (int h = 0; h < RN; h += 2) {
            const double2 q = *reinterpret_cast<const double2*>(p + h);
            v[h] = q.x; v[h + 1] = q.y;
        }
    }
}

// out[m][n] = sum_k A[m][k] B[k][n] for m < M, n < N (k = 0 .. Kd-1 in order); A has rup(M, kRM) rows,
// B has at least rup(N, kRN) columns; epi(m0, n0, acc) stores a block (and checks m < M, n < N).
template <class T, int kRM, int kRN, class Epi>
__device__ __forceinline__ void smem_mm(const T* A, int lda, const T* B, int ldb, int M, int N, int Kd, Epi&& epi) {
    const int nbn = (N + kRN - 1) / kRN;
    const int nblk = ((M + kRM - 1) / kRM) * nbn;
    for (int blk = threadIdx.x; blk < nblk; blk += blockDim.x) {
        const int m0 = (blk / nbn) * kRM, n0 = (blk % nbn) * kRN;
        T acc[kRM][kRN];
        for (int i = 0; i < kRM; ++i)
            for (int j = 0; j < kRN; ++j) acc[i][j] = T(0);
        const T* a = A + (size_t)m0 * lda;
        const T* b = B + n0;
#pragma unroll 4
        for (int k = 0; k < Kd; ++k) {
            T av[kRM], bv[kRN];
            for (int i = 0; i < kRM; ++i) av[i] = a[i * lda + k];
            ld_row<T, kRN>(b + (size_t)k * ldb, bv);
            for (int i = 0; i < kRM; ++i)
                for (int j = 0; j < kRN; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
        }
        epi(m0, n0, acc);
    }
}

template <class T, int kRM, int kRN>
__global__ void __launch_bounds__(kFdThreads) k_fdiag(FdiagArgs a) {
    extern __shared__ __align__(16) unsigned char fsm[];
    T* sm = reinterpret_cast<T*>(fsm);
    cg::cluster_group cl = cg::this_cluster();
    const int G = (int)cl.num_blocks();
    const int g = (int)cl.block_rank();
    const int sys = blockIdx.x / G;
    const int nx = a.nx, ny = a.ny, Kp = a.Kp;
    const FdLayout<kRM> lay(nx, ny, G);
    T* SX = sm + lay.osx;
    T* SY = sm + lay.osy;
    T* Bs = sm + lay.obs;
    T* R = sm + lay.orr;
    T* Cc = sm + lay.occ;
    T* Cd = sm + lay.ocd;
    uint64_t* bar = reinterpret_cast<uint64_t*>(fsm + lay.bar_offset(sizeof(T)));
    // the transforms do not depend on the previous kernel: their copy starts before waiting for it
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        mbar_fence_init();
        mbar_expect_tx(bar, (unsigned)lay.image_bytes(sizeof(T)));
        bulk_load(SX, a.simg, (unsigned)lay.image_bytes(sizeof(T)), bar);
    }
    const int y0 = g * lay.ry, ry = max(0, min(ny, y0 + lay.ry) - y0);
    const int c0 = g * lay.cx, cx = max(0, min(nx, c0 + lay.cx) - c0);
    const T d = reinterpret_cast<const T*>(a.dsh)[sys];
    pdl_wait();
    {
        const T* b = reinterpret_cast<const T*>(a.b);
        gather<T>(
            ry * nx, [&](int i) { return b[((size_t)y0 * nx + i) * Kp + sys]; },
            [&](int i, T v) {
                const int r = i / nx;
                Bs[r * lay.ldb + i - r * nx] = v;
            });
    }
    __syncthreads();  // the barrier's initialisation is visible to every thread
    {
        const long long budget = a.scal->wait_cycles > 0 ? a.scal->wait_cycles : kTmaWaitCycles;
        if (!mbar_wait_bounded(bar, 0, budget)) {
            // the copy did not arrive in time: flag the solve, and let it land before going on
            (void)mbar_wait_bounded(bar, 0, kTmaWaitCycles);
            atomicExch(&a.scal->fault, 1);
        }
    }
    // (A) R = (rows of B) S_x
    smem_mm<T, kRM, kRN>(Bs, lay.ldb, SX, lay.ldsx, ry, nx, nx, [&](int m0, int n0, const T(&acc)[kRM][kRN]) {
        for (int i = 0; i < kRM; ++i)
            for (int j = 0; j < kRN; ++j)
                if (m0 + i < ry && n0 + j < nx) R[(m0 + i) * lay.ldr + n0 + j] = acc[i][j];
    });
    cl.sync();
    // (B) the slab's columns of B S_x from every CTA's R
    if (cx > 0)
        gather<T>(
            ny * cx,
            [&](int i) {
                const int y = i / cx, owner = y / lay.ry;
                const T* src = cl.map_shared_rank(R, owner);
                return src[(y - owner * lay.ry) * lay.ldr + c0 + i - y * cx];
            },
            [&](int i, T v) {
                const int y = i / cx;
                Cc[y * lay.ldc + i - y * cx] = v;
            });
    __syncthreads();
    const T* lx = reinterpret_cast<const T*>(a.lx);
    const T* ly = reinterpret_cast<const T*>(a.ly);
    smem_mm<T, kRM, kRN>(SY, lay.ldsy, Cc, lay.ldc, ny, cx, ny, [&](int m0, int n0, const T(&acc)[kRM][kRN]) {
        for (int i = 0; i < kRM; ++i)
            for (int j = 0; j < kRN; ++j)
                if (m0 + i < ny && n0 + j < cx)
                    Cd[(m0 + i) * lay.ldc + n0 + j] = acc[i][j] / ((lx[c0 + n0 + j] + ly[m0 + i]) - d);
    });
    __syncthreads();
    smem_mm<T, kRM, kRN>(SY, lay.ldsy, Cd, lay.ldc, ny, cx, ny, [&](int m0, int n0, const T(&acc)[kRM][kRN]) {
        for (int i = 0; i < kRM; ++i)
            for (int j = 0; j < kRN; ++j)
                if (m0 + i < ny && n0 + j < cx) Cc[(m0 + i) * lay.ldc + n0 + j] = acc[i][j];
    });
    cl.sync();
    // (C) this CTA's rows of the result before the last transform, from every CTA's columns
    gather<T>(
        ry * nx,
        [&](int i) {
            const int r = i / nx, kx = i - r * nx, owner = kx / lay.cx;
            const T* src = cl.map_shared_rank(Cc, owner);
            return src[(y0 + r) * lay.ldc + kx - owner * lay.cx];
        },
        [&](int i, T v) {
            const int r = i / nx;
            Bs[r * lay.ldb + i - r * nx] = v;
        });
    cl.sync();  // every remote read of this CTA's shared memory is done before any CTA exits
    T* xo = reinterpret_cast<T*>(a.x);
    smem_mm<T, kRM, kRN>(Bs, lay.ldb, SX, lay.ldsx, ry, nx, nx, [&](int m0, int n0, const T(&acc)[kRM][kRN]) {
        for (int i = 0; i < kRM; ++i)
            for (int j = 0; j < kRN; ++j)
                if (m0 + i < ry && n0 + j < nx) xo[((size_t)(y0 + m0 + i) * nx + n0 + j) * Kp + sys] = acc[i][j];
    });
    pdl_trigger();
}

}  // namespace

bool fdiag_small(int nx, int ny) { return nx <= kFdSmallN && ny <= kFdSmallN; }

template <class T>
size_t fdiag_smem_bytes(int nx, int ny, int G) {
    return fdiag_small(nx, ny) ? FdLayout<1>(nx, ny, G).bytes(sizeof(T)) : FdLayout<2>(nx, ny, G).bytes(sizeof(T));
}

// the kernel of a level size: 1 x 2 blocks for small levels, 2 x 4 for large
template <class T>
auto fdiag_kernel(int nx, int ny) {
    return fdiag_small(nx, ny) ? k_fdiag<T, 1, 2> : k_fdiag<T, 2, 4>;
}

template <class T>
void fdiag_image(int nx, int ny, const double* sx, const double* sy, std::vector<T>& img) {
    // the positions of S_x and S_y do not depend on the block shape; the image's length (through the
    // last padding row of S_y) does
    const FdLayout<2> lay(nx, ny, 1);
    img.assign((size_t)(fdiag_small(nx, ny) ? FdLayout<1>(nx, ny, 1).obs : lay.obs), T(0));
    for (int i = 0; i < nx; ++i)
        for (int k = 0; k < nx; ++k) img[(size_t)lay.osx + (size_t)i * lay.ldsx + k] = (T)sx[(size_t)i * nx + k];
    for (int i = 0; i < ny; ++i)
        for (int k = 0; k < ny; ++k) img[(size_t)lay.osy + (size_t)i * lay.ldsy + k] = (T)sy[(size_t)i * ny + k];
}

// The dynamic shared-memory limit of a kernel variant on the current device is only ever raised: a
// captured graph of an earlier plan launches with its own (larger) size, and lowering the limit under
// it would make those launches fail.
template <class K>
cudaError_t raise_smem_limit(K fn, int variant, int bytes) {
    static std::mutex m;
    static int limit[4][kMaxDevices] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(m);
    if (bytes <= limit[variant][dev]) return cudaSuccess;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) limit[variant][dev] = bytes;
    return e;
}

template <class T>
cudaError_t fdiag_prepare(int nx, int ny, int nsys, int* G, size_t* smem) {
    auto fn = fdiag_kernel<T>(nx, ny);
    const int variant = (sizeof(T) == 8 ? 2 : 0) + (fdiag_small(nx, ny) ? 0 : 1);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    *G = 0;
    *smem = 0;
    int best = 0, bestG = 0;
    for (int c = 16; c >= 1; c /= 2) {
        if (c > nx || c > ny) continue;
        const size_t bytes = fdiag_smem_bytes<T>(nx, ny, c);
        if (bytes > 227 * 1024) continue;
        e = raise_smem_limit(fn, variant, (int)bytes);
        if (e != cudaSuccess) return e;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(c);
        cfg.blockDim = dim3(kFdThreads);
        cfg.dynamicSmemBytes = bytes;
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
        if (n >= nsys) { bestG = c; break; }  // the largest cluster with every system resident at once
        if (n * c > best) { best = n * c; bestG = c; }
    }
    if (bestG == 0) return cudaErrorInvalidConfiguration;
    *G = bestG;
    *smem = fdiag_smem_bytes<T>(nx, ny, bestG);
    return raise_smem_limit(fn, variant, (int)*smem);
}

template <class T>
cudaError_t fdiag_launch(const FdiagArgs& a, int G, size_t smem, int nsys, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nsys * G);
    cfg.blockDim = dim3(kFdThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = G;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    return cudaLaunchKernelEx(&cfg, fdiag_kernel<T>(a.nx, a.ny), a);
}

template size_t fdiag_smem_bytes<float>(int, int, int);
template size_t fdiag_smem_bytes<double>(int, int, int);
template void fdiag_image<float>(int, int, const double*, const double*, std::vector<float>&);
template void fdiag_image<double>(int, int, const double*, const double*, std::vector<double>&);
template cudaError_t fdiag_prepare<float>(int, int, int, int*, size_t*);
template cudaError_t fdiag_prepare<double>(int, int, int, int*, size_t*);
template cudaError_t fdiag_launch<float>(const FdiagArgs&, int, size_t, int, cudaStream_t);
template cudaError_t fdiag_launch<double>(const FdiagArgs&, int, size_t, int, cudaStream_t);

}  // namespace bura
