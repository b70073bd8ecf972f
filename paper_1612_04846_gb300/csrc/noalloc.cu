// Allocation-free entry point: per-system FP64 residual norms ||f - (A - d_j I) v_j||^2.
//
// Some callers cannot call cudaMalloc at all: code running inside a CUDA-graph capture that must
// not allocate, allocators that forbid foreign device allocations (a caller-owned memory pool or
// arena), or real-time loops that must never enter the driver's allocator.  This entry point
// serves them: its only scratch (the per-block partial sums of the grid reduction and the
// last-block ticket) lives in a file-scope __device__ array of fixed size, so a call allocates
// nothing.  The caller still passes every input and output.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/bura.h"
#include "guard.h"

namespace {

constexpr int kBlocks = BURA_NOALLOC_MAX_BLOCKS;
constexpr int kSys = BURA_NOALLOC_MAX_SYSTEMS;
constexpr int kThreads = 256;

// The scratch: kBlocks * kSys partial sums followed by the ticket counter (one 8-byte slot).
// 1024 * 16 * 8 B + 256 B = 131,328 bytes, held by every device that loads the library until exit.
static __device__ __align__(256) double g_noalloc_scratch[kBlocks * kSys + 32];

struct Shifts {
    double d[kSys];
};

__global__ void __launch_bounds__(kThreads) k_resnorm_noalloc(int nx, int ny, int nz, double wx, double wy,
                                                              double wz, int nsys, Shifts sh,
                                                              const double* __restrict__ f,
                                                              const double* __restrict__ V, double* __restrict__ out,
                                                              double* __restrict__ scratch) {
    const long long N = (long long)nx * ny * nz;
    const long long plane = (long long)nx * ny;
    double acc[kSys];
    for (int s = 0; s < kSys; ++s) acc[s] = 0.0;
    const double diag = 2.0 * (wx + wy + wz);
    for (long long P = blockIdx.x * (long long)kThreads + threadIdx.x; P < N; P += (long long)gridDim.x * kThreads) {
        const int i = (int)(P % nx);
        const long long rem = P / nx;
        const int j = (int)(rem % ny);
        const int l = (int)(rem / ny);
        const double fv = f[P];
        for (int s = 0; s < nsys; ++s) {
            const double* v = V + (size_t)s * N;
            double y = (diag - sh.d[s]) * v[P];
            if (i > 0) y -= wx * v[P - 1];
            if (i < nx - 1) y -= wx * v[P + 1];
            if (j > 0) y -= wy * v[P - nx];
            if (j < ny - 1) y -= wy * v[P + nx];
            if (l > 0) y -= wz * v[P - plane];
            if (l < nz - 1) y -= wz * v[P + plane];
            const double r = fv - y;
            acc[s] = fma(r, r, acc[s]);
        }
    }
    // block reduction in a fixed order: warps by shuffles, then the warp sums by thread s
    __shared__ double wsum[kThreads / 32][kSys];
    __shared__ int am_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int s = 0; s < nsys; ++s) {
        double v = acc[s];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) wsum[warp][s] = v;
    }
    __syncthreads();
    if (threadIdx.x < nsys) {
        double t = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) t += wsum[w][threadIdx.x];
        scratch[(size_t)blockIdx.x * kSys + threadIdx.x] = t;
    }
    __threadfence();
    __syncthreads();
    unsigned int* ticket = reinterpret_cast<unsigned int*>(scratch + (size_t)kBlocks * kSys);
    if (threadIdx.x == 0) am_last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    if (threadIdx.x < nsys) {
        double t = 0.0;
        for (int b = 0; b < (int)gridDim.x; ++b) t += __ldcg(scratch + (size_t)b * kSys + threadIdx.x);
        out[threadIdx.x] = t;
    }
    if (threadIdx.x == 0) *ticket = 0u;
}

// Device address of the scratch array, looked up once per device (with that device current).
std::mutex g_mu;
void* g_addr[256] = {nullptr};

int scratch_address(int dev, double** out) {
    if (dev < 0 || dev >= 256) return BURA_ECUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        // the lookup may load the module on this device: not beside another thread's graph capture
        std::shared_lock<std::shared_mutex> guard(bura::capture_guard());
        void* ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return BURA_ECUDA;
        g_addr[dev] = ptr;
    }
    *out = reinterpret_cast<double*>(g_addr[dev]);
    return BURA_OK;
}

}  // namespace

extern "C" int bura_residual_norms_noalloc(const bura_grid* grid, int nsys, const double* d, const double* f,
                                           const double* V, double* rr, void* stream) {
    if (!grid || !d || !f || !V || !rr || nsys < 1) return BURA_EINVAL;
    if (nsys > kSys) return BURA_ERANGE;
    if ((grid->dim != 2 && grid->dim != 3) || grid->coef_kind != BURA_COEF_CONSTANT) return BURA_EINVAL;
    int n[3] = {grid->n[0], grid->n[1], grid->dim == 3 ? grid->n[2] : 1};
    for (int a = 0; a < grid->dim; ++a)
        if (n[a] < 1) return BURA_EINVAL;
    const long long N = (long long)n[0] * n[1] * n[2];
    if (N >= (1LL << 31)) return BURA_ERANGE;
    // Gershgorin scale of the constant-coefficient operator and the scaled weights 1/(h^2 Lambda)
    double lam = 0.0, w[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < grid->dim; ++a) {
        const double h = 1.0 / (n[a] + 1);
        lam += (2.0 + (n[a] - 1 < 2 ? n[a] - 1 : 2)) / (h * h);
    }
    for (int a = 0; a < grid->dim; ++a) {
        const double h = 1.0 / (n[a] + 1);
        w[a] = 1.0 / (h * h * lam);
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return BURA_ECUDA;
    double* scratch = nullptr;
    int rc = scratch_address(dev, &scratch);
    if (rc != BURA_OK) return rc;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // the ticket must start at zero (the partial sums are overwritten before they are read)
    if (cudaMemsetAsync(scratch + (size_t)kBlocks * kSys, 0, 32 * sizeof(double), s) != cudaSuccess)
        return BURA_ECUDA;
    Shifts sh;
    for (int j = 0; j < kSys; ++j) sh.d[j] = j < nsys ? d[j] : 0.0;
    long long blocks = (N + kThreads - 1) / kThreads;
    if (blocks > kBlocks) blocks = kBlocks;
    k_resnorm_noalloc<<<(int)blocks, kThreads, 0, s>>>(n[0], n[1], n[2], w[0], w[1], w[2], nsys, sh, f, V, rr, scratch);
    return cudaGetLastError() == cudaSuccess ? BURA_OK : BURA_ECUDA;
}
