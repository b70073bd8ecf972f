// FP64 instantiation of the multi-shift MG-PCG kernels, plus the FP64 reduction and output kernels
// (norm of f, weighted sum, gather / scatter of the systems).
#include <cstddef>

#include "kernels_impl.cuh"

namespace bura {
template struct Ops<double>;

// ||f||^2 of a plain FP64 vector (red.out[0]); threads laid out as (1, 256) with two lanes of which
// the second stays zero, so the shared reduction machinery applies unchanged.
__global__ void k_norm2(int N, const double* __restrict__ f, Red red) {
    Accum<double> acc;
    for (int P = blockIdx.x * blockDim.y + threadIdx.y; P < N; P += gridDim.x * blockDim.y) {
        const double a[2] = {f[P], 0.0};
        acc.add(a, a);
    }
    reduce_finish<double>(acc, red, 2);
}

void launch_norm2(long long N, const double* f, const Red& red, int nsm, cudaStream_t s) {
    long long b = (N + 255) / 256;
    const int blocks = (int)(b < nsm * 8 ? (b > 0 ? b : 1) : nsm * 8);
    k_norm2<<<blocks, dim3(1, 256), 256 * 2 * sizeof(double), s>>>((int)N, f, red);
}

// u = sum_j c_j v_j (FP64, fixed order j = 0..K-1); one thread per point.
__global__ void k_weighted_sum(int N, int Kp, int K, const double* __restrict__ v, const double* __restrict__ c,
                               double* __restrict__ u) {
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
        u[P] = s;
    }
}

static int grid1(long long N, int bs) {
    long long b = (N + bs - 1) / bs;
    return (int)(b < 152 * 16 ? (b > 0 ? b : 1) : 152 * 16);
}

void launch_weighted_sum(long long N, int Kp, int K, const double* v, const double* c, double* u, cudaStream_t s) {
    k_weighted_sum<<<grid1(N, 256), 256, 0, s>>>((int)N, Kp, K, v, c, u);
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
