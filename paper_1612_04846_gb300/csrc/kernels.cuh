// Device kernels of the multi-shift multigrid-preconditioned CG (all k+1 shifted systems at once).
//
// Data layout ("interleaved k-vector"): a multi-shift vector holds, for every grid point P
// (lexicographic, x fastest), Kp consecutive values, one per shifted system (Kp = k+1 rounded up
// to a multiple of W = 16 bytes / sizeof(T)).  A thread owns one 16-byte chunk (W systems) of one
// point, so every load/store is a 128-bit vector access, a warp covers contiguous memory, and each
// stencil neighbour / face coefficient is fetched once for all systems of the point.
// Threads of a block form a (C = Kp/W) x PPB grid: threadIdx.x = chunk, threadIdx.y = point.
//
// Reductions (per system dot products) are deterministic: per-thread partials, a fixed-order
// block reduction in shared memory, per-block partials in global scratch and a fixed-order
// reduction by the last block to finish (threadfence + atomic ticket), which also applies the
// CG scalar updates for every system.  Accumulation is FP64 from the block level up; a thread's
// own partial is FP32 for FP32 data (at most a few tens of products) and FP64 for FP64 data.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>
#include <vector>

namespace bura {

constexpr int KMAXP = 16;  // largest padded number of systems per point

template <class T> struct VecT;
template <> struct VecT<double> { static constexpr int W = 2; using V = double2; using Acc = double; };
template <> struct VecT<float> { static constexpr int W = 4; using V = float4; using Acc = float; };

// Geometry and operator of one multigrid level (passed by value).
struct Lev {
    int nx, ny, nz;     // interior sizes (nz = 1 in 2D)
    long long N;        // nx*ny*nz
    long long plane;    // nx*ny
    double wx, wy, wz;  // constant-coefficient weights 1/(h^2 Lambda) per axis (wz = 0 in 2D)
    float wxf, wyf, wzf;  // the same rounded to FP32 (read by the FP32 kernels: no FP64 conversions)
    const void* fx;     // variable coefficients: face weights a/(h^2 Lambda), element type T (bf16 with cbf16)
    const void* fy;
    const void* fz;
    const void* dg;     // variable coefficients: the diagonal sum of a point's face weights, element type T
                        // (computed from the stored faces, so the operator stays consistent); null: summed
    int cbf16;          // 1: fx, fy, fz hold bfloat16 (FP32 kernels of the V-cycle levels only)
    // sparse operator (kernels instantiated with DIM = 0): row offsets, column indices and values of the
    // scaled matrix A, all entries of a row including its diagonal (which dg also holds), element type T
    const int* rowptr;
    const int* col;
    const void* val;
};

// Per-system CG state shared by the kernels (device memory).
struct Scal {
    double rz[KMAXP];     // r^T z of the current iteration
    double pq[KMAXP];     // p^T (A - dI) p
    double alpha[KMAXP];
    double beta[KMAXP];
    double rr[KMAXP];     // ||r||^2
    double thr[KMAXP];    // stop when rr <= thr
    double dsh[KMAXP];    // shifts d_j
    float alphaf[KMAXP];  // FP32 copies of alpha, beta and the shifts for the FP32 kernels (GB300's FP64
    float betaf[KMAXP];   // pipe is too slow for every thread of every launch to convert them)
    float dshf[KMAXP];
    int active[KMAXP];
    int iters[KMAXP];
    int nactive;
    int breakdown;
    unsigned int ticket;  // last-block ticket, reset by the last block
    int it;               // PCG iterations done in the current inner solve
    int max_it;           // cap on it (device-side loop control)
    int parity;           // which of the two direction buffers holds the current p
    int fault;            // set by a kernel whose bounded wait on its own copies gave up
    long long wait_cycles;  // SM clocks a TMA kernel waits for one stage of its ring before giving up
};

// Device-driven solve (the whole solve one captured graph): the per-plan constants of the refinement
// controller and the per-solve state it keeps (right-hand side and output addresses, tolerance, the
// FP64 thresholds and plan, the outcome).  Written by k_solve_params / the controller kernels only.
struct OuterCfg {
    double c[KMAXP], d[KMAXP];  // weights and shifts
    double lambda_lo;           // lower bound on lambda_min(A); 0: relative residual thresholds
    double inner_rtol;          // largest residual reduction asked of one FP32 inner solve
    long long wait_cycles;      // TMA ring wait budget of the inner solves (0: default)
    int K, max_outer, max_iters;
};
struct OuterState {
    const double* f;            // this solve's right-hand side (device)
    double tol;
    double fnorm2;
    double thr64[KMAXP];        // FP64 thresholds on ||r_j||^2
    double step[KMAXP];         // planned per-step residual reduction of each system
    double rr[KMAXP];           // latest FP64 ||r_j||^2
    int siters[KMAXP];          // iterations of each system over all inner solves
    int outer, total_it, status;  // refinement steps, PCG iterations, bura_status of the solve
    int done;                   // 1 once the controller has decided
};

// Chebyshev step coefficients of one level: d_m = c1 d_{m-1} + c2 Dinv res (c2 includes 1/(diag - d)
// for constant coefficients, where Dinv is a per-system scalar).
template <class C>
struct ChebStepT {
    const C* c1;  // [Kp] (null: c1 = 0)
    const C* c2;  // [Kp]
};

enum ReduceOp { RED_NONE = 0, RED_ALPHA = 1, RED_CONV = 2, RED_BETA = 3, RED_STORE = 4 };

// Grid reductions: every block writes its partial sums; on grids of up to kRedOneLevel blocks the last
// block to finish sums all block partials in block order.  Larger grids use two levels: blocks in groups
// of kRedGroup, the last block of a group sums the group's partials, and the last group to finish sums
// the group partials in group order.  Either way the order is fixed: results are deterministic.
constexpr int kRedGroup = 16;
constexpr int kRedOneLevel = 640;
constexpr int kRedFinBatch = 16;  // partials loaded at once per thread in the final step
struct Red {
    double* partial;          // [gridDim.x * Kp] block partials, then [groups * Kp] group partials
    unsigned int* tickets;    // [max groups + 1] counters, zero between reductions
    Scal* scal;
    double* out;              // RED_STORE destination [Kp]
    int op;
    unsigned long long cond;  // cudaGraphConditionalHandle of a captured PCG loop (0: none)
    int defer;                // 1: blocks only store their partials and block 0 the grid size in *nblk;
                              // a k_red_finish launched next on the stream sums them (no fences, no
                              // tickets, no serial tail in the producing grid)
    unsigned int* nblk;       // grid size of a deferred reduction's producer
};

// The final step of a deferred reduction: one CTA of kRedFinishThreads sums the producer's block
// partials in block order and applies op; launched right after the producer on the same stream.
constexpr int kRedFinishThreads = 256;
void launch_red_finish(const Red& red, int Kp, cudaStream_t s);

// One level of the single-CTA coarse V-cycle: its vectors live in the CTA's shared memory at the
// given byte offsets.  c1/c2 hold deg rows of Kp Chebyshev coefficients (global memory).
struct CoarseLevel {
    Lev L;
    unsigned int b, xa, xb, dd;  // shared-memory byte offsets
    unsigned int result;         // offset of the buffer holding this level's V-cycle result
    const void* c1;     // Chebyshev tables of the level, element type T
    const void* c2;
    unsigned int cofs;  // shared-memory byte offset of a copy of c1 then c2 (kNoCopy: read them from global)
    int deg;
};

// One level of the clustered coarse V-cycle (vectors in global memory, L2 resident).
struct ClusterLevel {
    Lev L;
    void* b;
    void* xa;
    void* xb;
    void* dd;
    const void* result;  // buffer holding this level's V-cycle result
    const void* c1;     // element type T
    const void* c2;
    int deg;
};

struct ClusterArgs {
    int nlev;
    int Kp;
    int exact;           // level solved with dense inverses (index in lev[]), -1: none
    const void* minv;
    const void* dsh;  // shifts, element type T
    ClusterLevel lev[16];
};
constexpr int kClusterThreads = 512;        // threads per CTA of the clustered coarse V-cycle
constexpr long long kClusterPoints = 16384; // levels with at most this many points run in the cluster

constexpr unsigned int kNoCopy = 0xffffffffu;
constexpr long long kExactPoints = 64;  // a coarse-CTA level this small is solved with dense inverses
// Most points per axis of the level solved exactly by fast diagonalization (2-D, constant coefficients):
// 63 in FP32 (measured on GB300: the 127^2 solve costs more than the two levels it replaces), 31 in FP64 (whose
// multiply-add rate on GB300 is a small fraction of FP32's).
#ifndef BURA_FDIAG_MAXN32
#define BURA_FDIAG_MAXN32 63
#endif
template <class T>
constexpr int kFdiagMaxN = sizeof(T) == 4 ? BURA_FDIAG_MAXN32 : 31;
constexpr int kMaxCoarseLevels = 16;
// Grid sweeps run CTAs of at most 256 threads; the register cap of 64 keeps 8 CTAs of 128 threads
// (or 4 of 256) resident per SM, so one wave covers the whole grid.
constexpr int kSweepThreads = 256;
constexpr int kSweepMinBlocks = 4;
constexpr int kCoarseThreads = 512;            // CTA size of the single-CTA coarse V-cycle
constexpr size_t kCoarseSmem = 200 * 1024;     // shared memory budget of that CTA's vectors
constexpr size_t kCoarseTables = 16 * 1024;    // and of its copies of the small Chebyshev tables
constexpr size_t kCoarseSmemMax = 227 * 1024;  // all of that CTA's dynamic shared memory
constexpr int kMaxDevices = 64;               // devices whose per-function launch limits are tracked
struct CoarseArgs {
    int nlev;
    int Kp;
    const void* dsh;  // shifts, element type T
    const void* b_in;  // right-hand side of the first coarse level (global)
    void* x_out;       // its V-cycle result (global)
    unsigned int smem_bytes;
    unsigned int dsh_ofs;  // shared-memory byte offset of a copy of the shifts (KMAXP doubles)
    int exact;             // level (index in lev[]) solved exactly by x = M_j b with dense inverses; -1: none
    const void* minv;      // M_j[(row * n + col) * Kp + j], n = points of that level (global, element type T)
    unsigned int minv_ofs; // shared-memory byte offset of the CTA's chunk of M, [row][col][W] (kNoCopy: read global)
    CoarseLevel lev[kMaxCoarseLevels];
};

struct Launch {
    int Kp, C, PPB, blocks;
};

// Prolongation and both post-smoothing steps of a 2-D constant-coefficient FP32 level as y-marching
// strips (strips.cu): items of 128 columns x SH rows, one CTA of Kp/4 x 132 threads per item.
struct StripGeo {
    int nx, ny, nxc, nyc, Kp;
    int SH;       // rows per item (even)
    int nstrips;  // strips across the level
    int items;    // strips x row segments
    float wx, wy;
};
StripGeo strip_geo(int nx, int ny, int nxc, int nyc, int Kp, float wx, float wy, int nsm);
size_t strip_smem_bytes(int Kp);
// Sets the strip kernel's dynamic shared-memory limit on the current device (a fixed size per Kp); called
// at plan setup, outside any stream capture.
cudaError_t strip_prepare(int Kp);
// x, b: the level's iterate and right-hand side; ec: the coarse correction ([nyc][nxc][Kp]); xout: the result
// (distinct from x and b); cs0 = (0, c2) of the first step, cs1 = (c1, c2) of the second; with red, b . xout.
cudaError_t launch_post2_strip(const StripGeo& g, int nsm, const float* x, const float* ec, const float* b, float* xout,
                               ChebStepT<float> cs0, ChebStepT<float> cs1, const float* dsh, const Red& red,
                               cudaStream_t s);

// The 3-D FP32 Chebyshev step with its inputs staged plane by plane in a shared-memory ring (sweep3d.cu);
// face weights in FP32 (not bf16).  cheb3s_prepare sets the kernel's shared-memory limit (plan setup).
#ifndef BURA_CHEB3S
#define BURA_CHEB3S 1
#endif
#ifndef BURA_CHEB3S_MIN_N
#define BURA_CHEB3S_MIN_N 127
#endif
constexpr bool kCheb3s = BURA_CHEB3S != 0;     // 3-D Chebyshev steps of levels >= kCheb3sMinN wide staged
constexpr int kCheb3sMinN = BURA_CHEB3S_MIN_N;  // in shared memory (else the z-marching grid sweep)
size_t cheb3s_smem_bytes(int Kp, bool var);
cudaError_t cheb3s_prepare(int Kp, bool var);
cudaError_t launch_cheb_step3s(const Lev& L, int Kp, bool var, int nsm, const float* xin, const float* din,
                               const float* b, float* xout, float* dout, ChebStepT<float> cs, const float* dsh,
                               const Red& red, cudaStream_t s);
// r = b - (A - d_j I) x with the same staging
cudaError_t launch_residual3s(const Lev& L, int Kp, bool var, int nsm, const float* x, const float* b, float* r,
                              const float* dsh, cudaStream_t s);

// Exact coarsest-level solve of a 2-D constant-coefficient operator by fast diagonalization (fdiag.cu):
// one thread-block cluster of G CTAs per shifted system; every array holds element type T.
struct FdiagArgs {
    int nx, ny, Kp;
    const void* b;     // right-hand sides, [ny][nx][Kp]
    void* x;           // solutions, [ny][nx][Kp]
    const void* simg;  // the orthonormal sine bases along x and y ([nx][nx], [ny][ny], symmetric) laid out
                       // as the kernel keeps them in shared memory (fdiag_image)
    const void* lx;    // eigenvalues of the x part of the level operator, [nx]
    const void* ly;    // and of the y part, [ny]
    const void* dsh;   // the shifts d_j, [Kp]
    Scal* scal;        // wait budget (wait_cycles) and fault flag
};
template <class T>
size_t fdiag_smem_bytes(int nx, int ny, int G);
// The shared-memory image of the two sine bases (given row-major in FP64), in T.
template <class T>
void fdiag_image(int nx, int ny, const double* sx, const double* sy, std::vector<T>& img);
// Largest cluster size G (16 .. 1, at most min(nx, ny)) with all nsys clusters resident at once (else the
// most CTAs resident), and its dynamic shared memory; sets the kernel's launch attributes.
template <class T>
cudaError_t fdiag_prepare(int nx, int ny, int nsys, int* G, size_t* smem);
template <class T>
cudaError_t fdiag_launch(const FdiagArgs& a, int G, size_t smem, int nsys, cudaStream_t s);

// ------------------------------------------------------------------ host launchers
template <class T>
struct Ops {
    static void broadcast(const Launch& g, const double* f, long long N, int K, T* r, T* x, T* p, cudaStream_t s,
                          const double* const* fp = nullptr);
    static void spmv_p(const Launch& g, const Lev& L, int dim, bool var, const T* z, T* pa, T* pb, T* q,
                       const Red& red, cudaStream_t s);
    static void cg_update(const Launch& g, long long N, T* x, T* r, const T* pa, const T* pb, const T* q,
                          const Red& red, cudaStream_t s);
    // the CG direction update and the operator apply of spmv_p as two sweeps (p = z + beta p; then
    // q = (A - dI) p with p.q): for operators whose stencil evaluation per neighbour is costly
    static void pupdate(const Launch& g, long long N, const T* z, T* pa, T* pb, const Red& red, cudaStream_t s);
    static void spmv_q(const Launch& g, const Lev& L, int dim, bool var, const T* pa, const T* pb, T* q, const Red& red,
                       cudaStream_t s);
    static void cheb_zero(const Launch& g, const Lev& L, int dim, bool var, const T* b, T* x, ChebStepT<T> cs,
                          const T* dsh, cudaStream_t s);
    static void cheb_step(const Launch& g, const Lev& L, int dim, bool var, const T* xin, const T* din, const T* b,
                          T* xout, T* dout, ChebStepT<T> cs, const T* dsh, const Red& red, cudaStream_t s);
    static void cheb_pre2(const Launch& g, const Lev& L, int dim, bool var, const T* b, T* xout, T* dout,
                          ChebStepT<T> cs0, ChebStepT<T> cs1, const T* dsh, cudaStream_t s);
    static void post_prolong(const Launch& g, const Lev& Lf, const Lev& Lc, int dim, bool var, const T* x,
                             const T* ec, const T* b, T* xout, T* dout, ChebStepT<T> cs, const T* dsh,
                             const Red& red, cudaStream_t s);
    static void restrict_res(const Launch& gc, const Lev& Lf, const Lev& Lc, int dim, bool var, const T* x,
                             const T* b, T* bc, const T* dsh, cudaStream_t s);
    static void prolong_add(const Launch& gf, const Lev& Lf, const Lev& Lc, int dim, const T* ec, T* x,
                            cudaStream_t s);
    // r = b - (A - dI) x, then bc = R r (full weighting): the residual restriction in two sweeps
    static void residual(const Launch& g, const Lev& L, int dim, bool var, const T* x, const T* b, T* r, const T* dsh,
                         cudaStream_t s);
    static void restrict_r(const Launch& gc, const Lev& Lf, const Lev& Lc, int dim, const T* r, T* bc, cudaStream_t s);
    static void coarse_cycle(const Launch& g1, int dim, bool var, const CoarseArgs& a, cudaStream_t s);
    static cudaError_t coarse_cluster(const Launch& g1, int csize, int dim, bool var, const ClusterArgs& a,
                                      cudaStream_t s);
    // Largest cluster size (16, 8, 4, 2 or 1) that the device can co-schedule for this kernel.
    static cudaError_t cluster_prepare(int dim, bool var, int threads, int want, int* csize);
    static cudaError_t prepare_coarse(int dim, bool var, size_t smem_bytes);
    static void apply_shifted(const Launch& g, const Lev& L, int dim, bool var, const T* x, T* y, const T* dsh,
                              cudaStream_t s);
    static void dot(const Launch& g, long long N, const T* a, const T* b, const Red& red, cudaStream_t s);
};

// Programmatic dependent launch: every kernel waits for its predecessor's completion (and memory
// flush) before touching dependent data, and lets its successor start launching early.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// FP64 refinement and output kernels.
// fp (optional): the address of a device pointer to the right-hand side, read by the kernel instead of f
// (a captured solve whose right-hand side changes from launch to launch)
void launch_residual64(const Launch& g, const Lev& L, int dim, bool var, const double* f, const double* v,
                       double* r, const Red& red, cudaStream_t s, const double* const* fp = nullptr);
void launch_cast_scaled(const Launch& g64, const Launch& g32, long long N, int K, const double* r64,
                        const double* scale, float* r32, float* x32, float* p32, cudaStream_t s);
void launch_correct64(const Launch& g64, const Launch& g32, long long N, int K, double* v, const float* e,
                      const double* scale, cudaStream_t s);
void launch_cast_f(const Launch& g32, long long N, int K, const double* f, const double* invscale, float* r32,
                   float* x32, float* p32, cudaStream_t s);
// u = sum_j c_j v_j (accumulate = 0) or u += sum_j c_j v_j (accumulate = 1), j = 0..K-1 in order.
void launch_weighted_sum(long long N, int Kp, int K, const double* v, const double* c, double* u, int accumulate,
                         cudaStream_t s);
void launch_norm2(long long N, const double* f, const Red& red, int nsm, cudaStream_t s,
                  const double* const* fp = nullptr);
void launch_gather_systems(long long N, int Kp, int K, const double* v, double* V, cudaStream_t s);
void launch_scatter_systems(long long N, int Kp, int K, const double* X, double* x, cudaStream_t s);
void launch_gather_systems_f(long long N, int Kp, int K, const float* v, double* V, cudaStream_t s);

// Device-side control of a captured solve (outer.cu).
void launch_solve_params(OuterState* st, const double* f, double tol, cudaStream_t s);
void launch_outer_begin(const OuterCfg* cfg, OuterState* st, const double* norm_partials, Scal* sc, double* scale,
                        double* invscale, unsigned long long cond_outer, unsigned long long cond_inner, int fp64,
                        cudaStream_t s);
void launch_outer_next(const OuterCfg* cfg, OuterState* st, const double* rr_partials, Scal* sc, double* scale,
                       double* invscale, unsigned long long cond_outer, cudaStream_t s);
void launch_outer_end_fp64(const OuterCfg* cfg, OuterState* st, const Scal* sc, cudaStream_t s);
void launch_cast_outer(const Launch& g64, const Launch& g32, long long N, int K, const OuterState* st,
                       const double* r64, const double* invscale, float* r32, float* x32, float* p32,
                       unsigned long long cond_inner, cudaStream_t s);

// Double-float refinement of the mixed path (kernels_df.cu).  DfOpHost holds device pointers and the
// hi/lo FP32 parts of the level-0 operator's coefficients.
struct DfOpHost {
    float w[3][2];                       // constant face weights (hi, lo)
    const float* ch = nullptr;           // diag - d_j (constant coefficients), Kp entries each
    const float* cl = nullptr;
    const float* dh = nullptr;           // d_j (variable coefficients)
    const float* dl = nullptr;
    const float* fh[3] = {nullptr, nullptr, nullptr};  // scaled face coefficients (variable coefficients)
    const float* fl[3] = {nullptr, nullptr, nullptr};
};
void launch_update_residual_df(const Launch& g, const Lev& L, int dim, bool var, const DfOpHost& h, const float* fh,
                               const float* fl, const float* vhin, const float* vlin, const float* x, float* vhout,
                               float* vlout, float* r32, float sf, const Red& red, cudaStream_t s);
void launch_cast_f_df(const Launch& g32, long long N, int K, const double* f, double sf, float* r32, float* x32,
                      float* p32, float* fh, float* fl, cudaStream_t s);
void launch_weighted_sum_df(long long N, int Kp, int K, const float* vh, const float* vl, const float* ch,
                            const float* cl, double* u, int accumulate, cudaStream_t s);
void launch_gather_df(long long N, int Kp, int K, const float* vh, const float* vl, double* V, cudaStream_t s);

}  // namespace bura
