// Internal definitions shared by the CUDA translation units of the random-walker library.
// Nothing here is part of the C ABI (include/rw.h).
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/rw.h"

#define RW_CHECK_CUDA(call)                                                     \
  do {                                                                          \
    cudaError_t e_ = (call);                                                    \
    if (e_ != cudaSuccess) {                                                    \
      rw_set_last_cuda_error(e_, #call, __FILE__, __LINE__);                    \
      return (e_ == cudaErrorMemoryAllocation) ? RW_ERR_OOM : RW_ERR_CUDA;      \
    }                                                                           \
  } while (0)

#define RW_TRY(expr)                        \
  do {                                      \
    rw_status s_ = (expr);                  \
    if (s_ < 0) return s_;                  \
  } while (0)

void rw_count_launch();
#define RW_LAUNCH_CHECK()  \
  do {                     \
    rw_count_launch();     \
    RW_CHECK_CUDA(cudaGetLastError()); \
  } while (0)

void rw_set_last_cuda_error(cudaError_t e, const char* what, const char* file, int line);

// Programmatic dependent launch.  A kernel launched with RW_LAUNCH may be scheduled while its
// predecessor in the stream is still running: it must call rw_grid_wait() before it reads
// anything an earlier kernel writes (the wait returns once the predecessor has completed and
// its memory is visible; it returns at once for a kernel launched without the attribute).
// rw_grid_trigger() lets the successor begin launching; it orders nothing.
__device__ __forceinline__ void rw_grid_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void rw_grid_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
static inline cudaError_t rw_launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block,
                                        size_t smem, cudaStream_t st, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}
#define RW_LAUNCH(kernel, grid, block, smem, st, ...)                                  \
  do {                                                                                 \
    RW_CHECK_CUDA(rw_launch_pdl(kernel, dim3(grid), dim3(block), smem, st, __VA_ARGS__)); \
    rw_count_launch();                                                                 \
  } while (0)
void rw_set_error_message(const char* msg);

// Device status word bits (ORed by kernels, read by the host).
enum : int {
  RW_DEV_BAD_SEED = 1,       // seed index out of range or label out of range
  RW_DEV_DUP_SEED = 2,       // two seeds on one voxel
  RW_DEV_ISOLATED = 4,       // degree 0 with the normalized Laplacian
  RW_DEV_SINGULAR = 8,       // zero pivot in a small dense factorization
  RW_DEV_EMPTY_LABEL = 16,   // a label without seeds (Gaussian priors need one)
  RW_DEV_NONFINITE = 32,     // NaN / Inf in an input
  RW_DEV_TIMEOUT = 64        // a bounded wait on an asynchronous copy gave up
};
rw_status rw_status_from_device_bits(int bits);

// A growable device buffer owned by a handle.  grow() may reallocate (synchronous).
struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
  rw_status grow(size_t bytes);
  void release();
  template <class T> T* as() const { return reinterpret_cast<T*>(p); }
};

struct PinnedBuf {
  void* p = nullptr;
  size_t cap = 0;
  rw_status grow(size_t bytes);
  void release();
  template <class T> T* as() const { return reinterpret_cast<T*>(p); }
};

enum { RW_GRAPH_GRID = 0, RW_GRAPH_CSR = 1 };

struct SolveWorkspace {
  DevBuf seedlab;   // int [N]: -1 unseeded, else label
  DevBuf seedpart;  // seed-side sums: fit (FP64) and per-block label sums
  bool seeds_clean = false;  // seedlab is all -1 (the last solve's final kernel cleared it)
  int seed_nsb = 0;          // scatter blocks of the last seed scatter (the priors fit reads them)
  DevBuf small;     // small per-solve arrays (stats, Q_s, X, products, Z, C, ...)
  DevBuf xhat[2];   // refinement iterates, N x lpad FP32
  DevBuf phat;      // hat-space priors, N x lpad FP32
  DevBuf pcg;       // PCG vectors
  DevBuf stage;     // device staging of the host-buffer entry point
  DevBuf grad;      // fast-path gradient scratch (grown on first use)
  DevBuf reg;       // unseeded (registration) solve: one label chunk of U, N x lpad FP32
  PinnedBuf host;   // info readback
  cudaEvent_t ev[8] = {};  // phase timing events (created on first use)
  int64_t small_cap_S = 0, small_cap_m = 0;
};

struct rw_graph {
  int kind = RW_GRAPH_GRID;
  int ndim = 2;
  int dims[3] = {1, 1, 1};
  int64_t N = 0;
  int64_t stride[3] = {1, 1, 1};
  double beta = 0.0;
  int form = RW_WEIGHT_SQ;
  int normalized = 1;
  // grid graphs: per-axis forward-edge arrays, entry axis*N + i
  float* J = nullptr;    // N intensities
  float* w = nullptr;    // ndim*N weights
  float* cw = nullptr;   // ndim*N operator coefficients: w * s_a * s_b (normalized) or w
  // csr graphs (aggregates): symmetric, no diagonal
  int32_t* rowptr = nullptr;
  int32_t* col = nullptr;
  float* wcsr = nullptr;  // weights
  float* ccsr = nullptr;  // operator coefficients
  int64_t nnz = 0;
  // per-node
  float* d = nullptr;     // degree
  float* s = nullptr;     // d^{-1/2} (normalized) or 1
  float* sq = nullptr;    // d^{1/2} (normalized) or 1
  int* status = nullptr;  // device status word
  double dsum = 0.0;      // sum of degrees (1^T D 1)
  int device = 0;         // CUDA device current when the handle was built
  SolveWorkspace ws;
  DevBuf upd;             // update scratch
};

struct rw_basis {
  int64_t N = 0;
  int m = 0;
  int ld32 = 0;           // row pitch of Q32 (multiple of 4)
  int ld16 = 0;           // row pitch of the 16-bit copies (multiple of 8)
  float* Q32 = nullptr;   // N x ld32
  __half* Q16 = nullptr;  // N x ld16, scaled by qscale (power of two), panel-major: column
                          // 8c + v of row i at ((c N + i) 8 + v)
  __nv_bfloat16* Qbf = nullptr;  // same layout, unscaled, built on first use
  float qscale = 1.f;
  double* lam = nullptr;  // m values on the device
  double* lam_host = nullptr;
  const rw_graph* owner = nullptr;
};

// ---- helpers shared across translation units -----------------------------------------
static inline int64_t rw_round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }
static inline unsigned rw_blocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }
static inline cudaStream_t rw_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

extern int g_rw_num_sms;
rw_status rw_device_init();

// graph.cu
rw_status rw_stencil_apply(const rw_graph* g, const float* X, int64_t ldx, float* Y,
                           int64_t ldy, int k, float alpha, float beta, const float* Z,
                           int64_t ldz, float gamma, cudaStream_t st);
rw_status rw_graph_coeffs(rw_graph* g, cudaStream_t st);
rw_status rw_graph_degree_sum(rw_graph* g, cudaStream_t st);  // sets g->dsum, synchronizes
rw_status rw_graph_reserve_scratch(rw_graph* g);
// every edge weight from an ndim x N edge-id array; degrees, scalings, coefficients (syncs)
rw_status rw_set_all_weights(rw_graph* g, const float* w_dev, cudaStream_t st);

// dense.cu (small / tall-skinny dense helpers)
// G (p x q, row-major, ldg, FP64) = (accumulate ? G : 0) + A^T B, A: N x p (lda), B: N x q (ldb)
rw_status rw_gram(const float* A, int64_t lda, const float* B, int64_t ldb, int64_t N, int p,
                  int q, double* G, int ldg, bool accumulate, cudaStream_t st);
// gram_tc.cu: the same G = (accumulate ? G : 0) + A^T B on the tensor cores (TF32 x 3 split,
// FP32 over 1024-row slices, FP64 over slices); scratch of rw_gram_tc_scratch_bytes(N, p, q)
// bytes, 256-byte aligned; status: device status word (RW_DEV_TIMEOUT on a failed wait)
size_t rw_gram_tc_scratch_bytes(int64_t N, int p, int q);
rw_status rw_gram_tc(const float* A, int64_t lda, const float* B, int64_t ldb, int64_t N, int p,
                     int q, double* G, int ldg, bool accumulate, void* scratch, int* status,
                     cudaStream_t st);
// Y (N x p) = alpha * A (N x q) * C (q x p, row-major FP32, ldc) + beta * Y
rw_status rw_gemm_tall(const float* A, int64_t lda, const float* C, int ldc, int64_t N, int q,
                       int p, float alpha, float beta, float* Y, int64_t ldy, cudaStream_t st);
// in place: A (n x n, row-major FP64) := upper-triangular R with R^T R = A + shift*I; returns
// via flag device word when a pivot is not positive
rw_status rw_cholesky_upper(double* A, int n, double shift, int* flag, cudaStream_t st);
// Rinv (n x n FP32 row-major) = inverse of the upper-triangular R (FP64)
rw_status rw_tri_inverse_upper(const double* R, int n, float* Rinv, cudaStream_t st);
// symmetric eigensolver (cyclic Jacobi, FP64): A (n x n) destroyed; w ascending; V columns
rw_status rw_sym_eig(double* A, int n, double* w, double* V, double* work, cudaStream_t st);
size_t rw_sym_eig_work_bytes(int n);
rw_status rw_copy_cols(const float* src, int64_t lds, float* dst, int64_t ldd, int64_t N,
                       const int* cols, int ncols, cudaStream_t st);
rw_status rw_f64_to_f32(const double* a, float* b, int64_t n, cudaStream_t st);

// Tensor-core passes over the 16-bit basis copy (csrc/proj_tc.cu).  rw_project_tc writes the
// projection partials scaled by kTcProjScale; both take nchunk_max <= 32, lp <= 32.
constexpr float kTcProjScale = 4096.f;
template <typename T>
rw_status rw_project_tc(const T* Qp, int64_t N, int nchunk_max, const float* phat, int lp,
                        const int* seedlab, const int* mdev, float* part, int nblk, int* status,
                        cudaStream_t st);
template <typename T>
rw_status rw_backproject_tc(const T* Qp, int64_t N, int nchunk_max, const float* C, int lp,
                            float cscale, const int* seedlab, const float* sq, const float* s,
                            int L, const int* mdev, float* xhat, float* U, uint8_t* labels,
                            int* clear, const float* nul, int* status, int nblk, cudaStream_t st);
// whether a basis pass (which = 1: projection, 2: back-projection) of a 16-bit copy with row
// pitch ld16 carrying lp padded labels runs on the tensor cores
bool rw_tc_passes(int ld16, int which, int lp);

// Seed bookkeeping shared by the fast solve, the PCG solve and the gradients: resets the label
// array when needed, scatters the seeds (per-block label statistics) and, unless deferred,
// launches the priors kernel; launch_priors launches it later (early = 1: other kernels were
// launched in between, see k_priors).
rw_status rw_solve_priors_internal(const rw_graph* g, const int32_t* seed_idx,
                                   const int32_t* seed_lab, int S, int L, int prior_mode,
                                   const float* priors, int lp, cudaStream_t st, float** phat_out,
                                   int** seedlab_out, double** fit64_out,
                                   bool defer_priors = false);
rw_status launch_priors(const rw_graph* g, int L, int prior_mode, const float* priors, int lp,
                        int early, cudaStream_t st);

// eig.cu: a basis handle from N x m columns X (pitch ldx, device) and m host values (syncs)
rw_status rw_make_basis(const rw_graph* g, int m, const float* X, int64_t ldx,
                        const double* lam_h, cudaStream_t st, rw_basis** out);

// update.cu: edge-sum Rayleigh quotients of every basis column under g -> b->lam (synchronizes)
rw_status rw_basis_rayleigh(const rw_graph* g, rw_basis* b, cudaStream_t st);
