// Offline precomputation (Sec. II-B, Eq. L_eigs): the m smallest eigenpairs of L-hat (or L),
// and the basis handle used online.
//
// The paper names no eigensolver.  This is a block solver with two kinds of outer step on the
// block X (m + guard columns):
// * a Chebyshev-filtered subspace step: X <- p(Op) X, p the scaled Chebyshev polynomial that
//   damps the spectrum above the block's largest Ritz value, then Cholesky-QR and an nb x nb
//   Rayleigh-Ritz;
// * an LOBPCG step on the basis [X | W | P]: W the residuals of the columns not yet converged
//   (soft locking), P the previous update directions, [W P] orthogonalized against X (block
//   Gram-Schmidt, two passes) and orthonormalized by shifted Cholesky-QR (two passes, FP64
//   Cholesky); the projected matrix S^T (Op S) is formed in FP64 and diagonalized by the FP64
//   Jacobi solver.
// Filtered steps run while they keep reducing the worst residual of the wanted columns (by at
// least 30% per step); LOBPCG steps take over when they stall.  In FP32-storage experiments
// (512^2 and 256^2 four-region images) the filtered steps alone reached 1e-5 in about a dozen
// steps, with nb x nb Rayleigh-Ritz problems instead of up to 3nb x 3nb ones; LOBPCG with the
// polynomial as a preconditioner of W (indefinite on the damped interval) stagnated near 1e-2.
// Bulk work (stencil, Gram, tall GEMMs) runs in FP32 on node-major N x k blocks.
#include "rw_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

namespace {

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ULL;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ULL;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBULL;
  return x ^ (x >> 31);
}

__global__ void k_random_block(float* X, int64_t ldx, int64_t N, int k, uint64_t seed) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * k) return;
  int64_t i = e / k;
  int j = (int)(e % k);
  uint64_t h = splitmix64(seed ^ splitmix64((uint64_t)e));
  X[i * ldx + j] = (float)((double)(h >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0);
}

__global__ void k_residual(const float* __restrict__ AX, const float* __restrict__ X, int64_t ld,
                           const float* __restrict__ lam, int64_t N, int k, float* __restrict__ R,
                           int64_t ldr) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * k) return;
  int64_t i = e / k;
  int j = (int)(e % k);
  R[i * ldr + j] = AX[i * ld + j] - lam[j] * X[i * ld + j];
}

__global__ void k_colnorms(const float* __restrict__ A, int64_t lda, int64_t N, int k,
                           int64_t rows_per_block, double* __restrict__ out) {
  int c = threadIdx.x + blockIdx.y * blockDim.x;
  if (c >= k) return;
  int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
  int64_t r1 = min(N, r0 + rows_per_block);
  float acc = 0.f;
  for (int64_t i = r0; i < r1; ++i) {
    float v = A[i * lda + c];
    acc = fmaf(v, v, acc);
  }
  atomicAdd(&out[c], (double)acc);
}

__global__ void k_scale_cols(float* __restrict__ Y, int64_t ld, int64_t N, int k,
                             const float* __restrict__ sc) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * k) return;
  int64_t i = e / k;
  int j = (int)(e % k);
  Y[i * ld + j] *= sc[j];
}

__global__ void k_symmetrize(double* H, int n) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * n) return;
  int i = (int)(e / n), j = (int)(e % n);
  if (j > i) {
    double a = 0.5 * (H[(int64_t)i * n + j] + H[(int64_t)j * n + i]);
    H[(int64_t)i * n + j] = a;
    H[(int64_t)j * n + i] = a;
  }
}

// C (n x k, FP32 row-major) = V[:, 0:k] with rows < zero_rows set to 0
__global__ void k_take_cols(const double* __restrict__ V, int n, int k, int zero_rows,
                            float* __restrict__ C) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * k) return;
  int i = (int)(e / k), j = (int)(e % k);
  C[e] = (i < zero_rows) ? 0.f : (float)V[(int64_t)i * n + j];
}

__global__ void k_to_basis(const float* __restrict__ X, int64_t ldx, int64_t N, int m,
                           float* __restrict__ Q32, int ld32, __half* __restrict__ Q16, int ld16,
                           float qscale) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * ld16) return;
  int64_t i = e / ld16;
  int c = (int)(e % ld16);
  float v = (c < m) ? X[i * ldx + c] : 0.f;
  if (c < ld32) Q32[i * ld32 + c] = v;
  Q16[((int64_t)(c / 8) * N + i) * 8 + (c % 8)] = __float2half_rn(v * qscale);  // panel-major
}

__global__ void k_maxf(const float* __restrict__ v, int64_t n, unsigned int* out) {
  float m = 0.f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    m = fmaxf(m, v[i]);
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffff, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));  // m >= 0
}

struct Work {
  cudaStream_t st;
  const rw_graph* g;
  int64_t N;
  DevBuf S, AS, T, Pb, small, gsc;   // gsc: scratch of the tensor-core Gram
  int ldS;
  double *H, *V, *w, *eigw, *G, *cn;
  float *C32, *Rinv, *lam32;
  int* flag;
  int* cols;
};

bool trace_on();
void trace_block(Work& W, const char* what, const float* A, int64_t lda, int k);
void trace_small(Work& W, const char* what, const double* M, int n);

// Gram of two N-row blocks: tensor cores (rw_gram_tc) for the eigensolver's projected
// matrices; its scratch grows once to the largest shape met
rw_status gram_into(Work& W, const float* A, int64_t lda, const float* B, int64_t ldb, int p,
                    int q, double* G) {
  RW_TRY(W.gsc.grow(rw_gram_tc_scratch_bytes(W.N, p, q)));
  return rw_gram_tc(A, lda, B, ldb, W.N, p, q, G, q, false, W.gsc.p, W.g->status, W.st);
}

rw_status colnorms(Work& W, const float* A, int64_t lda, int k, std::vector<double>& out);

// [Y] (k columns at Y, pitch ld) := orthonormal basis of its span.  The columns are first
// scaled to unit norm (the blocks mix residuals of very different sizes); then two passes of
// shifted Cholesky-QR.  Any shift keeps the span (R is invertible); the first (1e-5 on a unit
// diagonal, raised 100x and retried if a pivot still fails) is far above the rounding error of
// a Gram matrix of FP32 columns, and the second pass restores orthonormality to working
// precision.  Columns must be nonzero.
rw_status cholqr(Work& W, float* Y, int64_t ld, int k) {
  if (k <= 0) return RW_OK;
  {
    std::vector<double> nrm;
    RW_TRY(colnorms(W, Y, ld, k, nrm));
    std::vector<float> sc(k);
    for (int j = 0; j < k; ++j) sc[j] = nrm[j] > 0 ? (float)(1.0 / nrm[j]) : 0.f;
    RW_CHECK_CUDA(cudaMemcpyAsync(W.lam32 + W.ldS, sc.data(), sizeof(float) * k,
                                  cudaMemcpyHostToDevice, W.st));
    k_scale_cols<<<rw_blocks(W.N * k, 256), 256, 0, W.st>>>(Y, ld, W.N, k, W.lam32 + W.ldS);
    RW_LAUNCH_CHECK();
  }
  for (int pass = 0; pass < 2; ++pass) {
    double shift = pass == 0 ? 1e-5 : 1e-11;
    for (int attempt = 0;; ++attempt) {
      RW_TRY(gram_into(W, Y, ld, Y, ld, k, k, W.G));
      trace_small(W, "cholqr gram", W.G, k);
      RW_CHECK_CUDA(cudaMemsetAsync(W.flag, 0, sizeof(int), W.st));
      RW_TRY(rw_cholesky_upper(W.G, k, shift, W.flag, W.st));
      int bad = 0;
      RW_CHECK_CUDA(cudaMemcpyAsync(&bad, W.flag, sizeof(int), cudaMemcpyDeviceToHost, W.st));
      RW_CHECK_CUDA(cudaStreamSynchronize(W.st));
      if (!bad) break;
      if (attempt == 3) return RW_ERR_SINGULAR;
      shift *= 100.0;
    }
    trace_small(W, "cholqr R", W.G, k);
    RW_TRY(rw_tri_inverse_upper(W.G, k, W.Rinv, W.st));
    float* tmp = W.T.as<float>();
    RW_TRY(rw_gemm_tall(Y, ld, W.Rinv, k, W.N, k, k, 1.f, 0.f, tmp, W.ldS, W.st));
    RW_CHECK_CUDA(cudaMemcpy2DAsync(Y, sizeof(float) * ld, tmp, sizeof(float) * W.ldS,
                                    sizeof(float) * k, W.N, cudaMemcpyDeviceToDevice, W.st));
  }
  return RW_OK;
}

// Y (k cols) -= X (p cols) (X^T Y), twice
rw_status orth_against(Work& W, const float* X, int64_t ldx, int p, float* Y, int64_t ldy, int k) {
  if (k <= 0 || p <= 0) return RW_OK;
  for (int pass = 0; pass < 2; ++pass) {
    RW_TRY(gram_into(W, X, ldx, Y, ldy, p, k, W.G));
    RW_TRY(rw_f64_to_f32(W.G, W.Rinv, (int64_t)p * k, W.st));
    RW_TRY(rw_gemm_tall(X, ldx, W.Rinv, k, W.N, p, k, -1.f, 1.f, Y, ldy, W.st));
  }
  return RW_OK;
}

// scaled Chebyshev filter (degree deg) of the k columns at Y, damping [a, b]; a0 ~ lowest
// eigenvalue.  Uses two temporaries inside T.  Result left in Y.
rw_status cheb_filter(Work& W, float* Y, int64_t ld, int k, int deg, double a0, double a,
                      double b, int* applies) {
  if (deg <= 0 || k <= 0 || !(b > a) || !(a > a0)) return RW_OK;
  const double e = (b - a) / 2, c = (b + a) / 2;
  double sigma = e / (a0 - c);
  const double sigma1 = sigma;
  float* bufs[3] = {Y, W.T.as<float>(), W.T.as<float>() + W.ldS / 2};
  // T is N x ldS with ldS >= 2k: two k-wide slots (columns [0,k) and [ldS/2, ldS/2 + k))
  int64_t lds[3] = {ld, W.ldS, W.ldS};
  // Y1 = (sigma1 / e) (Op Y0 - c Y0)
  RW_TRY(rw_stencil_apply(W.g, bufs[0], lds[0], bufs[1], lds[1], k, (float)(sigma1 / e),
                          (float)(-sigma1 * c / e), nullptr, 0, 0.f, W.st));
  ++*applies;
  int i0 = 0, i1 = 1, i2 = 2;
  for (int it = 2; it <= deg; ++it) {
    double sigma2 = 1.0 / (2.0 / sigma1 - sigma);
    // Y2 = (2 sigma2 / e)(Op Y1 - c Y1) - sigma sigma2 Y0
    RW_TRY(rw_stencil_apply(W.g, bufs[i1], lds[i1], bufs[i2], lds[i2], k, (float)(2 * sigma2 / e),
                            (float)(-2 * sigma2 * c / e), bufs[i0], lds[i0],
                            (float)(-sigma * sigma2), W.st));
    ++*applies;
    sigma = sigma2;
    int t = i0; i0 = i1; i1 = i2; i2 = t;
  }
  if (bufs[i1] != Y)
    RW_CHECK_CUDA(cudaMemcpy2DAsync(Y, sizeof(float) * ld, bufs[i1], sizeof(float) * lds[i1],
                                    sizeof(float) * k, W.N, cudaMemcpyDeviceToDevice, W.st));
  return RW_OK;
}

rw_status colnorms(Work& W, const float* A, int64_t lda, int k, std::vector<double>& out);

// opt-in diagnostics (environment variable RW_TRACE_EIG): per-step column-norm ranges
bool trace_on() {
  static int on = -1;
  if (on < 0) on = getenv("RW_TRACE_EIG") ? 1 : 0;
  return on == 1;
}

void trace_block(Work& W, const char* what, const float* A, int64_t lda, int k) {
  if (!trace_on() || k <= 0) return;
  std::vector<double> v;
  if (colnorms(W, A, lda, k, v) != RW_OK) return;
  double lo = 1e300, hi = 0.0;
  int bad = -1;
  for (int j = 0; j < k; ++j) {
    if (!std::isfinite(v[j]) && bad < 0) bad = j;
    lo = std::min(lo, v[j]);
    hi = std::max(hi, v[j]);
  }
  fprintf(stderr, "[rw eig] %-14s k=%4d norms [%.3e, %.3e] first-nonfinite=%d\n", what, k, lo, hi,
          bad);
}

void trace_small(Work& W, const char* what, const double* M, int n) {
  if (!trace_on()) return;
  std::vector<double> h((size_t)n * n);
  cudaMemcpyAsync(h.data(), M, sizeof(double) * n * n, cudaMemcpyDeviceToHost, W.st);
  cudaStreamSynchronize(W.st);
  double mx = 0.0;
  int bad = -1;
  for (size_t e = 0; e < h.size(); ++e) {
    if (!std::isfinite(h[e]) && bad < 0) bad = (int)e;
    mx = std::max(mx, std::fabs(h[e]));
  }
  fprintf(stderr, "[rw eig] %-14s n=%4d max|.|=%.3e first-nonfinite=%d\n", what, n, mx, bad);
}

rw_status colnorms(Work& W, const float* A, int64_t lda, int k, std::vector<double>& out) {
  RW_CHECK_CUDA(cudaMemsetAsync(W.cn, 0, sizeof(double) * k, W.st));
  const int sms = g_rw_num_sms > 0 ? g_rw_num_sms : 148;
  int64_t rpb = std::max<int64_t>(256, (W.N + 2 * sms - 1) / (2 * sms));
  dim3 grid((unsigned)((W.N + rpb - 1) / rpb), (unsigned)((k + 255) / 256));
  k_colnorms<<<grid, 256, 0, W.st>>>(A, lda, W.N, k, rpb, W.cn);
  RW_LAUNCH_CHECK();
  out.resize(k);
  RW_CHECK_CUDA(cudaMemcpyAsync(out.data(), W.cn, sizeof(double) * k, cudaMemcpyDeviceToHost, W.st));
  RW_CHECK_CUDA(cudaStreamSynchronize(W.st));
  for (auto& v : out) v = std::sqrt(v);
  return RW_OK;
}

// Rayleigh-Ritz on the n orthonormal columns of S (AS = Op S): eigenvalues to host w_h,
// coefficients of the first k Ritz vectors -> C32 (n x k), rows < zero_rows zeroed.
rw_status rayleigh_ritz(Work& W, const float* S, const float* AS, int n, int k,
                        std::vector<double>& w_h) {
  RW_TRY(gram_into(W, S, W.ldS, AS, W.ldS, n, n, W.H));
  k_symmetrize<<<rw_blocks((int64_t)n * n, 256), 256, 0, W.st>>>(W.H, n);
  RW_LAUNCH_CHECK();
  trace_small(W, "rr H", W.H, n);
  RW_TRY(rw_sym_eig(W.H, n, W.w, W.V, W.eigw, W.st));
  trace_small(W, "rr V", W.V, n);
  w_h.resize(n);
  RW_CHECK_CUDA(cudaMemcpyAsync(w_h.data(), W.w, sizeof(double) * n, cudaMemcpyDeviceToHost, W.st));
  RW_CHECK_CUDA(cudaStreamSynchronize(W.st));
  (void)k;
  return RW_OK;
}

}  // namespace

static void basis_release(rw_basis* b) {
  if (!b) return;
  cudaFree(b->Q32); cudaFree(b->Q16); cudaFree(b->Qbf); cudaFree(b->lam);
  delete[] b->lam_host;
  delete b;
}

extern "C" void rw_basis_free(rw_basis* b) { basis_release(b); }
extern "C" int32_t rw_basis_m(const rw_basis* b) { return b ? b->m : 0; }

// allocates the basis and fills Q32/Q16 from an N x m block X (pitch ldx) and values lam_h
static rw_status make_basis(const rw_graph* g, int m, const float* X, int64_t ldx,
                            const double* lam_h, cudaStream_t st, rw_basis** out) {
  rw_basis* b = new (std::nothrow) rw_basis();
  if (!b) return RW_ERR_OOM;
  b->N = g->N;
  b->m = m;
  b->ld32 = (int)rw_round_up(m, 4);
  b->ld16 = (int)rw_round_up(m, 8);
  b->owner = g;
  // power-of-two scale near sqrt(N): entries of unit columns are O(1/sqrt(N))
  int e2 = (int)std::lround(0.5 * std::log2((double)g->N));
  e2 = std::max(0, std::min(e2, 14));
  b->qscale = std::ldexp(1.0f, e2);
  b->lam_host = new (std::nothrow) double[m];
  if (!b->lam_host) { basis_release(b); return RW_ERR_OOM; }
  memcpy(b->lam_host, lam_h, sizeof(double) * m);
  if (cudaMalloc(&b->Q32, sizeof(float) * g->N * b->ld32) != cudaSuccess ||
      cudaMalloc(&b->Q16, sizeof(__half) * g->N * b->ld16) != cudaSuccess ||
      cudaMalloc(&b->lam, sizeof(double) * b->ld32) != cudaSuccess) {
    basis_release(b);
    return RW_ERR_OOM;
  }
  cudaMemsetAsync(b->lam, 0, sizeof(double) * b->ld32, st);
  if (cudaMemcpyAsync(b->lam, lam_h, sizeof(double) * m, cudaMemcpyHostToDevice, st) != cudaSuccess) {
    basis_release(b);
    return RW_ERR_CUDA;
  }
  k_to_basis<<<rw_blocks(g->N * b->ld16, 256), 256, 0, st>>>(X, ldx, g->N, m, b->Q32, b->ld32,
                                                              b->Q16, b->ld16, b->qscale);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) {
    basis_release(b);
    return RW_ERR_CUDA;
  }
  *out = b;
  return RW_OK;
}

rw_status rw_make_basis(const rw_graph* g, int m, const float* X, int64_t ldx,
                        const double* lam_h, cudaStream_t st, rw_basis** out) {
  return make_basis(g, m, X, ldx, lam_h, st, out);
}

extern "C" rw_status rw_basis_create(const rw_graph* g, int32_t m, const float* Q_dev,
                                     const double* lambda_host, void* stream, rw_basis** out) {
  if (!g || !Q_dev || !lambda_host || !out || m < 1 || m > 4096) return RW_ERR_INVALID_ARG;
  *out = nullptr;
  return make_basis(g, m, Q_dev, m, lambda_host, rw_stream(stream), out);
}

extern "C" rw_status rw_basis_get(const rw_basis* b, float* Q_dev, double* lambda_host,
                                  void* stream) {
  if (!b) return RW_ERR_INVALID_ARG;
  cudaStream_t st = rw_stream(stream);
  if (Q_dev)
    RW_CHECK_CUDA(cudaMemcpy2DAsync(Q_dev, sizeof(float) * b->m, b->Q32, sizeof(float) * b->ld32,
                                    sizeof(float) * b->m, b->N, cudaMemcpyDeviceToDevice, st));
  if (lambda_host)
    RW_CHECK_CUDA(cudaMemcpyAsync(lambda_host, b->lam, sizeof(double) * b->m,
                                  cudaMemcpyDeviceToHost, st));
  RW_CHECK_CUDA(cudaStreamSynchronize(st));
  return RW_OK;
}

extern "C" rw_status rw_precompute(rw_graph* g, const rw_eig_opts* opts, void* stream,
                                   rw_basis** out, rw_eig_info* info) {
  if (!g || !opts || !out) return RW_ERR_INVALID_ARG;
  *out = nullptr;
  const int m = opts->m;
  if (m < 1 || m > 512 || m >= g->N) return RW_ERR_INVALID_ARG;
  int guard = opts->guard >= 0 ? opts->guard : std::max(8, m / 5);
  // block width a multiple of 4 so every column block starts 16-byte aligned
  int nb = (int)rw_round_up(m + guard, 4);
  if (nb > g->N) return RW_ERR_INVALID_ARG;
  const int max_iter = opts->max_iter > 0 ? opts->max_iter : 200;
  const double tol = opts->tol > 0 ? opts->tol : 1e-5;
  const int deg = opts->cheb_degree >= 0 ? opts->cheb_degree : 32;
  if (3 * nb > 1024 + 512) return RW_ERR_INVALID_ARG;
  RW_TRY(rw_device_init());
  Work W;
  W.st = rw_stream(stream);
  W.g = g;
  W.N = g->N;
  W.ldS = (int)rw_round_up(3 * nb, 8);  // ldS/2 is a multiple of 4 (second filter slot)
  const size_t blk = sizeof(float) * (size_t)g->N * W.ldS;
  struct Guard {
    Work& w;
    ~Guard() {
      w.S.release(); w.AS.release(); w.T.release(); w.Pb.release(); w.small.release();
      w.gsc.release();
    }
  } guard_rel{W};
  RW_TRY(W.S.grow(blk));
  RW_TRY(W.AS.grow(blk));
  RW_TRY(W.T.grow(blk));
  RW_TRY(W.Pb.grow(sizeof(float) * (size_t)g->N * W.ldS));
  const int nmax = 3 * nb;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t r = off; off += (bytes + 255) & ~size_t(255); return r; };
  size_t oH = take(sizeof(double) * nmax * nmax), oV = take(sizeof(double) * nmax * nmax),
         ow = take(sizeof(double) * nmax), oE = take(rw_sym_eig_work_bytes(nmax)),
         oG = take(sizeof(double) * nmax * nmax), ocn = take(sizeof(double) * nmax),
         oC = take(sizeof(float) * nmax * nmax), oR = take(sizeof(float) * nmax * nmax),
         oL = take(sizeof(float) * (2 * (size_t)W.ldS + nmax)), of = take(sizeof(int) * 16),
         oc = take(sizeof(int) * nmax);
  RW_TRY(W.small.grow(off));
  char* sb = W.small.as<char>();
  W.H = reinterpret_cast<double*>(sb + oH); W.V = reinterpret_cast<double*>(sb + oV);
  W.w = reinterpret_cast<double*>(sb + ow); W.eigw = reinterpret_cast<double*>(sb + oE);
  W.G = reinterpret_cast<double*>(sb + oG); W.cn = reinterpret_cast<double*>(sb + ocn);
  W.C32 = reinterpret_cast<float*>(sb + oC); W.Rinv = reinterpret_cast<float*>(sb + oR);
  W.lam32 = reinterpret_cast<float*>(sb + oL); W.flag = reinterpret_cast<int*>(sb + of);
  W.cols = reinterpret_cast<int*>(sb + oc);

  // spectrum upper bound: 2 for L-hat; 2 max(d) for L (Gershgorin)
  double upper = 2.0;
  if (!g->normalized) {
    unsigned int* mx = reinterpret_cast<unsigned int*>(W.flag);
    RW_CHECK_CUDA(cudaMemsetAsync(mx, 0, sizeof(unsigned int), W.st));
    k_maxf<<<256, 256, 0, W.st>>>(g->d, g->N, mx);
    RW_LAUNCH_CHECK();
    unsigned int h = 0;
    RW_CHECK_CUDA(cudaMemcpyAsync(&h, mx, sizeof(h), cudaMemcpyDeviceToHost, W.st));
    RW_CHECK_CUDA(cudaStreamSynchronize(W.st));
    float f;
    memcpy(&f, &h, sizeof(f));
    upper = 2.0 * f * 1.01;
  }

  float* S = W.S.as<float>();
  float* AS = W.AS.as<float>();
  const int64_t ld = W.ldS;
  int applies = 0;
  // initial block: random, orthonormalized, Rayleigh-Ritz
  k_random_block<<<rw_blocks(g->N * nb, 256), 256, 0, W.st>>>(S, ld, g->N, nb, opts->seed);
  RW_LAUNCH_CHECK();
  RW_TRY(cholqr(W, S, ld, nb));
  std::vector<double> lam(nb), res, wh;
  {
    RW_TRY(rw_stencil_apply(g, S, ld, AS, ld, nb, 1.f, 0.f, nullptr, 0, 0.f, W.st));
    ++applies;
    RW_TRY(rayleigh_ritz(W, S, AS, nb, nb, wh));
    k_take_cols<<<rw_blocks((int64_t)nb * nb, 256), 256, 0, W.st>>>(W.V, nb, nb, 0, W.C32);
    RW_LAUNCH_CHECK();
    float* T = W.T.as<float>();
    RW_TRY(rw_gemm_tall(S, ld, W.C32, nb, g->N, nb, nb, 1.f, 0.f, T, ld, W.st));
    RW_CHECK_CUDA(cudaMemcpy2DAsync(S, sizeof(float) * ld, T, sizeof(float) * ld,
                                    sizeof(float) * nb, g->N, cudaMemcpyDeviceToDevice, W.st));
    for (int j = 0; j < nb; ++j) lam[j] = wh[j];
  }
  int n_p = 0;
  int it = 0;
  int stalls = 0;                   // consecutive filtered steps that cut the residual < 30%
  double prev_maxres = 1e300;
  float* T = W.T.as<float>();
  int conv = 0;
  double maxres = 0.0;
  for (it = 0; it < max_iter; ++it) {
    // AX, residuals, norms
    RW_TRY(rw_stencil_apply(g, S, ld, AS, ld, nb, 1.f, 0.f, nullptr, 0, 0.f, W.st));
    ++applies;
    std::vector<float> lf(nb);
    for (int j = 0; j < nb; ++j) lf[j] = (float)lam[j];
    RW_CHECK_CUDA(cudaMemcpyAsync(W.lam32, lf.data(), sizeof(float) * nb, cudaMemcpyHostToDevice, W.st));
    k_residual<<<rw_blocks(g->N * nb, 256), 256, 0, W.st>>>(AS, S, ld, W.lam32, g->N, nb, T, ld);
    RW_LAUNCH_CHECK();
    RW_TRY(colnorms(W, T, ld, nb, res));
    for (double r : res)
      if (!std::isfinite(r)) return RW_ERR_NOT_CONVERGED;  // lost to rounding; no basis
    conv = 0;
    while (conv < m && res[conv] <= tol) ++conv;
    maxres = 0.0;
    for (int j = 0; j < m; ++j) maxres = std::max(maxres, res[j]);
    if (conv >= m) break;
    if (trace_on())
      fprintf(stderr, "[rw eig] it=%d conv=%d maxres=%.3e lam0=%.6e lam_nb=%.6e\n", it, conv, maxres,
              lam[0], lam[nb - 1]);
    if (deg > 0 && stalls < 2) {
      stalls = (maxres > 0.7 * prev_maxres) ? stalls + 1 : 0;
      prev_maxres = maxres;
      // filtered subspace step: X <- orth(p(Op) X), Rayleigh-Ritz on nb columns
      RW_TRY(cheb_filter(W, S, ld, nb, deg, std::min(lam[0], 0.0), lam[nb - 1], upper, &applies));
      trace_block(W, "filtered X", S, ld, nb);
      RW_TRY(cholqr(W, S, ld, nb));
      trace_block(W, "orth X", S, ld, nb);
      RW_TRY(rw_stencil_apply(g, S, ld, AS, ld, nb, 1.f, 0.f, nullptr, 0, 0.f, W.st));
      ++applies;
      RW_TRY(rayleigh_ritz(W, S, AS, nb, nb, wh));
      k_take_cols<<<rw_blocks((int64_t)nb * nb, 256), 256, 0, W.st>>>(W.V, nb, nb, 0, W.C32);
      RW_LAUNCH_CHECK();
      RW_TRY(rw_gemm_tall(S, ld, W.C32, nb, g->N, nb, nb, 1.f, 0.f, T, ld, W.st));
      RW_CHECK_CUDA(cudaMemcpy2DAsync(S, sizeof(float) * ld, T, sizeof(float) * ld,
                                      sizeof(float) * nb, g->N, cudaMemcpyDeviceToDevice, W.st));
      for (int j = 0; j < nb; ++j) lam[j] = wh[j];
      n_p = 0;
      continue;
    }
    std::vector<int> act;
    for (int j = 0; j < nb; ++j)
      if (!(res[j] <= tol)) act.push_back(j);
    const int n_act = (int)act.size();
    // W block = residuals of the active columns, at columns [nb, nb + n_act) of S
    RW_CHECK_CUDA(cudaMemcpyAsync(W.cols, act.data(), sizeof(int) * n_act, cudaMemcpyHostToDevice, W.st));
    RW_TRY(rw_copy_cols(T, ld, S + nb, ld, g->N, W.cols, n_act, W.st));
    // P block (previous directions of the active columns) after W
    int np_use = 0;
    if (n_p > 0) {
      std::vector<int> pc;
      for (int j : act) pc.push_back(j);
      np_use = (int)pc.size();
      RW_CHECK_CUDA(cudaMemcpyAsync(W.cols, pc.data(), sizeof(int) * np_use, cudaMemcpyHostToDevice, W.st));
      RW_TRY(rw_copy_cols(W.Pb.as<float>(), ld, S + nb + n_act, ld, g->N, W.cols, np_use, W.st));
    }
    int nw = n_act + np_use;
    {
      // drop columns that vanished (e.g. the previous direction of a column that stopped
      // moving); Cholesky-QR needs nonzero columns
      std::vector<double> nrm;
      RW_TRY(colnorms(W, S + nb, ld, nw, nrm));
      double mx = 0.0;
      for (double v : nrm) mx = std::max(mx, v);
      std::vector<int> keep;
      for (int j = 0; j < nw; ++j)
        if (nrm[j] > 1e-30 && nrm[j] > 1e-12 * mx) keep.push_back(j);
      if ((int)keep.size() < nw) {
        RW_CHECK_CUDA(cudaMemcpyAsync(W.cols, keep.data(), sizeof(int) * keep.size(),
                                      cudaMemcpyHostToDevice, W.st));
        RW_TRY(rw_copy_cols(S + nb, ld, T, ld, g->N, W.cols, (int)keep.size(), W.st));
        RW_CHECK_CUDA(cudaMemcpy2DAsync(S + nb, sizeof(float) * ld, T, sizeof(float) * ld,
                                        sizeof(float) * keep.size(), g->N,
                                        cudaMemcpyDeviceToDevice, W.st));
        nw = (int)keep.size();
      }
    }
    const int ntot = nb + nw;
    trace_block(W, "W P raw", S + nb, ld, nw);
    RW_TRY(orth_against(W, S, ld, nb, S + nb, ld, nw));
    trace_block(W, "W P orth", S + nb, ld, nw);
    RW_TRY(cholqr(W, S + nb, ld, nw));
    trace_block(W, "W P cholqr", S + nb, ld, nw);
    RW_TRY(rw_stencil_apply(g, S + nb, ld, AS + nb, ld, nw, 1.f, 0.f, nullptr, 0, 0.f, W.st));
    ++applies;
    RW_TRY(rayleigh_ritz(W, S, AS, ntot, nb, wh));
    // new X = S V[:, :nb]; new P = S[:, nb:] V[nb:, :nb]
    k_take_cols<<<rw_blocks((int64_t)ntot * nb, 256), 256, 0, W.st>>>(W.V, ntot, nb, 0, W.C32);
    RW_LAUNCH_CHECK();
    RW_TRY(rw_gemm_tall(S, ld, W.C32, nb, g->N, ntot, nb, 1.f, 0.f, T, ld, W.st));
    RW_TRY(rw_gemm_tall(S + nb, ld, W.C32 + (size_t)nb * nb, nb, g->N, nw, nb, 1.f, 0.f,
                        W.Pb.as<float>(), ld, W.st));
    RW_CHECK_CUDA(cudaMemcpy2DAsync(S, sizeof(float) * ld, T, sizeof(float) * ld,
                                    sizeof(float) * nb, g->N, cudaMemcpyDeviceToDevice, W.st));
    n_p = nb;
    for (int j = 0; j < nb; ++j) lam[j] = wh[j];
    // keep X orthonormal to working precision
    if ((it & 3) == 3) RW_TRY(cholqr(W, S, ld, nb));
  }
  // final Rayleigh-Ritz on X alone (FP64 projected matrix), residuals
  RW_TRY(cholqr(W, S, ld, nb));
  RW_TRY(rw_stencil_apply(g, S, ld, AS, ld, nb, 1.f, 0.f, nullptr, 0, 0.f, W.st));
  ++applies;
  RW_TRY(rayleigh_ritz(W, S, AS, nb, nb, wh));
  {
    k_take_cols<<<rw_blocks((int64_t)nb * nb, 256), 256, 0, W.st>>>(W.V, nb, nb, 0, W.C32);
    RW_LAUNCH_CHECK();
    RW_TRY(rw_gemm_tall(S, ld, W.C32, nb, g->N, nb, nb, 1.f, 0.f, T, ld, W.st));
    RW_TRY(rw_gemm_tall(AS, ld, W.C32, nb, g->N, nb, nb, 1.f, 0.f, T + nb, ld, W.st));
    std::vector<float> lf(nb);
    for (int j = 0; j < nb; ++j) lf[j] = (float)wh[j];
    RW_CHECK_CUDA(cudaMemcpyAsync(W.lam32, lf.data(), sizeof(float) * nb, cudaMemcpyHostToDevice, W.st));
    // residuals of the final vectors: AX' = T[:, nb:2nb], X' = T[:, :nb]
    k_residual<<<rw_blocks(g->N * nb, 256), 256, 0, W.st>>>(T + nb, T, ld, W.lam32, g->N, nb, AS, ld);
    RW_LAUNCH_CHECK();
    RW_TRY(colnorms(W, AS, ld, nb, res));
    conv = 0;
    while (conv < m && res[conv] <= tol) ++conv;
    maxres = 0.0;
    for (int j = 0; j < m; ++j) maxres = std::max(maxres, res[j]);
    for (double r : res)
      if (!std::isfinite(r)) return RW_ERR_NOT_CONVERGED;
    rw_basis* b = nullptr;
    RW_TRY(make_basis(g, m, T, ld, wh.data(), W.st, &b));
    // stored values: edge-sum Rayleigh quotients (Eq. z_ray) of the stored FP32 columns, so a
    // later update with unchanged weights reproduces them exactly
    rw_status rs = rw_basis_rayleigh(g, b, W.st);
    if (rs == RW_OK) rs = rw_last_device_status(g, W.st);  // e.g. a tensor-core wait gave up
    if (rs != RW_OK) { rw_basis_free(b); return rs; }
    *out = b;
  }
  if (info) {
    info->iterations = it;
    info->converged = conv;
    info->max_residual = maxres;
    info->stencil_applies = applies;
  }
  return conv >= m ? RW_OK : RW_WARN_NOT_CONVERGED;
}
