// Dense helpers for the block eigensolver and the seed-side products: Gram matrices A^T B of
// tall node-major blocks, tall-skinny products A C, and the small FP64 factorizations
// (Cholesky, triangular inverse, cyclic-Jacobi symmetric eigensolver).
#include "rw_internal.cuh"

#include <cooperative_groups.h>

#include <algorithm>

namespace cg = cooperative_groups;

// ---------------------------------------------------------------------------------------
// G += A^T B.  A: N x p, B: N x q (node-major FP32).  64 x 64 output tile per CTA, the N rows
// split across gridDim.z; FP32 partial sums over 256 rows, flushed into FP64 accumulators, and
// FP64 atomic accumulation across CTAs.
// ---------------------------------------------------------------------------------------
namespace {
constexpr int GT = 64, GK = 32;
}

__global__ void __launch_bounds__(256)
k_gram(const float* __restrict__ A, int64_t lda, const float* __restrict__ B, int64_t ldb,
       int64_t N, int p, int q, double* __restrict__ G, int ldg, int64_t rows_per_cta) {
  __shared__ float As[GK][GT + 4];
  __shared__ float Bs[GK][GT + 4];
  const int i0 = blockIdx.x * GT, j0 = blockIdx.y * GT;
  const int64_t r0 = (int64_t)blockIdx.z * rows_per_cta;
  const int64_t r1 = min(N, r0 + rows_per_cta);
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  float acc[4][4] = {};
  double accd[4][4] = {};
  int since_flush = 0;
  for (int64_t k0 = r0; k0 < r1; k0 += GK) {
    if (++since_flush == 8) {  // 256 rows
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) { accd[u][v] += acc[u][v]; acc[u][v] = 0.f; }
      since_flush = 0;
    }
    for (int e = threadIdx.x; e < GK * GT; e += 256) {
      int kk = e / GT, ii = e % GT;
      int64_t r = k0 + kk;
      bool rin = r < r1;
      As[kk][ii] = (rin && i0 + ii < p) ? A[r * lda + i0 + ii] : 0.f;
      Bs[kk][ii] = (rin && j0 + ii < q) ? B[r * ldb + j0 + ii] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < GK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) { a[u] = As[kk][ty * 4 + u]; b[u] = Bs[kk][tx * 4 + u]; }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(a[u], b[v], acc[u][v]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      int i = i0 + ty * 4 + u, j = j0 + tx * 4 + v;
      if (i < p && j < q) atomicAdd(&G[(int64_t)i * ldg + j], accd[u][v] + (double)acc[u][v]);
    }
}

rw_status rw_gram(const float* A, int64_t lda, const float* B, int64_t ldb, int64_t N, int p,
                  int q, double* G, int ldg, bool accumulate, cudaStream_t st) {
  if (p <= 0 || q <= 0) return RW_OK;
  if (!accumulate) {
    if (ldg == q) {
      RW_CHECK_CUDA(cudaMemsetAsync(G, 0, sizeof(double) * (size_t)p * q, st));
    } else {
      RW_CHECK_CUDA(cudaMemset2DAsync(G, sizeof(double) * ldg, 0, sizeof(double) * q, p, st));
    }
  }
  if (N <= 0) return RW_OK;
  const int ti = (p + GT - 1) / GT, tj = (q + GT - 1) / GT;
  const int sms = g_rw_num_sms > 0 ? g_rw_num_sms : 148;
  int64_t want = (int64_t)2 * sms / (ti * tj);
  if (want < 1) want = 1;
  int64_t maxz = (N + 255) / 256;  // at least 256 rows per CTA
  if (want > maxz) want = maxz;
  int64_t rpc = rw_round_up((N + want - 1) / want, GK);
  int64_t nz = (N + rpc - 1) / rpc;
  dim3 grid(ti, tj, (unsigned)nz);
  k_gram<<<grid, 256, 0, st>>>(A, lda, B, ldb, N, p, q, G, ldg, rpc);
  RW_LAUNCH_CHECK();
  return RW_OK;
}

// ---------------------------------------------------------------------------------------
// Y (N x p) = alpha A (N x q) C (q x p, FP32 row-major) + beta Y.  Y must not alias A.
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
k_gemm_tall(const float* __restrict__ A, int64_t lda, const float* __restrict__ C, int ldc,
            int64_t N, int q, int p, float alpha, float beta, float* __restrict__ Y,
            int64_t ldy) {
  __shared__ float As[GT][GK + 1];
  __shared__ float Cs[GK][GT + 4];
  const int64_t i0 = (int64_t)blockIdx.x * GT;
  const int j0 = blockIdx.y * GT;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < q; k0 += GK) {
    for (int e = threadIdx.x; e < GT * GK; e += 256) {
      int ii = e / GK, kk = e % GK;
      int64_t r = i0 + ii;
      As[ii][kk] = (r < N && k0 + kk < q) ? A[r * lda + k0 + kk] : 0.f;
    }
    for (int e = threadIdx.x; e < GK * GT; e += 256) {
      int kk = e / GT, jj = e % GT;
      Cs[kk][jj] = (k0 + kk < q && j0 + jj < p) ? C[(int64_t)(k0 + kk) * ldc + j0 + jj] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < GK; ++kk) {
      float a[4], c[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) { a[u] = As[ty * 4 + u][kk]; c[u] = Cs[kk][tx * 4 + u]; }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(a[u], c[v], acc[u][v]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    int64_t r = i0 + ty * 4 + u;
    if (r >= N) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      int j = j0 + tx * 4 + v;
      if (j < p) {
        float o = alpha * acc[u][v];
        if (beta != 0.f) o += beta * Y[r * ldy + j];
        Y[r * ldy + j] = o;
      }
    }
  }
}

rw_status rw_gemm_tall(const float* A, int64_t lda, const float* C, int ldc, int64_t N, int q,
                       int p, float alpha, float beta, float* Y, int64_t ldy, cudaStream_t st) {
  if (N <= 0 || p <= 0) return RW_OK;
  dim3 grid((unsigned)((N + GT - 1) / GT), (unsigned)((p + GT - 1) / GT));
  k_gemm_tall<<<grid, 256, 0, st>>>(A, lda, C, ldc, N, q, p, alpha, beta, Y, ldy);
  RW_LAUNCH_CHECK();
  return RW_OK;
}

// ---------------------------------------------------------------------------------------
// In-place Cholesky A + shift I = R^T R (R upper) of a small SPD FP64 matrix, one CTA.
// A zero or negative pivot sets *flag = 1 and continues with the pivot clamped to a tiny
// positive value (the caller decides what to do with the flag).
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_cholesky_upper(double* A, int n, double shift,
                                                         int* flag) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) A[(int64_t)i * n + i] += shift;
  __syncthreads();
  double scale = 0.0;
  for (int i = 0; i < n; ++i) scale = fmax(scale, fabs(A[(int64_t)i * n + i]));
  const double floor_piv = (scale > 0 ? scale : 1.0) * 1e-12;
  for (int k = 0; k < n; ++k) {
    __syncthreads();
    double piv = A[(int64_t)k * n + k];
    if (!(piv > 0.0)) {
      if (threadIdx.x == 0 && flag) *flag = 1;
      piv = floor_piv;  // keeps R finite; the caller sees the flag
    }
    const double r = sqrt(piv);
    __syncthreads();
    for (int j = k + 1 + threadIdx.x; j < n; j += blockDim.x) A[(int64_t)k * n + j] /= r;
    if (threadIdx.x == 0) A[(int64_t)k * n + k] = r;
    __syncthreads();
    const int m = n - k - 1;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
      int i = k + 1 + e / m, j = k + 1 + e % m;
      if (j >= i) A[(int64_t)i * n + j] -= A[(int64_t)k * n + i] * A[(int64_t)k * n + j];
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    int i = e / n, j = e % n;
    if (j < i) A[e] = 0.0;
  }
}

rw_status rw_cholesky_upper(double* A, int n, double shift, int* flag, cudaStream_t st) {
  k_cholesky_upper<<<1, 1024, 0, st>>>(A, n, shift, flag);
  RW_LAUNCH_CHECK();
  return RW_OK;
}

// Rinv = R^{-1} for upper-triangular R: thread j solves R x = e_j (x_i = 0 for i > j).
__global__ void k_tri_inverse_upper(const double* __restrict__ R, int n, double* __restrict__ W,
                                    float* __restrict__ Rinv) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  for (int i = n - 1; i > j; --i) W[(int64_t)i * n + j] = 0.0;
  for (int i = j; i >= 0; --i) {
    double sacc = (i == j) ? 1.0 : 0.0;
    for (int k = i + 1; k <= j; ++k) sacc -= R[(int64_t)i * n + k] * W[(int64_t)k * n + j];
    W[(int64_t)i * n + j] = sacc / R[(int64_t)i * n + i];
  }
  for (int i = 0; i < n; ++i) Rinv[(int64_t)i * n + j] = (float)W[(int64_t)i * n + j];
}

static DevBuf g_triw;  // FP64 scratch of the triangular inverse (offline path only)

rw_status rw_tri_inverse_upper(const double* R, int n, float* Rinv, cudaStream_t st) {
  RW_TRY(g_triw.grow(sizeof(double) * (size_t)n * n));
  k_tri_inverse_upper<<<rw_blocks(n, 128), 128, 0, st>>>(R, n, g_triw.as<double>(), Rinv);
  RW_LAUNCH_CHECK();
  return RW_OK;
}

// ---------------------------------------------------------------------------------------
// Symmetric eigensolver: parallel cyclic Jacobi with round-robin pairing.  Each round pairs
// all indices disjointly; phase 1 computes one rotation per pair from the current diagonal
// blocks; phase 2 applies J^T A J block by block (each 2x2 block of A belongs to one pair of
// pairs, so blocks update independently) and V := V J.  A cooperative grid runs the rounds
// with grid-wide barriers.  Sweeps stop when the off-diagonal mass is below 1e-26 of the
// total (or after 30 sweeps).
// ---------------------------------------------------------------------------------------
struct JacobiArgs {
  double* A;
  double* V;
  double* rot;   // per pair: c, s
  int* pairs;    // per pair: p, q  (index >= n means "no partner")
  double* off;   // [0] off-diagonal sum of squares, [1] total
  int n, ne;     // ne = n rounded up to even
};

__device__ __forceinline__ void rr_pair(int r, int i, int ne, int* p, int* q) {
  // players 0..ne-2 on a circle, player ne-1 fixed
  if (i == 0) {
    *p = r;
    *q = ne - 1;
  } else {
    *p = (r + i) % (ne - 1);
    *q = (r - i + (ne - 1)) % (ne - 1);
  }
  if (*p > *q) { int t = *p; *p = *q; *q = t; }
}

__global__ void k_jacobi(JacobiArgs a, int max_sweeps) {
  cg::grid_group grid = cg::this_grid();
  const int n = a.n, ne = a.ne, np = ne / 2;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    // convergence check
    if (tid == 0) { a.off[0] = 0.0; a.off[1] = 0.0; }
    grid.sync();
    {
      double so = 0.0, st = 0.0;
      for (int64_t e = tid; e < (int64_t)n * n; e += nth) {
        int i = (int)(e / n), j = (int)(e % n);
        double v = a.A[e] * a.A[e];
        st += v;
        if (i != j) so += v;
      }
      for (int o = 16; o > 0; o >>= 1) {
        so += __shfl_down_sync(0xffffffff, so, o);
        st += __shfl_down_sync(0xffffffff, st, o);
      }
      if ((threadIdx.x & 31) == 0) { atomicAdd(&a.off[0], so); atomicAdd(&a.off[1], st); }
    }
    grid.sync();
    if (a.off[0] <= 1e-26 * a.off[1] || a.off[1] == 0.0) break;
    for (int r = 0; r < ne - 1; ++r) {
      // phase 1: rotations
      for (int64_t i = tid; i < np; i += nth) {
        int p, q;
        rr_pair(r, (int)i, ne, &p, &q);
        double c = 1.0, s = 0.0;
        if (q < n) {
          double app = a.A[(int64_t)p * n + p], aqq = a.A[(int64_t)q * n + q];
          double apq = a.A[(int64_t)p * n + q];
          if (fabs(apq) > 1e-300 && fabs(apq) > 1e-18 * sqrt(fabs(app * aqq))) {
            double th = (aqq - app) / (2.0 * apq);
            double t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
            c = 1.0 / sqrt(t * t + 1.0);
            s = t * c;
          }
        }
        a.rot[2 * i] = c;
        a.rot[2 * i + 1] = s;
        a.pairs[2 * i] = p;
        a.pairs[2 * i + 1] = q;
      }
      grid.sync();
      // phase 2: A := J^T A J on 2x2 blocks (P1, P2), P1 <= P2; V := V J
      const int64_t nblk = (int64_t)np * (np + 1) / 2;
      for (int64_t e = tid; e < nblk + (int64_t)n * np; e += nth) {
        if (e < nblk) {
          // unrank e -> (u, v) with u <= v
          int u = (int)((sqrt(8.0 * (double)e + 1.0) - 1.0) / 2.0);
          while ((int64_t)u * (u + 1) / 2 > e) --u;
          while ((int64_t)(u + 1) * (u + 2) / 2 <= e) ++u;
          int v = (int)(e - (int64_t)u * (u + 1) / 2);  // v <= u
          int p1 = a.pairs[2 * v], q1 = a.pairs[2 * v + 1];
          int p2 = a.pairs[2 * u], q2 = a.pairs[2 * u + 1];
          double c1 = a.rot[2 * v], s1 = a.rot[2 * v + 1];
          double c2 = a.rot[2 * u], s2 = a.rot[2 * u + 1];
          bool h1 = q1 < n, h2 = q2 < n;
          double x00 = a.A[(int64_t)p1 * n + p2];
          double x01 = h2 ? a.A[(int64_t)p1 * n + q2] : 0.0;
          double x10 = h1 ? a.A[(int64_t)q1 * n + p2] : 0.0;
          double x11 = (h1 && h2) ? a.A[(int64_t)q1 * n + q2] : 0.0;
          // rows: [p1; q1] <- [c1 -s1; s1 c1]^T-applied: new_p = c x_p - s x_q, new_q = s x_p + c x_q
          double y00 = c1 * x00 - s1 * x10, y01 = c1 * x01 - s1 * x11;
          double y10 = s1 * x00 + c1 * x10, y11 = s1 * x01 + c1 * x11;
          // columns: same rotation with (c2, s2)
          double z00 = c2 * y00 - s2 * y01, z01 = s2 * y00 + c2 * y01;
          double z10 = c2 * y10 - s2 * y11, z11 = s2 * y10 + c2 * y11;
          if (u == v && h1) z01 = z10 = 0.5 * (z01 + z10);
          a.A[(int64_t)p1 * n + p2] = z00;
          if (h2) a.A[(int64_t)p1 * n + q2] = z01;
          if (h1) a.A[(int64_t)q1 * n + p2] = z10;
          if (h1 && h2) a.A[(int64_t)q1 * n + q2] = z11;
          if (u != v) {  // mirror block
            a.A[(int64_t)p2 * n + p1] = z00;
            if (h2) a.A[(int64_t)q2 * n + p1] = z01;
            if (h1) a.A[(int64_t)p2 * n + q1] = z10;
            if (h1 && h2) a.A[(int64_t)q2 * n + q1] = z11;
          }
        } else {
          int64_t f = e - nblk;
          int row = (int)(f / np), pi = (int)(f % np);
          int p = a.pairs[2 * pi], q = a.pairs[2 * pi + 1];
          if (q < n) {
            double c = a.rot[2 * pi], s = a.rot[2 * pi + 1];
            double vp = a.V[(int64_t)row * n + p], vq = a.V[(int64_t)row * n + q];
            a.V[(int64_t)row * n + p] = c * vp - s * vq;
            a.V[(int64_t)row * n + q] = s * vp + c * vq;
          }
        }
      }
      grid.sync();
    }
  }
}

// w ascending (ties by index), V columns permuted accordingly; W = previous V
__global__ void k_eig_sort(const double* __restrict__ A, const double* __restrict__ Vin, int n,
                           double* __restrict__ w, double* __restrict__ Vout) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double li = A[(int64_t)i * n + i];
  int rank = 0;
  for (int j = 0; j < n; ++j) {
    double lj = A[(int64_t)j * n + j];
    if (lj < li || (lj == li && j < i)) ++rank;
  }
  w[rank] = li;
  for (int r = 0; r < n; ++r) Vout[(int64_t)r * n + rank] = Vin[(int64_t)r * n + i];
}

__global__ void k_set_identity(double* V, int n) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < (int64_t)n * n) V[e] = (e / n == e % n) ? 1.0 : 0.0;
}

size_t rw_sym_eig_work_bytes(int n) {
  int ne = n + (n & 1);
  return sizeof(double) * ((size_t)n * n + (size_t)ne + 4) + sizeof(int) * (size_t)ne + 64;
}

rw_status rw_sym_eig(double* A, int n, double* w, double* V, double* work, cudaStream_t st) {
  if (n <= 0) return RW_OK;
  const int ne = n + (n & 1);
  double* Vtmp = work;
  double* rot = Vtmp + (size_t)n * n;
  double* off = rot + ne;
  int* pairs = reinterpret_cast<int*>(off + 4);
  k_set_identity<<<rw_blocks((int64_t)n * n, 256), 256, 0, st>>>(Vtmp, n);
  RW_LAUNCH_CHECK();
  int dev = 0, per_sm = 0;
  RW_CHECK_CUDA(cudaGetDevice(&dev));
  RW_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_jacobi, 256, 0));
  int sms = g_rw_num_sms > 0 ? g_rw_num_sms : 148;
  int64_t work_items = (int64_t)(ne / 2) * (ne / 2 + 1) / 2 + (int64_t)n * (ne / 2);
  int blocks = (int)std::min<int64_t>((int64_t)sms * std::max(per_sm, 1),
                                      std::max<int64_t>(1, (work_items + 255) / 256));
  if (blocks < 1) blocks = 1;
  JacobiArgs args{A, Vtmp, rot, pairs, off, n, ne};
  int max_sweeps = 30;
  void* kargs[] = {&args, &max_sweeps};
  RW_CHECK_CUDA(cudaLaunchCooperativeKernel((void*)k_jacobi, dim3(blocks), dim3(256), kargs, 0, st));
  rw_count_launch();
  k_eig_sort<<<rw_blocks(n, 128), 128, 0, st>>>(A, Vtmp, n, w, V);
  RW_LAUNCH_CHECK();
  return RW_OK;
}

// ---------------------------------------------------------------------------------------
__global__ void k_copy_cols(const float* __restrict__ src, int64_t lds, float* __restrict__ dst,
                            int64_t ldd, int64_t N, const int* __restrict__ cols, int ncols) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * ncols) return;
  int64_t r = e / ncols;
  int c = (int)(e % ncols);
  dst[r * ldd + c] = src[r * lds + cols[c]];
}

rw_status rw_copy_cols(const float* src, int64_t lds, float* dst, int64_t ldd, int64_t N,
                       const int* cols, int ncols, cudaStream_t st) {
  if (ncols <= 0 || N <= 0) return RW_OK;
  k_copy_cols<<<rw_blocks(N * ncols, 256), 256, 0, st>>>(src, lds, dst, ldd, N, cols, ncols);
  RW_LAUNCH_CHECK();
  return RW_OK;
}

__global__ void k_f64_to_f32(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

rw_status rw_f64_to_f32(const double* a, float* b, int64_t n, cudaStream_t st) {
  if (n <= 0) return RW_OK;
  k_f64_to_f32<<<rw_blocks(n, 256), 256, 0, st>>>(a, b, n);
  RW_LAUNCH_CHECK();
  return RW_OK;
}
