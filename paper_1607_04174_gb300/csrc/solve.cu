// Online fast random walker (Sec. II-B, Eqs. Fs and U_lin_comb, in the normalized form of
// Sec. II-C) with the number of eigenvectors chosen from the seeds (Sec. III-A-1, Eq. alpha_1),
// priors from a Gaussian fit to the seed intensities (Sec. IV-A), damped-Jacobi refinement on
// Eq. (rw_eq) and hard labels.
//
// Hat variables: U-hat = D^{1/2} U, P-hat = D^{1/2} P (sq = d^{1/2}, s = d^{-1/2}); with the
// unnormalized Laplacian sq = s = 1.  Operator coefficients c_ij = w_ij s_i s_j, so the seeded
// block of L-hat is B-hat_ij = -c_ij.
//
// Per solve (S seeds, m_max basis columns, l labels), every kernel launched with programmatic
// dependent launch (it waits on griddepcontrol before reading its predecessors' output):
//   seed labels, per-block seed statistics         -> k_seed_scatter
//   Q_s, X = B-hat Q_n (S x m_max), r0 = L-hat_s U-hat_s + gamma U-hat_s  -> k_seed_gather
//   K = Q_s^T X, h = Q_s^T r0, b = Q_s^T U-hat_s, G = Q_s^T Q_s (FP32)  -> k_seed_gram (cluster)
//   Gaussian fit, P-hat (N x lp)                    -> k_priors (beside the two before it)
//   m (incremental Cholesky over the nested candidates, trust region) and the LU of
//   M = diag(lambda + gamma) - K (left-looking, stopped at m)  -> k_adapt_lu (2-CTA cluster)
//   Z = Q_n^T P-hat_n (streams the 16-bit basis once)  -> k_project_tma, k_reduce_partials
//   C = M^{-1} (h + gamma Z)                          -> k_small_rhs (k_small_solve: pivoting)
//   U-hat_n = Q_n C (streams the basis again)          -> k_backproject_panel
//   refinement steps, U = s * U-hat, labels = argmax   -> k_jacobi_grid (k_jacobi_step on CSR)
// When the cluster's shared memory does not fit, k_adapt (or k_set_m) and k_small_solve run
// instead of k_adapt_lu and k_small_rhs.
#include "rw_internal.cuh"

#include <cooperative_groups.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <unordered_map>
#include <cstring>

namespace cg = cooperative_groups;

namespace {

constexpr int kMaxSmallM = 224;
constexpr int kMaxSeeds = 65536;   // seeds per solve (the validation's limit)

int lpad_of(int L) { return L <= 4 ? 4 : (L <= 8 ? 8 : 16); }

struct Layout {
  size_t mdev, Bcat, Gcat, Z, C, fu, lu, luinv, part, gnull, partw, wv, nul, lam0, total;
};

// wcat = 2 mp + 2 lp: the seed-side block [X | Q_s | r0 | U-hat_s] (S x wcat, one row per
// seed) and its product with Q_s, [K | G | h | b] = Q_s^T [X | Q_s | r0 | U-hat_s] (mp x wcat)
Layout make_layout(int S, int mp, int mq, int lp, int L, int ncand, int nblk_part) {
  (void)L;
  Layout o;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t r = off; off += (bytes + 255) & ~size_t(255); return r; };
  const size_t wcat = 2 * (size_t)mp + 2 * (size_t)lp;
  o.mdev = take(sizeof(int) * 8);
  o.Bcat = take(sizeof(float) * (size_t)S * wcat);
  o.Gcat = take(sizeof(float) * (size_t)mp * wcat);
  o.Z = take(sizeof(float) * (size_t)mq * lp + sizeof(float) * (size_t)mq);  // Z, lambda + gamma
  o.C = take(sizeof(float) * (size_t)mq * lp);
  o.fu = take(sizeof(double) * (size_t)(ncand + 1) * RW_MAX_LABELS + sizeof(double) * lp);
  o.lu = take(sizeof(float) * (size_t)mp * mp);   // LU factors of the m x m system, pitch mp
  o.luinv = take(sizeof(float) * (size_t)mp);     // 1 / U_ii
  o.part = take(sizeof(float) * (size_t)nblk_part * mq * lp);
  // gamma = 0: per seed (g_t, (B-hat g_n)_t), partial sums of Q_s^T g_s, w, the null
  // coefficients, the values with lambda_0 replaced
  o.gnull = take(sizeof(float) * 2 * (size_t)S);
  o.partw = take(sizeof(float) * 16 * (size_t)mq);
  o.wv = take(sizeof(float) * (size_t)mq);
  o.nul = take(sizeof(float) * RW_MAX_LABELS);
  o.lam0 = take(sizeof(double) * (size_t)mq);
  o.total = off;
  return o;
}

// cudaFuncSetAttribute(MaxDynamicSharedMemorySize) only when a kernel needs more than it was
// last given (host side; the per-solve call path stays free of attribute calls once warm)
template <typename F>
static cudaError_t ensure_smem(F* func, size_t bytes) {
  static std::mutex mu;
  static std::unordered_map<const void*, size_t> done[64];  // per device
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
    return cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  std::lock_guard<std::mutex> lock(mu);
  size_t& have = done[dev][reinterpret_cast<const void*>(func)];
  if (bytes <= have) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) have = bytes;
  return e;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffff, v, o);
  return v;
}

__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;"
               :: "r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(float* dst, const float* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;"
               :: "r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
// 16 bytes, or zeros when !valid (source size 0; src must still be a valid address)
__device__ __forceinline__ void cp_async16_zfill(void* dst, const void* src, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;"
               :: "r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src), "r"(valid ? 16 : 0) : "memory");
}

// mbarrier + bulk asynchronous copy (global -> shared, completion counted in bytes on the
// barrier).  Waits are bounded: a wait that gives up sets RW_DEV_TIMEOUT.
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
               :: "r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               :: "r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
               " selp.u32 %0, 1, 0, p;\n}" : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
  return ok != 0;
}
__device__ __forceinline__ void mbar_wait_bounded(uint64_t* bar, unsigned parity, int* status) {
  for (int it = 0; !mbar_try_wait(bar, parity); ++it) {
    if (it > (1 << 24)) {
      if (status) atomicOr(status, RW_DEV_TIMEOUT);
      return;
    }
  }
}

// ---------------------------------------------------------------------------------------
__global__ void k_seed_reset(int* __restrict__ seedlab, int64_t n, double* __restrict__ stats,
                             int nstats) {
  rw_grid_wait();
  rw_grid_trigger();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) seedlab[i] = -1;
  if (stats && i < nstats) stats[i] = 0.0;
}

// Marks the seeds (an index or label out of range or a voxel seeded twice sets a status bit)
// and writes, per block and label, the count, the mean and the sum of squared deviations from
// that mean of the seed intensities: bpart[block][3 k + {0, 1, 2}].  One warp per label, two
// passes (mean, then deviations) with fixed butterflies, so there is no cancellation and the
// result does not depend on scheduling.
__global__ void __launch_bounds__(256)
k_seed_scatter(const int32_t* __restrict__ idx, const int32_t* __restrict__ lab, int S, int L,
               int64_t N, const float* __restrict__ J, int* __restrict__ seedlab,
               float* __restrict__ bpart, int* status) {
  rw_grid_wait();
  rw_grid_trigger();
  __shared__ int sk[256];
  __shared__ float sv[256];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const int t = blockIdx.x * blockDim.x + tid;
  int k = -1;
  float v = 0.f;
  if (t < S) {
    const int i = idx[t];
    k = lab[t];
    if (i < 0 || (int64_t)i >= N || k < 0 || k >= L) {
      atomicOr(status, RW_DEV_BAD_SEED);
      k = -1;
    } else {
      if (atomicCAS(&seedlab[i], -1, k) != -1) atomicOr(status, RW_DEV_DUP_SEED);
      v = J ? J[i] : 0.f;
    }
  }
  sk[tid] = k;
  sv[tid] = v;
  __syncthreads();
  for (int kk = warp; kk < L; kk += nw) {
    float sum = 0.f, cnt = 0.f;
    for (int e = lane; e < 256; e += 32)
      if (sk[e] == kk) { sum += sv[e]; cnt += 1.f; }
    sum = warp_sum(sum);
    cnt = warp_sum(cnt);
    const float mean = cnt > 0.f ? sum / cnt : 0.f;
    float m2 = 0.f;
    for (int e = lane; e < 256; e += 32)
      if (sk[e] == kk) { const float d = sv[e] - mean; m2 = fmaf(d, d, m2); }
    m2 = warp_sum(m2);
    if (lane == 0) {
      float* o = bpart + ((size_t)blockIdx.x * L + kk) * 3;
      o[0] = cnt;
      o[1] = mean;
      o[2] = m2;
    }
  }
}

// The Gaussian fit of Sec. IV-A from the scatter blocks' (count, mean, squared deviations),
// merged in block order with the pairwise update of the mean and the sum of squared
// deviations: mu_k, 1/(2 sigma_k^2), log sigma_k with sigma_k = max(std, 1e-3) (maximum
// likelihood: the variance divides by the count).
__device__ void seed_fit(const float* __restrict__ bpart, int nsb, int L, int prior_mode,
                         float* fit, double* fit64, int* status) {
  const int k = threadIdx.x;
  if (k >= L) return;
  float n = 0.f, mean = 0.f, m2 = 0.f;
  for (int b = 0; b < nsb; ++b) {
    const float* o = bpart + ((size_t)b * L + k) * 3;
    const float nb = __ldcg(o);
    if (nb > 0.f) {
      const float nt = n + nb, delta = __ldcg(o + 1) - mean;
      mean += delta * (nb / nt);
      m2 += __ldcg(o + 2) + delta * delta * (n * nb / nt);
      n = nt;
    }
  }
  if (!(n > 0.f)) {
    if (prior_mode == 0 && status) atomicOr(status, RW_DEV_EMPTY_LABEL);
    fit[k] = 0.f; fit[16 + k] = 0.f; fit[32 + k] = 0.f;
    if (fit64) { fit64[k] = 0.0; fit64[16 + k] = 0.0; }
    return;
  }
  const float sig = fmaxf(sqrtf(fmaxf(m2 / n, 0.f)), 1e-3f);
  fit[k] = mean;
  fit[16 + k] = 0.5f / (sig * sig);
  fit[32 + k] = logf(sig);
  if (fit64) { fit64[k] = mean; fit64[16 + k] = sig; }
}

// P-hat rows (N x lp): Gaussian priors normalized per voxel, or caller priors, times d^{1/2}
template <int LP>
__global__ void __launch_bounds__(256)
k_priors(const float* __restrict__ J, const float* __restrict__ sq, int64_t N, int L,
         int prior_mode, const float* __restrict__ bpart, int nsb, double* __restrict__ fit64,
         const float* __restrict__ Pin, float* __restrict__ phat, int* status, int early) {
  // early: launched behind kernels that do not touch its inputs (they come from further back
  // and are complete once its predecessor has started), so it starts at once and waits for
  // its predecessor only before it exits; the kernels after it then see both
  if (!early) rw_grid_wait();
  rw_grid_trigger();
  __shared__ float fit[48];
  if (prior_mode == 0)
    seed_fit(bpart, nsb, L, prior_mode, fit, blockIdx.x == 0 ? fit64 : nullptr,
             blockIdx.x == 0 ? status : nullptr);
  else if (blockIdx.x == 0)
    seed_fit(bpart, nsb, L, prior_mode, fit, fit64, nullptr);
  __syncthreads();
  // grid-stride over groups of four consecutive voxels (16-byte loads of J and d^{1/2}, all of
  // a group's loads issued together; a few waves of blocks, so the fit above is amortized)
  const int64_t ng = (N + 3) / 4;
  for (int64_t gI = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gI < ng;
       gI += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i0 = 4 * gI;
    const bool full = i0 + 3 < N;
    float xv[4] = {0.f, 0.f, 0.f, 0.f}, rv[4] = {0.f, 0.f, 0.f, 0.f};
    float pin[4][LP];
    if (full) {
      const float4 r4 = *reinterpret_cast<const float4*>(sq + i0);
      rv[0] = r4.x; rv[1] = r4.y; rv[2] = r4.z; rv[3] = r4.w;
    } else {
#pragma unroll
      for (int u = 0; u < 4; ++u) rv[u] = i0 + u < N ? sq[i0 + u] : 0.f;
    }
    if (prior_mode == 0) {
      if (full) {
        const float4 j4 = *reinterpret_cast<const float4*>(J + i0);
        xv[0] = j4.x; xv[1] = j4.y; xv[2] = j4.z; xv[3] = j4.w;
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) xv[u] = i0 + u < N ? J[i0 + u] : 0.f;
      }
    } else {
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int k = 0; k < LP; ++k) pin[u][k] = (k < L && i0 + u < N) ? Pin[(i0 + u) * L + k] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t i = i0 + u;
      if (i >= N) break;
      float p[LP];
      if (prior_mode == 0) {
        float mx = -INFINITY;
#pragma unroll
        for (int k = 0; k < LP; ++k) {
          const float t = xv[u] - fit[k];
          p[k] = (k < L) ? -t * t * fit[16 + k] - fit[32 + k] : -INFINITY;
          mx = fmaxf(mx, p[k]);
        }
        float sum = 0.f;
#pragma unroll
        for (int k = 0; k < LP; ++k) {
          p[k] = (k < L) ? __expf(p[k] - mx) : 0.f;
          sum += p[k];
        }
        const float inv = 1.f / sum;
#pragma unroll
        for (int k = 0; k < LP; ++k) p[k] *= inv;
      } else {
#pragma unroll
        for (int k = 0; k < LP; ++k) {
          p[k] = pin[u][k];
          if (k < L && !isfinite(p[k])) atomicOr(status, RW_DEV_NONFINITE);
        }
      }
      float4* o = reinterpret_cast<float4*>(phat + i * LP);
#pragma unroll
      for (int k4 = 0; k4 < LP / 4; ++k4)
        o[k4] = make_float4(rv[u] * p[4 * k4], rv[u] * p[4 * k4 + 1], rv[u] * p[4 * k4 + 2],
                            rv[u] * p[4 * k4 + 3]);
    }
  }
  if (early) rw_grid_wait();
}

// One warp per seed: Q_s row, X = B-hat Q_n row, U-hat_s row, r0 = L-hat_s U-hat_s + g U-hat_s
__global__ void k_seed_gather(const int32_t* __restrict__ idx, const int32_t* __restrict__ lab,
                              int S, int L, int lp, int64_t N, const float* __restrict__ Q,
                              int ldq, int mp, const int* __restrict__ seedlab,
                              const float* __restrict__ cw, const float* __restrict__ d,
                              const float* __restrict__ sq, int normalized, int kind, int ndim,
                              int DX, int DY, int DZ, const int32_t* __restrict__ rowptr,
                              const int32_t* __restrict__ colv, const float* __restrict__ ccsr,
                              float gamma, float* __restrict__ Bcat, int ldb,
                              float* __restrict__ gnull, float ginv,
                              int* __restrict__ mflag) {
  rw_grid_wait();
  rw_grid_trigger();
  if (mflag && blockIdx.x == 0 && threadIdx.x == 0) *mflag = 0;   // m not yet published
  const int lane = threadIdx.x & 31;
  const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (t >= S) return;
  const int i = idx[t], k0 = lab[t];
  float* xs = Bcat + (int64_t)t * ldb;
  float* qs = xs + mp;
  float* R0 = qs + mp;
  float* Us = R0 + lp;
  if (i < 0 || (int64_t)i >= N || k0 < 0 || k0 >= L) {  // reported by k_seed_scatter
    for (int c = lane; c < mp; c += 32) { qs[c] = 0.f; xs[c] = 0.f; }
    if (lane < lp) { Us[lane] = 0.f; R0[lane] = 0.f; }
    if (gnull && lane < 2) gnull[2 * t + lane] = 0.f;
    return;
  }
  // gamma = 0: (B-hat g_n)_t = -sum over unseeded neighbours j of c_ij g_j, g = sq / ||sq||
  float bnull = 0.f;
  // X row = -sum over unseeded neighbours j of c_ij q_j, kept in registers (mp <= 224)
  const float* qi = Q + (int64_t)i * ldq;
  float acc[7], own[7];
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    const int c = lane + 32 * q;
    own[q] = c < mp ? qi[c] : 0.f;
    acc[q] = 0.f;
  }
  float r0 = 0.f;  // lane k accumulates column k of L-hat_s U-hat_s
  const float diag = normalized ? 1.f : d[i];
  if (lane == k0) r0 = diag * sq[i];
  auto visit = [&](int64_t j, float c, int lj) {
    if (lj < 0) {
      const float* qj = Q + j * ldq;
#pragma unroll
      for (int q = 0; q < 7; ++q) {
        const int cc = lane + 32 * q;
        if (cc < mp) acc[q] = fmaf(-c, qj[cc], acc[q]);
      }
      if (gnull) bnull -= c * sq[j];
    } else if (lane == lj) {
      r0 -= c * sq[j];
    }
  };
  if (kind == RW_GRAPH_GRID) {
    // all neighbours' indices, coefficients and labels first (independent loads)
    const int x = i % DX, y = (i / DX) % DY, z = i / (DX * DY);
    const int64_t st[3] = {1, (int64_t)DX, (int64_t)DX * DY};
    const int cc3[3] = {x, y, z};
    const int n3[3] = {DX, DY, DZ};
    int64_t nj[6];
    float nc[6];
    int nl[6];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const bool lo = a < ndim && cc3[a] > 0, hi = a < ndim && cc3[a] + 1 < n3[a];
      nj[2 * a] = lo ? i - st[a] : -1;
      nj[2 * a + 1] = hi ? i + st[a] : -1;
      nc[2 * a] = lo ? cw[a * N + i - st[a]] : 0.f;
      nc[2 * a + 1] = hi ? cw[a * N + i] : 0.f;
    }
    // the neighbours' rows of Q and d^{1/2} are requested together with their labels (one
    // round trip); a seeded neighbour's row is then dropped
    float qn[6][7], sn[6];
#pragma unroll
    for (int u = 0; u < 6; ++u) {
      nl[u] = nj[u] >= 0 ? seedlab[nj[u]] : -2;
      sn[u] = nj[u] >= 0 ? sq[nj[u]] : 0.f;
      const float* qj = Q + (nj[u] >= 0 ? nj[u] : 0) * ldq;
#pragma unroll
      for (int q = 0; q < 7; ++q) {
        const int cc = lane + 32 * q;
        qn[u][q] = (nj[u] >= 0 && cc < mp) ? qj[cc] : 0.f;
      }
    }
#pragma unroll
    for (int u = 0; u < 6; ++u) {
      if (nj[u] < 0) continue;
      if (nl[u] < 0) {
#pragma unroll
        for (int q = 0; q < 7; ++q) acc[q] = fmaf(-nc[u], qn[u][q], acc[q]);
        bnull -= nc[u] * sn[u];
      } else if (lane == nl[u]) {
        r0 -= nc[u] * sn[u];
      }
    }
  } else {
    for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) visit(colv[p], ccsr[p], seedlab[colv[p]]);
  }
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    const int c = lane + 32 * q;
    if (c < mp) { qs[c] = own[q]; xs[c] = acc[q]; }
  }
  // a fixed-m solve on a wider basis: the columns past 224 are never read (m <= 224)
  for (int c = 224 + lane; c < mp; c += 32) { qs[c] = 0.f; xs[c] = 0.f; }
  if (lane < lp) {
    float u = (lane == k0) ? sq[i] : 0.f;
    Us[lane] = u;
    R0[lane] = (lane < L) ? r0 + gamma * u : 0.f;
  }
  if (gnull && lane == 0) {
    gnull[2 * t] = sq[i] * ginv;
    gnull[2 * t + 1] = bnull * ginv;
  }
}

// ---------------------------------------------------------------------------------------
// Shared-memory FP32 dense kernels for one CTA (row stride ms, odd, so column walks are free
// of bank conflicts).
// ---------------------------------------------------------------------------------------
// A[i][j] -= sum_{q < kb} A[i][p0 + q] A[p0 + q][j] for i in [r1, m), j in [r1, ncol): warp tasks
// of 8 rows x 128 columns (lane = column within each 32-column group), k unrolled by 2 for ILP
__device__ void gemm_trailing(float* A, int ms, int m, int ncol, int r1, int p0, int kb) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int n = m - r1, nc = ncol - r1;
  const int nrt = (n + 7) / 8, nct = (nc + 127) / 128;
  for (int task = warp; task < nrt * nct; task += nw) {
    const int i0 = r1 + 8 * (task / nct), j0 = r1 + 128 * (task % nct) + lane;
    float acc[8][4];
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[u][v] = 0.f;
    const int ilast = m - 1;
#pragma unroll 2
    for (int q = 0; q < kb; ++q) {
      float av[8], bv[4];
#pragma unroll
      for (int u = 0; u < 8; ++u) av[u] = A[min(i0 + u, ilast) * ms + p0 + q];
#pragma unroll
      for (int v = 0; v < 4; ++v) bv[v] = A[(p0 + q) * ms + min(j0 + 32 * v, ncol - 1)];
#pragma unroll
      for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(av[u], bv[v], acc[u][v]);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const int i = i0 + u, j = j0 + 32 * v;
        if (i < m && j < ncol) A[i * ms + j] -= acc[u][v];
      }
  }
}

// A[i][j] -= sum_{q < 32} A[i][p0 + q] A[p0 + q][j] for i in [i0, i1), j in [j0, j1), for a row
// stride that is a multiple of 4 and p0, j0 multiples of 4: both operands move as 16-byte
// loads.  A warp task covers RU (32 / LC) rows x 4 LC columns: lane (lr = lane / LC,
// lc = lane % LC) owns rows ib + lr RU + u and the four columns jb + 4 lc ..; per four steps of
// q, RU loads of the row operand and four of the column operand feed 16 RU FMAs.
template <int RU, int LC>
__device__ void gemm4(float* A, int ms, int i0, int i1, int j0, int j1, int p0) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  constexpr int TR = RU * (32 / LC), TC = 4 * LC;
  const int n = i1 - i0, nc = j1 - j0;
  if (n <= 0 || nc <= 0) return;
  const int nrt = (n + TR - 1) / TR, nct = (nc + TC - 1) / TC;
  const int lr = lane / LC, lc = lane % LC;
  for (int task = warp; task < nrt * nct; task += nw) {
    const int ib = i0 + TR * (task / nct) + RU * lr, jb = j0 + TC * (task % nct) + 4 * lc;
    const int jl = min(jb, j1 - 1) & ~3;  // loads stay inside the row (ms >= round_up(j1, 4))
    float acc[RU][4];
#pragma unroll
    for (int u = 0; u < RU; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[u][v] = 0.f;
    const float* brow = A + (size_t)p0 * ms + jl;
    for (int q4 = 0; q4 < 8; ++q4) {
      float4 av[RU], bv[4];
#pragma unroll
      for (int u = 0; u < RU; ++u)
        av[u] = *reinterpret_cast<const float4*>(A + (size_t)min(ib + u, i1 - 1) * ms + p0 + 4 * q4);
#pragma unroll
      for (int qq = 0; qq < 4; ++qq)
        bv[qq] = *reinterpret_cast<const float4*>(brow + (size_t)(4 * q4 + qq) * ms);
#pragma unroll
      for (int u = 0; u < RU; ++u) {
        const float a4[4] = {av[u].x, av[u].y, av[u].z, av[u].w};
#pragma unroll
        for (int qq = 0; qq < 4; ++qq) {
          acc[u][0] = fmaf(a4[qq], bv[qq].x, acc[u][0]);
          acc[u][1] = fmaf(a4[qq], bv[qq].y, acc[u][1]);
          acc[u][2] = fmaf(a4[qq], bv[qq].z, acc[u][2]);
          acc[u][3] = fmaf(a4[qq], bv[qq].w, acc[u][3]);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < RU; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const int i = ib + u, j = jb + v;
        if (i < i1 && j < j1) A[(size_t)i * ms + j] -= acc[u][v];
      }
  }
}

// row stride of the LU CTA's matrix: a multiple of 4 (16-byte rows) that is an odd multiple of
// 4, so that column walks meet at most 4-way bank conflicts
__host__ __device__ inline int lu_stride(int m) {
  int s = (m + 3) / 4 * 4;
  if ((s / 4) % 2 == 0) s += 4;
  return s;
}

// one warp: U x = y for the upper factor held in A (uinv = 1 / diag(U)), one register group of
// 32 rows at a time.  Lane t keeps entries t + 32 q (m <= 224) in registers; each newly final
// entry is broadcast by shuffle.  The register group of the pivot is a compile-time index, so a
// step is one shuffle and a few independent FMAs.
template <int QI>
__device__ __forceinline__ void lu_bwd_group(const float* A, int m, int ms, const float* uinv,
                                             float (&y)[7], int lane) {
  if (32 * QI < m) {
    for (int li = min(31, m - 1 - 32 * QI); li >= 0; --li) {
      const int i = 32 * QI + li;
      const float xi = __shfl_sync(0xffffffff, y[QI], li) * uinv[i];
      if (lane == li) y[QI] = xi;
#pragma unroll
      for (int q = 0; q <= QI; ++q) {
        const int j = lane + 32 * q;
        if (j < i) y[q] = fmaf(-A[j * ms + i], xi, y[q]);
      }
    }
  }
}
// ---------------------------------------------------------------------------------------
// Compact single-warp factorizations of a 32 x 32 diagonal block.  Lane r keeps the not yet
// final part of row r in registers, shifted so that a[0] is always the current column: one
// step is a rank-1 update fused with the shift a[t] <- a[t + 1] - f b[t], b the broadcast
// column (or row) in shared memory read with 16-byte loads.  The step loop stays rolled (the
// kernels run once per launch on one SM, where code size costs more than loop overhead) and
// every register index is a constant.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void load_bcast(float4 (&v)[8], const float* b) {
#pragma unroll
  for (int t4 = 0; t4 < 8; ++t4) v[t4] = reinterpret_cast<const float4*>(b)[t4];
}
// a[t] <- a[t + 1] - f v[t] with the broadcast vector already in registers (its loads are
// issued before the scalar chain that produces f)
__device__ __forceinline__ void shift_update_r(float (&a)[32], float f, const float4 (&v)[8]) {
#pragma unroll
  for (int t4 = 0; t4 < 8; ++t4) {
    a[4 * t4 + 0] = fmaf(-f, v[t4].x, a[4 * t4 + 1]);
    a[4 * t4 + 1] = fmaf(-f, v[t4].y, a[4 * t4 + 2]);
    a[4 * t4 + 2] = fmaf(-f, v[t4].z, a[4 * t4 + 3]);
    a[4 * t4 + 3] = (t4 < 7) ? fmaf(-f, v[t4].w, a[4 * t4 + 4]) : 0.f;
  }
}

// Cholesky of the kb x kb diagonal block at (k0, k0), kb <= 32, by one warp.  buf: 128 floats,
// 16-byte aligned (two halves: the column below the pivot at [0, 32), the pivot at [32]).
// Every lane forms 1 / sqrt(pivot) beside the elimination (it only feeds the stores), so the
// entries of L are written final at their step.  On return the block holds L (lower, diagonal
// included) and dinv[0..kb) = 1 / L_cc.
__device__ void chol_diag_rot(float* A, int ms, int k0, int kb, float* dinv, float* buf, int* bad) {
  const int lane = threadIdx.x & 31;
  const bool live = lane < kb;
  float* row = A + (size_t)(k0 + (live ? lane : 0)) * ms + k0;
  float a[32];
#pragma unroll
  for (int c = 0; c < 32; ++c) {
    float v = (c == lane) ? 1.f : 0.f;
    if (live && c <= lane) v = row[c];
    a[c] = v;
  }
  for (int kk = 0; kk < kb; ++kk) {
    // every lane stores: a_lane,kk below the pivot at [lane - kk - 1], the pivot at [32], lanes
    // above it into the unused slots [33 + lane]
    float* b = buf + 64 * (kk & 1);
    b[lane > kk ? lane - kk - 1 : (lane == kk ? 32 : 33 + lane)] = a[0];
    __syncwarp();
    float d = b[32];
    float4 v[8];
    load_bcast(v, b);
    if (!(d > 0.f)) {
      if (lane == kk) *bad = 1;
      d = 1e-30f;
    }
    const float f = __fdividef(a[0], d);
    const float ri = rsqrtf(d);
    // L_lane,kk = a_lane,kk / sqrt(d) (the pivot lane writes sqrt(d)); lanes above the pivot
    // write into the block's unused upper triangle
    if (live) row[kk] = a[0] * ri;
    if (lane == kk) dinv[kk] = ri;
    shift_update_r(a, f, v);
  }
  __syncwarp();
}

// LU without pivoting of the kb x kb diagonal block at (k0, k0) by one warp: unit-lower
// multipliers below the diagonal, U on and above it; uinv[k0 + c] = 1 / U_cc.  Row kk is
// broadcast from lane kk by shuffles (one per register of the shifted row).  Also writes the
// shifted copies used by the panel solves: Ush[c][t] = U_c,c+1+t and Lsh[c][t] = L_c+1+t,c
// (32 x 32 each, zero outside the block).  A pivot below 1e-3 dref (the original row scale) sets
// *unstable (no check when dref is null; a zero pivot is replaced by 1e-30 either way).
__device__ void lu_diag_rot(float* A, int ms, int k0, int kb, float* buf, const float* dref,
                            float* uinv, float* Ush, float* Lsh, int* unstable) {
  const int lane = threadIdx.x & 31;
  const bool live = lane < kb;
  float* row = A + (size_t)(k0 + (live ? lane : 0)) * ms + k0;
  float a[32];
#pragma unroll
  for (int c = 0; c < 32; ++c) {
    float v = (c == lane) ? 1.f : 0.f;
    if (live) v = (c < kb) ? row[c] : 0.f;
    a[c] = v;
  }
#pragma unroll
  for (int t = 0; t < 32; ++t) Lsh[lane * 32 + t] = 0.f;
  for (int kk = 0; kk < kb; ++kk) {
    // the pivot lane publishes its row shifted by one (U_kk,kk+1+t at b[t]) and the pivot
    float* b = buf + 64 * (kk & 1);
    if (lane == kk) {
#pragma unroll
      for (int t4 = 0; t4 < 8; ++t4)
        reinterpret_cast<float4*>(b)[t4] =
            make_float4(a[4 * t4 + 1], a[4 * t4 + 2], a[4 * t4 + 3], t4 < 7 ? a[4 * t4 + 4] : 0.f);
      b[32] = a[0];
    }
    __syncwarp();
    float u = b[32];
    float4 v[8];
    load_bcast(v, b);
    if (dref && !(fabsf(u) >= 1e-3f * dref[k0 + kk]) && lane == 0) *unstable = 1;
    if (u == 0.f) u = 1e-30f;
    if (lane > kk) {
      const float f = __fdividef(a[0], u);
      if (live) {
        row[kk] = f;
        Lsh[kk * 32 + lane - kk - 1] = f;
      }
      shift_update_r(a, f, v);  // rows above and at the pivot keep their U rows
    }
  }
  __syncwarp();
  // lane r stopped shifting at step r: a[t] = U_r,r+t
#pragma unroll
  for (int t = 0; t < 32; ++t) Ush[lane * 32 + t] = 0.f;
  __syncwarp();
  if (live) {
#pragma unroll
    for (int t = 0; t < 32; ++t) {
      if (t < kb - lane) {
        row[lane + t] = a[t];
        if (t > 0) Ush[lane * 32 + t - 1] = a[t];
      }
    }
    uinv[k0 + lane] = 1.f / (a[0] == 0.f ? 1e-30f : a[0]);
  }
  __syncwarp();
}

// LU without pivoting of the kb x kb diagonal block at (k0, k0) by one warp, branch-free steps:
// lane r keeps row r in shifted registers; at step kk the pivot lane publishes its row (shifted
// by one) and the pivot through shared memory, every lane stores one entry of that U row into
// A, the lanes below write their multiplier, and every lane runs the shifted update (rows at or
// above the pivot only produce values that are never stored).  uinv[k0 + c] = 1 / U_cc; a zero
// pivot is replaced by 1e-30.  buf: 128 floats, 16-byte aligned.
__device__ void lu_diag_warp(float* A, int ms, int k0, int kb, float* buf, float* uinv) {
  const int lane = threadIdx.x & 31;
  const bool live = lane < kb;
  float* row = A + (size_t)(k0 + (live ? lane : 0)) * ms + k0;
  float a[32];
#pragma unroll
  for (int c = 0; c < 32; ++c) a[c] = (live && c < kb) ? row[c] : (c == lane ? 1.f : 0.f);
  for (int kk = 0; kk < kb; ++kk) {
    float* b = buf + 64 * (kk & 1);
    if (lane == kk) {
#pragma unroll
      for (int t4 = 0; t4 < 8; ++t4)
        reinterpret_cast<float4*>(b)[t4] =
            make_float4(a[4 * t4 + 1], a[4 * t4 + 2], a[4 * t4 + 3], t4 < 7 ? a[4 * t4 + 4] : 0.f);
      b[32] = a[0];
    }
    __syncwarp();
    float u = b[32];
    float4 v[8];
    load_bcast(v, b);
    if (u == 0.f) u = 1e-30f;
    const float ru = 1.f / u;
    // U_kk,kk+1+lane from the published row; the pivot itself by lane 0
    float* urow = A + (size_t)(k0 + kk) * ms + k0 + kk;
    if (lane + kk + 1 < kb) urow[1 + lane] = b[lane];
    if (lane == 0) { urow[0] = b[32]; uinv[k0 + kk] = ru; }
    const float f = a[0] * ru;
    if (live && lane > kk) row[kk] = f;  // multiplier L_lane,kk
    shift_update_r(a, f, v);
  }
  __syncwarp();
}

// ---------------------------------------------------------------------------------------
// Triangular solves of 32-row (32-column) panels on 128 threads: thread t keeps eight entries
// of row (or column) t / 4, the quarter t % 4, in registers, so a step is eight FMAs per
// thread; the value that every row needs comes by a shuffle inside the row's four lanes.  The
// step loop runs over the owning quarter (rolled) and the entry inside it (unrolled), so every
// register index is a constant.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void unpack8(const float4& v0, const float4& v1, float (&p)[8]) {
  p[0] = v0.x; p[1] = v0.y; p[2] = v0.z; p[3] = v0.w;
  p[4] = v1.x; p[5] = v1.y; p[6] = v1.z; p[7] = v1.w;
}

// Rows r0 .. r0 + nr of the 32 columns at c0 times U^{-1} (U the block at (c0, c0)): threads
// tb .. tb + 127, four per row.  U32[c][col] = U_c,col for col > c, else 0; ui = 1 / diag(U).
__device__ void trsm_rows_128(float* A, int ms, int r0, int nr, int c0, const float* U32,
                              const float* ui, int tb) {
  const int t = threadIdx.x - tb, r = t >> 2, g = t & 3, src = (t & 31) & ~3;
  const bool live = r < nr;
  float* row = A + (size_t)(r0 + (live ? r : 0)) * ms + c0 + 8 * g;
  float a[8], uv[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    a[q] = live ? row[q] : 0.f;
    uv[q] = ui[c0 + 8 * g + q];
  }
  for (int go = 0; go < 4; ++go) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int c = 8 * go + j;
      float w[8];
      unpack8(reinterpret_cast<const float4*>(U32 + c * 32)[2 * g],
              reinterpret_cast<const float4*>(U32 + c * 32)[2 * g + 1], w);
      const float x = __shfl_sync(0xffffffff, a[j] * uv[j], src | go);
      if (g == go) a[j] = x;
#pragma unroll
      for (int q = 0; q < 8; ++q) a[q] = fmaf(-x, w[q], a[q]);  // zero where col <= c
    }
  }
  if (live) {
#pragma unroll
    for (int q = 0; q < 8; ++q) row[q] = a[q];
  }
}

// Columns r0 .. r0 + nc of the 32 rows at c0 premultiplied by L^{-1} (L unit lower, the block at
// (c0, c0)): threads tb .. tb + 127, four per column.  L32T[r][row] = L_row,r for row > r, else 0.
__device__ void trsm_cols_128(float* A, int ms, int r0, int nc, int c0, const float* L32T, int tb) {
  const int t = threadIdx.x - tb, cc = t >> 2, g = t & 3, src = (t & 31) & ~3;
  const bool live = cc < nc;
  float* col = A + (size_t)(c0 + 8 * g) * ms + r0 + (live ? cc : 0);
  float a[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) a[q] = live ? col[(size_t)q * ms] : 0.f;
  for (int go = 0; go < 4; ++go) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int rr = 8 * go + j;
      float l[8];
      unpack8(reinterpret_cast<const float4*>(L32T + rr * 32)[2 * g],
              reinterpret_cast<const float4*>(L32T + rr * 32)[2 * g + 1], l);
      const float y = __shfl_sync(0xffffffff, a[j], src | go);
#pragma unroll
      for (int q = 0; q < 8; ++q) a[q] = fmaf(-y, l[q], a[q]);  // zero where row <= rr
    }
  }
  if (live) {
#pragma unroll
    for (int q = 0; q < 8; ++q) col[(size_t)q * ms] = a[q];
  }
}

// x = a U^{-1} for one row a (kb entries at ar), U the block whose shifted rows are in Ush and
// whose reciprocal diagonal is ui (right-looking, shifted registers)
__device__ __forceinline__ void trsm_row_rot(float* ar, int kb, const float* Ush, const float* ui) {
  float a[32];
#pragma unroll
  for (int c = 0; c < 32; ++c) a[c] = c < kb ? ar[c] : 0.f;
  for (int c = 0; c < kb; ++c) {
    float4 v[8];
    load_bcast(v, Ush + c * 32);
    const float x = a[0] * ui[c];
    ar[c] = x;
    shift_update_r(a, x, v);
  }
}

// y = L^{-1} a for one column a (kb entries, stride ms, at ac), L unit lower with shifted
// columns in Lsh
__device__ __forceinline__ void trsm_col_rot(float* ac, int ms, int kb, const float* Lsh) {
  float a[32];
#pragma unroll
  for (int r = 0; r < 32; ++r) a[r] = r < kb ? ac[r * ms] : 0.f;
  for (int r = 0; r < kb; ++r) {
    float4 v[8];
    load_bcast(v, Lsh + r * 32);
    const float y = a[0];
    ac[r * ms] = y;
    shift_update_r(a, y, v);
  }
}

// Cholesky of the kb x kb diagonal block at (k0, k0) by the whole CTA in shared memory.  Step
// kk uses the unscaled column (l_r l_c = a_r,kk a_c,kk / a_kk,kk), so one barrier per step
// suffices; the column scaling and the square roots follow in one pass.  dinv[0..kb) receives
// the reciprocals of the diagonal of L.
__device__ void chol_diag_block_cta(float* A, int ms, int k0, int kb, float* dinv, int* bad) {
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5, nty = blockDim.x >> 5;
  float* T = A + k0 * ms + k0;
  for (int kk = 0; kk < kb; ++kk) {
    float piv = T[kk * ms + kk];
    if (!(piv > 0.f)) piv = 1e-30f;
    const float inv = 1.f / piv;
    for (int r = kk + 1 + ty; r < kb; r += nty) {
      const int c = kk + 1 + tx;
      if (c <= r) T[r * ms + c] = fmaf(-T[r * ms + kk] * inv, T[c * ms + kk], T[r * ms + c]);
    }
    __syncthreads();
  }
  if (threadIdx.x < kb) {
    float piv = T[threadIdx.x * ms + threadIdx.x];
    if (!(piv > 0.f)) { *bad = 1; piv = 1e-30f; }
    const float d = sqrtf(piv);
    dinv[threadIdx.x] = 1.f / d;
  }
  __syncthreads();
  for (int r = ty; r < kb; r += nty) {
    const int c = tx;
    if (c < r) T[r * ms + c] *= dinv[c];
    else if (c == r) T[r * ms + c] = 1.f / dinv[c];
  }
  __syncthreads();
}

// Blocked right-looking Cholesky A = L L^T (lower, in place), 32-column panels.
__device__ bool chol_lower_smem(float* A, int m, int ms) {
  __shared__ int bad;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  if (tid == 0) bad = 0;
  __syncthreads();
  for (int k0 = 0; k0 < m; k0 += 32) {
    const int kb = min(32, m - k0);
    __shared__ float dloc[32];
    chol_diag_block_cta(A, ms, k0, kb, dloc, &bad);
    // L21 = A21 L11^{-T}: one thread per row below the panel
    for (int r = k0 + kb + tid; r < m; r += blockDim.x) {
      float* ar = A + r * ms + k0;
      for (int j = 0; j < kb; ++j) {
        const float* lj = A + (k0 + j) * ms + k0;
        float s = ar[j];
        for (int t = 0; t < j; ++t) s = fmaf(-ar[t], lj[t], s);
        ar[j] = s / lj[j];
      }
    }
    __syncthreads();
    // A22 -= L21 L21^T (lower): a warp per row, lanes over columns
    const int r0 = k0 + kb;
    for (int i = r0 + warp; i < m; i += nw) {
      const float* li = A + i * ms + k0;
      for (int j = r0 + lane; j <= i; j += 32) {
        const float* lj = A + j * ms + k0;
        float s = 0.f;
        for (int t = 0; t < kb; ++t) s = fmaf(li[t], lj[t], s);
        A[i * ms + j] -= s;
      }
    }
    __syncthreads();
  }
  return bad == 0;
}

// one warp: L z = b (forward, column-oriented: after z_i is known, every later entry is
// updated in parallel).  b and z may alias.
__device__ void fwd_lower_warp(const float* A, int m, int ms, const float* b, float* z) {
  const int lane = threadIdx.x & 31;
  for (int i = lane; i < m; i += 32) z[i] = b[i];
  __syncwarp();
  for (int i = 0; i < m; ++i) {
    const float zi = z[i] / A[i * ms + i];
    __syncwarp();
    if (lane == 0) z[i] = zi;
    for (int j = i + 1 + lane; j < m; j += 32) z[j] = fmaf(-A[j * ms + i], zi, z[j]);
    __syncwarp();
  }
}

// one warp: L^T x = z with the reciprocals of diag(L) given; lane t keeps x[t + 32 q] in
// registers (m <= 224), the newly final x_i is broadcast by shuffle; the register group of x_i
// is a compile-time index
template <int QI>
__device__ __forceinline__ void ltsolve_group(const float* __restrict__ A, int m, int ms,
                                              const float* __restrict__ dinv, float (&xr)[7],
                                              int lane) {
  if (32 * QI < m) {
    for (int li = min(31, m - 1 - 32 * QI); li >= 0; --li) {
      const int i = 32 * QI + li;
      const float xi = __shfl_sync(0xffffffff, xr[QI], li) * dinv[i];
      if (lane == li) xr[QI] = xi;
      const float* ai = A + i * ms;
#pragma unroll
      for (int q = 0; q <= QI; ++q) {
        const int j = lane + 32 * q;
        if (j < i) xr[q] = fmaf(-ai[j], xi, xr[q]);
      }
    }
  }
}
__device__ void bwd_lowerT_warp_reg(const float* __restrict__ A, int m, int ms,
                                    const float* __restrict__ dinv, const float* z, float* x) {
  const int lane = threadIdx.x & 31;
  float xr[7];
#pragma unroll
  for (int q = 0; q < 7; ++q) xr[q] = (lane + 32 * q < m) ? z[lane + 32 * q] : 0.f;
  ltsolve_group<6>(A, m, ms, dinv, xr, lane);
  ltsolve_group<5>(A, m, ms, dinv, xr, lane);
  ltsolve_group<4>(A, m, ms, dinv, xr, lane);
  ltsolve_group<3>(A, m, ms, dinv, xr, lane);
  ltsolve_group<2>(A, m, ms, dinv, xr, lane);
  ltsolve_group<1>(A, m, ms, dinv, xr, lane);
  ltsolve_group<0>(A, m, ms, dinv, xr, lane);
#pragma unroll
  for (int q = 0; q < 7; ++q)
    if (lane + 32 * q < m) x[lane + 32 * q] = xr[q];
  __syncwarp();
}

// one warp: L^T x = z (backward, column-oriented).  z and x may alias.
__device__ void bwd_lowerT_warp(const float* A, int m, int ms, const float* z, float* x) {
  const int lane = threadIdx.x & 31;
  for (int i = lane; i < m; i += 32) x[i] = z[i];
  __syncwarp();
  for (int i = m - 1; i >= 0; --i) {
    const float xi = x[i] / A[i * ms + i];
    __syncwarp();
    if (lane == 0) x[i] = xi;
    for (int j = lane; j < i; j += 32) x[j] = fmaf(-A[i * ms + j], xi, x[j]);
    __syncwarp();
  }
}

__device__ void load_shifted_gram(float* A, int m, int ms, const float* G, int ldg, float mu) {
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5, nty = blockDim.x >> 5;
  for (int i = ty; i < m; i += nty)
    for (int j = tx; j <= i; j += 32)
      A[i * ms + j] = G[(int64_t)i * ldg + j] + (i == j ? mu : 0.f);
}

// f_k = || Q_s^{(m)} alpha_k - u_k ||^2 over the seeds: a warp per seed row (lanes over the
// columns), all labels at once; result in fk[0..L)
__device__ void seed_residuals(const float* __restrict__ Qs, int ldq, const float* __restrict__ Us,
                               int ldu, int S, int L, int m, const float* al, float* fk, int alm) {
  // f_k = || Q_s^{(m)} alpha_k - u_k ||^2 over the seeds.  A warp takes 4 seeds at a time
  // (lanes over the columns), labels in groups of 4; the 16 (seed, label) dot products are
  // reduced across the warp by a reduce-scatter butterfly (even lane 2j holds sum j).
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __shared__ float wf[8 * RW_MAX_LABELS];  // per-warp sums (8 warps), added in warp order
  if (threadIdx.x < 8 * RW_MAX_LABELS) wf[threadIdx.x] = 0.f;
  __syncthreads();
  for (int k0 = 0; k0 < L; k0 += 4) {
    float acc = 0.f;  // lane 2j accumulates the squared residuals of entry j = 4 q + t
    for (int s0 = 4 * warp; s0 < S; s0 += 4 * nw) {
      float val[16];
#pragma unroll
      for (int e = 0; e < 16; ++e) val[e] = 0.f;
      for (int j = lane; j < m; j += 32) {
        float a[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) a[t] = (k0 + t < L) ? al[(k0 + t) * alm + j] : 0.f;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float qj = (s0 + q < S) ? Qs[(int64_t)(s0 + q) * ldq + j] : 0.f;
#pragma unroll
          for (int t = 0; t < 4; ++t) val[4 * q + t] = fmaf(qj, a[t], val[4 * q + t]);
        }
      }
#pragma unroll
      for (int half = 8, off = 16; half >= 1; half >>= 1, off >>= 1) {
        const bool up = (lane & off) != 0;
#pragma unroll
        for (int t = 0; t < half; ++t) {
          const float send = up ? val[t] : val[t + half];
          const float keep = up ? val[t + half] : val[t];
          val[t] = keep + __shfl_xor_sync(0xffffffff, send, off);
        }
      }
      const float sum = val[0] + __shfl_xor_sync(0xffffffff, val[0], 1);
      const int jj = lane >> 1, q = jj >> 2, t = jj & 3;
      if ((lane & 1) == 0 && s0 + q < S && k0 + t < L) {
        const float r = sum - Us[(int64_t)(s0 + q) * ldu + k0 + t];
        acc = fmaf(r, r, acc);
      }
    }
    // lanes 2j with j % 4 == t hold label k0 + t
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      float v = ((lane & 1) == 0 && ((lane >> 1) & 3) == t) ? acc : 0.f;
      v = warp_sum(v);
      if (lane == 0 && k0 + t < L) wf[warp * RW_MAX_LABELS + k0 + t] = v;
    }
  }
  __syncthreads();
  if (threadIdx.x < L) {
    float v = 0.f;
    for (int w = 0; w < nw; ++w) v += wf[w * RW_MAX_LABELS + threadIdx.x];
    fk[threadIdx.x] = v;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------------------
// [K | G | h | b] = Q_s^T [X | Q_s | r0 | U-hat_s] in FP32.  64 x 64 output tiles; the S seed
// rows are split over the CTAs of a thread-block cluster along z.  Each CTA keeps its partial
// tile in shared memory, and the rank-0 CTA of the cluster adds the partials in rank order
// through distributed shared memory, so the sums have a fixed order.  (S is a few thousand at
// most, so FP32 partial sums over S / cluster rows are accurate to a few ulps of the result.)
// ---------------------------------------------------------------------------------------
constexpr int kSgT = 64, kSgRows = 128, kSgMaxCluster = 8;

__global__ void __launch_bounds__(256)
k_seed_gram(const float* __restrict__ A, int lda, const float* __restrict__ B, int ldb, int S,
            int p, int q, float* __restrict__ Gout, int ldg) {
  rw_grid_wait();
  rw_grid_trigger();
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ float4 stage4[];          // As[kSgRows][17] | Bs[kSgRows][17] (float4)
  __shared__ float4 part[kSgT * kSgT / 4];
  float4* As = stage4;
  float4* Bs = stage4 + kSgRows * 17;
  const int i0 = blockIdx.x * kSgT, j0 = blockIdx.y * kSgT;
  const int nz = gridDim.z, rank = (int)cluster.block_rank();
  const int rpc = (S + nz - 1) / nz;
  const int r0 = rank * rpc, r1 = min(S, r0 + rpc);
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  float acc[4][4] = {};
  for (int k0 = r0; k0 < r1; k0 += kSgRows) {
    // the whole stage (kSgRows rows of the two 64-column tiles) requested at once (cp.async,
    // zero-filled outside the rows / columns), one round trip before one barrier
    for (int e = threadIdx.x; e < kSgRows * 16; e += 256) {
      const int kk = e / 16, c4 = e % 16;
      const int r = k0 + kk;
      const bool rin = r < r1;
      const bool ain = rin && i0 + 4 * c4 < p, bin = rin && j0 + 4 * c4 < q;
      cp_async16_zfill(As + kk * 17 + c4, ain ? A + (int64_t)r * lda + i0 + 4 * c4 : A, ain);
      cp_async16_zfill(Bs + kk * 17 + c4, bin ? B + (int64_t)r * ldb + j0 + 4 * c4 : B, bin);
    }
    cp_async_wait_all();
    __syncthreads();
    const int kn = min(kSgRows, r1 - k0);
#pragma unroll 4
    for (int kk = 0; kk < kn; ++kk) {
      const float4 av = As[kk * 17 + ty], bv = Bs[kk * 17 + tx];
      const float a[4] = {av.x, av.y, av.z, av.w}, b[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(a[u], b[v], acc[u][v]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
    part[(ty * 4 + u) * 16 + tx] = make_float4(acc[u][0], acc[u][1], acc[u][2], acc[u][3]);
  cluster.sync();
  // every rank sums its share of the tile's float4 entries over the ranks, in rank order
  const int per = (kSgT * kSgT / 4 + nz - 1) / nz;
  const int e0 = rank * per, e1 = min(kSgT * kSgT / 4, e0 + per);
  for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    float4 v[kSgMaxCluster];
#pragma unroll
    for (int r = 0; r < kSgMaxCluster; ++r)
      if (r < nz) v[r] = cluster.map_shared_rank(part, r)[e];
    float4 sum = v[0];
#pragma unroll
    for (int r = 1; r < kSgMaxCluster; ++r)
      if (r < nz) { sum.x += v[r].x; sum.y += v[r].y; sum.z += v[r].z; sum.w += v[r].w; }
    const int row = e / 16, c4 = e % 16;   // part[(ty * 4 + u) * 16 + tx]: row ty * 4 + u
    const int i = i0 + row;
    const float vals[4] = {sum.x, sum.y, sum.z, sum.w};
    if (i < p)
#pragma unroll
      for (int w = 0; w < 4; ++w) {
        const int j = j0 + c4 * 4 + w;
        if (j < q) Gout[(int64_t)i * ldg + j] = vals[w];
      }
  }
  cluster.sync();  // the peers' partial tiles stay alive until every rank has read them
}

// ---------------------------------------------------------------------------------------
// Adaptive m (Sec. III-A-1, Eq. alpha_1) in one CTA of 256 threads:
//   f_k(m) = min_{||a|| <= rho} || Q_s^{(m)} a - u_k ||^2,  candidates m = m_step, 2 m_step, ...
// The candidates are nested, so the Cholesky factor of G + mu0 I (G = Q_s^T Q_s, mu0 = 1e-6
// tr G / m_max) and z_k = L^{-1} b_k (b = Q_s^T U-hat_s) are grown 32 rows at a time
// (left-looking, "add eigenvectors and repeat") and stop at the first candidate whose worst
// label passes the unconstrained test f = ||u_k||^2 - ||z_k[:m]||^2 <= f_max.  That candidate
// is then checked exactly: a_k = L_m^{-T} z_k[:m] and f_k = ||u_k||^2 - ||z_k||^2 - mu0 ||a_k||^2,
// which is the squared residual ||Q_s a_k - u_k||^2 (a^T (G + mu0 I) a = z^T z = b^T a).  If
// some ||a_k|| > rho the constrained minimum can only be larger, and the
// trust-region solution (Newton on 1/||a(mu)|| - 1/rho, a Cholesky of G_m + mu I per step) is
// computed for it and, if it fails, for the following candidates.
// ---------------------------------------------------------------------------------------
// hint_remote / final_remote (null when the CTA runs alone): mailboxes in the shared memory of
// the LU CTA of the cluster, told the first passing candidate as soon as it is found and the
// final m at the end
template <int LP>
__device__ void adapt_body(const float* __restrict__ G, int ldg, const float* __restrict__ bv,
                           int ldb, const float* __restrict__ Qs, int ldq,
                           const float* __restrict__ Us, int ldu, int S, int L, int mmax,
                           int mstep, double rho, double fmax, int* __restrict__ mdev,
                           double* __restrict__ fsel, int* hint_remote, int* final_remote) {
  extern __shared__ float sm[];
  const int ms = mmax | 1;
  float* A = sm;                          // mmax x ms, lower factor
  float* z = A + (size_t)mmax * ms;       // L x mmax
  float* bb = z + (size_t)L * mmax;       // L x mmax
  float* al = bb + (size_t)L * mmax;      // L x mmax
  __shared__ float ck[RW_MAX_LABELS], zz[RW_MAX_LABELS], fk[RW_MAX_LABELS], nk[RW_MAX_LABELS];
  __shared__ float wpart[8 * RW_MAX_LABELS + 8];  // per-warp partial sums (8 warps)
  __shared__ float dinv[kMaxSmallM];  // reciprocals of diag(L)
  __shared__ __align__(16) float colbuf[128];
  __shared__ float mu0s, red;
  __shared__ int chosen, bad, done, capped;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const int ncand = (mmax + mstep - 1) / mstep;
  auto cand_m = [&](int c) { return min((c + 1) * mstep, mmax); };
  // ||u_k||^2, mu0, right-hand sides
  if (tid < RW_MAX_LABELS) { ck[tid] = 0.f; zz[tid] = 0.f; }
  if (tid == 0) { chosen = -1; bad = 0; done = 0; capped = 0; }
  __syncthreads();
  if (tid == 0) red = 0.f;
  __syncthreads();
  {
    float acc[LP];
#pragma unroll
    for (int k = 0; k < LP; ++k) acc[k] = 0.f;
#pragma unroll 4
    for (int s = tid; s < S; s += blockDim.x)
#pragma unroll
      for (int k = 0; k < LP; ++k)
        if (k < L) { float u = Us[(int64_t)s * ldu + k]; acc[k] = fmaf(u, u, acc[k]); }
#pragma unroll
    for (int k = 0; k < LP; ++k) {
      float v = warp_sum(acc[k]);
      if (lane == 0 && k < L) wpart[warp * RW_MAX_LABELS + k] = v;
    }
    // trace of G (for mu0): one diagonal entry per thread
    float tr = 0.f;
    for (int i = tid; i < mmax; i += blockDim.x) tr += G[(int64_t)i * ldg + i];
    tr = warp_sum(tr);
    if (lane == 0) wpart[8 * RW_MAX_LABELS + warp] = tr;
  }
  __syncthreads();
  // the warps' sums added in warp order (deterministic)
  if (tid < L) {
    float v = 0.f;
    for (int w = 0; w < nw; ++w) v += wpart[w * RW_MAX_LABELS + tid];
    ck[tid] = v;
  } else if (tid == RW_MAX_LABELS) {
    float v = 0.f;
    for (int w = 0; w < nw; ++w) v += wpart[8 * RW_MAX_LABELS + w];
    red = v;
  }
#pragma unroll 4
  for (int e = tid; e < L * mmax; e += blockDim.x) {
    const int k = e / mmax, i = e % mmax;
    bb[e] = bv[(int64_t)i * ldb + k];
  }
  __syncthreads();
  if (tid == 0) mu0s = 1e-6f * red / mmax;
  __syncthreads();
  const float mu0 = mu0s;
  for (int K = 0; K * 32 < mmax; ++K) {
    const int r0 = K * 32, nr = min(32, mmax - r0);
    // tile row K of G + mu0 I (columns 0 .. r0 + nr): every element requested at once
    // (cp.async), then the shift on the diagonal
    for (int i = r0 + warp; i < r0 + nr; i += nw)
      for (int j = lane; j <= i; j += 32) cp_async4(A + i * ms + j, G + (int64_t)i * ldg + j);
    cp_async_wait_all();
    __syncthreads();
    if (tid < nr) A[(r0 + tid) * ms + r0 + tid] += mu0;
    __syncthreads();
    // off-diagonal tiles L_KJ = (A_KJ - sum_{t<J} L_Kt L_Jt^T) L_JJ^{-T}, J = 0..K-1 in order
    for (int J = 0; J < K; ++J) {
      const int c0 = J * 32;
      // each warp owns rows r0 + warp + nw * q, q = 0..3 (32 rows / 8 warps): their
      // dot products and triangular solves run interleaved
      float y[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int r = r0 + warp + nw * q;
        y[q] = (r < r0 + nr) ? A[r * ms + c0 + lane] : 0.f;
      }
      const float* lrow = A + (c0 + lane) * ms;
      for (int t = 0; t < c0; ++t) {
        const float l = lrow[t];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int r = r0 + warp + nw * q;
          if (r < r0 + nr) y[q] = fmaf(-A[r * ms + t], l, y[q]);
        }
      }
      const float* lrow_j = A + (c0 + lane) * ms + c0;  // row c0 + lane of block J
      for (int u = 0; u < 32; ++u) {  // branch-free: loads for every lane, selects below
        const float du = dinv[c0 + u];
        const float lu = lrow_j[u];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          y[q] = lane == u ? y[q] * du : y[q];
          const float xu = __shfl_sync(0xffffffff, y[q], u);
          const float yn = fmaf(-xu, lu, y[q]);
          y[q] = lane > u ? yn : y[q];
        }
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int r = r0 + warp + nw * q;
        if (r < r0 + nr) A[r * ms + c0 + lane] = y[q];
      }
      __syncthreads();
    }
    // diagonal tile: A_KK -= sum_{t<K} L_Kt L_Kt^T, then its Cholesky by one warp
    for (int r = r0 + warp; r < r0 + nr; r += nw) {
      const int c = r0 + lane;
      if (c <= r) {
        float y = A[r * ms + c];
        for (int t = 0; t < r0; ++t) y = fmaf(-A[r * ms + t], A[c * ms + t], y);
        A[r * ms + c] = y;
      }
    }
    __syncthreads();
    if (warp == 0) chol_diag_rot(A, ms, r0, nr, dinv + r0, colbuf, &bad);
    __syncthreads();
    // z_k on tile K: z = L_KK^{-1} (b_K - sum_J L_KJ z_J), one warp per label
    for (int k = warp; k < L; k += nw) {
      float y = 0.f;
      if (lane < nr) {
        y = bb[k * mmax + r0 + lane];
        for (int t = 0; t < r0; ++t) y = fmaf(-A[(r0 + lane) * ms + t], z[k * mmax + t], y);
      }
      const float* zrow = A + (r0 + (lane < nr ? lane : 0)) * ms + r0;
      for (int u = 0; u < nr; ++u) {  // branch-free: loads for every lane, selects below
        const float du = dinv[r0 + u];
        const float a = zrow[u];
        y = lane == u ? y * du : y;
        const float zu = __shfl_sync(0xffffffff, y, u);
        const float yn = fmaf(-zu, a, y);
        y = (lane > u && lane < nr) ? yn : y;
      }
      if (lane < nr) z[k * mmax + r0 + lane] = y;
      // prefix sums of z^2 inside the tile; f_u(m) = ck - zz - prefix
      float sq = (lane < nr) ? y * y : 0.f;
      for (int o = 1; o < 32; o <<= 1) {
        const float v = __shfl_up_sync(0xffffffff, sq, o);
        if (lane >= o) sq += v;
      }
      // candidates inside (r0, r0 + nr]: m - r0 - 1 is the lane whose inclusive prefix applies
      for (int c = 0; c < ncand; ++c) {
        const int m = cand_m(c);
        if (m <= r0 || m > r0 + nr) continue;
        const float pre = __shfl_sync(0xffffffff, sq, m - r0 - 1);
        if (lane == 0) al[k * mmax + c] = ck[k] - (zz[k] + pre);  // f_u(candidate c), label k
      }
      const float tot = __shfl_sync(0xffffffff, sq, 31);
      if (lane == 0) zz[k] += tot;
    }
    __syncthreads();
    if (warp == 0) {  // the first candidate inside this tile that passes for every label
      for (int cb = 0; cb < ncand; cb += 32) {
        const int c = cb + lane, m = cand_m(c);
        bool pass = c < ncand && m > r0 && m <= r0 + nr && !bad;
        for (int k = 0; k < L && pass; ++k)
          if (!(al[k * mmax + c] <= (float)fmax)) pass = false;
        const unsigned bal = __ballot_sync(0xffffffff, pass);
        if (bal) {
          if (lane == 0) chosen = cb + __ffs(bal) - 1;
          break;
        }
      }
    }
    __syncthreads();
    if (chosen >= 0) {
      if (tid == 0 && hint_remote) *reinterpret_cast<volatile int*>(hint_remote) = cand_m(chosen);
      break;
    }
  }
  if (tid == 0 && chosen < 0) { chosen = ncand - 1; capped = 1; }
  __syncthreads();
  // exact check of the chosen candidate: a_k = L_m^{-T} z_k[:m], ||a_k||, direct residual
  int c = chosen;
  int m = cand_m(c);
  // ||a_k|| from the back-substitution; f_k = ||u_k||^2 - ||z_k[:m]||^2 - mu0 ||a_k||^2, the
  // squared residual of the (mu0-regularized) fit, since L^T a = z and L z = b.
  for (int k = warp; k < L; k += nw) {
    bwd_lowerT_warp_reg(A, m, ms, dinv, z + k * mmax, al + k * mmax);
    float s2 = 0.f, zz2 = 0.f;
    for (int i = lane; i < m; i += 32) {
      s2 = fmaf(al[k * mmax + i], al[k * mmax + i], s2);
      zz2 = fmaf(z[k * mmax + i], z[k * mmax + i], zz2);
    }
    s2 = warp_sum(s2);
    zz2 = warp_sum(zz2);
    if (lane == 0) {
      nk[k] = sqrtf(s2);
      fk[k] = ck[k] - zz2 - mu0 * s2;
    }
  }
  __syncthreads();
  bool inside = true;
  for (int k = 0; k < L; ++k)
    if (!(nk[k] <= (float)rho)) inside = false;
  if (!inside) {
    // trust region for candidates c, c + 1, ... (the fit leaves the ball: few seeds, m > S).
    // Each label's Newton starts from the mu it reached on the previous candidate (the
    // constrained solution's mu grows with m, so the warm start stays on the left of the root,
    // where the iteration is monotone).
    __shared__ float s_muw[RW_MAX_LABELS];
    __shared__ int cand_fail;
    const float fail_thr = 1.05f * (float)fmax;
    if (tid < RW_MAX_LABELS) s_muw[tid] = 0.f;
    __syncthreads();
    for (; c < ncand; ++c) {
      m = cand_m(c);
      const int mss = m | 1;
      float* B2 = A;  // reuse the factor storage: G_m + mu I, stride mss
      load_shifted_gram(B2, m, mss, G, ldg, mu0);
      __syncthreads();
      bool okc = chol_lower_smem(B2, m, mss);
      for (int k = warp; k < L; k += nw) {
        for (int i = lane; i < m; i += 32) z[k * mmax + i] = bv[(int64_t)i * ldb + k];
        __syncwarp();
        fwd_lower_warp(B2, m, mss, z + k * mmax, z + k * mmax);
        bwd_lowerT_warp(B2, m, mss, z + k * mmax, al + k * mmax);
        float s2 = 0.f;
        for (int i = lane; i < m; i += 32) s2 = fmaf(al[k * mmax + i], al[k * mmax + i], s2);
        s2 = warp_sum(s2);
        if (lane == 0) nk[k] = sqrtf(s2);
      }
      // Lower bounds of f_k by Lagrangian duality: for a shift mu >= 0 and a = (G + mu I)^{-1} b,
      // f_k >= ||u_k||^2 - a^T b - mu rho^2.  One label whose bound exceeds f_max (with a 5%
      // margin for the FP32 arithmetic) fails the candidate whatever the others give, so the
      // Newton iterations of a failing candidate stop there; a passing candidate is solved
      // exactly as before.
      if (tid == 0) cand_fail = 0;
      __syncthreads();
      for (int k = warp; k < L; k += nw) {
        if (!(nk[k] > (float)rho)) continue;
        float t = 0.f;
        for (int i = lane; i < m; i += 32) t = fmaf(al[k * mmax + i], bv[(int64_t)i * ldb + k], t);
        t = warp_sum(t);
        if (lane == 0 && ck[k] - t - mu0 * (float)(rho * rho) > fail_thr) cand_fail = 1;
      }
      __syncthreads();
      if (cand_fail) continue;   // (uniform) the next candidate
      bool refactored = false;   // B2 still holds the factor of G_m + mu0 I
      for (int k = 0; k < L && okc; ++k) {
        if (!(nk[k] > (float)rho)) continue;
        // Newton from the left converges quadratically; in FP32 an ill-conditioned G_m + mu I
        // can keep ||a|| from settling below 1e-5 rho, so stop at 1e-4 rho or after 12 steps
        // (each step refactors the m x m matrix on one CTA; 40 steps cost milliseconds)
        float mu = fmaxf(mu0, s_muw[k]);
        if (mu > mu0 || refactored) {   // factor and solve at this label's starting mu
          __syncthreads();
          load_shifted_gram(B2, m, mss, G, ldg, mu);
          __syncthreads();
          if (!chol_lower_smem(B2, m, mss)) { okc = false; break; }
          if (warp == 0) {
            for (int i = lane; i < m; i += 32) z[k * mmax + i] = bv[(int64_t)i * ldb + k];
            __syncwarp();
            fwd_lower_warp(B2, m, mss, z + k * mmax, z + k * mmax);
            bwd_lowerT_warp(B2, m, mss, z + k * mmax, al + k * mmax);
            float s2 = 0.f, t = 0.f;
            for (int i = lane; i < m; i += 32) {
              s2 = fmaf(al[k * mmax + i], al[k * mmax + i], s2);
              t = fmaf(al[k * mmax + i], bv[(int64_t)i * ldb + k], t);
            }
            s2 = warp_sum(s2);
            t = warp_sum(t);
            if (lane == 0) {
              nk[k] = sqrtf(s2);
              if (ck[k] - t - mu * (float)(rho * rho) > fail_thr) cand_fail = 1;   // dual bound
            }
          }
          __syncthreads();
          if (cand_fail) break;
        }
        refactored = true;
        for (int it = 0; it < 12; ++it) {
          __syncthreads();
          const float na = nk[k];
          if (fabsf(na - (float)rho) <= 1e-4f * (float)rho) break;
          if (warp == 0) {  // ||q||^2 with L q = a
            fwd_lower_warp(B2, m, mss, al + k * mmax, bb + k * mmax);
            float s2 = 0.f;
            for (int i = lane; i < m; i += 32) s2 = fmaf(bb[k * mmax + i], bb[k * mmax + i], s2);
            s2 = warp_sum(s2);
            if (lane == 0) red = s2;
          }
          __syncthreads();
          mu = fmaxf(mu + (na * na / fmaxf(red, 1e-30f)) * ((na - (float)rho) / (float)rho), mu0);
          load_shifted_gram(B2, m, mss, G, ldg, mu);
          __syncthreads();
          if (!chol_lower_smem(B2, m, mss)) { okc = false; break; }
          if (warp == 0) {
            float t = 0.f;
            for (int i = lane; i < m; i += 32) {
              const float bi = bv[(int64_t)i * ldb + k];
              z[k * mmax + i] = bi;
            }
            __syncwarp();
            fwd_lower_warp(B2, m, mss, z + k * mmax, z + k * mmax);
            bwd_lowerT_warp(B2, m, mss, z + k * mmax, al + k * mmax);
            float s2 = 0.f;
            for (int i = lane; i < m; i += 32) {
              s2 = fmaf(al[k * mmax + i], al[k * mmax + i], s2);
              t = fmaf(al[k * mmax + i], bv[(int64_t)i * ldb + k], t);
            }
            s2 = warp_sum(s2);
            t = warp_sum(t);
            if (lane == 0) {
              nk[k] = sqrtf(s2);
              if (ck[k] - t - mu * (float)(rho * rho) > fail_thr) cand_fail = 1;   // dual bound
            }
          }
          __syncthreads();
          if (cand_fail) break;
        }
        __syncthreads();
        if (tid == 0) s_muw[k] = mu;   // the next candidate's start for this label
        if (cand_fail) break;
      }
      __syncthreads();
      if (cand_fail) continue;
      seed_residuals(Qs, ldq, Us, ldu, S, L, m, al, fk, mmax);
      bool pass = okc;
      for (int k = 0; k < L; ++k)
        if (!(fk[k] <= (float)fmax)) pass = false;
      if (pass) break;
      __syncthreads();
    }
    if (c >= ncand) { c = ncand - 1; if (tid == 0) capped = 1; }
  }
  __syncthreads();
  if (tid == 0) {
    mdev[0] = cand_m(c);
    mdev[1] = capped;
    for (int k = 0; k < L; ++k) fsel[k] = fk[k];
    if (final_remote) {
      *reinterpret_cast<volatile int*>(hint_remote) = cand_m(c);
      *reinterpret_cast<volatile int*>(final_remote) = cand_m(c);
    }
  }
}

template <int LP>
__global__ void __launch_bounds__(256, 1)
k_adapt(const float* __restrict__ G, int ldg, const float* __restrict__ bv, int ldb,
        const float* __restrict__ Qs, int ldq, const float* __restrict__ Us, int ldu, int S,
        int L, int mmax, int mstep, double rho, double fmax, int* __restrict__ mdev,
        double* __restrict__ fsel) {
  rw_grid_wait();
  rw_grid_trigger();
  adapt_body<LP>(G, ldg, bv, ldb, Qs, ldq, Us, ldu, S, L, mmax, mstep, rho, fmax, mdev, fsel,
                 nullptr, nullptr);
}

__global__ void k_set_m(int* mdev, int m) {
  rw_grid_wait();
  rw_grid_trigger();
  if (threadIdx.x == 0) { mdev[0] = m; mdev[1] = 0; }
}

// ---------------------------------------------------------------------------------------
// Z = Q_n^T P-hat_n.  Thread (row r, chunk c) of a block reads 16 bytes of row i's basis
// entries; cpr threads cover one row, R rows per block step.  Per-thread FP32 sums, reduced
// within the block and written as per-block partials (no atomics), then k_reduce.
// ---------------------------------------------------------------------------------------
template <typename T> struct Vec16;
template <> struct Vec16<__half> {
  static constexpr int V = 8;
  __device__ static void unpack(const uint4& u, float* o) {
    const __half2* h = reinterpret_cast<const __half2*>(&u);
#pragma unroll
    for (int t = 0; t < 4; ++t) { float2 f = __half22float2(h[t]); o[2 * t] = f.x; o[2 * t + 1] = f.y; }
  }
  __device__ static void load(const __half* p, float* o) {
    unpack(__ldg(reinterpret_cast<const uint4*>(p)), o);
  }
};
template <> struct Vec16<__nv_bfloat16> {
  static constexpr int V = 8;
  __device__ static void unpack(const uint4& u, float* o) {
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
    for (int t = 0; t < 4; ++t) { float2 f = __bfloat1622float2(h[t]); o[2 * t] = f.x; o[2 * t + 1] = f.y; }
  }
  __device__ static void load(const __nv_bfloat16* p, float* o) {
    unpack(__ldg(reinterpret_cast<const uint4*>(p)), o);
  }
};
template <> struct Vec16<float> {
  static constexpr int V = 4;
  __device__ static void load(const float* p, float* o) {
    float4 u = __ldg(reinterpret_cast<const float4*>(p));
    o[0] = u.x; o[1] = u.y; o[2] = u.z; o[3] = u.w;
  }
};

// One warp per basis row (lane c reads 16-byte chunk c, c + 32, ... of the row), rows strided
// across the grid with 4 rows in flight per warp; per-lane FP32 sums, reduced over the warps
// of a block in a fixed order and written as per-block partials (deterministic).
template <typename T, int LP, int CPL>
__global__ void __launch_bounds__(256)
k_project(const T* __restrict__ Q, int ldq, int cpr, const float* __restrict__ phat,
          const int* __restrict__ seedlab, int64_t N, const int* __restrict__ mdev,
          float* __restrict__ part) {
  rw_grid_wait();
  rw_grid_trigger();
  constexpr int V = Vec16<T>::V;
  constexpr int U = 4;  // rows per warp iteration
  extern __shared__ float zacc[];  // ldq * LP
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int m = mdev[0];
  float acc[CPL][V][LP];
#pragma unroll
  for (int t = 0; t < CPL; ++t)
#pragma unroll
    for (int v = 0; v < V; ++v)
#pragma unroll
      for (int k = 0; k < LP; ++k) acc[t][v][k] = 0.f;
  const int64_t stride = (int64_t)gridDim.x * nw;
  for (int64_t i0 = (int64_t)blockIdx.x * nw + warp; i0 < N; i0 += stride * U) {
    float q[U][CPL][V];
    float p[U][LP];
    bool use[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = i0 + u * stride;
      use[u] = i < N && __ldg(seedlab + i) < 0;
#pragma unroll
      for (int t = 0; t < CPL; ++t) {
        const int c = lane + 32 * t;
        if (use[u] && c < cpr && c * V < m) {
          Vec16<T>::load(Q + i * ldq + c * V, q[u][t]);
        } else {
#pragma unroll
          for (int v = 0; v < V; ++v) q[u][t][v] = 0.f;
        }
      }
      if (use[u]) {
#pragma unroll
        for (int k4 = 0; k4 < LP / 4; ++k4) {
          float4 pv = __ldg(reinterpret_cast<const float4*>(phat + i * LP) + k4);
          p[u][4 * k4] = pv.x; p[u][4 * k4 + 1] = pv.y; p[u][4 * k4 + 2] = pv.z; p[u][4 * k4 + 3] = pv.w;
        }
      } else {
#pragma unroll
        for (int k = 0; k < LP; ++k) p[u][k] = 0.f;
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int t = 0; t < CPL; ++t)
#pragma unroll
        for (int v = 0; v < V; ++v)
#pragma unroll
          for (int k = 0; k < LP; ++k) acc[t][v][k] = fmaf(q[u][t][v], p[u][k], acc[t][v][k]);
  }
  for (int e = threadIdx.x; e < ldq * LP; e += blockDim.x) zacc[e] = 0.f;
  for (int w = 0; w < nw; ++w) {
    __syncthreads();
    if (warp == w) {
#pragma unroll
      for (int t = 0; t < CPL; ++t) {
        const int c = lane + 32 * t;
        if (c < cpr)
#pragma unroll
          for (int v = 0; v < V; ++v)
#pragma unroll
            for (int k = 0; k < LP; ++k) zacc[(c * V + v) * LP + k] += acc[t][v][k];
      }
    }
  }
  __syncthreads();
  float* out = part + (int64_t)blockIdx.x * ldq * LP;
  for (int e = threadIdx.x; e < ldq * LP; e += blockDim.x) out[e] = zacc[e];
}

// Z (mq x lp, FP64) = scale * sum over blocks of the partials; one warp per entry, fixed order
__global__ void k_reduce_partials(const float* __restrict__ part, int nblk, int ldq, int lp,
                                  int mq, float scale, float* __restrict__ Z,
                                  const double* __restrict__ lam, double gamma, int m,
                                  float* __restrict__ lgam, int wait_first) {
  // The small solve's prologue reads the factors of k_adapt_lu.  Behind an ordinary
  // projection they are complete once the projection has started, so the trigger comes first;
  // behind an early one (started before k_adapt_lu ends, waiting for it before it exits) they
  // are complete only once the projection has ended, so the wait comes first.
  if (wait_first) {
    rw_grid_wait();
    rw_grid_trigger();
  } else {
    rw_grid_trigger();
    rw_grid_wait();
  }
  // one warp per entry of Z: lane l adds the partials l, l + 32, ... in order, then a fixed
  // butterfly; also lgam = lambda + gamma in FP32 for the small system
  const int lane = threadIdx.x & 31;
  const int e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (e < m && lane == 0) lgam[e] = (float)(lam[e] + gamma);
  if (e >= mq * lp) return;
  const int row = e / lp;
  float s = 0.f;
  if (row < ldq) {  // up to 16 partials per lane requested at once, added in block order
    for (int b0 = lane; b0 < nblk; b0 += 32 * 16) {
      float v[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int b = b0 + 32 * u;
        v[u] = b < nblk ? part[(int64_t)b * ldq * lp + e] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < 16; ++u) s += v[u];
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffff, s, o);
  if (lane == 0) Z[e] = s * scale;
}

// ---------------------------------------------------------------------------------------
// Small system of Eq. (Fs) in Woodbury form, one CTA:
//   M = diag(lambda + gamma) - K_m,  M y = h + gamma K (Lambda_gamma Z),  C = y + gamma Lambda_gamma Z
// LU in FP32 shared memory.  M is diagonally dominant in practice (its off-diagonal part is
// Q_s^T X, small next to lambda + gamma), so the elimination first runs without pivoting,
// blocked by 32-column panels.  If a pivot falls below 1e-3 of the largest entry of its
// original row, M is reloaded and eliminated with partial pivoting (rows permuted through an
// index array).
// ---------------------------------------------------------------------------------------
__device__ void load_M(float* M, int m, int ms, const float* __restrict__ K, int ldk,
                       const float* __restrict__ lgam) {
  // M = diag(lambda + gamma) - K: a warp per row, the row's loads (m <= 224: at most 7 per
  // lane) issued together
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = warp; i < m; i += nw) {
    const float* kr = K + (int64_t)i * ldk;
    float v[7];
#pragma unroll
    for (int q = 0; q < 7; ++q) {
      const int j = lane + 32 * q;
      v[q] = j < m ? kr[j] : 0.f;
    }
#pragma unroll
    for (int q = 0; q < 7; ++q) {
      const int j = lane + 32 * q;
      if (j < m) M[i * ms + j] = (j == i ? lgam[i] : 0.f) - v[q];
    }
  }
}

template <int LP>
__device__ void small_solve_body(const float* __restrict__ K, int ldk, const float* __restrict__ h,
                                 int ldh, const float* __restrict__ Z,
                                 const float* __restrict__ lgam, float gamma, int L, int lp,
                                 int mq, const int* __restrict__ mdev, float* __restrict__ C,
                                 int* status) {
  extern __shared__ float sm[];
  const int m = mdev[0];
  const int na = m + L;                // augmented columns: [M | B]
  const int ms = na | 1;
  float* M = sm;                       // m x ms : M, then the right-hand sides in columns m..
  float* W = M + (size_t)m * ms;       // m x L : Lambda_gamma Z (row-major)
  float* B = W + (size_t)m * L;        // L x m : right-hand sides (label-major), kept for the
                                       //         pivoting fallback
  int* perm = reinterpret_cast<int*>(B + (size_t)m * L);  // m
  float* dref = reinterpret_cast<float*>(perm + m);       // m : row scales before elimination
  __shared__ float uinv[kMaxSmallM];
  __shared__ __align__(16) float buf[128];
  __shared__ __align__(16) float Ush[32 * 32], Lsh[32 * 32];
  __shared__ int bad, unstable;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5, nty = blockDim.x >> 5;
  const int warp = ty, lane = tx;
  if (threadIdx.x == 0) { bad = 0; unstable = 0; }
  for (int e = threadIdx.x; e < m * L; e += blockDim.x) {
    const int i = e / L, k = e % L;
    W[i * L + k] = __fdividef(Z[(int64_t)i * lp + k], lgam[i]);
    B[k * m + i] = h[(int64_t)i * ldh + k];
  }
  load_M(M, m, ms, K, ldk, lgam);
  __syncthreads();
  for (int i = threadIdx.x; i < m; i += blockDim.x) perm[i] = i;
  for (int i = warp; i < m; i += nty) {  // row scale max_j |M_ij| before elimination
    float mx = 0.f;
    for (int j = lane; j < m; j += 32) mx = fmaxf(mx, fabsf(M[(size_t)i * ms + j]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffff, mx, o));
    if (lane == 0) dref[i] = mx;
  }
  // B += gamma K W, with K read back from the shared copy of M (K_ij = -M_ij off the diagonal,
  // K_ii = lambda_i + gamma - M_ii): one thread per (row, label), the row walked in order; the
  // result also goes to the augmented columns of M
  for (int e = threadIdx.x; e < m * L; e += blockDim.x) {
    const int i = e % m, k = e / m;
    const float* mi = M + (size_t)i * ms;
    float acc0 = 0.f, acc1 = 0.f;
    int j = 0;
    for (; j + 1 < m; j += 2) {
      acc0 = fmaf(-mi[j], W[j * L + k], acc0);
      acc1 = fmaf(-mi[j + 1], W[(j + 1) * L + k], acc1);
    }
    if (j < m) acc0 = fmaf(-mi[j], W[j * L + k], acc0);
    const float kii_extra = lgam[i] * W[i * L + k];   // diagonal: K_ii = lgam_i - M_ii
    const float rhs = B[k * m + i] + gamma * (acc0 + acc1 + kii_extra);
    B[k * m + i] = rhs;
    M[(size_t)i * ms + m + k] = rhs;
  }
  __syncthreads();
  // blocked LU without pivoting of [M | B], 32-column panels: the diagonal block on one warp
  // in registers, the two triangular solves one row / column per thread (the column solves
  // also cover the right-hand sides), the trailing update in 8 x 4 register tiles.  The
  // right-hand-side columns end as L^{-1} B, so only the upper solve remains.
  for (int p0 = 0; p0 < m; p0 += 32) {
    const int kb = min(32, m - p0);
    if (warp == 0) lu_diag_rot(M, ms, p0, kb, buf, dref, uinv, Ush, Lsh, &unstable);
    __syncthreads();
    const int r1 = p0 + kb, n = m - r1, nc = na - r1;
    for (int t = threadIdx.x; t < n + nc; t += blockDim.x) {
      if (t < n) trsm_row_rot(M + (size_t)(r1 + t) * ms + p0, kb, Ush, uinv + p0);
      else trsm_col_rot(M + (size_t)p0 * ms + r1 + (t - n), ms, kb, Lsh);
    }
    __syncthreads();
    if (n > 0) {
      gemm_trailing(M, ms, m, na, r1, p0, kb);
      __syncthreads();
    }
  }
  if (!unstable) {
    // U x = y per label (warp per label); C = x + gamma Lambda_gamma Z written directly
    for (int k = warp; k < L; k += nty) {
      float y[7];
#pragma unroll
      for (int q = 0; q < 7; ++q) {
        const int i = lane + 32 * q;
        y[q] = i < m ? M[(size_t)i * ms + m + k] : 0.f;
      }
      lu_bwd_group<6>(M, m, ms, uinv, y, lane);
      lu_bwd_group<5>(M, m, ms, uinv, y, lane);
      lu_bwd_group<4>(M, m, ms, uinv, y, lane);
      lu_bwd_group<3>(M, m, ms, uinv, y, lane);
      lu_bwd_group<2>(M, m, ms, uinv, y, lane);
      lu_bwd_group<1>(M, m, ms, uinv, y, lane);
      lu_bwd_group<0>(M, m, ms, uinv, y, lane);
#pragma unroll
      for (int q = 0; q < 7; ++q) {
        const int i = lane + 32 * q;
        if (i < m) C[(size_t)i * lp + k] = y[q] + gamma * W[i * L + k];
      }
    }
    for (int e = threadIdx.x; e < mq * lp; e += blockDim.x) {  // padding rows / labels
      const int i = e / lp, k = e % lp;
      if (i >= m || k >= L) C[e] = 0.f;
    }
  } else {
    // a pivot fell below 1e-3 of its original diagonal: partial pivoting from the original M
    __syncthreads();
    load_M(M, m, ms, K, ldk, lgam);
    for (int k = 0; k < m; ++k) {
      __syncthreads();
      if (warp == 0) {  // pivot among the rows perm[k..m-1]
        float best = -1.f;
        int bi = k;
        for (int i = k + lane; i < m; i += 32) {
          float a = fabsf(M[perm[i] * ms + k]);
          if (a > best) { best = a; bi = i; }
        }
        for (int o = 16; o > 0; o >>= 1) {
          float ob = __shfl_xor_sync(0xffffffff, best, o);
          int oi = __shfl_xor_sync(0xffffffff, bi, o);
          if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (lane == 0) {
          if (!(best > 0.f)) bad = 1;
          int t = perm[k]; perm[k] = perm[bi]; perm[bi] = t;
        }
      }
      __syncthreads();
      const int pk = perm[k];
      float pv = M[pk * ms + k];
      if (pv == 0.f) pv = 1e-30f;
      const float inv = 1.f / pv;
      for (int r = k + 1 + ty; r < m; r += nty) {
        const int pr = perm[r];
        const float a = M[pr * ms + k] * inv;
        for (int j = k + 1 + tx; j < m; j += 32) M[pr * ms + j] = fmaf(-a, M[pk * ms + j], M[pr * ms + j]);
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += blockDim.x) uinv[i] = 1.f / M[perm[i] * ms + i];
    __syncthreads();
    // forward (unit lower, multipliers a_ij / u_jj) and backward (upper) substitution on the
    // permuted rows, one warp per label, in place in B's row for the label (the original
    // right-hand sides are first moved to row order by a copy into the augmented columns)
    for (int e = threadIdx.x; e < m * L; e += blockDim.x) {
      const int i = e % m, k = e / m;
      M[(size_t)i * ms + m + k] = B[k * m + perm[i]];
    }
    __syncthreads();
    for (int k = warp; k < L; k += nty) {
      float* y = B + (size_t)k * m;
      for (int i = lane; i < m; i += 32) y[i] = M[(size_t)i * ms + m + k];
      __syncwarp();
      for (int j = 0; j < m; ++j) {
        const float f = y[j] * uinv[j];
        for (int i = j + 1 + lane; i < m; i += 32) y[i] = fmaf(-M[perm[i] * ms + j], f, y[i]);
        __syncwarp();
      }
      for (int i = m - 1; i >= 0; --i) {
        const float yi = y[i] * uinv[i];
        __syncwarp();
        if (lane == 0) y[i] = yi;
        for (int j = lane; j < i; j += 32) y[j] = fmaf(-M[perm[j] * ms + i], yi, y[j]);
        __syncwarp();
      }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < mq * lp; e += blockDim.x) {
      const int i = e / lp, k = e % lp;
      float v = 0.f;
      if (i < m && k < L) v = B[(size_t)k * m + i] + gamma * W[i * L + k];
      C[e] = v;
    }
  }
  if (threadIdx.x == 0 && bad) atomicOr(status, RW_DEV_SINGULAR);
}

template <int LP>
__global__ void __launch_bounds__(256, 1)
k_small_solve(const float* __restrict__ K, int ldk, const float* __restrict__ h, int ldh,
              const float* __restrict__ Z, const float* __restrict__ lgam, float gamma,
              int L, int lp, int mq, const int* __restrict__ mdev, float* __restrict__ C,
              int* status) {
  rw_grid_wait();
  rw_grid_trigger();
  small_solve_body<LP>(K, ldk, h, ldh, Z, lgam, gamma, L, lp, mq, mdev, C, status);
}

// ---------------------------------------------------------------------------------------
// The adaptive choice of m and the factorization of the m x m system as one cluster of two
// CTAs.  M = diag(lambda + gamma) - K does not depend on the projection, and an LU without
// pivoting of M restricted to its leading rows and columns is the leading part of the LU of M,
// so the LU CTA factors M tile by tile (left-looking) while the other CTA grows its Cholesky
// over the candidates; it stops at the first tile boundary past the m it is told.  After the
// projection, C = M^{-1} (h + gamma Z) needs only the two triangular solves (with
// K = diag(lambda + gamma) - M and W = Lambda_gamma Z, h + gamma K W = h + gamma Z - gamma M W,
// so y + gamma W = M^{-1} (h + gamma Z)).
// ---------------------------------------------------------------------------------------
constexpr int kLuTiles = kMaxSmallM / 32;  // column tiles per row of the stability maxima

__device__ __forceinline__ void bar_sync_id(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" :: "r"(id), "r"(nthreads) : "memory");
}

// Tile T of the left-looking LU held in A (stride ms, a multiple of 4; K's pitch ldk too).
// lu_load_border: the border of M (rows [r0, r1) x columns [0, r1) and rows [0, r0) x columns
// [r0, r1)) by warps w0.. of the CTA: every 16-byte piece of K is requested at once
// (cp.async, one round trip), then, after a barrier of those warps (id 2), a thread per (row,
// column tile) forms M = diag(lambda + gamma) - K in place and dmax[i][q] = max_j |M_ij| over
// column tile q (the stability check's row scale).  Whole 16-byte pieces past r1 may be copied
// (inside the row; never read).
__device__ void lu_load_border(float* A, int ms, int T, int mmax, const float* __restrict__ Kg,
                               int ldk, const float* lg, float* dmax, int w0) {
  const int lane = threadIdx.x & 31, warp = (threadIdx.x >> 5) - w0, nw = (blockDim.x >> 5) - w0;
  const int t = threadIdx.x - 32 * w0, nt = 32 * nw;
  const int r0 = 32 * T, nr = min(32, mmax - r0), r1 = r0 + nr;
  const int w4 = (r1 + 3) / 4, c4 = (nr + 3) / 4;
  for (int i = r0 + warp; i < r1; i += nw)  // row block: a warp per row
    for (int c = lane; c < w4; c += 32)
      cp_async16(A + (size_t)i * ms + 4 * c, Kg + (int64_t)i * ldk + 4 * c);
  for (int ib = 4 * warp; ib < r0; ib += 4 * nw) {  // column block: four rows per warp step
    const int i = ib + (lane >> 3), c = lane & 7;
    if (i < r0 && c < c4) cp_async16(A + (size_t)i * ms + r0 + 4 * c, Kg + (int64_t)i * ldk + r0 + 4 * c);
  }
  cp_async_wait_all();
  bar_sync_id(2, nt);
  const int nrb = nr * (T + 1);
  for (int e = t; e < nrb + r0; e += nt) {
    int i, q;
    if (e < nrb) { i = r0 + e / (T + 1); q = e % (T + 1); }
    else { i = e - nrb; q = T; }
    float* ar = A + (size_t)i * ms + 32 * q;
    const int cnt = min(32, r1 - 32 * q), rot = cnt == 32 ? (e & 31) : 0;  // rotation: spread banks
    const int dg = i - 32 * q;  // diagonal position inside the tile (if any)
    float mx = 0.f;
    for (int k = 0; k < cnt; ++k) {
      int kk = k + rot;
      if (kk >= cnt) kk -= cnt;
      const float v = (kk == dg ? lg[i] : 0.f) - ar[kk];
      ar[kk] = v;
      mx = fmaxf(mx, fabsf(v));
    }
    dmax[i * kLuTiles + q] = mx;
  }
}

// lu_solve_border: the loaded border against the factored blocks J < T in order (the row block
// against U_JJ, the column block against L_JJ, each solve followed by the update of the rest of
// the border), all warps; ends with a barrier.  The diagonal block is then factored by one warp
// (lu_diag_rot) while the other warps load the next tile's border, which no step of this tile
// reads or writes.
__device__ void lu_solve_border(float* A, int ms, int T, int mmax, float* Ush, float* Lsh,
                                const float* uinv) {
  const int tid = threadIdx.x;
  const int r0 = 32 * T, nr = min(32, mmax - r0), r1 = r0 + nr;
  for (int J = 0; J < T; ++J) {
    const int c0 = 32 * J;
    // U32[c][col] = U_c,col (col > c) and L32T[r][row] = L_row,r (row > r) of block J, else 0
    for (int e = tid; e < 1024; e += blockDim.x) {
      const int c = e >> 5, o = e & 31;
      Ush[e] = o > c ? A[(c0 + c) * ms + c0 + o] : 0.f;
      Lsh[e] = o > c ? A[(c0 + o) * ms + c0 + c] : 0.f;
    }
    __syncthreads();
    if (tid < 128) trsm_rows_128(A, ms, r0, nr, c0, Ush, uinv, 0);
    else trsm_cols_128(A, ms, r0, nr, c0, Lsh, 128);
    __syncthreads();
    gemm4<8, 32>(A, ms, r0, r1, c0 + 32, r1, c0);   // row block, columns past block J
    gemm4<4, 8>(A, ms, c0 + 32, r0, r0, r1, c0);    // column block, rows past block J
    __syncthreads();
  }
}

// The LU CTA: tiles until the adaptive CTA's hint (the first passing candidate) is covered,
// then the cluster barrier (after which the final m is in the mailbox), then any tiles still
// missing.  Writes the leading m x m factors (F, pitch ldf), 1 / U_ii and mdev[2] = 1 when a
// pivot falls below 1e-3 of the largest |M_ij| of its row over the first ceil(m / 32) column
// tiles (the solve then pivots from the original matrix).
__device__ void lu_body(cg::cluster_group& cl, int mmax, const float* __restrict__ Kg, int ldk,
                        const double* __restrict__ lam, double gamma, float* __restrict__ F,
                        int ldf, float* __restrict__ luinv, int* __restrict__ mdev,
                        const int* hint, const int* fin) {
  extern __shared__ float sm[];
  const int tid = threadIdx.x;
  const int ms = lu_stride(mmax);
  float* A = sm;
  float* dmax = A + (size_t)mmax * ms;
  __shared__ float lg[kMaxSmallM], uinv[kMaxSmallM];
  __shared__ __align__(16) float Ush[32 * 32], Lsh[32 * 32];
  __shared__ __align__(16) float buf[128];
  __shared__ int dec, unstable;
  for (int i = tid; i < mmax; i += blockDim.x) lg[i] = (float)(lam[i] + gamma);
  if (tid == 0) unstable = 0;
  __syncthreads();
  lu_load_border(A, ms, 0, mmax, Kg, ldk, lg, dmax, 0);
  __syncthreads();
  int T = 0, covered = 0, target = mmax;
  bool synced = false;
  for (;;) {
    if (!synced) {
      if (tid == 0) {
        int hv;  // the mailbox is this CTA's own shared memory, written remotely by the other CTA
        asm volatile("ld.volatile.shared.u32 %0, [%1];"
                     : "=r"(hv) : "r"((unsigned)__cvta_generic_to_shared(hint)));
        dec = (covered >= mmax || (hv > 0 && covered >= hv)) ? 1 : 0;
      }
      __syncthreads();
      if (dec) {
        cl.sync();
        synced = true;
        target = *reinterpret_cast<const volatile int*>(fin);
      }
    }
    if (synced && covered >= target) break;
    lu_solve_border(A, ms, T, mmax, Ush, Lsh, uinv);
    if (threadIdx.x < 32)
      lu_diag_warp(A, ms, 32 * T, min(32, mmax - 32 * T), buf, uinv);
    else if (threadIdx.x >= 128 && 32 * (T + 1) < mmax)
      lu_load_border(A, ms, T + 1, mmax, Kg, ldk, lg, dmax, 4);
    __syncthreads();
    ++T;
    covered = min(32 * T, mmax);
  }
  const int m = target, nt = (m + 31) / 32;
  for (int i = tid; i < m; i += blockDim.x) {
    float d = 0.f;
    for (int q = 0; q < nt; ++q) d = fmaxf(d, dmax[i * kLuTiles + q]);
    const float u = A[i * ms + i];
    if (u == 0.f || !(fabsf(u) >= 1e-3f * d)) unstable = 1;
    luinv[i] = uinv[i];
  }
  for (int e = tid; e < m * m; e += blockDim.x) {
    const int i = e / m, j = e - i * m;
    F[(int64_t)i * ldf + j] = A[i * ms + j];
  }
  __syncthreads();
  if (tid == 0) mdev[2] = unstable;
}

template <int LP>
__global__ void __launch_bounds__(256, 1)
k_adapt_lu(const float* __restrict__ G, int ldg, const float* __restrict__ bv, int ldb,
           const float* __restrict__ Qs, int ldq, const float* __restrict__ Us, int ldu, int S,
           int L, int mmax, int mstep, double rho, double fmax, int adaptive,
           const float* __restrict__ Kg, int ldk, const double* __restrict__ lam, double gamma,
           float* __restrict__ F, int ldf, float* __restrict__ luinv, int* __restrict__ mdev,
           double* __restrict__ fsel) {
  rw_grid_wait();
  rw_grid_trigger();
  cg::cluster_group cl = cg::this_cluster();
  __shared__ int s_hint, s_final;  // mailboxes of the LU CTA
  if (threadIdx.x == 0) { s_hint = 0; s_final = 0; }
  cl.sync();  // both CTAs running, mailboxes cleared
  if (cl.block_rank() == 0) {
    int* rh = cl.map_shared_rank(&s_hint, 1);
    int* rf = cl.map_shared_rank(&s_final, 1);
    if (adaptive) {
      adapt_body<LP>(G, ldg, bv, ldb, Qs, ldq, Us, ldu, S, L, mmax, mstep, rho, fmax, mdev, fsel,
                     rh, rf);
    } else if (threadIdx.x == 0) {
      mdev[0] = mmax;
      mdev[1] = 0;
      *reinterpret_cast<volatile int*>(rh) = mmax;
      *reinterpret_cast<volatile int*>(rf) = mmax;
    }
    // m is final (thread 0 wrote mdev[0] above): publish it for a projection that starts
    // before this kernel ends (k_project_tma with early = 1); the factors are not covered
    if (threadIdx.x == 0)
      asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(mdev + 3), "r"(1) : "memory");
    cl.sync();
  } else {
    lu_body(cl, mmax, Kg, ldk, lam, gamma, F, ldf, luinv, mdev, &s_hint, &s_final);
  }
}

// C = M^{-1} (h + gamma Z) from the factors of k_adapt_lu.  Before the grid dependency wait
// (the factors come from two launches back and are complete when this kernel starts: behind an
// ordinary projection, which started after k_adapt_lu ended; behind an early one,
// k_reduce_partials lets this kernel start only after its own wait) the factors are copied in; after it the substitutions run by 32-row blocks: one warp solves the
// diagonal block for all labels (lane = row, labels in registers), then all threads update the
// remaining rows.  When the factorization was flagged unstable the whole pivoting solve runs
// instead.
template <int LP>
__global__ void __launch_bounds__(256, 1)
k_small_rhs(const float* __restrict__ K, int ldk, const float* __restrict__ h, int ldh,
            const float* __restrict__ Z, const float* __restrict__ lgam, float gamma, int L,
            int lp, int mq, const int* __restrict__ mdev, const float* __restrict__ F, int ldf,
            const float* __restrict__ luinv, float* __restrict__ C, int* status) {
  if (__ldcg(mdev + 2)) {
    rw_grid_wait();
    rw_grid_trigger();
    small_solve_body<LP>(K, ldk, h, ldh, Z, lgam, gamma, L, lp, mq, mdev, C, status);
    return;
  }
  extern __shared__ float sm[];
  const int tid = threadIdx.x, warp = tid >> 5, nw = blockDim.x >> 5;
  const int m = __ldcg(mdev), ms = lu_stride(m), nt = (m + 31) / 32;
  float* A = sm;                              // m x ms factors
  float* Y = A + (size_t)m * ms;              // LP x m right-hand sides / solution (label-major)
  __shared__ float ui[kMaxSmallM];
  // the factors: every 16-byte piece requested at once (ldf and ms are multiples of 4; whole
  // pieces past column m are copied and never read)
  const int g4 = (m + 3) / 4;
  for (int i = warp; i < m; i += nw)
    for (int c = tid & 31; c < g4; c += 32) cp_async16(A + (size_t)i * ms + 4 * c, F + (int64_t)i * ldf + 4 * c);
  cp_async_wait_all();
  for (int i = tid; i < m; i += blockDim.x) ui[i] = __ldcg(luinv + i);
  __syncthreads();
  rw_grid_wait();
  rw_grid_trigger();
  // one warp per label, independent of the others: its vector y (label-major in Y) is solved by
  // 32-row blocks: the diagonal block by a chain over the lanes (lane = row, one shuffle per
  // step), then the rows past it (forward) or before it (backward) by the block's product
  const int lane = tid & 31;
  for (int k = warp; k < L; k += nw) {
    float* y = Y + (size_t)k * m;
    for (int i = lane; i < m; i += 32) y[i] = fmaf(gamma, Z[(int64_t)i * lp + k], h[(int64_t)i * ldh + k]);
    __syncwarp();
    for (int I = 0; I < nt; ++I) {  // L y = b, L unit lower
      const int r0 = 32 * I, kb = min(32, m - r0), r1 = r0 + kb;
      const bool live = lane < kb;
      const float* lr = A + (size_t)(r0 + (live ? lane : 0)) * ms + r0;
      float yi = live ? y[r0 + lane] : 0.f;
      for (int c = 0; c < kb; ++c) {
        const float lc = lr[c];  // inside the row for every lane; used below the diagonal only
        const float yn = fmaf(-lc, __shfl_sync(0xffffffff, yi, c), yi);
        yi = lane > c ? yn : yi;
      }
      if (live) y[r0 + lane] = yi;
      __syncwarp();
      for (int j = r1 + lane; j < m; j += 32) {
        const float* ar = A + (size_t)j * ms + r0;
        float s0 = y[j], s1 = 0.f;
        int c = 0;
        for (; c + 1 < kb; c += 2) {
          s0 = fmaf(-ar[c], y[r0 + c], s0);
          s1 = fmaf(-ar[c + 1], y[r0 + c + 1], s1);
        }
        if (c < kb) s0 = fmaf(-ar[c], y[r0 + c], s0);
        y[j] = s0 + s1;
      }
      __syncwarp();
    }
    for (int I = nt - 1; I >= 0; --I) {  // U x = y, 1 / U_ii in ui
      const int r0 = 32 * I, kb = min(32, m - r0);
      const bool live = lane < kb;
      const float* ur = A + (size_t)(r0 + (live ? lane : 0)) * ms + r0;
      const float uii = live ? ui[r0 + lane] : 0.f;
      float yi = live ? y[r0 + lane] : 0.f;
      for (int c = kb - 1; c >= 0; --c) {
        const float uc = ur[c];  // inside the row for every lane; used above the diagonal only
        const float xc = __shfl_sync(0xffffffff, yi * uii, c);
        const float yn = fmaf(-uc, xc, yi);
        yi = lane == c ? xc : (lane < c ? yn : yi);
      }
      if (live) y[r0 + lane] = yi;
      __syncwarp();
      for (int j = lane; j < r0; j += 32) {
        const float* ar = A + (size_t)j * ms + r0;
        float s0 = y[j], s1 = 0.f;
        int c = 0;
        for (; c + 1 < kb; c += 2) {
          s0 = fmaf(-ar[c], y[r0 + c], s0);
          s1 = fmaf(-ar[c + 1], y[r0 + c + 1], s1);
        }
        if (c < kb) s0 = fmaf(-ar[c], y[r0 + c], s0);
        y[j] = s0 + s1;
      }
      __syncwarp();
    }
  }
  __syncthreads();
  for (int e = tid; e < mq * lp; e += blockDim.x) {
    const int i = e / lp, k = e % lp;
    C[e] = (i < m && k < L) ? Y[(size_t)k * m + i] : 0.f;
  }
}

// ---------------------------------------------------------------------------------------
// U-hat_n = Q_n C on the row-major FP32 basis.  One warp per group of RB rows (RB = 16 / LP, so every warp iteration
// produces 16 (row, label) sums); lane c holds chunk c of each row and the matching rows of C
// in registers.  The 16 partial sums are reduced across the warp by a reduce-scatter
// butterfly (each exchange halves the values a lane keeps; 16 shuffles in all), after which
// the even lane 2j holds sum j = (row j / LP, label j % LP).  Writes either the refinement
// start (hat space, seeds = d^{1/2} one-hot) or the final U / labels.
// ---------------------------------------------------------------------------------------
template <typename T, int LP, int CPL>
__global__ void __launch_bounds__(256)
k_backproject(const T* __restrict__ Q, int ldq, int cpr, const float* __restrict__ Cg,
              float cscale, const int* __restrict__ seedlab, const float* __restrict__ sq,
              const float* __restrict__ s, int64_t N, int L, const int* __restrict__ mdev,
              float* __restrict__ xhat, float* __restrict__ U, uint8_t* __restrict__ labels, int* clear_seedlab,
              const float* __restrict__ nul) {
  rw_grid_wait();
  rw_grid_trigger();
  constexpr int V = Vec16<T>::V;
  constexpr int RB = 16 / LP;  // rows per warp iteration
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int m = mdev[0];
  float creg[CPL][V][LP];
#pragma unroll
  for (int t = 0; t < CPL; ++t) {
    const int c = lane + 32 * t;
#pragma unroll
    for (int v = 0; v < V; ++v)
#pragma unroll
      for (int k = 0; k < LP; ++k)
        creg[t][v][k] = (c < cpr) ? __ldg(Cg + (c * V + v) * LP + k) * cscale : 0.f;
  }
  const int64_t ngroups = (N + RB - 1) / RB;
  for (int64_t grp = (int64_t)blockIdx.x * nw + warp; grp < ngroups;
       grp += (int64_t)gridDim.x * nw) {
    const int64_t i0 = grp * RB;
    float val[16];
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      const int64_t i = i0 + r;
      float acc[LP];
#pragma unroll
      for (int k = 0; k < LP; ++k) acc[k] = 0.f;
      if (i < N) {
#pragma unroll
        for (int t = 0; t < CPL; ++t) {
          const int c = lane + 32 * t;
          if (c < cpr && c * V < m) {
            float q[V];
            Vec16<T>::load(Q + i * ldq + c * V, q);
#pragma unroll
            for (int v = 0; v < V; ++v)
#pragma unroll
              for (int k = 0; k < LP; ++k) acc[k] = fmaf(q[v], creg[t][v][k], acc[k]);
          }
        }
      }
#pragma unroll
      for (int k = 0; k < LP; ++k) val[r * LP + k] = acc[k];
    }
    // reduce-scatter: 16 -> 8 -> 4 -> 2 -> 1 values per lane, then the last pair
#pragma unroll
    for (int half = 8, off = 16; half >= 1; half >>= 1, off >>= 1) {
      const bool up = (lane & off) != 0;
#pragma unroll
      for (int t = 0; t < half; ++t) {
        const float send = up ? val[t] : val[t + half];
        const float keep = up ? val[t + half] : val[t];
        val[t] = keep + __shfl_xor_sync(0xffffffff, send, off);
      }
    }
    float sum = val[0] + __shfl_xor_sync(0xffffffff, val[0], 1);
    // even lane 2j holds entry j = r * LP + k
    const int j = lane >> 1;
    const int r = j / LP, k = j % LP;
    const int64_t i = i0 + r;
    const bool writer = (lane & 1) == 0 && i < N;
    int sl = -1;
    if (writer) sl = seedlab[i];
    if (nul && writer && sl < 0) sum = fmaf(sq[i], __ldg(nul + k), sum);  // gamma = 0: + g_i c_eff
    if (xhat) {
      if (writer) xhat[i * LP + k] = (k >= L) ? 0.f : ((sl >= 0) ? (k == sl ? sq[i] : 0.f) : sum);
    } else {
      float u = 0.f;
      if (writer && k < L) {
        u = (sl >= 0) ? (k == sl ? 1.f : 0.f) : sum * s[i];
        U[i * L + k] = u;
      }
      if (labels) {
        // lanes 2 (r LP + k), k = 0..LP-1, hold row r: argmax over the first L, ties -> lowest
        int best = 0;
        float bv = __shfl_sync(0xffffffff, u, (lane & ~(2 * LP - 1)));
        for (int kk = 1; kk < LP; ++kk) {
          const float o = __shfl_sync(0xffffffff, u, (lane & ~(2 * LP - 1)) + 2 * kk);
          if (kk < L && o > bv) { bv = o; best = kk; }
        }
        if (writer && k == 0) labels[i] = (uint8_t)best;
      }
      if (clear_seedlab && writer && k == 0 && sl >= 0) clear_seedlab[i] = -1;
    }
  }
}

// ---------------------------------------------------------------------------------------
// 16-bit basis copies are stored panel-major: for each 8-column chunk c an N x 8 panel of
// 16-byte rows, element (i, 8c + v) at ((c N + i) 8 + v).  Using the first m columns reads the
// first ceil(m / 8) panels end to end.
// ---------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void load8(const T* p, float* o) { Vec16<T>::load(p, o); }

// Z partials on the panel layout, chunk-major: a block owns a range of rows, split into
// kParts parts; warps take (chunk, part) items, a lane walks the item's rows (8 rows of 16 bytes
// in flight per lane) and keeps the 8 x LPG products of one label group in registers; a single
// reduce-scatter butterfly per item, then the parts are added in part order in shared memory.
// Block partials part[block][8 c + v][k] (the layout k_reduce_partials reads).
constexpr int kParts = 4;

// butterfly: after it, lane j holds the warp sum of val[j] (val has 32 entries)
__device__ __forceinline__ float reduce_scatter32(float (&val)[32], int lane) {
#pragma unroll
  for (int half = 16, off = 16; half >= 1; half >>= 1, off >>= 1) {
    const bool up = (lane & off) != 0;
#pragma unroll
    for (int t = 0; t < half; ++t) {
      const float send = up ? val[t] : val[t + half];
      const float keep = up ? val[t + half] : val[t];
      val[t] = keep + __shfl_xor_sync(0xffffffff, send, off);
    }
  }
  return val[0];
}

template <typename T, int LP>
__global__ void __launch_bounds__(256, 2)
k_project_cw(const T* __restrict__ Qp, int64_t N, int nchunk_max, const float* __restrict__ phat,
             const int* __restrict__ seedlab, const int* __restrict__ mdev, int64_t rows_per_block,
             float* __restrict__ part) {
  rw_grid_wait();
  rw_grid_trigger();
  constexpr int LPG = LP < 4 ? LP : 4;   // labels per pass: 8 x 4 = 32 products per lane
  constexpr int NG = LP / LPG;
  extern __shared__ float red[];        // kParts x nchunk_max x 8 x LP
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int m = mdev[0];
  const int nch = min((m + 7) / 8, nchunk_max);
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
  const int64_t r1 = min(N, r0 + rows_per_block);
  const int64_t plen = (r1 - r0 + kParts - 1) / kParts;
  const int items = nch * kParts * NG;
  for (int it = warp; it < items; it += nw) {
    const int c = it % nch, rest = it / nch, pt = rest % kParts, g = rest / kParts;
    const int64_t a0 = r0 + pt * plen, a1 = min(r1, a0 + plen);
    const T* qc = Qp + (int64_t)c * N * 8;
    float acc[32];
#pragma unroll
    for (int t = 0; t < 32; ++t) acc[t] = 0.f;
    for (int64_t i0 = a0 + lane; i0 < a1; i0 += 32 * 8) {
      uint4 raw[8];            // 8 rows of this chunk in flight, converted at use
      float p[8][LPG];
      // the basis row, the prior row and the seed flag are loaded together (one round trip);
      // seed rows are masked afterwards
      int sl[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int64_t i = i0 + 32 * u;
        const bool inb = i < a1;
        sl[u] = inb ? __ldg(seedlab + i) : 0;
        raw[u] = inb ? __ldg(reinterpret_cast<const uint4*>(qc + i * 8)) : make_uint4(0, 0, 0, 0);
        if constexpr (LPG == 4) {
          const float4 pv = inb ? __ldg(reinterpret_cast<const float4*>(phat + i * LP + g * LPG))
                                : make_float4(0.f, 0.f, 0.f, 0.f);
          p[u][0] = pv.x; p[u][1] = pv.y; p[u][2] = pv.z; p[u][3] = pv.w;
        } else {
#pragma unroll
          for (int k = 0; k < LPG; ++k) p[u][k] = inb ? __ldg(phat + i * LP + g * LPG + k) : 0.f;
        }
      }
#pragma unroll
      for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int k = 0; k < LPG; ++k) p[u][k] = sl[u] < 0 ? p[u][k] : 0.f;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        float q[8];
        Vec16<T>::unpack(raw[u], q);
#pragma unroll
        for (int v = 0; v < 8; ++v)
#pragma unroll
          for (int k = 0; k < LPG; ++k) acc[v * LPG + k] = fmaf(q[v], p[u][k], acc[v * LPG + k]);
      }
    }
    const float sum = reduce_scatter32(acc, lane);  // lane j: product j = (v = j / LPG, k = j % LPG)
    if (lane < 8 * LPG) {
      const int v = lane / LPG, k = lane % LPG;
      red[((size_t)pt * nchunk_max + c) * 8 * LP + v * LP + g * LPG + k] = sum;
    }
  }
  __syncthreads();
  float* pb = part + (int64_t)blockIdx.x * nchunk_max * 8 * LP;
  for (int e = threadIdx.x; e < nchunk_max * 8 * LP; e += blockDim.x) {
    const int c = e / (8 * LP);
    float v = 0.f;
    if (c < nch)
      for (int pt = 0; pt < kParts; ++pt) v += red[(size_t)pt * nchunk_max * 8 * LP + e];
    pb[e] = v;
  }
}

// U-hat_n = Q_n C on the panel layout: lane = row, the chunk's 8 x LP coefficients come from
// shared memory as broadcasts; no cross-lane reduction.
// Z partials with the basis streamed through shared memory by bulk asynchronous copies: a
// block owns a range of rows, taken in tiles of kPtRows rows; for each tile the masked priors
// of a thread's rows are loaded once (registers) and the tile's 16-byte rows of every
// chunk arrive in a kPtStages-deep ring (one bulk copy per (tile, chunk), completion on an
// mbarrier).  Per step a thread forms its rows' 8 x LP products, a reduce-scatter butterfly
// sums them over the warp and the warp adds them to its own accumulator (step order: fixed);
// the warps are added in order at the end.  Block partials as k_project_cw writes them.
constexpr int kPtRows = 1024, kPtStages = 4, kPtRowsPerThread = kPtRows / 256;
constexpr int kEarlyPolls = 1 << 16;   // x (up to 2 us + an L2 round trip): about 0.15 s

template <typename T, int LP>
__global__ void __launch_bounds__(256, 2)
k_project_tma(const T* __restrict__ Qp, int64_t N, int nchunk_max, const float* __restrict__ phat,
              const int* __restrict__ seedlab, const int* __restrict__ mdev,
              int64_t rows_per_block, float* __restrict__ part, int* status, int early) {
  // early: the preceding kernel is k_adapt_lu, whose LU half may still run after m is final.
  // Its other inputs (basis, priors, seed labels) are complete once it has started, so the
  // block starts as soon as mdev[3] says m is published (a bounded poll; on time-out, the
  // ordinary grid wait) and waits for the whole predecessor only before it exits, so that
  // the kernels after it still see every output of k_adapt_lu.
  __shared__ int s_m;
  if (early) {
    if (threadIdx.x == 0) {
      int v = 0, mm = -1;
      unsigned ns = 128;   // back-off doubling to 2 us: few L2 requests while a long choice runs
      for (int it = 0; it < kEarlyPolls; ++it) {
        asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(mdev + 3) : "memory");
        if (v) break;
        __nanosleep(ns);
        ns = ns < 2048u ? 2u * ns : 2048u;
      }
      if (v) asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(mm) : "l"(mdev) : "memory");
      s_m = mm;
    }
    __syncthreads();
    if (s_m < 0) rw_grid_wait();
  } else {
    rw_grid_wait();
  }
  rw_grid_trigger();
  constexpr int NV = 8 * LP, NG = NV / 32;
  extern __shared__ __align__(16) unsigned char smraw[];
  uint4* stage = reinterpret_cast<uint4*>(smraw);                      // kPtStages x kPtRows
  float* red = reinterpret_cast<float*>(stage + kPtStages * kPtRows);  // nw x nchunk_max x NV
  __shared__ __align__(8) uint64_t bar[kPtStages];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const int m = (early && s_m >= 0) ? s_m : mdev[0];
  const int nch = min((m + 7) / 8, nchunk_max);
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
  const int64_t r1 = min(N, r0 + rows_per_block);
  const int ntile = r1 > r0 ? (int)((r1 - r0 + kPtRows - 1) / kPtRows) : 0;
  const int nsteps = ntile * nch;
  float* wred = red + (size_t)warp * nchunk_max * NV;
  for (int e = lane; e < nchunk_max * NV; e += 32) wred[e] = 0.f;
  if (tid == 0)
    for (int s = 0; s < kPtStages; ++s) mbar_init(&bar[s], 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  __syncthreads();
  auto issue = [&](int q) {  // step q = (tile q / nch, chunk q % nch) into stage q % kPtStages
    const int t = q / nch, c = q % nch;
    const int64_t i0 = r0 + (int64_t)t * kPtRows;
    const unsigned bytes = (unsigned)(min((int64_t)kPtRows, r1 - i0) * 16);
    uint64_t* b = &bar[q % kPtStages];
    mbar_expect_tx(b, bytes);
    bulk_g2s(stage + (q % kPtStages) * kPtRows, Qp + ((int64_t)c * N + i0) * 8, bytes, b);
  };
  if (tid == 0)
    for (int q = 0; q < min(kPtStages, nsteps); ++q) issue(q);
  float p[kPtRowsPerThread][LP];
  for (int q = 0; q < nsteps; ++q) {
    const int t = q / nch, c = q % nch;
    const int64_t i0 = r0 + (int64_t)t * kPtRows;
    const int rows = (int)min((int64_t)kPtRows, r1 - i0);
    if (c == 0) {  // the tile's priors, seeds masked, for rows tid + 256 u
#pragma unroll
      for (int u = 0; u < kPtRowsPerThread; ++u) {
        const int r = tid + 256 * u;
        const bool use = r < rows && __ldg(seedlab + i0 + r) < 0;
#pragma unroll
        for (int k4 = 0; k4 < LP / 4; ++k4) {
          const float4 v = r < rows ? __ldg(reinterpret_cast<const float4*>(phat + (i0 + r) * LP) + k4)
                                    : make_float4(0.f, 0.f, 0.f, 0.f);
          p[u][4 * k4 + 0] = use ? v.x : 0.f;
          p[u][4 * k4 + 1] = use ? v.y : 0.f;
          p[u][4 * k4 + 2] = use ? v.z : 0.f;
          p[u][4 * k4 + 3] = use ? v.w : 0.f;
        }
      }
    }
    mbar_wait_bounded(&bar[q % kPtStages], (unsigned)((q / kPtStages) & 1), status);
    const uint4* sq = stage + (q % kPtStages) * kPtRows;
    float acc[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) acc[j] = 0.f;
#pragma unroll
    for (int u = 0; u < kPtRowsPerThread; ++u) {
      const int r = tid + 256 * u;
      if (r < rows) {
        float qv[8];
        Vec16<T>::unpack(sq[r], qv);
#pragma unroll
        for (int v = 0; v < 8; ++v)
#pragma unroll
          for (int k = 0; k < LP; ++k) acc[v * LP + k] = fmaf(qv[v], p[u][k], acc[v * LP + k]);
      }
    }
#pragma unroll
    for (int gq = 0; gq < NG; ++gq) {
      float val[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) val[j] = acc[32 * gq + j];
      const float sum = reduce_scatter32(val, lane);  // lane j: product 32 gq + j
      wred[c * NV + 32 * gq + lane] += sum;
    }
    __syncthreads();  // stage q % kPtStages consumed
    if (tid == 0 && q + kPtStages < nsteps) issue(q + kPtStages);
  }
  __syncthreads();
  float* pb = part + (int64_t)blockIdx.x * nchunk_max * NV;
  for (int e = tid; e < nchunk_max * NV; e += blockDim.x) {
    float v = 0.f;
    if (e / NV < nch)
      for (int w = 0; w < nw; ++w) v += red[(size_t)w * nchunk_max * NV + e];
    pb[e] = v;
  }
  if (early) rw_grid_wait();
}

constexpr int kBackChunks = 8;  // 16-byte chunks per row in flight in the back-projection

// VPI voxels per loop iteration, kBackChunks / VPI chunks of each in flight (all of an
// iteration's loads issued before its arithmetic): VPI > 1 when few chunks are used, so that a
// thread still keeps kBackChunks 16-byte loads in flight
template <typename T, int LP, int VPI>
__device__ __forceinline__ void backproject_rows(const T* __restrict__ Qp, int64_t N, int nch,
                                                 const float* Cs, const int* __restrict__ seedlab,
                                                 const float* __restrict__ sq,
                                                 const float* __restrict__ s, int L,
                                                 float* __restrict__ xhat, float* __restrict__ U,
                                                 uint8_t* __restrict__ labels, int* clear_seedlab,
                                                 const float* nul) {
  constexpr int CPI = kBackChunks / VPI;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < N; i0 += VPI * stride) {
    int sl[VPI];
    float acc[VPI][LP];
#pragma unroll
    for (int w = 0; w < VPI; ++w) {
      const int64_t i = i0 + w * stride;
      sl[w] = i < N ? __ldg(seedlab + i) : 0;
#pragma unroll
      for (int k = 0; k < LP; ++k) acc[w][k] = 0.f;
    }
    for (int c = 0; c < nch; c += CPI) {
      uint4 raw[VPI][CPI];
#pragma unroll
      for (int w = 0; w < VPI; ++w) {
        const int64_t i = i0 + w * stride;
#pragma unroll
        for (int u = 0; u < CPI; ++u)
          raw[w][u] = (i < N && c + u < nch)
              ? __ldg(reinterpret_cast<const uint4*>(Qp + ((int64_t)(c + u) * N + i) * 8))
              : make_uint4(0, 0, 0, 0);
      }
#pragma unroll
      for (int u = 0; u < CPI; ++u) {
        if (c + u < nch) {  // uniform over the block
#pragma unroll
          for (int w = 0; w < VPI; ++w) {
            float q[8];
            Vec16<T>::unpack(raw[w][u], q);
#pragma unroll
            for (int v = 0; v < 8; ++v) {
              const float4* cr = reinterpret_cast<const float4*>(Cs + ((c + u) * 8 + v) * LP);
#pragma unroll
              for (int k4 = 0; k4 < LP / 4; ++k4) {
                const float4 cv = cr[k4];
                acc[w][4 * k4 + 0] = fmaf(q[v], cv.x, acc[w][4 * k4 + 0]);
                acc[w][4 * k4 + 1] = fmaf(q[v], cv.y, acc[w][4 * k4 + 1]);
                acc[w][4 * k4 + 2] = fmaf(q[v], cv.z, acc[w][4 * k4 + 2]);
                acc[w][4 * k4 + 3] = fmaf(q[v], cv.w, acc[w][4 * k4 + 3]);
              }
            }
          }
        }
      }
    }
    if (nul) {  // gamma = 0: + g_i c_eff on the unseeded rows (g_i = sq_i / ||sq||, in nul)
#pragma unroll
      for (int w = 0; w < VPI; ++w) {
        const int64_t i = i0 + w * stride;
        if (i < N && sl[w] < 0) {
          const float sqi = sq[i];
#pragma unroll
          for (int k = 0; k < LP; ++k) acc[w][k] = fmaf(sqi, nul[k], acc[w][k]);
        }
      }
    }
#pragma unroll
    for (int w = 0; w < VPI; ++w) {
      const int64_t i = i0 + w * stride;
      if (i >= N) break;
      if (xhat) {
        float4* xo = reinterpret_cast<float4*>(xhat + i * LP);
#pragma unroll
        for (int k4 = 0; k4 < LP / 4; ++k4) {
          float o[4];
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            const int k = 4 * k4 + t;
            o[t] = (k >= L) ? 0.f : ((sl[w] >= 0) ? (k == sl[w] ? sq[i] : 0.f) : acc[w][k]);
          }
          xo[k4] = make_float4(o[0], o[1], o[2], o[3]);
        }
      } else {
        const float si = s[i];
        int best = 0;
        float bv = -INFINITY;
#pragma unroll
        for (int k = 0; k < LP; ++k) {
          if (k < L) {
            const float u = (sl[w] >= 0) ? (k == sl[w] ? 1.f : 0.f) : acc[w][k] * si;
            U[i * L + k] = u;
            if (u > bv) { bv = u; best = k; }
          }
        }
        if (labels) labels[i] = (uint8_t)best;
        if (clear_seedlab && sl[w] >= 0) clear_seedlab[i] = -1;
      }
    }
  }
}

template <typename T, int LP>
__global__ void __launch_bounds__(256, 3)
k_backproject_panel(const T* __restrict__ Qp, int64_t N, int nchunk_max,
                    const float* __restrict__ Cg, float cscale, const int* __restrict__ seedlab,
                    const float* __restrict__ sq, const float* __restrict__ s, int L,
                    const int* __restrict__ mdev, float* __restrict__ xhat,
                    float* __restrict__ U, uint8_t* __restrict__ labels, int* clear_seedlab,
                    const float* __restrict__ nulg) {
  rw_grid_wait();
  rw_grid_trigger();
  extern __shared__ float Cs[];  // (8 nchunk_max, rounded up to kBackChunks chunks) x LP, + LP
  const int m = mdev[0];
  const int nch = min((m + 7) / 8, nchunk_max);
  const int ncs = (nchunk_max + kBackChunks - 1) / kBackChunks * kBackChunks;
  for (int e = threadIdx.x; e < ncs * 8 * LP; e += blockDim.x)
    Cs[e] = e < nchunk_max * 8 * LP ? Cg[e] * cscale : 0.f;
  float* nul = nulg ? Cs + ncs * 8 * LP : nullptr;
  if (nulg && threadIdx.x < LP) nul[threadIdx.x] = nulg[threadIdx.x];
  __syncthreads();
  // seed rows discard the products (their flag is loaded with the first chunks)
  if constexpr (LP <= 8) {  // (16 labels: the four-voxel form would spill)
    if (nch <= kBackChunks / 4) {
      backproject_rows<T, LP, 4>(Qp, N, nch, Cs, seedlab, sq, s, L, xhat, U, labels, clear_seedlab, nul);
      return;
    }
  }
  if (nch <= kBackChunks / 2)
    backproject_rows<T, LP, 2>(Qp, N, nch, Cs, seedlab, sq, s, L, xhat, U, labels, clear_seedlab, nul);
  else
    backproject_rows<T, LP, 1>(Qp, N, nch, Cs, seedlab, sq, s, L, xhat, U, labels, clear_seedlab, nul);
}

// ---------------------------------------------------------------------------------------
// Damped Jacobi on Eq. (rw_eq) in hat variables: for an unseeded voxel
//   x_i <- (1 - omega) x_i + omega / a_ii (gamma p-hat_i + sum_j c_ij x_j),
// a_ii = 1 + gamma (L-hat) or d_i + gamma (L); seeded voxels keep x = U-hat_s.  The last step
// writes U = s * x (seeds one-hot) and the argmax labels.
// ---------------------------------------------------------------------------------------
template <int LP>
__global__ void __launch_bounds__(256)
k_jacobi_step(const float* __restrict__ xin, float* __restrict__ xout,
              const float* __restrict__ phat, const int* __restrict__ seedlab,
              const float* __restrict__ cw, const float* __restrict__ d,
              const float* __restrict__ s, int normalized, int kind, int ndim, int DX, int DY,
              int DZ, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colv,
              const float* __restrict__ ccsr, int64_t N, int L, float gamma, float omega,
              int last, float* __restrict__ U, uint8_t* __restrict__ labels, int* clear_seedlab) {
  rw_grid_wait();
  rw_grid_trigger();
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  constexpr int NV = LP / 4;
  const float4* xi4 = reinterpret_cast<const float4*>(xin);
  float4 x[NV];
#pragma unroll
  for (int t = 0; t < NV; ++t) x[t] = xi4[i * NV + t];
  const int sl = seedlab[i];
  if (sl < 0) {
    float4 acc[NV];
#pragma unroll
    for (int t = 0; t < NV; ++t) acc[t] = make_float4(0.f, 0.f, 0.f, 0.f);
    auto add = [&](int64_t j, float c) {
#pragma unroll
      for (int t = 0; t < NV; ++t) {
        float4 v = xi4[j * NV + t];
        acc[t].x = fmaf(c, v.x, acc[t].x); acc[t].y = fmaf(c, v.y, acc[t].y);
        acc[t].z = fmaf(c, v.z, acc[t].z); acc[t].w = fmaf(c, v.w, acc[t].w);
      }
    };
    if (kind == RW_GRAPH_GRID) {
      const int64_t st[3] = {1, (int64_t)DX, (int64_t)DX * DY};
      const int cc[3] = {(int)(i % DX), (int)((i / DX) % DY), (int)(i / ((int64_t)DX * DY))};
      const int n[3] = {DX, DY, DZ};
      for (int a = 0; a < ndim; ++a) {
        if (cc[a] > 0) add(i - st[a], cw[a * N + i - st[a]]);
        if (cc[a] + 1 < n[a]) add(i + st[a], cw[a * N + i]);
      }
    } else {
      for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) add(colv[p], ccsr[p]);
    }
    const float aii = (normalized ? 1.f : d[i]) + gamma;
    const float f = omega / aii, keep = 1.f - omega;
    const float4* p4 = reinterpret_cast<const float4*>(phat);
#pragma unroll
    for (int t = 0; t < NV; ++t) {
      float4 pv = p4[i * NV + t];
      x[t].x = keep * x[t].x + f * fmaf(gamma, pv.x, acc[t].x);
      x[t].y = keep * x[t].y + f * fmaf(gamma, pv.y, acc[t].y);
      x[t].z = keep * x[t].z + f * fmaf(gamma, pv.z, acc[t].z);
      x[t].w = keep * x[t].w + f * fmaf(gamma, pv.w, acc[t].w);
    }
  }
  if (!last) {
    float4* xo4 = reinterpret_cast<float4*>(xout);
#pragma unroll
    for (int t = 0; t < NV; ++t) xo4[i * NV + t] = x[t];
    return;
  }
  const float* xv = reinterpret_cast<const float*>(x);
  const float si = s[i];
  int best = 0;
  float bv = -INFINITY;
#pragma unroll
  for (int k = 0; k < LP; ++k) {
    if (k < L) {
      const float u = (sl >= 0) ? (k == sl ? 1.f : 0.f) : xv[k] * si;
      U[i * L + k] = u;
      if (u > bv) { bv = u; best = k; }
    }
  }
  if (labels) labels[i] = (uint8_t)best;
  if (clear_seedlab && sl >= 0) clear_seedlab[i] = -1;  // the label array is all -1 again for the next call
}

// The same damped-Jacobi step on a grid graph, launched as a 3-D grid (x in threads, y and z
// in blocks) so a thread finds its voxel and its neighbours without integer division.
template <int LP>
__global__ void __launch_bounds__(128)
k_jacobi_grid(const float* __restrict__ xin, float* __restrict__ xout,
              const float* __restrict__ phat, const int* __restrict__ seedlab,
              const float* __restrict__ cw, const float* __restrict__ d, const float* __restrict__ s,
              int normalized, int ndim, int DX, int DY, int DZ, int64_t N, int L, float gamma,
              float omega, int last, float* __restrict__ U, uint8_t* __restrict__ labels, int* clear_seedlab) {
  rw_grid_wait();
  rw_grid_trigger();
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= DX) return;
  const int y = blockIdx.y, z = blockIdx.z;
  const int64_t sy = DX, sz = (int64_t)DX * DY;
  const int64_t i = x + sy * y + sz * z;
  constexpr int NV = LP / 4;
  const float4* xi4 = reinterpret_cast<const float4*>(xin);
  float4 xv[NV];
#pragma unroll
  for (int t = 0; t < NV; ++t) xv[t] = xi4[i * NV + t];
  // every load of the step is issued before the seed flag is tested (one round trip); seed
  // rows keep their value
  const int sl = seedlab[i];
  float4 acc[NV];
#pragma unroll
  for (int t = 0; t < NV; ++t) acc[t] = make_float4(0.f, 0.f, 0.f, 0.f);
  auto add = [&](int64_t j, float c) {
#pragma unroll
    for (int t = 0; t < NV; ++t) {
      const float4 v = xi4[j * NV + t];
      acc[t].x = fmaf(c, v.x, acc[t].x); acc[t].y = fmaf(c, v.y, acc[t].y);
      acc[t].z = fmaf(c, v.z, acc[t].z); acc[t].w = fmaf(c, v.w, acc[t].w);
    }
  };
  if (x > 0) add(i - 1, cw[i - 1]);
  if (x + 1 < DX) add(i + 1, cw[i]);
  if (y > 0) add(i - sy, cw[N + i - sy]);
  if (y + 1 < DY) add(i + sy, cw[N + i]);
  if (ndim == 3) {
    if (z > 0) add(i - sz, cw[2 * N + i - sz]);
    if (z + 1 < DZ) add(i + sz, cw[2 * N + i]);
  }
  const float aii = (normalized ? 1.f : d[i]) + gamma;
  const float4* p4 = reinterpret_cast<const float4*>(phat);
  float4 pv[NV];
#pragma unroll
  for (int t = 0; t < NV; ++t) pv[t] = p4[i * NV + t];
  if (sl < 0) {
    const float f = omega / aii, keep = 1.f - omega;
#pragma unroll
    for (int t = 0; t < NV; ++t) {
      xv[t].x = keep * xv[t].x + f * fmaf(gamma, pv[t].x, acc[t].x);
      xv[t].y = keep * xv[t].y + f * fmaf(gamma, pv[t].y, acc[t].y);
      xv[t].z = keep * xv[t].z + f * fmaf(gamma, pv[t].z, acc[t].z);
      xv[t].w = keep * xv[t].w + f * fmaf(gamma, pv[t].w, acc[t].w);
    }
  }
  if (!last) {
    float4* xo4 = reinterpret_cast<float4*>(xout);
#pragma unroll
    for (int t = 0; t < NV; ++t) xo4[i * NV + t] = xv[t];
    return;
  }
  const float* xf = reinterpret_cast<const float*>(xv);
  const float si = s[i];
  int best = 0;
  float bv = -INFINITY;
#pragma unroll
  for (int k = 0; k < LP; ++k) {
    if (k < L) {
      const float u = (sl >= 0) ? (k == sl ? 1.f : 0.f) : xf[k] * si;
      U[i * L + k] = u;
      if (u > bv) { bv = u; best = k; }
    }
  }
  if (labels) labels[i] = (uint8_t)best;
  if (clear_seedlab && sl >= 0) clear_seedlab[i] = -1;  // the label array is all -1 again for the next call
}

// A damped-Jacobi step for wide rows (LP >= 16 labels) on a grid graph: one thread per (voxel,
// 4-label chunk), so that the row loads of a warp are contiguous; the neighbour terms are added
// in the order of k_jacobi_grid (same result).  The last step writes U = s * x (seeds one-hot)
// for the first L labels; it does not form the hard labels (a row spans several threads).
template <int LP>
__global__ void __launch_bounds__(256)
k_jacobi_wide(const float* __restrict__ xin, float* __restrict__ xout,
              const float* __restrict__ phat, const int* __restrict__ seedlab,
              const float* __restrict__ cw, const float* __restrict__ d,
              const float* __restrict__ s, int normalized, int ndim, int DX, int DY, int DZ,
              int64_t N, float gamma, float omega, int L, float* __restrict__ U) {
  rw_grid_wait();
  rw_grid_trigger();
  constexpr int NV = LP / 4;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= DX * NV) return;
  const int x = t / NV, c = t % NV;
  const int y = blockIdx.y, z = blockIdx.z;
  const int64_t sy = DX, sz = (int64_t)DX * DY;
  const int64_t i = x + sy * y + sz * z;
  const float4* x4 = reinterpret_cast<const float4*>(xin);
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  const bool hx0 = x > 0, hx1 = x + 1 < DX, hy0 = y > 0, hy1 = y + 1 < DY;
  const bool hz0 = ndim == 3 && z > 0, hz1 = ndim == 3 && z + 1 < DZ;
  const float4 xo = x4[i * NV + c];
  const float4 v0 = hx0 ? x4[(i - 1) * NV + c] : zero, v1 = hx1 ? x4[(i + 1) * NV + c] : zero;
  const float4 v2 = hy0 ? x4[(i - sy) * NV + c] : zero, v3 = hy1 ? x4[(i + sy) * NV + c] : zero;
  const float4 v4 = hz0 ? x4[(i - sz) * NV + c] : zero, v5 = hz1 ? x4[(i + sz) * NV + c] : zero;
  const float c0 = hx0 ? cw[i - 1] : 0.f, c1 = hx1 ? cw[i] : 0.f;
  const float c2 = hy0 ? cw[N + i - sy] : 0.f, c3 = hy1 ? cw[N + i] : 0.f;
  const float c4 = hz0 ? cw[2 * N + i - sz] : 0.f, c5 = hz1 ? cw[2 * N + i] : 0.f;
  const float4 pv = reinterpret_cast<const float4*>(phat)[i * NV + c];
  const int sl = seedlab[i];
  const float aii = (normalized ? 1.f : d[i]) + gamma;
  float4 acc = zero;
  auto add = [&](bool h, float cc, float4 v) {
    if (!h) return;
    acc.x = fmaf(cc, v.x, acc.x); acc.y = fmaf(cc, v.y, acc.y);
    acc.z = fmaf(cc, v.z, acc.z); acc.w = fmaf(cc, v.w, acc.w);
  };
  add(hx0, c0, v0); add(hx1, c1, v1); add(hy0, c2, v2); add(hy1, c3, v3);
  add(hz0, c4, v4); add(hz1, c5, v5);
  float4 o = xo;
  if (sl < 0) {
    const float f = omega / aii, keep = 1.f - omega;
    o.x = keep * xo.x + f * fmaf(gamma, pv.x, acc.x);
    o.y = keep * xo.y + f * fmaf(gamma, pv.y, acc.y);
    o.z = keep * xo.z + f * fmaf(gamma, pv.z, acc.z);
    o.w = keep * xo.w + f * fmaf(gamma, pv.w, acc.w);
  }
  if (!U) {
    reinterpret_cast<float4*>(xout)[i * NV + c] = o;
    return;
  }
  const float si = s[i];
  const float ov[4] = {o.x, o.y, o.z, o.w};
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const int k = 4 * c + t;
    if (k < L) U[i * L + k] = (sl >= 0) ? (k == sl ? 1.f : 0.f) : ov[t] * si;
  }
}

template <int LP>
rw_status launch_jacobi(const rw_graph* g, const float* xin, float* xout, const float* phat,
                        const int* seedlab, int L, float gamma, float omega, int last,
                        float* U, uint8_t* labels, int* clear, cudaStream_t st) {
  if (g->kind == RW_GRAPH_GRID && LP >= 16 && (!last || (!labels && !clear))) {
    const dim3 grid((unsigned)((g->dims[0] * (LP / 4) + 255) / 256), (unsigned)g->dims[1],
                    (unsigned)g->dims[2]);
    RW_LAUNCH((k_jacobi_wide<LP>), grid, 256, 0, st, xin, xout, phat, seedlab, g->cw, g->d, g->s,
              g->normalized, g->ndim, g->dims[0], g->dims[1], g->dims[2], g->N, gamma, omega, L,
              last ? U : nullptr);
    return RW_OK;
  }
  if (g->kind == RW_GRAPH_GRID) {
    const dim3 grid((unsigned)((g->dims[0] + 127) / 128), (unsigned)g->dims[1], (unsigned)g->dims[2]);
    RW_LAUNCH((k_jacobi_grid<LP>), grid, 128, 0, st, xin, xout, phat, seedlab, g->cw, g->d, g->s,
              g->normalized, g->ndim, g->dims[0], g->dims[1], g->dims[2], g->N, L, gamma, omega,
              last, U, labels, clear);
    return RW_OK;
  }
  RW_LAUNCH((k_jacobi_step<LP>), rw_blocks(g->N, 256), 256, 0, st,
      xin, xout, phat, seedlab, g->cw, g->d, g->s, g->normalized, g->kind, g->ndim, g->dims[0],
      g->dims[1], g->dims[2], g->rowptr, g->col, g->ccsr, g->N, L, gamma, omega, last, U,
      labels, clear);
  return RW_OK;
}

rw_status jacobi(const rw_graph* g, int lp, const float* xin, float* xout, const float* phat,
                 const int* seedlab, int L, float gamma, float omega, int last, float* U,
                 uint8_t* labels, int* clear, cudaStream_t st) {
  switch (lp) {
    case 4: return launch_jacobi<4>(g, xin, xout, phat, seedlab, L, gamma, omega, last, U, labels, clear, st);
    case 8: return launch_jacobi<8>(g, xin, xout, phat, seedlab, L, gamma, omega, last, U, labels, clear, st);
    case 16: return launch_jacobi<16>(g, xin, xout, phat, seedlab, L, gamma, omega, last, U, labels, clear, st);
    default: return launch_jacobi<32>(g, xin, xout, phat, seedlab, L, gamma, omega, last, U, labels, clear, st);
  }
}

template <typename T, int LP>
rw_status launch_proj_back(bool back, const T* Q, int ldq, const float* phat,
                           const int* seedlab, const rw_graph* g, const int* mdev, float* part,
                           int nblk, const float* C, float cscale, float* xhat, float* U,
                           uint8_t* labels, int L, int* clear, const float* nul, cudaStream_t st,
                           int early = 0) {
  constexpr int V = Vec16<T>::V;
  const int cpr = ldq / V;
  if constexpr (V == 8) {  // 16-bit copies: panel-major layout, ldq = 8 x chunks
    const int nchunk = ldq / 8;
    if (rw_tc_passes(ldq, back ? 2 : 1, LP)) {   // tensor cores (the caller sized nblk, scale)
      if (!back)
        return rw_project_tc<T>(Q, g->N, nchunk, phat, LP, seedlab, mdev, part, nblk, g->status, st);
      return rw_backproject_tc<T>(Q, g->N, nchunk, C, LP, cscale, seedlab, g->sq, g->s, L, mdev,
                                  xhat, U, labels, clear, nul, g->status, nblk, st);
    }
    if (!back) {
      const int64_t rpb = (g->N + nblk - 1) / nblk;
      if constexpr (LP <= 8) {
        const size_t shm = sizeof(uint4) * kPtStages * kPtRows + sizeof(float) * 8 * (size_t)nchunk * 8 * LP;
        RW_CHECK_CUDA(ensure_smem(k_project_tma<T, LP>, shm));
        RW_LAUNCH((k_project_tma<T, LP>), nblk, 256, shm, st, Q, g->N, nchunk, phat, seedlab, mdev,
                  rpb, part, g->status, early);
      } else {
        const size_t shm = sizeof(float) * kParts * (size_t)nchunk * 8 * LP;
        if (shm > 48 * 1024)
          RW_CHECK_CUDA(ensure_smem(k_project_cw<T, LP>, shm));
        RW_LAUNCH((k_project_cw<T, LP>), nblk, 256, shm, st, Q, g->N, nchunk, phat, seedlab, mdev,
                  rpb, part);
      }
    } else {
      const size_t shm = sizeof(float) * ((size_t)((nchunk + kBackChunks - 1) / kBackChunks * kBackChunks) * 8 * LP + LP);
      RW_LAUNCH((k_backproject_panel<T, LP>), nblk, 256, shm, st, Q, g->N, nchunk, C, cscale, seedlab,
                                                        g->sq, g->s, L, mdev, xhat, U, labels, clear, nul);
    }
    RW_LAUNCH_CHECK();
    return RW_OK;
  } else {
  if (!back) {
    size_t shm = sizeof(float) * ldq * LP;
    if (cpr <= 32)
      RW_LAUNCH((k_project<T, LP, 1>), nblk, 256, shm, st, Q, ldq, cpr, phat, seedlab, g->N, mdev, part);
    else if (cpr <= 64)
      RW_LAUNCH((k_project<T, LP, 2>), nblk, 256, shm, st, Q, ldq, cpr, phat, seedlab, g->N, mdev, part);
    else
      return RW_ERR_UNSUPPORTED;
  } else {
    if (cpr <= 32)
      RW_LAUNCH((k_backproject<T, LP, 1>), nblk, 256, 0, st, Q, ldq, cpr, C, cscale, seedlab, g->sq, g->s,
                                                   g->N, L, mdev, xhat, U, labels, clear, nul);
    else if (cpr <= 64)
      RW_LAUNCH((k_backproject<T, LP, 2>), nblk, 256, 0, st, Q, ldq, cpr, C, cscale, seedlab, g->sq, g->s,
                                                   g->N, L, mdev, xhat, U, labels, clear, nul);
    else
      return RW_ERR_UNSUPPORTED;
  }
  RW_LAUNCH_CHECK();
  return RW_OK;
  }
}

template <typename T>
rw_status proj_back(int lp, bool back, const T* Q, int ldq, const float* phat, const int* seedlab,
                    const rw_graph* g, const int* mdev, float* part, int nblk, const float* C,
                    float cscale, float* xhat, float* U, uint8_t* labels, int L, cudaStream_t st, int* clear = nullptr,
                    const float* nul = nullptr, int early = 0) {
  switch (lp) {
    case 4: return launch_proj_back<T, 4>(back, Q, ldq, phat, seedlab, g, mdev, part, nblk, C, cscale, xhat, U, labels, L, clear, nul, st, early);
    case 8: return launch_proj_back<T, 8>(back, Q, ldq, phat, seedlab, g, mdev, part, nblk, C, cscale, xhat, U, labels, L, clear, nul, st, early);
    case 16: return launch_proj_back<T, 16>(back, Q, ldq, phat, seedlab, g, mdev, part, nblk, C, cscale, xhat, U, labels, L, clear, nul, st);
    default:   // 32 labels per pass: the tensor-core kernels only
      if constexpr (Vec16<T>::V == 8) {
        if (rw_tc_passes(ldq, back ? 2 : 1, 32)) {
          if (!back)
            return rw_project_tc<T>(Q, g->N, ldq / 8, phat, 32, seedlab, mdev, part, nblk, g->status, st);
          return rw_backproject_tc<T>(Q, g->N, ldq / 8, C, 32, cscale, seedlab, g->sq, g->s, L, mdev,
                                      xhat, U, labels, clear, nul, g->status, nblk, st);
        }
      }
      return RW_ERR_UNSUPPORTED;
  }
}

// ---------------------------------------------------------------------------------------
// gamma = 0 (Sec. II-B, after Eq. Fs): L-hat has the null vector g = sq / ||sq|| and E is its
// pseudo-inverse, so the seeded system gains the column sums c = g^T U-hat as unknowns.  The
// stored column 0 is taken as the null direction and replaced by g, the other columns are
// projected orthogonal to g (Q' = Q - g w^T, w_j = g^T q_j), and row 0 of the m x m system
// becomes the column-sum equation:
//   k_seed_gather  also writes g_t and (B-hat g_n)_t per seed
//   k_null_fill    P-hat column 0 := g (the projection then gives w^n = Q_n^T g_n)
//   k_null_w       partial sums of p = Q_s^T g_s (fixed order)
//   k_null_rows    w = w^n + p; seed rows Q_s' = [g_s, Q_s - g_s w^T], X' = [B g_n, X - B g_n w^T]
//   (seed Gram: K, G, h, b on the basis [g, Q'])
//   k_null_row0    s = g_s^T g_s; M_00 = s, M_0j = -(w^n_j - w_j (1 - s)), h_0 = g_s^T U-hat_s
//   (adaptive m, LU, C = M^{-1} h)
//   k_null_coef    c_eff = c - w^T C' (C row 0 := 0), added as g_i c_eff by the back-projection
// ---------------------------------------------------------------------------------------
template <int LP>
__global__ void k_null_fill(float* __restrict__ phat, const float* __restrict__ sq, int64_t N,
                            float ginv) {
  rw_grid_wait();
  rw_grid_trigger();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    float4* row = reinterpret_cast<float4*>(phat + i * LP);
    row[0] = make_float4(sq[i] * ginv, 0.f, 0.f, 0.f);
#pragma unroll
    for (int k4 = 1; k4 < LP / 4; ++k4) row[k4] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

constexpr int kNullSplit = 16;   // seed ranges of the p = Q_s^T g_s partial sums (the layout's partw)

// grid (ceil(mmax / 32), ny): block (x, y) sums g_t Q_s[t, c] over seed range y for the 32
// columns c of x; warps take seeds strided by 8 and are added in order
__global__ void __launch_bounds__(256)
k_null_w(const float* __restrict__ Qs, int ldb, const float* __restrict__ gnull, int S, int mmax,
         float* __restrict__ partw, int mq) {
  rw_grid_wait();
  rw_grid_trigger();
  __shared__ float red[8][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = blockIdx.x * 32 + lane;
  const int chunk = (S + gridDim.y - 1) / gridDim.y;
  const int t0 = blockIdx.y * chunk, t1 = min(S, t0 + chunk);
  float acc = 0.f;
  if (c < mmax)
    for (int t = t0 + warp; t < t1; t += 8) acc = fmaf(gnull[2 * t], Qs[(int64_t)t * ldb + c], acc);
  red[warp][lane] = acc;
  __syncthreads();
  if (warp == 0 && c < mmax) {
    float v = 0.f;
#pragma unroll
    for (int w = 0; w < 8; ++w) v += red[w][lane];
    partw[(size_t)blockIdx.y * mq + c] = v;
  }
}

__global__ void __launch_bounds__(256)
k_null_rows(float* __restrict__ Bcat, int ldb, int mp, const float* __restrict__ gnull, int S,
            int mmax, const float* __restrict__ partw, int ny, int mq,
            const float* __restrict__ Z, int lp, float* __restrict__ wv) {
  rw_grid_wait();
  rw_grid_trigger();
  __shared__ float w[kMaxSmallM];
  for (int j = threadIdx.x; j < mmax; j += blockDim.x) {
    float v = Z[(size_t)j * lp];                       // w^n_j
    for (int y = 0; y < ny; ++y) v += partw[(size_t)y * mq + j];
    w[j] = j == 0 ? 0.f : v;
    if (blockIdx.x == 0) wv[j] = w[j];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  for (int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < S;
       t += (gridDim.x * blockDim.x) >> 5) {
    const float gt = gnull[2 * t], bt = gnull[2 * t + 1];
    float* xs = Bcat + (int64_t)t * ldb;
    float* qs = xs + mp;
    for (int c = lane; c < mmax; c += 32) {
      if (c == 0) {
        xs[0] = bt;
        qs[0] = gt;
      } else {
        xs[c] = fmaf(-bt, w[c], xs[c]);
        qs[c] = fmaf(-gt, w[c], qs[c]);
      }
    }
  }
}

// one CTA: row 0 of K, h (M = diag(lambda0) - K, lambda0_0 = s) after the seed Gram; Z zeroed
// once w^n is read (gamma Z = 0 then needs no 0 x inf guard)
__global__ void __launch_bounds__(256)
k_null_row0(float* __restrict__ Gcat, int mp, int lp, int mmax, const float* __restrict__ wv,
            float* __restrict__ Z, int mq, const double* __restrict__ lam,
            double* __restrict__ lam0, float* __restrict__ lgam) {
  rw_grid_wait();
  rw_grid_trigger();
  const float sv = Gcat[mp];          // G_00 = g_s^T g_s
  for (int j = threadIdx.x; j < mmax; j += blockDim.x) {
    Gcat[j] = j == 0 ? 0.f : Z[(size_t)j * lp] - wv[j] * (1.f - sv);
    lam0[j] = j == 0 ? (double)sv : lam[j];
  }
  if (threadIdx.x < lp) Gcat[2 * mp + threadIdx.x] = Gcat[2 * mp + lp + threadIdx.x];
  if (threadIdx.x == 0) lgam[0] = sv;
  __syncthreads();
  for (int e = threadIdx.x; e < mq * lp; e += blockDim.x) Z[e] = 0.f;
}

// one CTA, a warp per label: c_eff_k = C_0k - sum_{j >= 1} w_j C_jk (lanes strided, butterfly),
// nul_k = c_eff_k / ||sq||, C_0k := 0
__global__ void __launch_bounds__(256)
k_null_coef(float* __restrict__ C, int lp, int L, const int* __restrict__ mdev,
            const float* __restrict__ wv, float ginv, float* __restrict__ nul) {
  rw_grid_wait();
  rw_grid_trigger();
  __shared__ float ce[RW_MAX_LABELS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int m = mdev[0];
  for (int k = warp; k < lp; k += nw) {
    float v = 0.f;
    for (int j = 1 + lane; j < m; j += 32) v = fmaf(wv[j], C[(size_t)j * lp + k], v);
    v = warp_sum(v);
    if (lane == 0) ce[k] = k < L ? (C[k] - v) * ginv : 0.f;
  }
  __syncthreads();
  if (threadIdx.x < lp) {
    nul[threadIdx.x] = ce[threadIdx.x];
    C[threadIdx.x] = 0.f;
  }
}

// An empty launch between k_adapt_lu and k_small_rhs when no projection runs between them
// (gamma = 0): k_small_rhs copies the factors in ahead of its own grid dependency wait, which
// is safe only two launches behind their producer.
__global__ void k_pdl_fence(int) {
  rw_grid_wait();
  rw_grid_trigger();
}

// BF16 copy in the panel-major layout of the 16-bit basis copies
__global__ void k_f32_to_bf16(const float* __restrict__ a, int64_t N, int m, int lda,
                              __nv_bfloat16* __restrict__ b, int ldb) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * ldb) return;
  int64_t r = e / ldb;
  int col = (int)(e % ldb);
  b[((int64_t)(col / 8) * N + r) * 8 + (col % 8)] = __float2bfloat16(col < m ? a[r * lda + col] : 0.f);
}

}  // namespace


// launches k_seed_gram with the seed rows split over a cluster of up to 8 CTAs along z
// The cluster-fused adaptive choice + LU (k_adapt_lu) when both CTAs' shared memory fits;
// otherwise the caller runs k_adapt / k_set_m and the one-CTA k_small_solve.
template <int LP>
static bool adapt_lu_fits(size_t dyn) {
  static int optin = -1, stat = -1;
  if (optin < 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
      optin = 0;
    cudaFuncAttributes fa;
    stat = cudaFuncGetAttributes(&fa, k_adapt_lu<LP>) == cudaSuccess ? (int)fa.sharedSizeBytes : 1 << 30;
    cudaGetLastError();
  }
  return dyn + (size_t)stat <= (size_t)optin;
}

template <int LP>
static rw_status launch_adapt_lu(size_t shm, cudaStream_t st, const float* G, const float* bv,
                                 const float* Qs, const float* Us, int wcat, int S, int L,
                                 int m_max, int m_step, double rho, double fmax, int adaptive,
                                 const float* K, const double* lam, double gamma, float* F,
                                 int ldf, float* luinv, int* mdev, double* fsel) {
  RW_CHECK_CUDA(ensure_smem(k_adapt_lu<LP>, shm));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2, 1, 1);
  cfg.blockDim = dim3(256, 1, 1);
  cfg.dynamicSmemBytes = shm;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  RW_CHECK_CUDA(cudaLaunchKernelEx(&cfg, k_adapt_lu<LP>, G, wcat, bv, wcat, Qs, wcat, Us, wcat, S,
                                   L, m_max, m_step, rho, fmax, adaptive, K, wcat, lam, gamma, F,
                                   ldf, luinv, mdev, fsel));
  rw_count_launch();
  return RW_OK;
}

static rw_status seed_gram(const float* A, int lda, const float* B, int ldb, int S, int p, int q,
                           float* G, int ldg, cudaStream_t st) {
  // enough CTAs along z that each holds at most one stage of rows (up to the cluster limit)
  const int nz = std::max(1, std::min(kSgMaxCluster, (S + kSgRows - 1) / kSgRows));
  const size_t shm = sizeof(float4) * 2 * kSgRows * 17;
  RW_CHECK_CUDA(ensure_smem(k_seed_gram, shm));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((p + kSgT - 1) / kSgT, (q + kSgT - 1) / kSgT, nz);
  cfg.blockDim = dim3(256, 1, 1);
  cfg.dynamicSmemBytes = shm;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 1;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = nz;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  RW_CHECK_CUDA(cudaLaunchKernelEx(&cfg, k_seed_gram, A, lda, B, ldb, S, p, q, G, ldg));
  rw_count_launch();
  return RW_OK;
}

// ---------------------------------------------------------------------------------------
// Seed bookkeeping and priors, shared by the fast solve, the PCG solve and the gradients
// ---------------------------------------------------------------------------------------
rw_status rw_solve_priors_internal(const rw_graph* g, const int32_t* seed_idx,
                                   const int32_t* seed_lab, int S, int L, int prior_mode,
                                   const float* priors, int lp, cudaStream_t st, float** phat_out,
                                   int** seedlab_out, double** fit64_out, bool defer_priors) {
  rw_graph* gm = const_cast<rw_graph*>(g);
  SolveWorkspace& ws = gm->ws;
  if (S > kMaxSeeds || S < 0) return RW_ERR_INVALID_ARG;
  if (S == 0 && prior_mode != 1) return RW_ERR_INVALID_ARG;   // no seeds: priors are given
  const size_t cap0 = ws.seedlab.cap;
  RW_TRY(ws.seedlab.grow(sizeof(int) * g->N));
  if (ws.seedlab.cap != cap0) ws.seeds_clean = false;
  RW_TRY(ws.phat.grow(sizeof(float) * g->N * lp));
  const int nsb = (S + 255) / 256;
  const size_t need = 4096 + sizeof(float) * (size_t)nsb * 3 * L;
  RW_TRY(ws.seedpart.grow(need));
  float* bpart = reinterpret_cast<float*>(ws.seedpart.as<char>() + 4096);
  double* fit64 = ws.seedpart.as<double>();
  int* seedlab = ws.seedlab.as<int>();
  // the labels array is all -1 between calls when the previous call's last kernel cleared its
  // seeds (rw_solve does); otherwise reset it here
  if (!ws.seeds_clean)
    RW_LAUNCH(k_seed_reset, rw_blocks(g->N, 256), 256, 0, st, seedlab, g->N, nullptr, 0);
  ws.seeds_clean = S == 0;   // nothing scattered: the label array stays all -1
  ws.seed_nsb = nsb;
  if (S > 0)
    RW_LAUNCH(k_seed_scatter, nsb, 256, 0, st, seed_idx, seed_lab, S, L, g->N,
              g->J ? g->J : nullptr, seedlab, bpart, g->status);
  if (!defer_priors) RW_TRY(launch_priors(g, L, prior_mode, priors, lp, 0, st));
  *phat_out = ws.phat.as<float>();
  *seedlab_out = seedlab;
  if (fit64_out) *fit64_out = fit64;
  return RW_OK;
}

// The priors kernel for the seeds scattered by the last rw_solve_priors_internal call on g;
// early = 1 when other kernels were launched in between (see k_priors).
rw_status launch_priors(const rw_graph* g, int L, int prior_mode, const float* priors, int lp,
                        int early, cudaStream_t st) {
  SolveWorkspace& ws = const_cast<rw_graph*>(g)->ws;
  const int nsb = ws.seed_nsb;
  float* bpart = reinterpret_cast<float*>(ws.seedpart.as<char>() + 4096);
  double* fit64 = ws.seedpart.as<double>();
  const int sms = g_rw_num_sms > 0 ? g_rw_num_sms : 148;
  const int pblk = (int)std::min<int64_t>(rw_blocks((g->N + 3) / 4, 256), 8 * sms);
  if (lp == 4)
    RW_LAUNCH(k_priors<4>, pblk, 256, 0, st, g->J, g->sq, g->N, L, prior_mode,
              bpart, nsb, fit64, priors, ws.phat.as<float>(), g->status, early);
  else if (lp == 8)
    RW_LAUNCH(k_priors<8>, pblk, 256, 0, st, g->J, g->sq, g->N, L, prior_mode,
              bpart, nsb, fit64, priors, ws.phat.as<float>(), g->status, early);
  else
    RW_LAUNCH(k_priors<16>, pblk, 256, 0, st, g->J, g->sq, g->N, L, prior_mode,
              bpart, nsb, fit64, priors, ws.phat.as<float>(), g->status, early);
  return RW_OK;
}

// Which 16-bit basis passes run on the tensor cores (csrc/proj_tc.cu), set by rw_set_tc_passes:
// bit 0 the projection, bit 1 the back-projection, bit 2 (the default) both for passes that
// carry 16 or more padded labels; copies wider than 256 columns keep the CUDA-core kernels.
namespace {
std::atomic<int> g_tc_passes{4};
}
bool rw_tc_passes(int ld16, int which, int lp) {
  const int mode = g_tc_passes.load(std::memory_order_relaxed);
  return ld16 <= 256 && ((mode & which) != 0 || ((mode & 4) != 0 && lp >= 16));
}
extern "C" rw_status rw_set_tc_passes(int32_t mask) {
  if (mask < 0 || mask > 4) return RW_ERR_INVALID_ARG;
  g_tc_passes.store(mask);
  return RW_OK;
}

// Launch shapes of the two 16-bit basis passes (blocks per SM), per graph-size class: entry k
// applies to graphs with N <= nmax_k (the first such entry, classes ascending).  Set by
// rw_set_launch_shape from a table the project's autotuner measures; without an entry the
// projection takes 2 blocks per SM and the back-projection 3.
namespace {
struct ShapeEntry { int64_t nmax; int proj, back; };
std::mutex g_shape_mu;
ShapeEntry g_shapes[16];
int g_nshapes = 0;

void launch_shape(int64_t N, int* proj, int* back) {
  std::lock_guard<std::mutex> lock(g_shape_mu);
  *proj = 2;
  *back = 3;
  for (int k = 0; k < g_nshapes; ++k)
    if (N <= g_shapes[k].nmax) { *proj = g_shapes[k].proj; *back = g_shapes[k].back; return; }
}
}  // namespace

extern "C" rw_status rw_set_launch_shape(int64_t n_max, int32_t proj_per_sm,
                                         int32_t back_per_sm) {
  std::lock_guard<std::mutex> lock(g_shape_mu);
  if (n_max <= 0) { g_nshapes = 0; return RW_OK; }
  if (proj_per_sm < 1 || proj_per_sm > 4 || back_per_sm < 1 || back_per_sm > 8)
    return RW_ERR_INVALID_ARG;
  int k = 0;
  while (k < g_nshapes && g_shapes[k].nmax < n_max) ++k;
  if (k < g_nshapes && g_shapes[k].nmax == n_max) {
    g_shapes[k].proj = proj_per_sm;
    g_shapes[k].back = back_per_sm;
    return RW_OK;
  }
  if (g_nshapes == 16) return RW_ERR_INVALID_ARG;
  for (int j = g_nshapes; j > k; --j) g_shapes[j] = g_shapes[j - 1];
  g_shapes[k] = ShapeEntry{n_max, proj_per_sm, back_per_sm};
  ++g_nshapes;
  return RW_OK;
}

static rw_status validate_solve(const rw_graph* g, const rw_basis* b, const int32_t* si,
                                const int32_t* sl, int S, int L, const float* priors,
                                const rw_solve_opts* o, const void* prob) {
  if (!g || !b || !si || !sl || !o || !prob) return RW_ERR_INVALID_ARG;
  if (b->N != g->N) return RW_ERR_INVALID_ARG;
  if (S < 1 || S > 65536 || L < 1 || L > RW_MAX_LABELS) return RW_ERR_INVALID_ARG;
  if (!(o->gamma >= 0.0)) return RW_ERR_INVALID_ARG;   // negative or NaN
  if (o->m < 0 || o->m > b->m) return RW_ERR_INVALID_ARG;
  if (o->refine_steps < 0 || o->refine_steps > 100000) return RW_ERR_INVALID_ARG;
  if (o->prior_mode != 0 && o->prior_mode != 1) return RW_ERR_INVALID_ARG;
  if (o->gamma > 0.0) {   // gamma = 0 takes no priors
    if (o->prior_mode == 1 && !priors) return RW_ERR_INVALID_ARG;
    if (o->prior_mode == 0 && !g->J) return RW_ERR_INVALID_ARG;
  }
  if (o->basis_format < RW_BASIS_F16 || o->basis_format > RW_BASIS_F32) return RW_ERR_INVALID_ARG;
  if (o->refine_mode != RW_REFINE_JACOBI && o->refine_mode != RW_REFINE_PCG) return RW_ERR_INVALID_ARG;
  int mmax = o->m > 0 ? o->m : b->m;
  if (mmax > kMaxSmallM) return RW_ERR_UNSUPPORTED;
  // one CTA holds an m x m FP32 matrix plus label-sized vectors in shared memory
  const size_t shm_adapt = sizeof(float) * ((size_t)mmax * (mmax | 1) + 3 * (size_t)L * mmax);
  const size_t shm_small = sizeof(float) * ((size_t)mmax * ((mmax + L) | 1) + 2 * (size_t)L * mmax + mmax) +
                           sizeof(int) * mmax;
  // + the kernels' static shared arrays (reciprocal diagonals, broadcast buffers, the
  // shifted copies of the LU panel's diagonal block)
  constexpr size_t kStaticShm = 12 * 1024;
  if (std::max(o->m == 0 ? shm_adapt : 0, shm_small) + kStaticShm > 227 * 1024) return RW_ERR_UNSUPPORTED;
  return RW_OK;
}

rw_status rw_pcg_from(const rw_graph* g, const float* phat, const int* seedlab, int L, int lp,
                      double gamma, float* xhat0, int iters, double tol, float* U,
                      uint8_t* labels, int* iters_done, cudaStream_t st);
rw_status rw_unhat_priors(const rw_graph* g, const float* phat, int lp, int L, float* P,
                          cudaStream_t st);

extern "C" rw_status rw_solve(const rw_graph* g, const rw_basis* b, const int32_t* seed_idx_dev,
                              const int32_t* seed_lab_dev, int32_t S, int32_t n_labels,
                              const float* priors_dev, const rw_solve_opts* opts,
                              float* prob_dev, uint8_t* labels_dev, rw_solve_info* info,
                              void* stream) {
  RW_TRY(validate_solve(g, b, seed_idx_dev, seed_lab_dev, S, n_labels, priors_dev, opts, prob_dev));
  cudaStream_t st = rw_stream(stream);
  rw_graph* gm = const_cast<rw_graph*>(g);
  SolveWorkspace& ws = gm->ws;
  const int L = n_labels, lp = lpad_of(L);
  const int mp = b->ld32;
  const double gamma = opts->gamma;
  const bool g0 = gamma == 0.0;   // no priors: the null-vector form of Sec. II-B
  const int m_step = opts->m_step > 0 ? opts->m_step : 10;
  const double eps = opts->eps > 0 ? opts->eps : 0.1;
  const float omega = (float)(opts->omega > 0 ? std::min(opts->omega, 1.0) : 0.8);
  const bool adaptive = opts->m == 0;
  const int m_max = adaptive ? b->m : opts->m;
  // adaptive candidates: m_step, 2 m_step, ..., m_max (m_max last)
  const int ncand = adaptive ? (m_max + m_step - 1) / m_step : 0;
  const int sms = g_rw_num_sms > 0 ? g_rw_num_sms : 148;
  const int nblk = 4 * sms;  // blocks of the two basis passes (partials of the projection)
  const int mq = std::max(b->ld16, b->ld32);  // rows of Z, C and the partials
  Layout lay = make_layout(S, mp, mq, lp, L, std::max(ncand, 1), nblk);
  RW_TRY(ws.small.grow(lay.total));
  char* base = ws.small.as<char>();
  auto P = [&](size_t off) { return base + off; };
  int* mdev = reinterpret_cast<int*>(P(lay.mdev));

  const bool phases = opts->record_phases && info;
  if (phases) {
    for (auto& e : ws.ev)
      if (!e) RW_CHECK_CUDA(cudaEventCreate(&e));
    RW_CHECK_CUDA(cudaEventRecord(ws.ev[0], st));
  }
  auto mark = [&](int k) -> rw_status {
    if (phases) RW_CHECK_CUDA(cudaEventRecord(ws.ev[k], st));
    return RW_OK;
  };
  float* phat = nullptr;
  int* seedlab = nullptr;
  double* fit64 = nullptr;
  // seeds scattered now; the priors kernel runs behind the seed-side products (it only needs
  // the scatter) and overlaps them
  RW_TRY(rw_solve_priors_internal(g, seed_idx_dev, seed_lab_dev, S, L, opts->prior_mode,
                                  priors_dev, lp, st, &phat, &seedlab, &fit64, true));

  RW_TRY(mark(1));
  const int wcat = 2 * mp + 2 * lp;
  float* Bcat = reinterpret_cast<float*>(P(lay.Bcat));
  float* Gcat = reinterpret_cast<float*>(P(lay.Gcat));
  float* Qs = Bcat + mp;               // S x m_max, row pitch wcat
  float* Us = Bcat + 2 * mp + lp;      // S x lp
  float* K = Gcat;                     // Q_s^T X
  float* G = Gcat + mp;                // Q_s^T Q_s
  float* h = Gcat + 2 * mp;            // Q_s^T r0
  float* bv = Gcat + 2 * mp + lp;      // Q_s^T U-hat_s
  // rho = sqrt(1^T D 1) with the normalized Laplacian (Sec. III-A-1), else sqrt(N); the unit
  // null vector of L-hat is sq / rho
  const double rho = g->normalized ? sqrt(g->dsum) : sqrt((double)g->N);
  const float ginv = (float)(1.0 / rho);
  float* gnull = g0 ? reinterpret_cast<float*>(P(lay.gnull)) : nullptr;
  float* wv = reinterpret_cast<float*>(P(lay.wv));
  float* nul = reinterpret_cast<float*>(P(lay.nul));
  double* lam0 = reinterpret_cast<double*>(P(lay.lam0));
  RW_LAUNCH(k_seed_gather, rw_blocks((int64_t)S * 32, 256), 256, 0, st, 
      seed_idx_dev, seed_lab_dev, S, L, lp, g->N, b->Q32, b->ld32, mp, seedlab, g->cw, g->d,
      g->sq, g->normalized, g->kind, g->ndim, g->dims[0], g->dims[1], g->dims[2], g->rowptr,
      g->col, g->ccsr, (float)gamma, Bcat, wcat, gnull, ginv, mdev + 3);
  float* part = reinterpret_cast<float*>(P(lay.part));
  float* Z = reinterpret_cast<float*>(P(lay.Z));
  float* lgam = Z + (size_t)mq * lp;
  int fmt = opts->basis_format;
  if (fmt == RW_BASIS_BF16 && !b->Qbf) {
    rw_basis* bm = const_cast<rw_basis*>(b);
    RW_CHECK_CUDA(cudaMalloc(&bm->Qbf, sizeof(__nv_bfloat16) * b->N * b->ld16));
    k_f32_to_bf16<<<rw_blocks(b->N * b->ld16, 256), 256, 0, st>>>(b->Q32, b->N, b->m, b->ld32,
                                                                   bm->Qbf, b->ld16);
    RW_LAUNCH_CHECK();
  }
  int ldq_e = fmt == RW_BASIS_F32 ? b->ld32 : b->ld16;
  // projection blocks: the chunk-major 16-bit kernel takes the tuned count per SM (2 by
  // default: more rows per block, fewer partials to add); the FP32 row kernel 4 per SM
  int proj_per_sm = 2, back_per_sm = 3;
  launch_shape(g->N, &proj_per_sm, &back_per_sm);
  // the tensor-core passes hold one CTA per SM and write partials scaled by kTcProjScale
  const bool tc_p = fmt != RW_BASIS_F32 && rw_tc_passes(b->ld16, 1, lp);
  const bool tc_b = fmt != RW_BASIS_F32 && rw_tc_passes(b->ld16, 2, lp);
  const int nblk_p = fmt == RW_BASIS_F32 ? nblk : (tc_p ? sms : proj_per_sm * sms);
  float zscale = (fmt == RW_BASIS_F16 ? 1.f / b->qscale : 1.f) / (tc_p ? kTcProjScale : 1.f);
  float cscale = fmt == RW_BASIS_F16 ? 1.f / b->qscale : 1.f;
  // early (behind the fused k_adapt_lu at a fixed m, on the bulk-copy kernel only): m is
  // published as the kernel starts, so the projection runs beside the whole LU of the m x m
  // system; two SMs hold that cluster, so the grid leaves them out and every block is
  // resident at once.  (With m chosen adaptively the choice ends only a few microseconds
  // before the LU, and the overlap measured no faster.)
  auto project = [&](bool early) -> rw_status {
    const int nb = early ? proj_per_sm * (sms - 2) : nblk_p;
    const int ef = early ? 1 : 0;
    if (fmt == RW_BASIS_F16)
      RW_TRY(proj_back<__half>(lp, false, b->Q16, ldq_e, phat, seedlab, g, mdev, part, nb, nullptr, 0.f, nullptr, nullptr, nullptr, L, st, nullptr, nullptr, ef));
    else if (fmt == RW_BASIS_BF16)
      RW_TRY(proj_back<__nv_bfloat16>(lp, false, b->Qbf, ldq_e, phat, seedlab, g, mdev, part, nb, nullptr, 0.f, nullptr, nullptr, nullptr, L, st, nullptr, nullptr, ef));
    else
      RW_TRY(proj_back<float>(lp, false, b->Q32, ldq_e, phat, seedlab, g, mdev, part, nb, nullptr, 0.f, nullptr, nullptr, nullptr, L, st));
    RW_LAUNCH(k_reduce_partials, rw_blocks((int64_t)std::max(mq * lp, m_max) * 32, 256), 256, 0, st, 
        part, nb, ldq_e, lp, mq, zscale, Z, b->lam, gamma, m_max, lgam, ef);
    return RW_OK;
  };
  if (g0) {
    // w^n = Q_n^T g_n over all m_max columns (P-hat column 0 := g), then the seed rows of the
    // basis [g, Q']
    const int fblk = (int)std::min<int64_t>(rw_blocks(g->N, 256), 8 * sms);
    if (lp == 4) RW_LAUNCH(k_null_fill<4>, fblk, 256, 0, st, phat, g->sq, g->N, ginv);
    else if (lp == 8) RW_LAUNCH(k_null_fill<8>, fblk, 256, 0, st, phat, g->sq, g->N, ginv);
    else RW_LAUNCH(k_null_fill<16>, fblk, 256, 0, st, phat, g->sq, g->N, ginv);
    RW_LAUNCH(k_set_m, 1, 32, 0, st, mdev, m_max);
    RW_TRY(project(false));
    float* partw = reinterpret_cast<float*>(P(lay.partw));
    const int ny = std::max(1, std::min(kNullSplit, (S + 255) / 256));
    RW_LAUNCH(k_null_w, dim3((m_max + 31) / 32, ny), 256, 0, st, Qs, wcat, gnull, S, m_max,
              partw, mq);
    const int rblk = (int)std::min<int64_t>((S + 7) / 8, 2 * sms);
    RW_LAUNCH(k_null_rows, rblk, 256, 0, st, Bcat, wcat, mp, gnull, S, m_max, partw, ny, mq, Z,
              lp, wv);
  }
  RW_TRY(seed_gram(Qs, wcat, Bcat, wcat, S, m_max, wcat, Gcat, wcat, st));
  if (g0)
    RW_LAUNCH(k_null_row0, 1, 256, 0, st, Gcat, mp, lp, m_max, wv, Z, mq, b->lam, lam0, lgam);
  else
    RW_TRY(launch_priors(g, L, opts->prior_mode, priors_dev, lp, phases ? 0 : 1, st));
  const double* lamv = g0 ? lam0 : b->lam;
  double* fu = reinterpret_cast<double*>(P(lay.fu));
  double* fsel = fu + (size_t)(ncand + 1) * RW_MAX_LABELS;
  RW_TRY(mark(2));
  const double fmax = (double)S * eps * eps;
  float* Fac = reinterpret_cast<float*>(P(lay.lu));
  float* luinv = reinterpret_cast<float*>(P(lay.luinv));
  const size_t shm_fused =
      sizeof(float) * std::max((size_t)m_max * (m_max | 1) + 3 * (size_t)L * m_max,
                               (size_t)m_max * lu_stride(m_max) + (size_t)kLuTiles * m_max);
  const bool fused = lp == 4 ? adapt_lu_fits<4>(shm_fused)
                             : (lp == 8 ? adapt_lu_fits<8>(shm_fused) : adapt_lu_fits<16>(shm_fused));
  if (fused) {
    if (lp == 4)
      RW_TRY(launch_adapt_lu<4>(shm_fused, st, G, bv, Qs, Us, wcat, S, L, m_max, m_step, rho, fmax,
                                adaptive, K, lamv, gamma, Fac, mp, luinv, mdev, fsel));
    else if (lp == 8)
      RW_TRY(launch_adapt_lu<8>(shm_fused, st, G, bv, Qs, Us, wcat, S, L, m_max, m_step, rho, fmax,
                                adaptive, K, lamv, gamma, Fac, mp, luinv, mdev, fsel));
    else
      RW_TRY(launch_adapt_lu<16>(shm_fused, st, G, bv, Qs, Us, wcat, S, L, m_max, m_step, rho,
                                 fmax, adaptive, K, lamv, gamma, Fac, mp, luinv, mdev, fsel));
  } else if (adaptive) {
    const size_t shm = sizeof(float) * ((size_t)m_max * (m_max | 1) + 3 * (size_t)L * m_max);
    if (lp == 4) {
      RW_CHECK_CUDA(ensure_smem(k_adapt<4>, shm));
      RW_LAUNCH((k_adapt<4>), 1, 256, shm, st, G, wcat, bv, wcat, Qs, wcat, Us, wcat, S, L, m_max, m_step,
                                      rho, fmax, mdev, fsel);
    } else if (lp == 8) {
      RW_CHECK_CUDA(ensure_smem(k_adapt<8>, shm));
      RW_LAUNCH((k_adapt<8>), 1, 256, shm, st, G, wcat, bv, wcat, Qs, wcat, Us, wcat, S, L, m_max, m_step,
                                      rho, fmax, mdev, fsel);
    } else {
      RW_CHECK_CUDA(ensure_smem(k_adapt<16>, shm));
      RW_LAUNCH((k_adapt<16>), 1, 256, shm, st, G, wcat, bv, wcat, Qs, wcat, Us, wcat, S, L, m_max, m_step,
                                       rho, fmax, mdev, fsel);
    }
    RW_LAUNCH_CHECK();
  } else {
    RW_LAUNCH(k_set_m, 1, 32, 0, st, mdev, m_max);
  }
  RW_TRY(mark(3));
  // Z = Q_n^T P-hat_n (gamma = 0: no priors; Z was zeroed by k_null_row0)
  if (!g0) RW_TRY(project(fused && !adaptive && fmt != RW_BASIS_F32 && !tc_p && lp <= 8 && sms > 8));
  else if (fused) RW_LAUNCH(k_pdl_fence, 1, 32, 0, st, 0);
  RW_TRY(mark(4));
  // small system
  float* C = reinterpret_cast<float*>(P(lay.C));
  {
    size_t shm = sizeof(float) * ((size_t)m_max * ((m_max + L) | 1) + 2 * (size_t)L * m_max + m_max) +
                 sizeof(int) * m_max;
    if (fused)  // the factors, the right-hand sides and one block of them
      shm = std::max(shm, sizeof(float) * ((size_t)m_max * lu_stride(m_max) + (size_t)(m_max + 32) * lp));
    if (fused) {
      if (lp == 4) {
        RW_CHECK_CUDA(ensure_smem(k_small_rhs<4>, shm));
        RW_LAUNCH((k_small_rhs<4>), 1, 256, shm, st, K, wcat, h, wcat, Z, lgam, (float)gamma, L, lp, mq,
                  mdev, Fac, mp, luinv, C, g->status);
      } else if (lp == 8) {
        RW_CHECK_CUDA(ensure_smem(k_small_rhs<8>, shm));
        RW_LAUNCH((k_small_rhs<8>), 1, 256, shm, st, K, wcat, h, wcat, Z, lgam, (float)gamma, L, lp, mq,
                  mdev, Fac, mp, luinv, C, g->status);
      } else {
        RW_CHECK_CUDA(ensure_smem(k_small_rhs<16>, shm));
        RW_LAUNCH((k_small_rhs<16>), 1, 256, shm, st, K, wcat, h, wcat, Z, lgam, (float)gamma, L, lp, mq,
                  mdev, Fac, mp, luinv, C, g->status);
      }
    } else if (lp == 4) {
      RW_CHECK_CUDA(ensure_smem(k_small_solve<4>, shm));
      RW_LAUNCH((k_small_solve<4>), 1, 256, shm, st, K, wcat, h, wcat, Z, lgam, (float)gamma, L, lp, mq, mdev, C,
                                            g->status);
    } else if (lp == 8) {
      RW_CHECK_CUDA(ensure_smem(k_small_solve<8>, shm));
      RW_LAUNCH((k_small_solve<8>), 1, 256, shm, st, K, wcat, h, wcat, Z, lgam, (float)gamma, L, lp, mq, mdev, C,
                                            g->status);
    } else {
      RW_CHECK_CUDA(ensure_smem(k_small_solve<16>, shm));
      RW_LAUNCH((k_small_solve<16>), 1, 256, shm, st, K, wcat, h, wcat, Z, lgam, (float)gamma, L, lp, mq,
                                             mdev, C, g->status);
    }
    RW_LAUNCH_CHECK();
  }
  if (g0) RW_LAUNCH(k_null_coef, 1, 256, 0, st, C, lp, L, mdev, wv, ginv, nul);
  RW_TRY(mark(5));
  // back-projection (+ refinement); the 16-bit kernel holds three blocks per SM
  const int nblk_b = fmt == RW_BASIS_F32 ? nblk : (tc_b ? sms : back_per_sm * sms);
  const int steps = opts->refine_steps;
  float* xh0 = nullptr;
  float* xh1 = nullptr;
  if (steps > 0) {
    RW_TRY(ws.xhat[0].grow(sizeof(float) * g->N * lp));
    RW_TRY(ws.xhat[1].grow(sizeof(float) * g->N * lp));
    xh0 = ws.xhat[0].as<float>();
    xh1 = ws.xhat[1].as<float>();
  }
  const float* nulp = g0 ? nul : nullptr;
  if (fmt == RW_BASIS_F16)
    RW_TRY(proj_back<__half>(lp, true, b->Q16, ldq_e, phat, seedlab, g, mdev, part, nblk_b, C, cscale, xh0, prob_dev, labels_dev, L, st, steps == 0 ? seedlab : nullptr, nulp));
  else if (fmt == RW_BASIS_BF16)
    RW_TRY(proj_back<__nv_bfloat16>(lp, true, b->Qbf, ldq_e, phat, seedlab, g, mdev, part, nblk_b, C, cscale, xh0, prob_dev, labels_dev, L, st, steps == 0 ? seedlab : nullptr, nulp));
  else
    RW_TRY(proj_back<float>(lp, true, b->Q32, ldq_e, phat, seedlab, g, mdev, part, nblk_b, C, cscale, xh0, prob_dev, labels_dev, L, st, steps == 0 ? seedlab : nullptr, nulp));
  RW_TRY(mark(6));
  if (steps > 0) {
    if (opts->refine_mode == RW_REFINE_JACOBI) {
      float* a = xh0;
      float* c = xh1;
      for (int t = 0; t < steps; ++t) {
        int last = (t == steps - 1);
        RW_TRY(jacobi(g, lp, a, c, phat, seedlab, L, (float)gamma, omega, last,
                      last ? prob_dev : nullptr, last ? labels_dev : nullptr,
                      last ? seedlab : nullptr, st));
        std::swap(a, c);
      }
    } else {
      RW_TRY(rw_pcg_from(g, phat, seedlab, L, lp, gamma, xh0, steps, 0.0, prob_dev, labels_dev,
                         nullptr, st));
    }
  }
  // the final kernel (last Jacobi step, or the back-projection without refinement) cleared the
  // seeds from the label array
  if (steps == 0 || opts->refine_mode == RW_REFINE_JACOBI) ws.seeds_clean = true;
  RW_TRY(mark(7));
  if (info) {
    RW_TRY(ws.host.grow(4096));
    char* hb = ws.host.as<char>();
    RW_CHECK_CUDA(cudaMemcpyAsync(hb, mdev, sizeof(int) * 2, cudaMemcpyDeviceToHost, st));
    RW_CHECK_CUDA(cudaMemcpyAsync(hb + 64, fsel, sizeof(double) * lp, cudaMemcpyDeviceToHost, st));
    RW_CHECK_CUDA(cudaMemcpyAsync(hb + 256, fit64, sizeof(double) * 32, cudaMemcpyDeviceToHost, st));
    RW_CHECK_CUDA(cudaMemcpyAsync(hb + 1024, g->status, sizeof(int), cudaMemcpyDeviceToHost, st));
    RW_CHECK_CUDA(cudaMemsetAsync(g->status, 0, sizeof(int), st));
    RW_CHECK_CUDA(cudaStreamSynchronize(st));
    memset(info, 0, sizeof(*info));
    const int* mi = reinterpret_cast<const int*>(hb);
    info->m_used = mi[0];
    info->capped = adaptive ? mi[1] : 0;
    info->f_max = (double)S * eps * eps;
    const double* fh = reinterpret_cast<const double*>(hb + 64);
    const double* f64 = reinterpret_cast<const double*>(hb + 256);
    for (int k = 0; k < L; ++k) {
      info->f[k] = adaptive ? fh[k] : 0.0;
      info->mu[k] = g0 ? 0.0 : f64[k];          // no Gaussian fit without priors
      info->sigma[k] = g0 ? 0.0 : f64[16 + k];
    }
    if (phases)
      for (int k = 0; k < RW_NUM_PHASES; ++k)
        RW_CHECK_CUDA(cudaEventElapsedTime(&info->phase_ms[k], ws.ev[k], ws.ev[k + 1]));
    int bits = *reinterpret_cast<const int*>(hb + 1024);
    rw_status ds = rw_status_from_device_bits(bits);
    info->device_status = ds;
    if (ds != RW_OK) return ds;
    if (info->capped) return RW_WARN_M_CAPPED;
  }
  return RW_OK;
}

static rw_status solve_host(const rw_graph* g, const rw_basis* b, const int32_t* seed_idx_host,
                            const int32_t* seed_lab_host, int32_t S, int32_t n_labels,
                            const float* priors_host, const rw_solve_opts* opts,
                            float* prob_host, uint8_t* labels_host, rw_solve_info* info,
                            void* stream, bool sync) {
  if (!g || !b || !seed_idx_host || !seed_lab_host || !opts || !prob_host) return RW_ERR_INVALID_ARG;
  if (S < 1 || S > 65536 || n_labels < 1 || n_labels > RW_MAX_LABELS) return RW_ERR_INVALID_ARG;
  cudaStream_t st = rw_stream(stream);
  rw_graph* gm = const_cast<rw_graph*>(g);
  // device staging: seeds, priors, probabilities, labels (kept in the graph's scratch)
  size_t n_pri = (opts->prior_mode == 1 && priors_host) ? (size_t)g->N * n_labels : 0;
  size_t off_seed = 0, off_lab = rw_round_up((int64_t)S * 4, 256);
  size_t off_pri = off_lab + rw_round_up((int64_t)S * 4, 256);
  size_t off_prob = off_pri + rw_round_up((int64_t)n_pri * 4, 256);
  size_t off_labels = off_prob + rw_round_up((int64_t)g->N * n_labels * 4, 256);
  size_t total = off_labels + rw_round_up(g->N, 256);
  RW_TRY(gm->ws.stage.grow(total));
  char* d = gm->ws.stage.as<char>();
  RW_CHECK_CUDA(cudaMemcpyAsync(d + off_seed, seed_idx_host, S * 4, cudaMemcpyHostToDevice, st));
  RW_CHECK_CUDA(cudaMemcpyAsync(d + off_lab, seed_lab_host, S * 4, cudaMemcpyHostToDevice, st));
  if (n_pri)
    RW_CHECK_CUDA(cudaMemcpyAsync(d + off_pri, priors_host, n_pri * 4, cudaMemcpyHostToDevice, st));
  rw_status s = rw_solve(g, b, reinterpret_cast<int32_t*>(d + off_seed),
                         reinterpret_cast<int32_t*>(d + off_lab), S, n_labels,
                         n_pri ? reinterpret_cast<float*>(d + off_pri) : nullptr, opts,
                         reinterpret_cast<float*>(d + off_prob),
                         labels_host ? reinterpret_cast<uint8_t*>(d + off_labels) : nullptr,
                         info, stream);
  if (s < 0) return s;
  RW_CHECK_CUDA(cudaMemcpyAsync(prob_host, d + off_prob, (size_t)g->N * n_labels * 4,
                                cudaMemcpyDeviceToHost, st));
  if (labels_host)
    RW_CHECK_CUDA(cudaMemcpyAsync(labels_host, d + off_labels, g->N, cudaMemcpyDeviceToHost, st));
  if (sync) RW_CHECK_CUDA(cudaStreamSynchronize(st));
  return s;
}

extern "C" rw_status rw_solve_host(const rw_graph* g, const rw_basis* b,
                                   const int32_t* seed_idx_host, const int32_t* seed_lab_host,
                                   int32_t S, int32_t n_labels, const float* priors_host,
                                   const rw_solve_opts* opts, float* prob_host,
                                   uint8_t* labels_host, rw_solve_info* info, void* stream) {
  return solve_host(g, b, seed_idx_host, seed_lab_host, S, n_labels, priors_host, opts,
                    prob_host, labels_host, info, stream, true);
}

extern "C" rw_status rw_solve_host_async(const rw_graph* g, const rw_basis* b,
                                         const int32_t* seed_idx_host,
                                         const int32_t* seed_lab_host, int32_t S,
                                         int32_t n_labels, const float* priors_host,
                                         const rw_solve_opts* opts, float* prob_host,
                                         uint8_t* labels_host, rw_solve_info* info,
                                         void* stream) {
  return solve_host(g, b, seed_idx_host, seed_lab_host, S, n_labels, priors_host, opts,
                    prob_host, labels_host, info, stream, false);
}

extern "C" rw_status rw_solve_priors(const rw_graph* g, const int32_t* seed_idx_dev,
                                     const int32_t* seed_lab_dev, int32_t S, int32_t n_labels,
                                     float* priors_dev, void* stream) {
  if (!g || !seed_idx_dev || !seed_lab_dev || !priors_dev || !g->J) return RW_ERR_INVALID_ARG;
  if (S < 1 || n_labels < 1 || n_labels > RW_MAX_LABELS) return RW_ERR_INVALID_ARG;
  cudaStream_t st = rw_stream(stream);
  float* phat;
  int* seedlab;
  const int lp = lpad_of(n_labels);
  RW_TRY(rw_solve_priors_internal(g, seed_idx_dev, seed_lab_dev, S, n_labels, 0, nullptr, lp, st,
                                  &phat, &seedlab, nullptr));
  RW_TRY(rw_unhat_priors(g, phat, lp, n_labels, priors_dev, st));
  return rw_last_device_status(g, stream);
}

// ---------------------------------------------------------------------------------------
// Unseeded solve (registration, Sec. II-A with no landmarks): with S = 0, Eq. (U_lin_comb)
// reads U-hat = Q Lambda_gamma (gamma Z), Z = Q^T P-hat, and the refinement is the damped
// Jacobi of Eq. (rw_eq) without seeded rows.  The K labels (displacements) run in chunks of
// lp = 8 (4 when K <= 4) through the same basis passes; m is given or chosen by Eq. (g),
// g_k(m) = ||p-hat_k||^2 - ||Z_k[:m]||^2 (Q orthonormal), the smallest candidate with
// max_k g_k <= g_max = 1^T D 1 eps^2 (normalized form).
// ---------------------------------------------------------------------------------------
namespace {

// P-hat chunk: phat[i][j] = d_i^{1/2} P[i][k0 + j] (j < Lc, zero above); optionally the squared
// norms of the chunk's P-hat columns, per block in FP64, one atomic per block and label.
// P-hat rows of one chunk of labels: phat[i][j] = d_i^{1/2} P[i][k0 + j] (zero past Lc), one
// thread per entry so that both the reads of P and the writes of P-hat are coalesced; with
// pnorm, also adds ||P-hat column||^2 (per-thread FP64 sums: the grid is a multiple of LP
// threads, so a thread always meets the same column; warp, then block, then one atomic per
// column and block).
template <int LP>
__global__ void __launch_bounds__(256)
k_hat_chunk(const float* __restrict__ P, int K, int k0, int Lc,
            const float* __restrict__ sq, int64_t N, float* __restrict__ phat,
            double* __restrict__ pnorm) {
  __shared__ double red[8][LP];
  double acc = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N * LP; e += stride) {
    const int64_t i = e / LP;
    const int j = (int)(e % LP);
    const float v = j < Lc ? __ldg(sq + i) * __ldg(P + i * K + k0 + j) : 0.f;
    phat[e] = v;
    acc += (double)v * v;
  }
  if (!pnorm) return;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int o = 16; o >= LP; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane < LP) red[w][lane] = acc;
  __syncthreads();
  if (threadIdx.x < Lc) {
    double t = 0.0;
    for (int ww = 0; ww < 8; ++ww) t += red[ww][threadIdx.x];
    atomicAdd(&pnorm[k0 + threadIdx.x], t);
  }
}

static rw_status hat_chunk(int lp, unsigned nblk, cudaStream_t st, const float* P, int K, int k0,
                           int Lc, const float* sq, int64_t N, float* phat, double* pnorm) {
  switch (lp) {
    case 4: k_hat_chunk<4><<<nblk, 256, 0, st>>>(P, K, k0, Lc, sq, N, phat, pnorm); break;
    case 8: k_hat_chunk<8><<<nblk, 256, 0, st>>>(P, K, k0, Lc, sq, N, phat, pnorm); break;
    case 16: k_hat_chunk<16><<<nblk, 256, 0, st>>>(P, K, k0, Lc, sq, N, phat, pnorm); break;
    default: k_hat_chunk<32><<<nblk, 256, 0, st>>>(P, K, k0, Lc, sq, N, phat, pnorm); break;
  }
  RW_LAUNCH_CHECK();
  return RW_OK;
}

__global__ void k_store_z(const float* __restrict__ Z, int lp, int Lc, int k0, int rows, int K,
                          float* __restrict__ Zall) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rows * Lc) return;
  const int i = e / Lc, j = e - i * Lc;
  Zall[(int64_t)i * K + k0 + j] = Z[i * lp + j];
}

// Eq. (g) over the candidates m_step, 2 m_step, ..., m_max: running sums of Z^2 per label in
// FP64, first candidate whose worst label passes (m_max, flagged, when none does)
__global__ void __launch_bounds__(256)
k_choose_m_g(const float* __restrict__ Zall, int K, int m_max, int m_step,
             const double* __restrict__ pnorm, double gmax, int* __restrict__ mdev,
             double* __restrict__ gout) {
  __shared__ double wmax[8];
  __shared__ int done;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (threadIdx.x == 0) done = 0;
  int m_prev = 0;
  for (int mc = m_step < m_max ? m_step : m_max;; mc = (mc + m_step < m_max ? mc + m_step : m_max)) {
    double worst = 0.0;
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
      double c = 0.0;
      for (int i = m_prev; i < mc; ++i) {
        const double z = Zall[(int64_t)i * K + k];
        c += z * z;
      }
      gout[k] = (m_prev == 0 ? pnorm[k] : gout[k]) - c;
      worst = fmax(worst, gout[k]);
    }
    for (int o = 16; o > 0; o >>= 1) worst = fmax(worst, __shfl_xor_sync(0xffffffffu, worst, o));
    __syncthreads();
    if (lane == 0) wmax[w] = worst;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int ww = 0; ww < (int)(blockDim.x >> 5); ++ww) t = fmax(t, wmax[ww]);
      if (t <= gmax || mc == m_max) {
        mdev[0] = mc;
        mdev[1] = t <= gmax ? 0 : 1;
        done = 1;
      }
    }
    __syncthreads();
    if (done) return;
    m_prev = mc;
  }
}

// C = gamma Lambda_gamma Z[:m] for one chunk (rows >= m and labels >= Lc zero)
__global__ void k_c_unseeded(const float* __restrict__ Zall, int K, int k0, int Lc, int lp,
                             const double* __restrict__ lam, double gamma,
                             const int* __restrict__ mdev, int rows, float* __restrict__ C) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rows * lp) return;
  const int i = e / lp, j = e - i * lp;
  const int m = mdev[0];
  C[e] = (i < m && j < Lc) ? (float)(gamma * Zall[(int64_t)i * K + k0 + j] / (lam[i] + gamma))
                           : 0.f;
}

__global__ void k_scatter_cols(const float* __restrict__ Uc, int Lc, int64_t N,
                               float* __restrict__ prob, int K, int k0) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * Lc) return;
  const int64_t i = e / Lc;
  const int j = (int)(e - i * Lc);
  prob[i * K + k0 + j] = Uc[e];
}

// hard labels (largest probability, ties to the lowest label) and the expected displacement
__global__ void k_reg_finish(const float* __restrict__ prob, int K, int64_t N,
                             uint8_t* __restrict__ labels, const int32_t* __restrict__ disp,
                             int dd, float* __restrict__ field) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const float* p = prob + i * K;
  int best = 0;
  float bv = -INFINITY;
  float f[3] = {0.f, 0.f, 0.f};
  for (int k = 0; k < K; ++k) {
    const float u = p[k];
    if (u > bv) { bv = u; best = k; }
    if (field)
      for (int a = 0; a < dd; ++a) f[a] = fmaf(u, (float)disp[k * dd + a], f[a]);
  }
  if (labels) labels[i] = (uint8_t)best;
  if (field)
    for (int a = 0; a < dd; ++a) field[i * dd + a] = f[a];
}

}  // namespace

template <typename T>
static rw_status unseeded_passes(const rw_graph* g, const rw_basis* b, const T* Q, int ldq,
                                 float zscale, float cscale, const float* priors, int K, int lp,
                                 const rw_solve_opts* opts, float* prob, cudaStream_t st,
                                 int* mall, int* mdev, float* Z, float* lgam, float* C,
                                 float* Zall, double* pnorm, double* gout, float* part,
                                 int mq, int nblk_p, int nblk_b) {
  rw_graph* gm = const_cast<rw_graph*>(g);
  SolveWorkspace& ws = gm->ws;
  const int64_t N = g->N;
  const double gamma = opts->gamma;
  const bool adaptive = opts->m == 0;
  const int m_max = adaptive ? b->m : opts->m;
  const int steps = opts->refine_steps;
  const float omega = (float)(opts->omega > 0 ? std::min(opts->omega, 1.0) : 0.8);
  const int nchunks = (K + lp - 1) / lp;
  float* phat = ws.phat.as<float>();
  int* seedlab = ws.seedlab.as<int>();
  const int sms = g_rw_num_sms > 0 ? g_rw_num_sms : 148;
  const unsigned hblk = (unsigned)std::min<int64_t>(rw_blocks(N, 256), 4 * sms);
  // Z of every chunk over all m_max columns (and the norms of P-hat for Eq. g)
  RW_CHECK_CUDA(cudaMemsetAsync(pnorm, 0, sizeof(double) * K, st));
  RW_LAUNCH(k_set_m, 1, 32, 0, st, mall, m_max);
  for (int c = 0; c < nchunks; ++c) {
    const int k0 = c * lp, Lc = std::min(lp, K - k0);
    RW_TRY(hat_chunk(lp, hblk, st, priors, K, k0, Lc, g->sq, N, phat, adaptive ? pnorm : nullptr));
    RW_TRY(proj_back<T>(lp, false, Q, ldq, phat, seedlab, g, mall, part, nblk_p, nullptr, 0.f,
                        nullptr, nullptr, nullptr, Lc, st));
    RW_LAUNCH(k_reduce_partials, rw_blocks((int64_t)std::max(mq * lp, m_max) * 32, 256), 256, 0,
              st, part, nblk_p, ldq, lp, mq, zscale, Z, b->lam, gamma, m_max, lgam, 0);
    k_store_z<<<rw_blocks((int64_t)m_max * Lc, 256), 256, 0, st>>>(Z, lp, Lc, k0, m_max, K, Zall);
    RW_LAUNCH_CHECK();
  }
  if (adaptive) {
    const int m_step = opts->m_step > 0 ? opts->m_step : 10;
    const double eps = opts->eps > 0 ? opts->eps : 0.1;
    const double gmax = (g->normalized ? g->dsum : (double)N) * eps * eps;
    k_choose_m_g<<<1, 256, 0, st>>>(Zall, K, m_max, m_step, pnorm, gmax, mdev, gout);
    RW_LAUNCH_CHECK();
  } else {
    RW_LAUNCH(k_set_m, 1, 32, 0, st, mdev, m_max);
  }
  float* xh0 = steps > 0 ? ws.xhat[0].as<float>() : nullptr;
  float* xh1 = steps > 0 ? ws.xhat[1].as<float>() : nullptr;
  // one chunk holding every label writes prob directly (same layout); else a chunk buffer
  float* Uc = nchunks == 1 ? prob : ws.reg.as<float>();
  for (int c = 0; c < nchunks; ++c) {
    const int k0 = c * lp, Lc = std::min(lp, K - k0);
    if (nchunks > 1)   // with one chunk the P-hat rows of the first loop are still in place
      RW_TRY(hat_chunk(lp, hblk, st, priors, K, k0, Lc, g->sq, N, phat, nullptr));
    k_c_unseeded<<<rw_blocks((int64_t)mq * lp, 256), 256, 0, st>>>(Zall, K, k0, Lc, lp, b->lam,
                                                                 gamma, mdev, mq, C);
    RW_LAUNCH_CHECK();
    RW_TRY(proj_back<T>(lp, true, Q, ldq, phat, seedlab, g, mdev, part, nblk_b, C, cscale, xh0,
                        steps > 0 ? nullptr : Uc, nullptr, Lc, st));
    if (steps > 0) {
      float* a = xh0;
      float* o = xh1;
      for (int t = 0; t < steps; ++t) {
        const int last = t == steps - 1;
        RW_TRY(jacobi(g, lp, a, o, phat, seedlab, Lc, (float)gamma, omega, last,
                      last ? Uc : nullptr, nullptr, nullptr, st));
        std::swap(a, o);
      }
    }
    if (nchunks > 1) {
      k_scatter_cols<<<rw_blocks(N * Lc, 256), 256, 0, st>>>(Uc, Lc, N, prob, K, k0);
      RW_LAUNCH_CHECK();
    }
  }
  return RW_OK;
}

extern "C" rw_status rw_solve_unseeded(const rw_graph* g, const rw_basis* b,
                                       const float* priors_dev, int32_t K,
                                       const rw_solve_opts* opts, float* prob_dev,
                                       uint8_t* labels_dev, const int32_t* disp_dev,
                                       int32_t disp_dim, float* field_dev, int32_t* m_used,
                                       void* stream) {
  if (!g || !b || !priors_dev || !opts || !prob_dev) return RW_ERR_INVALID_ARG;
  if (b->N != g->N || K < 1 || K > 4096 || (labels_dev && K > 255)) return RW_ERR_INVALID_ARG;
  if (!(opts->gamma > 0.0)) return opts->gamma == 0.0 ? RW_ERR_UNSUPPORTED : RW_ERR_INVALID_ARG;
  if (opts->m < 0 || opts->m > b->m || opts->refine_steps < 0 || opts->refine_steps > 100000)
    return RW_ERR_INVALID_ARG;
  if (field_dev && (!disp_dev || disp_dim < 1 || disp_dim > 3)) return RW_ERR_INVALID_ARG;
  if (opts->basis_format != RW_BASIS_F16 && opts->basis_format != RW_BASIS_F32)
    return RW_ERR_UNSUPPORTED;
  if (opts->basis_format == RW_BASIS_F32 && b->ld32 > 256) return RW_ERR_UNSUPPORTED;
  if (g_rw_num_sms <= 0) RW_TRY(rw_device_init());
  cudaStream_t st = rw_stream(stream);
  rw_graph* gm = const_cast<rw_graph*>(g);
  SolveWorkspace& ws = gm->ws;
  const int64_t N = g->N;
  // labels per pass: 8 on the CUDA cores; with both basis passes on the tensor cores up to 32
  // (one pass over the basis for every 32 labels)
  const bool tc_all = rw_tc_passes(b->ld16, 1, 32) && rw_tc_passes(b->ld16, 2, 32) &&
                      opts->basis_format != RW_BASIS_F32;
  const int lp = K <= 4 ? 4 : (K <= 8 || !tc_all ? 8 : (K <= 16 ? 16 : 32));
  const int sms = g_rw_num_sms;
  const int nblk = 4 * sms;
  const int mq = std::max(b->ld16, b->ld32);
  // scratch: label array (all unseeded), P-hat and iterate chunks, and the small arrays
  const size_t cap0 = ws.seedlab.cap;
  RW_TRY(ws.seedlab.grow(sizeof(int) * N));
  if (ws.seedlab.cap != cap0) ws.seeds_clean = false;
  RW_TRY(ws.phat.grow(sizeof(float) * N * lp));
  RW_TRY(ws.reg.grow(sizeof(float) * N * lp));
  if (opts->refine_steps > 0) {
    RW_TRY(ws.xhat[0].grow(sizeof(float) * N * lp));
    RW_TRY(ws.xhat[1].grow(sizeof(float) * N * lp));
  }
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t r = off; off += (bytes + 255) & ~size_t(255); return r; };
  const size_t o_mall = take(sizeof(int) * 8), o_mdev = take(sizeof(int) * 8);
  const size_t o_Z = take(sizeof(float) * mq * lp), o_lgam = take(sizeof(float) * mq);
  const size_t o_C = take(sizeof(float) * mq * lp), o_Zall = take(sizeof(float) * mq * K);
  const size_t o_pn = take(sizeof(double) * K), o_g = take(sizeof(double) * K);
  const size_t o_part = take(sizeof(float) * (size_t)nblk * mq * lp);
  RW_TRY(ws.small.grow(off));
  char* base = ws.small.as<char>();
  int* mall = reinterpret_cast<int*>(base + o_mall);
  int* mdev = reinterpret_cast<int*>(base + o_mdev);
  float* Z = reinterpret_cast<float*>(base + o_Z);
  float* lgam = reinterpret_cast<float*>(base + o_lgam);
  float* C = reinterpret_cast<float*>(base + o_C);
  float* Zall = reinterpret_cast<float*>(base + o_Zall);
  double* pnorm = reinterpret_cast<double*>(base + o_pn);
  double* gout = reinterpret_cast<double*>(base + o_g);
  float* part = reinterpret_cast<float*>(base + o_part);
  if (!ws.seeds_clean)
    RW_LAUNCH(k_seed_reset, rw_blocks(N, 256), 256, 0, st, ws.seedlab.as<int>(), N, nullptr, 0);
  ws.seeds_clean = true;   // no seed is placed
  int proj_per_sm = 2, back_per_sm = 3;
  launch_shape(N, &proj_per_sm, &back_per_sm);
  if (opts->basis_format == RW_BASIS_F16) {
    const float sc = 1.f / b->qscale;
    const bool tc_p = rw_tc_passes(b->ld16, 1, lp), tc_b = rw_tc_passes(b->ld16, 2, lp);
    RW_TRY(unseeded_passes<__half>(g, b, b->Q16, b->ld16, tc_p ? sc / kTcProjScale : sc, sc,
                                   priors_dev, K, lp, opts,
                                   prob_dev, st, mall, mdev, Z, lgam, C, Zall, pnorm, gout, part,
                                   mq, tc_p ? sms : proj_per_sm * sms,
                                   tc_b ? sms : back_per_sm * sms));
  } else {
    RW_TRY(unseeded_passes<float>(g, b, b->Q32, b->ld32, 1.f, 1.f, priors_dev, K, lp, opts,
                                  prob_dev, st, mall, mdev, Z, lgam, C, Zall, pnorm, gout, part,
                                  mq, nblk, nblk));
  }
  if (labels_dev || field_dev) {
    k_reg_finish<<<rw_blocks(N, 256), 256, 0, st>>>(prob_dev, K, N, labels_dev, disp_dev,
                                                   disp_dim, field_dev);
    RW_LAUNCH_CHECK();
  }
  if (m_used) {
    int h = 0;
    RW_CHECK_CUDA(cudaMemcpyAsync(&h, mdev, sizeof(int), cudaMemcpyDeviceToHost, st));
    RW_CHECK_CUDA(cudaStreamSynchronize(st));
    *m_used = h;
    return rw_last_device_status(g, stream);
  }
  return RW_OK;
}
