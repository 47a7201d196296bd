// Online fast random walker (Sec. II-B, Eqs. Fs and U_lin_comb, in the normalized form of
// Sec. II-C) with the number of eigenvectors chosen from the seeds (Sec. III-A-1, Eq. alpha_1),
// priors from a Gaussian fit to the seed intensities (Sec. IV-A), damped-Jacobi refinement on
// Eq. (rw_eq) and hard labels.
//
// Hat variables: U-hat = D^{1/2} U, P-hat = D^{1/2} P (sq = d^{1/2}, s = d^{-1/2}); with the
// unnormalized Laplacian sq = s = 1.  Operator coefficients c_ij = w_ij s_i s_j, so the seeded
// block of L-hat is B-hat_ij = -c_ij.
//
// Per solve (S seeds, m_max basis columns, l labels):
//   scatter seeds, Gaussian fit, P-hat (N x lp)                    -> k_seed_scatter, k_fit,
//                                                                     k_priors
//   Q_s, X = B-hat Q_n (S x m_max), r0 = L-hat_s U-hat_s + gamma U-hat_s  -> k_seed_gather
//   K = Q_s^T X, h = Q_s^T r0, b = Q_s^T U-hat_s, G = Q_s^T Q_s     -> rw_gram (FP64 out)
//   m (adaptive: one CTA per candidate m, trust-region least squares) -> k_adapt, k_pick
//   Z = Q_n^T P-hat_n (streams the 16-bit basis once)                -> k_project, k_reduce
//   (diag(lambda + gamma) - K) y = h + gamma K Lambda_gamma Z, C = y + gamma Lambda_gamma Z
//                                                                    -> k_small_solve
//   U-hat_n = Q_n C (streams the basis again)                        -> k_backproject
//   refinement steps, U = s * U-hat, labels = argmax                 -> k_jacobi_step
#include "rw_internal.cuh"

#include <algorithm>
#include <cstring>

namespace {

constexpr int kMaxSmallM = 224;  // m x m FP32 factorizations live in one CTA's shared memory

int lpad_of(int L) { return L <= 4 ? 4 : (L <= 8 ? 8 : 16); }

struct Layout {
  size_t stats, fit, cnt, mdev, Qs, Xs, Us, R0, G, K, bv, h, cu, Z, C, fc, pass, cand, lam,
      fit64, part, total;
};

Layout make_layout(int S, int mp, int mq, int lp, int ncand, int nblk_part) {
  Layout o;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t r = off; off += (bytes + 255) & ~size_t(255); return r; };
  o.stats = take(sizeof(double) * 16 * 3);
  o.fit = take(sizeof(float) * 16 * 3);
  o.cnt = take(sizeof(int) * 16);
  o.mdev = take(sizeof(int) * 8);
  o.Qs = take(sizeof(float) * (size_t)S * mp);
  o.Xs = take(sizeof(float) * (size_t)S * mp);
  o.Us = take(sizeof(float) * (size_t)S * lp);
  o.R0 = take(sizeof(float) * (size_t)S * lp);
  o.G = take(sizeof(double) * (size_t)mp * mp);
  o.K = take(sizeof(double) * (size_t)mp * mp);
  o.bv = take(sizeof(double) * (size_t)mp * lp);
  o.h = take(sizeof(double) * (size_t)mp * lp);
  o.cu = take(sizeof(double) * (size_t)lp * lp);
  o.Z = take(sizeof(double) * (size_t)mq * lp);
  o.C = take(sizeof(float) * (size_t)mq * lp);
  o.fc = take(sizeof(double) * (size_t)(ncand + 1) * lp);
  o.pass = take(sizeof(int) * (size_t)(ncand + 1));
  o.cand = take(sizeof(int) * (size_t)(ncand + 1));
  o.lam = take(sizeof(float) * (size_t)mp);
  o.fit64 = take(sizeof(double) * 16 * 2);
  o.part = take(sizeof(float) * (size_t)nblk_part * mq * lp);
  o.total = off;
  return o;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffff, v, o);
  return v;
}

// ---------------------------------------------------------------------------------------
__global__ void k_fill_i32(int* p, int64_t n, int v) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

__global__ void k_seed_scatter(const int32_t* __restrict__ idx, const int32_t* __restrict__ lab,
                               int S, int L, int64_t N, const float* __restrict__ J,
                               int* __restrict__ seedlab, double* __restrict__ stats,
                               int* status) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= S) return;
  int i = idx[t], k = lab[t];
  if (i < 0 || (int64_t)i >= N || k < 0 || k >= L) {
    atomicOr(status, RW_DEV_BAD_SEED);
    return;
  }
  int old = atomicCAS(&seedlab[i], -1, k);
  if (old != -1) {
    atomicOr(status, RW_DEV_DUP_SEED);
    return;
  }
  double v = J ? (double)J[i] : 0.0;
  atomicAdd(&stats[3 * k + 0], v);
  atomicAdd(&stats[3 * k + 1], v * v);
  atomicAdd(&stats[3 * k + 2], 1.0);
}

// mu_k, 1/(2 sigma_k^2), log sigma_k with sigma_k = max(std, 1e-3) (ML estimates, Sec. IV-A)
__global__ void k_fit(const double* __restrict__ stats, int L, int prior_mode,
                      float* __restrict__ fit, double* __restrict__ fit64, int* status) {
  int k = threadIdx.x;
  if (k >= L) return;
  double n = stats[3 * k + 2];
  if (n <= 0.0) {
    if (prior_mode == 0) atomicOr(status, RW_DEV_EMPTY_LABEL);
    fit[k] = 0.f; fit[16 + k] = 0.f; fit[32 + k] = 0.f;
    fit64[k] = 0.0; fit64[16 + k] = 0.0;
    return;
  }
  double mu = stats[3 * k] / n;
  double var = stats[3 * k + 1] / n - mu * mu;
  double sig = fmax(sqrt(fmax(var, 0.0)), 1e-3);
  fit[k] = (float)mu;
  fit[16 + k] = (float)(0.5 / (sig * sig));
  fit[32 + k] = (float)log(sig);
  fit64[k] = mu;
  fit64[16 + k] = sig;
}

// P-hat rows (N x lp): Gaussian priors normalized per voxel, or caller priors, times d^{1/2}
__global__ void k_priors(const float* __restrict__ J, const float* __restrict__ sq, int64_t N,
                         int L, int lp, int prior_mode, const float* __restrict__ fit,
                         const float* __restrict__ Pin, float* __restrict__ phat, int* status) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  float p[RW_MAX_LABELS];
  if (prior_mode == 0) {
    float x = J[i], mx = -INFINITY;
    for (int k = 0; k < L; ++k) {
      float t = x - fit[k];
      p[k] = -t * t * fit[16 + k] - fit[32 + k];
      mx = fmaxf(mx, p[k]);
    }
    float sum = 0.f;
    for (int k = 0; k < L; ++k) { p[k] = expf(p[k] - mx); sum += p[k]; }
    float inv = 1.f / sum;
    for (int k = 0; k < L; ++k) p[k] *= inv;
  } else {
    for (int k = 0; k < L; ++k) {
      p[k] = Pin[i * L + k];
      if (!isfinite(p[k])) atomicOr(status, RW_DEV_NONFINITE);
    }
  }
  float r = sq[i];
  float* o = phat + i * lp;
  for (int k = 0; k < lp; ++k) o[k] = (k < L) ? r * p[k] : 0.f;
}

// One warp per seed: Q_s row, X = B-hat Q_n row, U-hat_s row, r0 = L-hat_s U-hat_s + g U-hat_s
__global__ void k_seed_gather(const int32_t* __restrict__ idx, const int32_t* __restrict__ lab,
                              int S, int L, int lp, int64_t N, const float* __restrict__ Q,
                              int ldq, int mp, const int* __restrict__ seedlab,
                              const float* __restrict__ cw, const float* __restrict__ d,
                              const float* __restrict__ sq, int normalized, int kind, int ndim,
                              int DX, int DY, int DZ, const int32_t* __restrict__ rowptr,
                              const int32_t* __restrict__ colv, const float* __restrict__ ccsr,
                              float gamma, float* __restrict__ Qs, float* __restrict__ Xs,
                              float* __restrict__ Us, float* __restrict__ R0) {
  const int lane = threadIdx.x & 31;
  const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (t >= S) return;
  const int i = idx[t], k0 = lab[t];
  float* qs = Qs + (int64_t)t * mp;
  float* xs = Xs + (int64_t)t * mp;
  if (i < 0 || (int64_t)i >= N || k0 < 0 || k0 >= L) {  // reported by k_seed_scatter
    for (int c = lane; c < mp; c += 32) { qs[c] = 0.f; xs[c] = 0.f; }
    if (lane < lp) { Us[t * lp + lane] = 0.f; R0[t * lp + lane] = 0.f; }
    return;
  }
  const float* qi = Q + (int64_t)i * ldq;
  for (int c = lane; c < mp; c += 32) { qs[c] = qi[c]; xs[c] = 0.f; }
  float r0 = 0.f;  // lane k accumulates column k of L-hat_s U-hat_s
  const float diag = normalized ? 1.f : d[i];
  if (lane == k0) r0 = diag * sq[i];
  auto visit = [&](int64_t j, float c) {
    int lj = seedlab[j];
    if (lj < 0) {
      const float* qj = Q + j * ldq;
      for (int cc = lane; cc < mp; cc += 32) xs[cc] = fmaf(-c, qj[cc], xs[cc]);
    } else if (lane == lj) {
      r0 -= c * sq[j];
    }
  };
  if (kind == RW_GRAPH_GRID) {
    const int64_t st[3] = {1, (int64_t)DX, (int64_t)DX * DY};
    const int cc[3] = {(int)(i % DX), (int)((i / DX) % DY), (int)(i / ((int64_t)DX * DY))};
    const int n[3] = {DX, DY, DZ};
    for (int a = 0; a < ndim; ++a) {
      if (cc[a] > 0) visit(i - st[a], cw[a * N + i - st[a]]);
      if (cc[a] + 1 < n[a]) visit(i + st[a], cw[a * N + i]);
    }
  } else {
    for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) visit(colv[p], ccsr[p]);
  }
  if (lane < lp) {
    float u = (lane == k0) ? sq[i] : 0.f;
    Us[t * lp + lane] = u;
    R0[t * lp + lane] = (lane < L) ? r0 + gamma * u : 0.f;
  }
}

// ---------------------------------------------------------------------------------------
// Shared-memory FP32 helpers for one CTA (row stride ms, odd to avoid bank conflicts)
// ---------------------------------------------------------------------------------------
__device__ bool chol_lower_smem(float* A, int m, int ms) {
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  for (int k = 0; k < m; ++k) {
    __syncthreads();
    float piv = A[k * ms + k];
    if (!(piv > 0.f)) {
      if (threadIdx.x == 0) bad = 1;
      piv = 1e-30f;
    }
    const float r = sqrtf(piv);
    __syncthreads();
    for (int i = k + 1 + threadIdx.x; i < m; i += blockDim.x) A[i * ms + k] /= r;
    if (threadIdx.x == 0) A[k * ms + k] = r;
    __syncthreads();
    const int w = m - k - 1;
    for (int e = threadIdx.x; e < w * w; e += blockDim.x) {
      int i = k + 1 + e / w, j = k + 1 + e % w;
      if (j <= i) A[i * ms + j] = fmaf(-A[i * ms + k], A[j * ms + k], A[i * ms + j]);
    }
  }
  __syncthreads();
  return bad == 0;
}

// one warp: L z = b (forward), L lower with stride ms
__device__ void fwd_lower_warp(const float* A, int m, int ms, const float* b, float* z) {
  const int lane = threadIdx.x & 31;
  for (int i = 0; i < m; ++i) {
    float s = 0.f;
    for (int j = lane; j < i; j += 32) s = fmaf(A[i * ms + j], z[j], s);
    s = warp_sum(s);
    if (lane == 0) z[i] = (b[i] - s) / A[i * ms + i];
    __syncwarp();
  }
}

// one warp: L^T x = z (backward)
__device__ void bwd_lowerT_warp(const float* A, int m, int ms, const float* z, float* x) {
  const int lane = threadIdx.x & 31;
  for (int i = m - 1; i >= 0; --i) {
    float s = 0.f;
    for (int j = i + 1 + lane; j < m; j += 32) s = fmaf(A[j * ms + i], x[j], s);
    s = warp_sum(s);
    if (lane == 0) x[i] = (z[i] - s) / A[i * ms + i];
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------------------
// Adaptive m (Sec. III-A-1, Eq. alpha_1).  One CTA per candidate m: f_k(m) =
// min_{||a|| <= rho} ||Q_s^{(m)} a - u-hat_s^k||^2.  G_m + mu0 I = L L^T (FP32, mu0 a tiny
// relative shift); a = (G_m + mu I)^{-1} b_k with mu = mu0 if ||a|| <= rho, else mu from Newton
// on 1/||a(mu)|| - 1/rho (More-Sorensen); f evaluated directly as the squared residual over
// the S seeds.
// ---------------------------------------------------------------------------------------
__device__ void load_shifted_gram(float* A, int m, int ms, const double* G, int ldg, float mu) {
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    int i = e / m, j = e % m;
    A[i * ms + j] = (float)G[(int64_t)i * ldg + j] + (i == j ? mu : 0.f);
  }
}

__global__ void __launch_bounds__(1024)
k_adapt(const double* __restrict__ G, int ldg, const double* __restrict__ bv, int lp,
        const float* __restrict__ Qs, int mp, const float* __restrict__ Us, int S, int L,
        const int* __restrict__ cand, double rho, double fmax, double* __restrict__ fout,
        int* __restrict__ pass) {
  extern __shared__ float sm[];
  const int m = cand[blockIdx.x];
  const int ms = m | 1;
  float* A = sm;                       // m x ms
  float* al = A + (size_t)m * ms;      // L x m   solutions
  float* z = al + (size_t)L * m;       // L x m   temporaries
  float* bb = z + (size_t)L * m;       // L x m   right-hand sides
  __shared__ float mu0s, red[32];
  __shared__ float fk[RW_MAX_LABELS], nrm[RW_MAX_LABELS];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int e = threadIdx.x; e < L * m; e += blockDim.x) {
    int k = e / m, i = e % m;
    bb[k * m + i] = (float)bv[(int64_t)i * lp + k];
  }
  if (threadIdx.x == 0) {
    double tr = 0.0;
    for (int i = 0; i < m; ++i) tr += G[(int64_t)i * ldg + i];
    mu0s = (float)(1e-6 * tr / m);
  }
  __syncthreads();
  const float mu0 = mu0s;
  load_shifted_gram(A, m, ms, G, ldg, mu0);
  bool ok = chol_lower_smem(A, m, ms);
  for (int k = warp; k < L; k += nw) {
    fwd_lower_warp(A, m, ms, bb + k * m, z + k * m);
    bwd_lowerT_warp(A, m, ms, z + k * m, al + k * m);
    float s = 0.f;
    for (int i = lane; i < m; i += 32) s = fmaf(al[k * m + i], al[k * m + i], s);
    s = warp_sum(s);
    if (lane == 0) nrm[k] = sqrtf(s);
  }
  __syncthreads();
  // labels whose minimum-norm solution leaves the ball: Newton on the secular equation
  for (int k = 0; k < L && ok; ++k) {
    if (!(nrm[k] > (float)rho)) continue;
    float mu = mu0;
    for (int it = 0; it < 40; ++it) {
      __syncthreads();
      float na = nrm[k];
      if (fabsf(na - (float)rho) <= 1e-5f * (float)rho) break;
      // q: L q = alpha, ||q||^2 = alpha^T (G + mu I)^{-1} alpha
      if (warp == 0) {
        fwd_lower_warp(A, m, ms, al + k * m, z + k * m);
        float s = 0.f;
        for (int i = lane; i < m; i += 32) s = fmaf(z[k * m + i], z[k * m + i], s);
        s = warp_sum(s);
        if (lane == 0) red[0] = s;
      }
      __syncthreads();
      float nq2 = red[0];
      float step = (na * na / fmaxf(nq2, 1e-30f)) * ((na - (float)rho) / (float)rho);
      mu = fmaxf(mu + step, mu0);
      __syncthreads();
      load_shifted_gram(A, m, ms, G, ldg, mu);
      if (!chol_lower_smem(A, m, ms)) { ok = false; break; }
      if (warp == 0) {
        fwd_lower_warp(A, m, ms, bb + k * m, z + k * m);
        bwd_lowerT_warp(A, m, ms, z + k * m, al + k * m);
        float s = 0.f;
        for (int i = lane; i < m; i += 32) s = fmaf(al[k * m + i], al[k * m + i], s);
        s = warp_sum(s);
        if (lane == 0) nrm[k] = sqrtf(s);
      }
    }
    __syncthreads();
  }
  // f_k = ||Q_s a_k - u_k||^2 over the seeds
  if (threadIdx.x < RW_MAX_LABELS) fk[threadIdx.x] = 0.f;
  __syncthreads();
  for (int k = 0; k < L; ++k) {
    float acc = 0.f;
    for (int s = threadIdx.x; s < S; s += blockDim.x) {
      const float* q = Qs + (int64_t)s * mp;
      float r = -Us[(int64_t)s * lp + k];
      for (int j = 0; j < m; ++j) r = fmaf(q[j], al[k * m + j], r);
      acc = fmaf(r, r, acc);
    }
    acc = warp_sum(acc);
    if (lane == 0) atomicAdd(&fk[k], acc);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    bool p = ok;
    for (int k = 0; k < L; ++k) {
      double f = ok ? (double)fk[k] : INFINITY;
      fout[(int64_t)blockIdx.x * lp + k] = f;
      if (!(f <= fmax)) p = false;
    }
    pass[blockIdx.x] = p ? 1 : 0;
  }
}

__global__ void k_pick(const int* __restrict__ cand, const int* __restrict__ pass, int ncand,
                       const double* __restrict__ fc, int lp, int* mdev, double* fsel) {
  if (threadIdx.x != 0) return;
  int c = ncand - 1, capped = 1;
  for (int i = 0; i < ncand; ++i)
    if (pass[i]) { c = i; capped = 0; break; }
  mdev[0] = cand[c];
  mdev[1] = capped;
  for (int k = 0; k < lp; ++k) fsel[k] = fc[(int64_t)c * lp + k];
}

__global__ void k_set_m(int* mdev, int m) {
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
  __device__ static void load(const __half* p, float* o) {
    uint4 u = __ldg(reinterpret_cast<const uint4*>(p));
    const __half2* h = reinterpret_cast<const __half2*>(&u);
#pragma unroll
    for (int t = 0; t < 4; ++t) { float2 f = __half22float2(h[t]); o[2 * t] = f.x; o[2 * t + 1] = f.y; }
  }
};
template <> struct Vec16<__nv_bfloat16> {
  static constexpr int V = 8;
  __device__ static void load(const __nv_bfloat16* p, float* o) {
    uint4 u = __ldg(reinterpret_cast<const uint4*>(p));
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
    for (int t = 0; t < 4; ++t) { float2 f = __bfloat1622float2(h[t]); o[2 * t] = f.x; o[2 * t + 1] = f.y; }
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
                                  int mq, double scale, double* __restrict__ Z) {
  const int lane = threadIdx.x & 31;
  const int e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (e >= mq * lp) return;
  const int row = e / lp;
  double s = 0.0;
  if (row < ldq)
    for (int b = lane; b < nblk; b += 32) s += (double)part[(int64_t)b * ldq * lp + e];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffff, s, o);
  if (lane == 0) Z[e] = s * scale;
}

// ---------------------------------------------------------------------------------------
// Small system of Eq. (Fs) in Woodbury form, one CTA:
//   M = diag(lambda + gamma) - K_m,  M y = h + gamma K (Lambda_gamma Z),  C = y + gamma Lambda_gamma Z
// LU with partial pivoting in FP32 shared memory.
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(1024)
k_small_solve(const double* __restrict__ K, int ldk, const double* __restrict__ h,
              const double* __restrict__ Z, const double* __restrict__ lam, double gamma,
              int L, int lp, int mp, const int* __restrict__ mdev, float* __restrict__ C,
              int* status) {
  extern __shared__ float sm[];
  const int m = mdev[0];
  const int ms = m | 1;
  float* M = sm;                       // m x ms
  float* W = M + (size_t)m * ms;       // m x L : Lambda_gamma Z
  float* B = W + (size_t)m * L;        // m x L : right-hand sides -> y
  __shared__ int piv_row, bad;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) bad = 0;
  for (int e = threadIdx.x; e < m * L; e += blockDim.x) {
    int i = e / L, k = e % L;
    W[i * L + k] = (float)(Z[(int64_t)i * lp + k] / (lam[i] + gamma));
  }
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    int i = e / m, j = e % m;
    float v = -(float)K[(int64_t)i * ldk + j];
    if (i == j) v += (float)(lam[i] + gamma);
    M[i * ms + j] = v;
  }
  __syncthreads();
  // B = h + gamma K W
  for (int e = threadIdx.x; e < m * L; e += blockDim.x) {
    int i = e / L, k = e % L;
    float s = 0.f;
    for (int j = 0; j < m; ++j) s = fmaf((float)K[(int64_t)i * ldk + j], W[j * L + k], s);
    B[i * L + k] = (float)h[(int64_t)i * lp + k] + (float)gamma * s;
  }
  // LU with partial pivoting
  for (int k = 0; k < m; ++k) {
    __syncthreads();
    if (warp == 0) {
      float best = -1.f;
      int bi = k;
      for (int i = k + lane; i < m; i += 32) {
        float a = fabsf(M[i * ms + k]);
        if (a > best) { best = a; bi = i; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        float ob = __shfl_xor_sync(0xffffffff, best, o);
        int oi = __shfl_xor_sync(0xffffffff, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (lane == 0) {
        piv_row = bi;
        if (!(best > 0.f)) bad = 1;
      }
    }
    __syncthreads();
    const int p = piv_row;
    if (p != k) {
      for (int j = threadIdx.x; j < m; j += blockDim.x) {
        float t = M[k * ms + j]; M[k * ms + j] = M[p * ms + j]; M[p * ms + j] = t;
      }
      for (int j = threadIdx.x; j < L; j += blockDim.x) {
        float t = B[k * L + j]; B[k * L + j] = B[p * L + j]; B[p * L + j] = t;
      }
      __syncthreads();
    }
    float pv = M[k * ms + k];
    if (pv == 0.f) pv = 1e-30f;
    const float inv = 1.f / pv;
    const int w = m - k - 1;
    for (int i = k + 1 + threadIdx.x; i < m; i += blockDim.x) M[i * ms + k] *= inv;
    __syncthreads();
    for (int e = threadIdx.x; e < w * w; e += blockDim.x) {
      int i = k + 1 + e / w, j = k + 1 + e % w;
      M[i * ms + j] = fmaf(-M[i * ms + k], M[k * ms + j], M[i * ms + j]);
    }
  }
  __syncthreads();
  // forward (unit lower) and backward (upper) substitution, one warp per label
  for (int k = warp; k < L; k += nw) {
    for (int i = 0; i < m; ++i) {
      float s = 0.f;
      for (int j = lane; j < i; j += 32) s = fmaf(M[i * ms + j], B[j * L + k], s);
      s = warp_sum(s);
      if (lane == 0) B[i * L + k] -= s;
      __syncwarp();
    }
    for (int i = m - 1; i >= 0; --i) {
      float s = 0.f;
      for (int j = i + 1 + lane; j < m; j += 32) s = fmaf(M[i * ms + j], B[j * L + k], s);
      s = warp_sum(s);
      if (lane == 0) B[i * L + k] = (B[i * L + k] - s) / M[i * ms + i];
      __syncwarp();
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < mp * lp; e += blockDim.x) {
    int i = e / lp, k = e % lp;
    float v = 0.f;
    if (i < m && k < L) v = B[i * L + k] + (float)gamma * W[i * L + k];
    C[e] = v;
  }
  if (threadIdx.x == 0 && bad) atomicOr(status, RW_DEV_SINGULAR);
}

// ---------------------------------------------------------------------------------------
// U-hat_n = Q_n C.  Same thread mapping as k_project; per-(row, chunk) partial dot products
// go to shared memory and are summed per row.  Writes either the refinement start (hat
// space, seeds = d^{1/2} one-hot) or the final U / labels.
// ---------------------------------------------------------------------------------------
template <typename T, int LP>
__global__ void __launch_bounds__(1024)
k_backproject(const T* __restrict__ Q, int ldq, int cpr, int R, const float* __restrict__ Cg,
              float cscale, const int* __restrict__ seedlab, const float* __restrict__ sq,
              const float* __restrict__ s, int64_t N, int L, const int* __restrict__ mdev,
              float* __restrict__ xhat, float* __restrict__ U, uint8_t* __restrict__ labels) {
  constexpr int V = Vec16<T>::V;
  extern __shared__ float smem[];
  float* Cs = smem;                    // ldq x LP
  float* part = Cs + ldq * LP;         // R x cpr x LP
  const int c = threadIdx.x % cpr, r = threadIdx.x / cpr;
  const int m = mdev[0];
  for (int e = threadIdx.x; e < ldq * LP; e += blockDim.x) Cs[e] = Cg[e] * cscale;
  __syncthreads();
  const bool active = r < R && c * V < m;
  for (int64_t base = (int64_t)blockIdx.x * R; base < N; base += (int64_t)gridDim.x * R) {
    const int64_t i = base + r;
    if (r < R) {
      float acc[LP];
#pragma unroll
      for (int k = 0; k < LP; ++k) acc[k] = 0.f;
      if (active && i < N) {
        float q[V];
        Vec16<T>::load(Q + i * ldq + c * V, q);
#pragma unroll
        for (int v = 0; v < V; ++v)
#pragma unroll
          for (int k = 0; k < LP; ++k) acc[k] = fmaf(q[v], Cs[(c * V + v) * LP + k], acc[k]);
      }
#pragma unroll
      for (int k = 0; k < LP; ++k) part[(r * cpr + c) * LP + k] = acc[k];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < R * LP; e += blockDim.x) {
      int rr = e / LP, k = e % LP;
      int64_t ii = base + rr;
      if (ii >= N) continue;
      float v = 0.f;
      for (int cc = 0; cc < cpr; ++cc) v += part[(rr * cpr + cc) * LP + k];
      int sl = seedlab[ii];
      if (sl >= 0) v = (k == sl) ? sq[ii] : 0.f;
      if (k >= L) v = 0.f;
      if (xhat) {
        xhat[ii * LP + k] = v;
      } else if (k < L) {
        U[ii * L + k] = (sl >= 0) ? ((k == sl) ? 1.f : 0.f) : v * s[ii];
      }
    }
    if (!xhat && labels) {
      __syncthreads();
      for (int rr = threadIdx.x; rr < R; rr += blockDim.x) {
        int64_t ii = base + rr;
        if (ii >= N) continue;
        int best = 0;
        float bv = U[ii * L];
        for (int k = 1; k < L; ++k) {
          float v = U[ii * L + k];
          if (v > bv) { bv = v; best = k; }
        }
        labels[ii] = (uint8_t)best;
      }
    }
    __syncthreads();
  }
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
              int last, float* __restrict__ U, uint8_t* __restrict__ labels) {
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
  for (int k = 0; k < L; ++k) {
    float u = (sl >= 0) ? (k == sl ? 1.f : 0.f) : xv[k] * si;
    U[i * L + k] = u;
    if (u > bv) { bv = u; best = k; }
  }
  if (labels) labels[i] = (uint8_t)best;
}

template <int LP>
rw_status launch_jacobi(const rw_graph* g, const float* xin, float* xout, const float* phat,
                        const int* seedlab, int L, float gamma, float omega, int last,
                        float* U, uint8_t* labels, cudaStream_t st) {
  k_jacobi_step<LP><<<rw_blocks(g->N, 256), 256, 0, st>>>(
      xin, xout, phat, seedlab, g->cw, g->d, g->s, g->normalized, g->kind, g->ndim, g->dims[0],
      g->dims[1], g->dims[2], g->rowptr, g->col, g->ccsr, g->N, L, gamma, omega, last, U,
      labels);
  RW_LAUNCH_CHECK();
  return RW_OK;
}

rw_status jacobi(const rw_graph* g, int lp, const float* xin, float* xout, const float* phat,
                 const int* seedlab, int L, float gamma, float omega, int last, float* U,
                 uint8_t* labels, cudaStream_t st) {
  switch (lp) {
    case 4: return launch_jacobi<4>(g, xin, xout, phat, seedlab, L, gamma, omega, last, U, labels, st);
    case 8: return launch_jacobi<8>(g, xin, xout, phat, seedlab, L, gamma, omega, last, U, labels, st);
    default: return launch_jacobi<16>(g, xin, xout, phat, seedlab, L, gamma, omega, last, U, labels, st);
  }
}

template <typename T, int LP>
rw_status launch_proj_back(bool back, const T* Q, int ldq, const float* phat,
                           const int* seedlab, const rw_graph* g, const int* mdev, float* part,
                           int nblk, const float* C, float cscale, float* xhat, float* U,
                           uint8_t* labels, int L, cudaStream_t st) {
  constexpr int V = Vec16<T>::V;
  const int cpr = ldq / V;
  const int R = std::max(1, 1024 / cpr);
  const int threads = cpr * R;
  if (!back) {
    size_t shm = sizeof(float) * ldq * LP;
    if (cpr <= 32)
      k_project<T, LP, 1><<<nblk, 256, shm, st>>>(Q, ldq, cpr, phat, seedlab, g->N, mdev, part);
    else if (cpr <= 64)
      k_project<T, LP, 2><<<nblk, 256, shm, st>>>(Q, ldq, cpr, phat, seedlab, g->N, mdev, part);
    else
      return RW_ERR_UNSUPPORTED;
  } else {
    size_t shm = sizeof(float) * ((size_t)ldq * LP + (size_t)R * cpr * LP);
    if (shm > 48 * 1024)
      cudaFuncSetAttribute(k_backproject<T, LP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    k_backproject<T, LP><<<nblk, threads, shm, st>>>(Q, ldq, cpr, R, C, cscale, seedlab, g->sq,
                                                     g->s, g->N, L, mdev, xhat, U, labels);
  }
  RW_LAUNCH_CHECK();
  return RW_OK;
}

template <typename T>
rw_status proj_back(int lp, bool back, const T* Q, int ldq, const float* phat, const int* seedlab,
                    const rw_graph* g, const int* mdev, float* part, int nblk, const float* C,
                    float cscale, float* xhat, float* U, uint8_t* labels, int L, cudaStream_t st) {
  switch (lp) {
    case 4: return launch_proj_back<T, 4>(back, Q, ldq, phat, seedlab, g, mdev, part, nblk, C, cscale, xhat, U, labels, L, st);
    case 8: return launch_proj_back<T, 8>(back, Q, ldq, phat, seedlab, g, mdev, part, nblk, C, cscale, xhat, U, labels, L, st);
    default: return launch_proj_back<T, 16>(back, Q, ldq, phat, seedlab, g, mdev, part, nblk, C, cscale, xhat, U, labels, L, st);
  }
}

__global__ void k_f32_to_bf16(const float* __restrict__ a, int64_t N, int m, int lda,
                              __nv_bfloat16* __restrict__ b, int ldb) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * ldb) return;
  int64_t r = e / ldb;
  int c = (int)(e % ldb);
  b[e] = __float2bfloat16(c < m ? a[r * lda + c] : 0.f);
}

}  // namespace

rw_status rw_solve_priors_internal(const rw_graph* g, const int32_t* seed_idx,
                                   const int32_t* seed_lab, int S, int L, int prior_mode,
                                   const float* priors, int lp, cudaStream_t st, float** phat_out,
                                   int** seedlab_out, double** fit64_out);

// ---------------------------------------------------------------------------------------
// Seed bookkeeping and priors, shared by the fast solve, the PCG solve and the gradients
// ---------------------------------------------------------------------------------------
rw_status rw_solve_priors_internal(const rw_graph* g, const int32_t* seed_idx,
                                   const int32_t* seed_lab, int S, int L, int prior_mode,
                                   const float* priors, int lp, cudaStream_t st, float** phat_out,
                                   int** seedlab_out, double** fit64_out) {
  rw_graph* gm = const_cast<rw_graph*>(g);
  SolveWorkspace& ws = gm->ws;
  RW_TRY(ws.seedlab.grow(sizeof(int) * g->N));
  RW_TRY(ws.phat.grow(sizeof(float) * g->N * lp));
  // stats (48 doubles) + fit (48 floats) + fit64 (32 doubles) live in ws.pcg's head? use own buffer
  static_assert(sizeof(double) * 48 + sizeof(float) * 48 + sizeof(double) * 32 < 2048, "");
  if (gm->upd.cap < 4096) return RW_ERR_OOM;
  double* stats = gm->upd.as<double>();
  float* fit = reinterpret_cast<float*>(stats + 48);
  double* fit64 = reinterpret_cast<double*>(fit + 48);
  int* seedlab = ws.seedlab.as<int>();
  k_fill_i32<<<rw_blocks(g->N, 256), 256, 0, st>>>(seedlab, g->N, -1);
  RW_LAUNCH_CHECK();
  RW_CHECK_CUDA(cudaMemsetAsync(stats, 0, sizeof(double) * 48, st));
  k_seed_scatter<<<rw_blocks(S, 256), 256, 0, st>>>(seed_idx, seed_lab, S, L, g->N, g->J ? g->J : nullptr,
                                                    seedlab, stats, g->status);
  RW_LAUNCH_CHECK();
  k_fit<<<1, 32, 0, st>>>(stats, L, prior_mode, fit, fit64, g->status);
  RW_LAUNCH_CHECK();
  k_priors<<<rw_blocks(g->N, 256), 256, 0, st>>>(g->J, g->sq, g->N, L, lp, prior_mode, fit, priors,
                                                 ws.phat.as<float>(), g->status);
  RW_LAUNCH_CHECK();
  *phat_out = ws.phat.as<float>();
  *seedlab_out = seedlab;
  if (fit64_out) *fit64_out = fit64;
  return RW_OK;
}

static rw_status validate_solve(const rw_graph* g, const rw_basis* b, const int32_t* si,
                                const int32_t* sl, int S, int L, const float* priors,
                                const rw_solve_opts* o, const void* prob) {
  if (!g || !b || !si || !sl || !o || !prob) return RW_ERR_INVALID_ARG;
  if (b->N != g->N) return RW_ERR_INVALID_ARG;
  if (S < 1 || S > 65536 || L < 1 || L > RW_MAX_LABELS) return RW_ERR_INVALID_ARG;
  if (!(o->gamma > 0.0)) return o->gamma == 0.0 ? RW_ERR_UNSUPPORTED : RW_ERR_INVALID_ARG;
  if (o->m < 0 || o->m > b->m) return RW_ERR_INVALID_ARG;
  if (o->refine_steps < 0 || o->refine_steps > 100000) return RW_ERR_INVALID_ARG;
  if (o->prior_mode == 1 && !priors) return RW_ERR_INVALID_ARG;
  if (o->prior_mode != 0 && o->prior_mode != 1) return RW_ERR_INVALID_ARG;
  if (o->prior_mode == 0 && !g->J) return RW_ERR_INVALID_ARG;
  if (o->basis_format < RW_BASIS_F16 || o->basis_format > RW_BASIS_F32) return RW_ERR_INVALID_ARG;
  if (o->refine_mode != RW_REFINE_JACOBI && o->refine_mode != RW_REFINE_PCG) return RW_ERR_INVALID_ARG;
  int mmax = o->m > 0 ? o->m : b->m;
  if (mmax > kMaxSmallM) return RW_ERR_UNSUPPORTED;
  // one CTA holds an m x m FP32 matrix plus label-sized vectors in shared memory
  const size_t shm_adapt = sizeof(float) * ((size_t)mmax * (mmax | 1) + 3 * (size_t)L * mmax);
  const size_t shm_small = sizeof(float) * ((size_t)mmax * (mmax | 1) + 2 * (size_t)L * mmax);
  if (std::max(o->m == 0 ? shm_adapt : 0, shm_small) > 227 * 1024) return RW_ERR_UNSUPPORTED;
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
  const int m_step = opts->m_step > 0 ? opts->m_step : 10;
  const double eps = opts->eps > 0 ? opts->eps : 0.1;
  const float omega = (float)(opts->omega > 0 ? std::min(opts->omega, 1.0) : 0.8);
  const bool adaptive = opts->m == 0;
  const int m_max = adaptive ? b->m : opts->m;
  // adaptive candidates: m_step, 2 m_step, ..., m_max (m_max last)
  int cand_h[2048];
  int ncand = 0;
  if (adaptive) {
    for (int m = m_step; m < m_max && ncand < 2047; m += m_step) cand_h[ncand++] = m;
    cand_h[ncand++] = m_max;
  }
  const int sms = g_rw_num_sms > 0 ? g_rw_num_sms : 148;
  const int nblk = 4 * sms;  // blocks of the two basis passes (partials of the projection)
  const int mq = std::max(b->ld16, b->ld32);  // rows of Z, C and the partials
  Layout lay = make_layout(S, mp, mq, lp, std::max(ncand, 1), nblk);
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
  RW_TRY(rw_solve_priors_internal(g, seed_idx_dev, seed_lab_dev, S, L, opts->prior_mode,
                                  priors_dev, lp, st, &phat, &seedlab, &fit64));

  RW_TRY(mark(1));
  float* Qs = reinterpret_cast<float*>(P(lay.Qs));
  float* Xs = reinterpret_cast<float*>(P(lay.Xs));
  float* Us = reinterpret_cast<float*>(P(lay.Us));
  float* R0 = reinterpret_cast<float*>(P(lay.R0));
  k_seed_gather<<<rw_blocks((int64_t)S * 32, 256), 256, 0, st>>>(
      seed_idx_dev, seed_lab_dev, S, L, lp, g->N, b->Q32, b->ld32, mp, seedlab, g->cw, g->d,
      g->sq, g->normalized, g->kind, g->ndim, g->dims[0], g->dims[1], g->dims[2], g->rowptr,
      g->col, g->ccsr, (float)gamma, Qs, Xs, Us, R0);
  RW_LAUNCH_CHECK();
  double* G = reinterpret_cast<double*>(P(lay.G));
  double* K = reinterpret_cast<double*>(P(lay.K));
  double* bv = reinterpret_cast<double*>(P(lay.bv));
  double* h = reinterpret_cast<double*>(P(lay.h));
  RW_TRY(rw_gram(Qs, mp, Xs, mp, S, m_max, m_max, K, mp, false, st));
  RW_TRY(rw_gram(Qs, mp, R0, lp, S, m_max, lp, h, lp, false, st));
  double* fsel = reinterpret_cast<double*>(P(lay.fc)) + (size_t)ncand * lp;
  if (adaptive) {
    RW_TRY(rw_gram(Qs, mp, Qs, mp, S, m_max, m_max, G, mp, false, st));
    RW_TRY(rw_gram(Qs, mp, Us, lp, S, m_max, lp, bv, lp, false, st));
  }
  RW_TRY(mark(2));
  if (adaptive) {
    int* cand = reinterpret_cast<int*>(P(lay.cand));
    int* pass = reinterpret_cast<int*>(P(lay.pass));
    double* fc = reinterpret_cast<double*>(P(lay.fc));
    RW_CHECK_CUDA(cudaMemcpyAsync(cand, cand_h, sizeof(int) * ncand, cudaMemcpyHostToDevice, st));
    // rho = sqrt(1^T D 1) (normalized, Sec. III-A-1) or sqrt(N): needs the degree sum
    const double rho = g->normalized ? sqrt(g->dsum) : sqrt((double)g->N);
    const double fmax = (double)S * eps * eps;
    size_t shm = sizeof(float) * ((size_t)m_max * (m_max | 1) + 3 * (size_t)L * m_max);
    cudaFuncSetAttribute(k_adapt, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    k_adapt<<<ncand, 1024, shm, st>>>(G, mp, bv, lp, Qs, mp, Us, S, L, cand, rho, fmax, fc, pass);
    RW_LAUNCH_CHECK();
    k_pick<<<1, 32, 0, st>>>(cand, pass, ncand, fc, lp, mdev, fsel);
    RW_LAUNCH_CHECK();
  } else {
    k_set_m<<<1, 32, 0, st>>>(mdev, m_max);
    RW_LAUNCH_CHECK();
  }
  RW_TRY(mark(3));
  // Z = Q_n^T P-hat_n
  float* part = reinterpret_cast<float*>(P(lay.part));
  double* Z = reinterpret_cast<double*>(P(lay.Z));
  int fmt = opts->basis_format;
  if (fmt == RW_BASIS_BF16 && !b->Qbf) {
    rw_basis* bm = const_cast<rw_basis*>(b);
    RW_CHECK_CUDA(cudaMalloc(&bm->Qbf, sizeof(__nv_bfloat16) * b->N * b->ld16));
    k_f32_to_bf16<<<rw_blocks(b->N * b->ld16, 256), 256, 0, st>>>(b->Q32, b->N, b->m, b->ld32,
                                                                   bm->Qbf, b->ld16);
    RW_LAUNCH_CHECK();
  }
  int ldq_e = fmt == RW_BASIS_F32 ? b->ld32 : b->ld16;
  double zscale = fmt == RW_BASIS_F16 ? 1.0 / b->qscale : 1.0;
  float cscale = fmt == RW_BASIS_F16 ? 1.f / b->qscale : 1.f;
  if (fmt == RW_BASIS_F16)
    RW_TRY(proj_back<__half>(lp, false, b->Q16, ldq_e, phat, seedlab, g, mdev, part, nblk, nullptr, 0.f, nullptr, nullptr, nullptr, L, st));
  else if (fmt == RW_BASIS_BF16)
    RW_TRY(proj_back<__nv_bfloat16>(lp, false, b->Qbf, ldq_e, phat, seedlab, g, mdev, part, nblk, nullptr, 0.f, nullptr, nullptr, nullptr, L, st));
  else
    RW_TRY(proj_back<float>(lp, false, b->Q32, ldq_e, phat, seedlab, g, mdev, part, nblk, nullptr, 0.f, nullptr, nullptr, nullptr, L, st));
  k_reduce_partials<<<rw_blocks((int64_t)mq * lp * 32, 256), 256, 0, st>>>(part, nblk, ldq_e, lp, mq, zscale, Z);
  RW_LAUNCH_CHECK();
  RW_TRY(mark(4));
  // small system
  float* C = reinterpret_cast<float*>(P(lay.C));
  {
    size_t shm = sizeof(float) * ((size_t)m_max * (m_max | 1) + 2 * (size_t)L * m_max);
    cudaFuncSetAttribute(k_small_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    k_small_solve<<<1, 1024, shm, st>>>(K, mp, h, Z, b->lam, gamma, L, lp, mq, mdev, C, g->status);
    RW_LAUNCH_CHECK();
  }
  RW_TRY(mark(5));
  // back-projection (+ refinement)
  const int steps = opts->refine_steps;
  float* xh0 = nullptr;
  float* xh1 = nullptr;
  if (steps > 0) {
    RW_TRY(ws.xhat[0].grow(sizeof(float) * g->N * lp));
    RW_TRY(ws.xhat[1].grow(sizeof(float) * g->N * lp));
    xh0 = ws.xhat[0].as<float>();
    xh1 = ws.xhat[1].as<float>();
  }
  if (fmt == RW_BASIS_F16)
    RW_TRY(proj_back<__half>(lp, true, b->Q16, ldq_e, phat, seedlab, g, mdev, part, nblk, C, cscale, xh0, prob_dev, labels_dev, L, st));
  else if (fmt == RW_BASIS_BF16)
    RW_TRY(proj_back<__nv_bfloat16>(lp, true, b->Qbf, ldq_e, phat, seedlab, g, mdev, part, nblk, C, cscale, xh0, prob_dev, labels_dev, L, st));
  else
    RW_TRY(proj_back<float>(lp, true, b->Q32, ldq_e, phat, seedlab, g, mdev, part, nblk, C, cscale, xh0, prob_dev, labels_dev, L, st));
  RW_TRY(mark(6));
  if (steps > 0) {
    if (opts->refine_mode == RW_REFINE_JACOBI) {
      float* a = xh0;
      float* c = xh1;
      for (int t = 0; t < steps; ++t) {
        int last = (t == steps - 1);
        RW_TRY(jacobi(g, lp, a, c, phat, seedlab, L, (float)gamma, omega, last,
                      last ? prob_dev : nullptr, last ? labels_dev : nullptr, st));
        std::swap(a, c);
      }
    } else {
      RW_TRY(rw_pcg_from(g, phat, seedlab, L, lp, gamma, xh0, steps, 0.0, prob_dev, labels_dev,
                         nullptr, st));
    }
  }
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
      info->mu[k] = f64[k];
      info->sigma[k] = f64[16 + k];
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

extern "C" rw_status rw_solve_host(const rw_graph* g, const rw_basis* b,
                                   const int32_t* seed_idx_host, const int32_t* seed_lab_host,
                                   int32_t S, int32_t n_labels, const float* priors_host,
                                   const rw_solve_opts* opts, float* prob_host,
                                   uint8_t* labels_host, rw_solve_info* info, void* stream) {
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
  RW_CHECK_CUDA(cudaStreamSynchronize(st));
  return s;
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
