// Gradient of a loss on the label probabilities through the eigenvector (fast) solve of
// Sec. II-B in the normalized form of Sec. II-C, with respect to the edge weights and beta.
//
// The basis Q (first m columns) is held fixed; its values are the Rayleigh quotients of
// Eq. (z_ray) under the current weights, lambda-hat_i = sum_e w_e (q_ia s_a - q_ib s_b)^2 /
// |q_i|^2, s = d^{-1/2}.  Forward, with c_ab = w_ab s_a s_b, Lambda = diag(1/(lambda-hat+gamma)),
// U-hat_s = d_s^{1/2} onehot, P-hat = d^{1/2} P:
//   X = B-hat Q_n = -C_sn Q_n,  Z = Q_n^T P-hat_n,  L-hat_s U-hat_s = U-hat_s - C_ss U-hat_s,
//   rhs = L-hat_s U-hat_s + gamma (U-hat_s + X Lambda Z)                     Eq. (Fs)
//   K = Lambda^{-1} - Q_s^T X,  y = K^{-1} Q_s^T rhs,  F_s = rhs + X y        (Woodbury form)
//   C = y + gamma Lambda Z = Lambda (Q_s^T F_s + gamma Z),  x_0 = Q_n C        Eq. (U_lin_comb)
//   x_{t+1} = (1 - omega) x_t + a (C_nn x_t + b),  b = gamma P-hat_n + C_ns U-hat_s,
//   a = omega / (1 + gamma)   (damped Jacobi on (L-hat_n + gamma I) U-hat_n = b),
//   U_n = s_n x_k.
// Reverse (G = d loss / d U):
//   x-bar_k = s G;  x-bar_{t-1} = (1 - omega) x-bar_t + a C_nn x-bar_t;  b-bar = a sum_t x-bar_t
//   C-bar = Q_n^T x-bar_0;  Y-bar = Lambda C-bar;  F_s-bar = Q_s Y-bar
//   rhs-bar = M^{-T} F_s-bar = F_s-bar + Q_s K^{-T} X^T F_s-bar   (M = I - X Lambda Q_s^T)
//   X-bar = rhs-bar C^T,  so the seed-to-free edge term is -rhs-bar_a . x_0,b
//   Lambda-bar_i = sum_k [C-bar (Lambda^{-1} C) + (X^T rhs-bar)(Lambda^{-1} y + gamma Z)]_ik
//   Z-bar = gamma Y-bar + gamma Lambda X^T rhs-bar,  P-hat-bar_n = gamma b-bar + Q_n Z-bar
// and from there through the Rayleigh values, c_ab = w s_a s_b, d^{-1/2}, d^{1/2} and d to w
// and beta (Eq. W).  The same steps are restated in FP64 by the oracle; here the N-sized passes
// are FP32 and the m x m work FP64.
#include "rw_internal.cuh"

#include <algorithm>
#include <vector>


namespace {

constexpr int kBetaBlocks = 1024;

struct Grid3 {
  int ndim, DX, DY, DZ;
  int64_t N;
  __device__ void coords(int64_t i, int c[3]) const {
    c[0] = (int)(i % DX);
    c[1] = (int)((i / DX) % DY);
    c[2] = (int)(i / ((int64_t)DX * DY));
  }
  __device__ int64_t stride(int a) const {
    return a == 0 ? 1 : (a == 1 ? (int64_t)DX : (int64_t)DX * DY);
  }
  __device__ int extent(int a) const { return a == 0 ? DX : (a == 1 ? DY : DZ); }
};

// visit every neighbour j of i: fn(j, edge id)
template <class F>
__device__ __forceinline__ void for_each_nbr(const Grid3& G, int64_t i, F fn) {
  int c[3];
  G.coords(i, c);
  for (int a = 0; a < G.ndim; ++a) {
    const int64_t st = G.stride(a);
    if (c[a] > 0) fn(i - st, a * G.N + i - st);
    if (c[a] + 1 < G.extent(a)) fn(i + st, a * G.N + i);
  }
}

__device__ __forceinline__ float dotl(const float* a, const float* b, int L) {
  float s = 0.f;
  for (int k = 0; k < L; ++k) s = fmaf(a[k], b[k], s);
  return s;
}

__global__ void k_posmap(const int32_t* __restrict__ seed_idx, int S, int* __restrict__ pos) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < S) pos[seed_idx[t]] = t;
}

__global__ void k_fill(int* p, int64_t n, int v) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

// one warp per seed t (node i, label l): Q_s row, X row = -sum_{free j} c_ij q_j,
// U-hat_s row = d_i^{1/2} e_l, (L-hat_s U-hat_s) row = U-hat_s row - sum_{seeded j} c_ij U-hat_j
__global__ void k_fg_seed_rows(Grid3 G, const int32_t* __restrict__ seed_idx,
                               const int* __restrict__ seedlab, const float* __restrict__ cw,
                               const float* __restrict__ sq, const float* __restrict__ Q,
                               int64_t ldq, int m, int S, int lp, float* __restrict__ Qs,
                               float* __restrict__ X, int ldx, float* __restrict__ Ush,
                               float* __restrict__ LsUs) {
  const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (t >= S) return;
  const int64_t i = seed_idx[t];
  const int l = seedlab[i];
  for (int c = lane; c < ldx; c += 32) {
    Qs[(int64_t)t * ldx + c] = c < m ? Q[i * ldq + c] : 0.f;
    X[(int64_t)t * ldx + c] = 0.f;
  }
  float ls = (lane == l) ? sq[i] : 0.f;
  __syncwarp();
  for_each_nbr(G, i, [&](int64_t j, int64_t e) {
    const float c = cw[e];
    const int lj = seedlab[j];
    if (lj < 0) {
      for (int cc = lane; cc < m; cc += 32) X[(int64_t)t * ldx + cc] -= c * Q[j * ldq + cc];
    } else if (lane == lj) {
      ls -= c * sq[j];
    }
  });
  if (lane < lp) {
    Ush[(int64_t)t * lp + lane] = (lane == l) ? sq[i] : 0.f;
    LsUs[(int64_t)t * lp + lane] = ls;
  }
}

// rows of seeded nodes zeroed (a copy of P-hat restricted to the free nodes)
__global__ void k_mask_rows(const float* __restrict__ src, const int* __restrict__ seedlab,
                            int64_t N, int lp, float* __restrict__ dst) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * lp) return;
  dst[e] = seedlab[e / lp] < 0 ? src[e] : 0.f;
}

// K = diag(lambda-hat + gamma) - Q_s^T X (in place on the Gram), lgZ = Lambda Z (FP32 m x lp)
__global__ void k_fg_K(double* __restrict__ K, int m, const double* __restrict__ lam,
                       double gamma, const double* __restrict__ Z, int lp,
                       float* __restrict__ lgZ) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < m * m) {
    const int i = e / m, j = e % m;
    K[e] = (i == j ? lam[i] + gamma : 0.0) - K[e];
  }
  if (e < m * lp) {
    const int i = e / lp;
    lgZ[e] = (float)(Z[e] / (lam[i] + gamma));
  }
}

// rhs = LsUs + gamma (Ush + XlgZ)
__global__ void k_fg_rhs(const float* __restrict__ LsUs, const float* __restrict__ Ush,
                         const float* __restrict__ XlgZ, int n, float gamma,
                         float* __restrict__ rhs) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) rhs[e] = LsUs[e] + gamma * (Ush[e] + XlgZ[e]);
}

// In-place LU with partial pivoting of an m x m FP64 matrix (row-major) by one CTA; piv[k]
// is the row swapped with k at step k.  A zero pivot sets *bad.
__global__ void __launch_bounds__(256) k_lu64(double* __restrict__ A, int m, int* __restrict__ piv,
                                              int* __restrict__ bad) {
  __shared__ double vbest[8];
  __shared__ int ibest[8];
  __shared__ int prow;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int k = 0; k < m; ++k) {
    double bv = -1.0;
    int bi = k;
    for (int r = k + tid; r < m; r += blockDim.x) {
      const double v = fabs(A[(int64_t)r * m + k]);
      if (v > bv) { bv = v; bi = r; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffff, bv, o);
      const int oi = __shfl_xor_sync(0xffffffff, bi, o);
      if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
    }
    if (lane == 0) { vbest[warp] = bv; ibest[warp] = bi; }
    __syncthreads();
    if (tid == 0) {
      double v = vbest[0];
      int r = ibest[0];
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
        if (vbest[w] > v || (vbest[w] == v && ibest[w] < r)) { v = vbest[w]; r = ibest[w]; }
      prow = r;
      piv[k] = r;
      if (!(v > 0.0)) *bad = 1;
    }
    __syncthreads();
    const int r = prow;
    if (r != k)
      for (int c = tid; c < m; c += blockDim.x) {
        const double t = A[(int64_t)k * m + c];
        A[(int64_t)k * m + c] = A[(int64_t)r * m + c];
        A[(int64_t)r * m + c] = t;
      }
    __syncthreads();
    double p = A[(int64_t)k * m + k];
    if (p == 0.0) p = 1e-300;
    for (int rr = k + 1 + tid; rr < m; rr += blockDim.x) A[(int64_t)rr * m + k] /= p;
    __syncthreads();
    const int rem = m - k - 1;
    for (int e = tid; e < rem * rem; e += blockDim.x) {
      const int rr = k + 1 + e / rem, c = k + 1 + e % rem;
      A[(int64_t)rr * m + c] -= A[(int64_t)rr * m + k] * A[(int64_t)k * m + c];
    }
    __syncthreads();
  }
}

// Solve K x = b (trans = 0) or K^T x = b (trans = 1) from the LU of k_lu64, for nr right-hand
// sides stored m x ldb (FP64, in place).  One CTA, one thread per right-hand side column.
__global__ void k_lu64_solve(const double* __restrict__ A, int m, const int* __restrict__ piv,
                             double* __restrict__ B, int ldb, int nr, int trans) {
  const int c = threadIdx.x;
  if (c >= nr) return;
  auto b = [&](int i) -> double& { return B[(int64_t)i * ldb + c]; };
  if (!trans) {
    for (int k = 0; k < m; ++k)
      if (piv[k] != k) { double t = b(k); b(k) = b(piv[k]); b(piv[k]) = t; }
    for (int i = 0; i < m; ++i) {  // L (unit) forward
      double s = b(i);
      for (int j = 0; j < i; ++j) s -= A[(int64_t)i * m + j] * b(j);
      b(i) = s;
    }
    for (int i = m - 1; i >= 0; --i) {  // U backward
      double s = b(i);
      for (int j = i + 1; j < m; ++j) s -= A[(int64_t)i * m + j] * b(j);
      b(i) = s / A[(int64_t)i * m + i];
    }
  } else {
    // P K = L U  =>  K^T = U^T L^T P ;  solve U^T z = b, L^T w = z, x = P^T w
    for (int i = 0; i < m; ++i) {
      double s = b(i);
      for (int j = 0; j < i; ++j) s -= A[(int64_t)j * m + i] * b(j);
      b(i) = s / A[(int64_t)i * m + i];
    }
    for (int i = m - 1; i >= 0; --i) {
      double s = b(i);
      for (int j = i + 1; j < m; ++j) s -= A[(int64_t)j * m + i] * b(j);
      b(i) = s;
    }
    for (int k = m - 1; k >= 0; --k)
      if (piv[k] != k) { double t = b(k); b(k) = b(piv[k]); b(piv[k]) = t; }
  }
}

// C = y + gamma Lambda Z (FP64 and FP32 copies); y in place
__global__ void k_fg_C(const double* __restrict__ y, const double* __restrict__ Z,
                       const double* __restrict__ lam, double gamma, int m, int lp,
                       double* __restrict__ C64, float* __restrict__ C32, float* __restrict__ y32) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m * lp) return;
  const int i = e / lp;
  const double c = y[e] + gamma * Z[e] / (lam[i] + gamma);
  C64[e] = c;
  C32[e] = (float)c;
  y32[e] = (float)y[e];
}

// free rows: b = gamma P-hat + sum_{seeded j} c_ij U-hat_j; seeded rows 0
__global__ void k_fg_b(Grid3 G, const float* __restrict__ phat, const int* __restrict__ seedlab,
                       const float* __restrict__ cw, const float* __restrict__ sq, int lp,
                       float gamma, float* __restrict__ b) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= G.N) return;
  float acc[16];
  for (int k = 0; k < lp; ++k) acc[k] = 0.f;
  if (seedlab[i] < 0) {
    for (int k = 0; k < lp; ++k) acc[k] = gamma * phat[i * lp + k];
    for_each_nbr(G, i, [&](int64_t j, int64_t e) {
      const int lj = seedlab[j];
      if (lj >= 0) acc[lj] = fmaf(cw[e], sq[j], acc[lj]);
    });
  }
  for (int k = 0; k < lp; ++k) b[i * lp + k] = acc[k];
}

// seeded rows of x zeroed (the tall product also wrote them)
__global__ void k_zero_seeded(float* __restrict__ x, const int* __restrict__ seedlab, int64_t N,
                              int lp) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < N * lp && seedlab[e / lp] >= 0) x[e] = 0.f;
}

// one damped-Jacobi step on the free rows: y = (1 - omega) x + a (C_nn x + b)
__global__ void k_fg_jacobi(Grid3 G, const float* __restrict__ x, const float* __restrict__ b,
                            const int* __restrict__ seedlab, const float* __restrict__ cw, int lp,
                            float omega, float a, float* __restrict__ y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= G.N) return;
  float acc[16];
  for (int k = 0; k < lp; ++k) acc[k] = 0.f;
  if (seedlab[i] < 0) {
    for (int k = 0; k < lp; ++k) acc[k] = b[i * lp + k];
    for_each_nbr(G, i, [&](int64_t j, int64_t e) {
      if (seedlab[j] < 0) {
        const float c = cw[e];
        for (int k = 0; k < lp; ++k) acc[k] = fmaf(c, x[j * lp + k], acc[k]);
      }
    });
    for (int k = 0; k < lp; ++k) acc[k] = (1.f - omega) * x[i * lp + k] + a * acc[k];
  }
  for (int k = 0; k < lp; ++k) y[i * lp + k] = acc[k];
}

// U = s x on free rows, one-hot on seeds (the forward result, N x L)
__global__ void k_fg_U(const float* __restrict__ x, const int* __restrict__ seedlab,
                       const float* __restrict__ s, int64_t N, int L, int lp,
                       float* __restrict__ U) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * L) return;
  const int64_t i = e / L;
  const int k = (int)(e % L);
  const int sl = seedlab[i];
  U[e] = sl >= 0 ? (k == sl ? 1.f : 0.f) : s[i] * x[i * lp + k];
}

// x-bar_k = s G (free rows), s-bar = sum_k G x_k (free rows)
__global__ void k_fg_out_rev(const float* __restrict__ Gd, const float* __restrict__ xk,
                             const int* __restrict__ seedlab, const float* __restrict__ s,
                             int64_t N, int L, int lp, float* __restrict__ xbar,
                             float* __restrict__ sbar) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const bool fr = seedlab[i] < 0;
  float acc = 0.f;
  for (int k = 0; k < lp; ++k) {
    const float gk = (fr && k < L) ? Gd[i * L + k] : 0.f;
    xbar[i * lp + k] = s[i] * gk;
    acc = fmaf(gk, xk[i * lp + k], acc);
  }
  sbar[i] = acc;
}

// reverse of one Jacobi step: xb_out = (1 - omega) xb + a C_nn xb; bbar += a xb;
// cbar[e] += a (xb_i . xprev_j + xb_j . xprev_i) on forward edges between free nodes
__global__ void k_fg_jacobi_rev(Grid3 G, const float* __restrict__ xb,
                                const float* __restrict__ xprev, const int* __restrict__ seedlab,
                                const float* __restrict__ cw, int lp, float omega, float a,
                                float* __restrict__ xb_out, float* __restrict__ bbar,
                                float* __restrict__ cbar) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= G.N) return;
  float acc[16];
  for (int k = 0; k < lp; ++k) acc[k] = 0.f;
  const bool fi = seedlab[i] < 0;
  if (fi) {
    for_each_nbr(G, i, [&](int64_t j, int64_t e) {
      if (seedlab[j] < 0) {
        const float c = cw[e];
        for (int k = 0; k < lp; ++k) acc[k] = fmaf(c, xb[j * lp + k], acc[k]);
        if (j > i)
          cbar[e] += a * (dotl(xb + i * lp, xprev + j * lp, lp) + dotl(xb + j * lp, xprev + i * lp, lp));
      }
    });
    for (int k = 0; k < lp; ++k) {
      const float v = xb[i * lp + k];
      bbar[i * lp + k] += a * v;
      acc[k] = (1.f - omega) * v + a * acc[k];
    }
  }
  for (int k = 0; k < lp; ++k) xb_out[i * lp + k] = acc[k];
}

// Ybar32 = Lambda Cbar, lgbar = sum_k Cbar (Lambda^{-1} C)
__global__ void k_fg_small1(const double* __restrict__ Cbar, const double* __restrict__ C64,
                            const double* __restrict__ lam, double gamma, int m, int lp,
                            float* __restrict__ Ybar32, double* __restrict__ lgbar) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const double li = lam[i] + gamma;
  double acc = 0.0;
  for (int k = 0; k < lp; ++k) {
    const double cb = Cbar[i * lp + k];
    Ybar32[i * lp + k] = (float)(cb / li);
    acc += cb * li * C64[i * lp + k];
  }
  lgbar[i] = acc;
}

// v32 = FP32 copy of the K^{-T} solve
__global__ void k_f64_to_f32_n(const double* __restrict__ a, float* __restrict__ b, int n) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) b[e] = (float)a[e];
}

// with t3 = X^T rhs-bar: lgbar += sum_k t3 (Lambda^{-1} y + gamma Z);
// Zbar32 = gamma (Ybar + Lambda t3); coef = -lgbar Lambda^2 / |q|^2 (Rayleigh weights)
__global__ void k_fg_small2(const double* __restrict__ t3, const double* __restrict__ y,
                            const double* __restrict__ Z, const float* __restrict__ Ybar32,
                            const double* __restrict__ lam, const double* __restrict__ qn2,
                            double gamma, int m, int lp, double* __restrict__ lgbar,
                            float* __restrict__ Zbar32, float* __restrict__ coef) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const double li = lam[i] + gamma;
  double acc = lgbar[i];
  for (int k = 0; k < lp; ++k) {
    const double t = t3[i * lp + k];
    acc += t * (li * y[i * lp + k] + gamma * Z[i * lp + k]);
    Zbar32[i * lp + k] = (float)(gamma * ((double)Ybar32[i * lp + k] + t / li));
  }
  lgbar[i] = acc;
  coef[i] = (float)(-acc / (li * li) / qn2[i]);
}

// per seed t (node i, label l): U-hat_s-bar[t][l] = (1 + gamma) rhsbar[t][l]
//   - sum_{seeded j} c_ij rhsbar[pos j][l] + sum_{free j} c_ij bbar[j][l]  -> sqbar[i]
__global__ void k_fg_seed_rev(Grid3 G, const int32_t* __restrict__ seed_idx,
                              const int* __restrict__ seedlab, const int* __restrict__ pos,
                              const float* __restrict__ cw, const float* __restrict__ rbar,
                              const float* __restrict__ bbar, int S, int lp, float gamma,
                              float* __restrict__ sqbar) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= S) return;
  const int64_t i = seed_idx[t];
  const int l = seedlab[i];
  float acc = (1.f + gamma) * rbar[(int64_t)t * lp + l];
  for_each_nbr(G, i, [&](int64_t j, int64_t e) {
    const float c = cw[e];
    if (seedlab[j] >= 0) acc -= c * rbar[(int64_t)pos[j] * lp + l];
    else acc += c * bbar[j * lp + l];
  });
  sqbar[i] = acc;
}

// free rows: sqbar = sum_k (gamma bbar + QZbar) P (P-hat = d^{1/2} P)
__global__ void k_fg_sqbar_free(const float* __restrict__ QZbar, const float* __restrict__ bbar,
                                const float* __restrict__ P, const int* __restrict__ seedlab,
                                int64_t N, int L, int lp, float gamma, float* __restrict__ sqbar) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N || seedlab[i] >= 0) return;
  float acc = 0.f;
  for (int k = 0; k < L; ++k)
    acc = fmaf(fmaf(gamma, bbar[i * lp + k], QZbar[i * lp + k]), P[i * L + k], acc);
  sqbar[i] = acc;
}

// coefficient gradient on edges with a seeded end (forward edges e = (i, j)):
//   free i, seeded j: bbar_i . U-hat_j - rhsbar_j . x0_i   (and mirrored)
//   both seeded:      -(rhsbar_i . U-hat_j + rhsbar_j . U-hat_i)
__global__ void k_fg_cbar_seed(Grid3 G, const int* __restrict__ seedlab,
                               const int* __restrict__ pos, const float* __restrict__ sq,
                               const float* __restrict__ bbar, const float* __restrict__ x0,
                               const float* __restrict__ rbar, int lp,
                               float* __restrict__ cbar) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= G.N) return;
  const int li = seedlab[i];
  int c[3];
  G.coords(i, c);
  for (int a = 0; a < G.ndim; ++a) {
    if (c[a] + 1 >= G.extent(a)) continue;
    const int64_t j = i + G.stride(a), e = a * G.N + i;
    const int lj = seedlab[j];
    if (li < 0 && lj < 0) continue;
    float v;
    if (li < 0) {
      v = bbar[i * lp + lj] * sq[j] - dotl(rbar + (int64_t)pos[j] * lp, x0 + i * lp, lp);
    } else if (lj < 0) {
      v = bbar[j * lp + li] * sq[i] - dotl(rbar + (int64_t)pos[i] * lp, x0 + j * lp, lp);
    } else {
      v = -(rbar[(int64_t)pos[i] * lp + lj] * sq[j] + rbar[(int64_t)pos[j] * lp + li] * sq[i]);
    }
    cbar[e] += v;
  }
}

// Rayleigh part, one warp per node a: for each incident edge (a, b) with D = q_a s_a - q_b s_b,
// sbar_a += 2 w sum_i coef_i D_i q_ia; on forward edges wray_e = sum_i coef_i D_i^2
__global__ void k_fg_rayleigh_rev(Grid3 G, const float* __restrict__ Q, int64_t ldq, int m,
                                  const float* __restrict__ w, const float* __restrict__ s,
                                  const float* __restrict__ coef, float* __restrict__ sray,
                                  float* __restrict__ wray) {
  const int64_t a = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (a >= G.N) return;
  const float sa = s[a];
  float sacc = 0.f;
  for_each_nbr(G, a, [&](int64_t b, int64_t e) {
    const float sb = s[b], we = w[e];
    float t1 = 0.f, t2 = 0.f;
    for (int i = lane; i < m; i += 32) {
      const float qa = Q[a * ldq + i], qb = Q[b * ldq + i];
      const float D = qa * sa - qb * sb, cd = coef[i] * D;
      t1 = fmaf(cd, D, t1);
      t2 = fmaf(cd, qa, t2);
    }
    for (int o = 16; o > 0; o >>= 1) {
      t1 += __shfl_xor_sync(0xffffffff, t1, o);
      t2 += __shfl_xor_sync(0xffffffff, t2, o);
    }
    sacc = fmaf(2.f * we, t2, sacc);
    if (b > a && lane == 0) wray[e] = t1;
  });
  if (lane == 0) sray[a] = sacc;
}

// dbar = sbar_total (-1/2 d^{-3/2}) + sqbar (1/2 d^{-1/2}),
// sbar_total = sbar + sray + sum_{e at a} cbar_e w_e s_other
__global__ void k_fg_node(Grid3 G, const float* __restrict__ sbar, const float* __restrict__ sray,
                          const float* __restrict__ sqbar, const float* __restrict__ cbar,
                          const float* __restrict__ w, const float* __restrict__ s,
                          float* __restrict__ dbar) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= G.N) return;
  float acc = sbar[i] + sray[i];
  for_each_nbr(G, i, [&](int64_t j, int64_t e) { acc = fmaf(cbar[e] * w[e], s[j], acc); });
  const float si = s[i];  // s^3 = d^{-3/2}
  dbar[i] = acc * (-0.5f * si * si * si) + sqbar[i] * (0.5f * si);
}

// gw_e = wray_e + cbar_e s_a s_b + dbar_a + dbar_b; beta partials (FP64)
__global__ void __launch_bounds__(256)
k_fg_edge(Grid3 G, const float* __restrict__ wray, const float* __restrict__ cbar,
          const float* __restrict__ dbar, const float* __restrict__ s,
          const float* __restrict__ J, const float* __restrict__ w, int form,
          float* __restrict__ gw, double* __restrict__ part) {
  double accb = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < G.N;
       i += (int64_t)gridDim.x * blockDim.x) {
    int c[3];
    G.coords(i, c);
    for (int a = 0; a < G.ndim; ++a) {
      const int64_t e = a * G.N + i;
      if (c[a] + 1 >= G.extent(a)) { gw[e] = 0.f; continue; }
      const int64_t j = i + G.stride(a);
      const float g = wray[e] + cbar[e] * s[i] * s[j] + dbar[i] + dbar[j];
      gw[e] = g;
      if (J) {
        const float dJ = J[i] - J[j];
        const float dwdb = form == RW_WEIGHT_SQ ? -(dJ * dJ) * w[e] : -fabsf(dJ) * w[e];
        accb += (double)g * (double)dwdb;
      }
    }
  }
  __shared__ double red[256];
  red[threadIdx.x] = accb;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void k_sum_part(const double* __restrict__ part, int n, double* __restrict__ out) {
  __shared__ double red[256];
  double a = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) a += part[i];
  red[threadIdx.x] = a;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = red[0];
}

__global__ void k_qn2(const float* __restrict__ Q, int64_t ldq, int64_t N, int m,
                      double* __restrict__ out) {
  // one block per column: sum of squares in FP64, fixed order
  const int c = blockIdx.x;
  __shared__ double red[256];
  double a = 0.0;
  for (int64_t i = threadIdx.x; i < N; i += blockDim.x) {
    const double v = Q[i * ldq + c];
    a += v * v;
  }
  red[threadIdx.x] = a;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[c] = red[0];
}

// bump allocator over one device buffer
struct Arena {
  char* base;
  size_t off = 0;
  template <class T> T* take(size_t n) {
    T* p = reinterpret_cast<T*>(base + off);
    off += (sizeof(T) * n + 255) & ~size_t(255);
    return p;
  }
};

}  // namespace

extern "C" rw_status rw_grad_fast(const rw_graph* g, const rw_basis* b,
                                  const int32_t* seed_idx_dev, const int32_t* seed_lab_dev,
                                  int32_t S, int32_t n_labels, const float* priors_dev,
                                  double gamma, int32_t m, int32_t refine_steps, double omega,
                                  const float* dloss_dU_dev, float* U_out_dev, float* grad_w_dev,
                                  double* grad_beta_host, void* stream) {
  if (!g || !b || !seed_idx_dev || !seed_lab_dev || !priors_dev || !dloss_dU_dev || !grad_w_dev)
    return RW_ERR_INVALID_ARG;
  if (b->N != g->N) return RW_ERR_INVALID_ARG;
  if (S < 1 || S > 65536 || n_labels < 1 || n_labels > RW_MAX_LABELS) return RW_ERR_INVALID_ARG;
  if (m < 1 || m > b->m || m > 1024) return RW_ERR_INVALID_ARG;
  if (refine_steps < 0 || refine_steps > 1000) return RW_ERR_INVALID_ARG;
  if (!(omega > 0.0 && omega <= 1.0)) return RW_ERR_INVALID_ARG;
  if (!(gamma > 0.0)) return gamma == 0.0 ? RW_ERR_UNSUPPORTED : RW_ERR_INVALID_ARG;
  if (g->kind != RW_GRAPH_GRID || !g->normalized) {
    rw_set_error_message("rw_grad_fast: normalized grid graphs only");
    return RW_ERR_UNSUPPORTED;
  }
  if (grad_beta_host && !g->J) return RW_ERR_INVALID_ARG;
  cudaStream_t st = rw_stream(stream);
  rw_graph* gm = const_cast<rw_graph*>(g);
  const int L = n_labels;
  const int lp = L <= 4 ? 4 : (L <= 8 ? 8 : 16);
  const int64_t N = g->N;
  const int ldx = (int)rw_round_up(m, 4);
  const int K = refine_steps;
  Grid3 G{g->ndim, g->dims[0], g->dims[1], g->dims[2], N};
  const float gf = (float)gamma, om = (float)omega, aa = (float)(omega / (1.0 + gamma));
  float* phat;
  int* seedlab;
  RW_TRY(rw_solve_priors_internal(g, seed_idx_dev, seed_lab_dev, S, L, 1, priors_dev, lp, st,
                                  &phat, &seedlab, nullptr));
  // scratch
  const size_t Nl = (size_t)N * lp, E = (size_t)g->ndim * N;
  size_t need = 0;
  {
    auto r = [](size_t bytes) { return (bytes + 255) & ~size_t(255); };
    need += r(sizeof(int) * N);                                   // pos
    need += 2 * r(sizeof(float) * (size_t)S * ldx);               // Qs, X
    need += 7 * r(sizeof(float) * (size_t)S * lp);                // Ush LsUs XlgZ rhs Fs rbar Fsbar
    need += r(sizeof(double) * (size_t)m * m) + r(sizeof(int) * (m + 2));  // K, piv + flag
    need += 7 * r(sizeof(double) * (size_t)m * lp);               // Z t1 C Cbar t2 t3 qn2
    need += 6 * r(sizeof(float) * (size_t)m * lp) + r(sizeof(float) * m) +
            r(sizeof(double) * m);                                // FP32 copies, coef, lgbar
    need += (size_t)(K + 1) * r(sizeof(float) * Nl);              // x_0..x_K
    need += 6 * r(sizeof(float) * Nl);                            // phn, b, xbar x2, bbar, QZbar
    need += 2 * r(sizeof(float) * E);                             // cbar, wray
    need += 4 * r(sizeof(float) * N);                             // sbar, sray, sqbar, dbar
    need += r(sizeof(double) * (kBetaBlocks + 8));
  }
  RW_TRY(gm->ws.grad.grow(need));
  Arena ar{gm->ws.grad.as<char>()};
  int* pos = ar.take<int>(N);
  float* Qs = ar.take<float>((size_t)S * ldx);
  float* X = ar.take<float>((size_t)S * ldx);
  float* Ush = ar.take<float>((size_t)S * lp);
  float* LsUs = ar.take<float>((size_t)S * lp);
  float* XlgZ = ar.take<float>((size_t)S * lp);
  float* rhs = ar.take<float>((size_t)S * lp);
  float* Fs = ar.take<float>((size_t)S * lp);
  float* rbar = ar.take<float>((size_t)S * lp);
  float* Fsbar = ar.take<float>((size_t)S * lp);
  double* Km = ar.take<double>((size_t)m * m);
  int* piv = ar.take<int>(m + 2);
  int* bad = piv + m;
  double* Z = ar.take<double>((size_t)m * lp);
  double* t1 = ar.take<double>((size_t)m * lp);   // becomes y
  double* C64 = ar.take<double>((size_t)m * lp);
  double* Cbar = ar.take<double>((size_t)m * lp);
  double* t2 = ar.take<double>((size_t)m * lp);   // becomes v = K^{-T} X^T Fsbar
  double* t3 = ar.take<double>((size_t)m * lp);
  double* qn2 = ar.take<double>((size_t)m * lp);   // m used
  float* lgZ = ar.take<float>((size_t)m * lp);
  float* C32 = ar.take<float>((size_t)m * lp);
  float* y32 = ar.take<float>((size_t)m * lp);
  float* Ybar32 = ar.take<float>((size_t)m * lp);
  float* v32 = ar.take<float>((size_t)m * lp);
  float* Zbar32 = ar.take<float>((size_t)m * lp);
  float* coef = ar.take<float>(m);
  double* lgbar = ar.take<double>(m);
  std::vector<float*> xs(K + 1);
  for (int t = 0; t <= K; ++t) xs[t] = ar.take<float>(Nl);
  float* phn = ar.take<float>(Nl);
  float* bv = ar.take<float>(Nl);
  float* xb0 = ar.take<float>(Nl);
  float* xb1 = ar.take<float>(Nl);
  float* bbar = ar.take<float>(Nl);
  float* QZbar = ar.take<float>(Nl);
  float* cbar = ar.take<float>(E);
  float* wray = ar.take<float>(E);
  float* sbar = ar.take<float>(N);
  float* sray = ar.take<float>(N);
  float* sqbar = ar.take<float>(N);
  float* dbar = ar.take<float>(N);
  double* part = ar.take<double>(kBetaBlocks + 8);
  double* gbeta_dev = part + kBetaBlocks;
  const double* lam = b->lam;
  const float* Q = b->Q32;
  const int64_t ldq = b->ld32;
  const unsigned TB = 256;

  // ---- forward ----
  k_fill<<<rw_blocks(N, TB), TB, 0, st>>>(pos, N, -1);
  RW_LAUNCH_CHECK();
  k_posmap<<<rw_blocks(S, TB), TB, 0, st>>>(seed_idx_dev, S, pos);
  RW_LAUNCH_CHECK();
  k_fg_seed_rows<<<rw_blocks((int64_t)S * 32, TB), TB, 0, st>>>(
      G, seed_idx_dev, seedlab, g->cw, g->sq, Q, ldq, m, S, lp, Qs, X, ldx, Ush, LsUs);
  RW_LAUNCH_CHECK();
  k_mask_rows<<<rw_blocks(Nl, TB), TB, 0, st>>>(phat, seedlab, N, lp, phn);
  RW_LAUNCH_CHECK();
  RW_TRY(rw_gram(Q, ldq, phn, lp, N, m, lp, Z, lp, false, st));          // Z = Q_n^T P-hat_n
  RW_TRY(rw_gram(Qs, ldx, X, ldx, S, m, m, Km, m, false, st));           // Q_s^T X
  k_fg_K<<<rw_blocks((int64_t)m * std::max(m, lp), TB), TB, 0, st>>>(Km, m, lam, gamma, Z, lp, lgZ);
  RW_LAUNCH_CHECK();
  RW_TRY(rw_gemm_tall(X, ldx, lgZ, lp, S, m, lp, 1.f, 0.f, XlgZ, lp, st));
  k_fg_rhs<<<rw_blocks((int64_t)S * lp, TB), TB, 0, st>>>(LsUs, Ush, XlgZ, S * lp, gf, rhs);
  RW_LAUNCH_CHECK();
  RW_TRY(rw_gram(Qs, ldx, rhs, lp, S, m, lp, t1, lp, false, st));        // Q_s^T rhs
  RW_CHECK_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), st));
  k_lu64<<<1, 256, 0, st>>>(Km, m, piv, bad);
  RW_LAUNCH_CHECK();
  k_lu64_solve<<<1, 32, 0, st>>>(Km, m, piv, t1, lp, lp, 0);             // y = K^{-1} Q_s^T rhs
  RW_LAUNCH_CHECK();
  k_fg_C<<<rw_blocks((int64_t)m * lp, TB), TB, 0, st>>>(t1, Z, lam, gamma, m, lp, C64, C32, y32);
  RW_LAUNCH_CHECK();
  RW_CHECK_CUDA(cudaMemcpyAsync(Fs, rhs, sizeof(float) * S * lp, cudaMemcpyDeviceToDevice, st));
  RW_TRY(rw_gemm_tall(X, ldx, y32, lp, S, m, lp, 1.f, 1.f, Fs, lp, st));  // F_s = rhs + X y
  RW_TRY(rw_gemm_tall(Q, ldq, C32, lp, N, m, lp, 1.f, 0.f, xs[0], lp, st));  // x_0 = Q C
  k_zero_seeded<<<rw_blocks(Nl, TB), TB, 0, st>>>(xs[0], seedlab, N, lp);
  RW_LAUNCH_CHECK();
  k_fg_b<<<rw_blocks(N, TB), TB, 0, st>>>(G, phat, seedlab, g->cw, g->sq, lp, gf, bv);
  RW_LAUNCH_CHECK();
  for (int t = 0; t < K; ++t) {
    k_fg_jacobi<<<rw_blocks(N, TB), TB, 0, st>>>(G, xs[t], bv, seedlab, g->cw, lp, om, aa, xs[t + 1]);
    RW_LAUNCH_CHECK();
  }
  if (U_out_dev) {
    k_fg_U<<<rw_blocks((int64_t)N * L, TB), TB, 0, st>>>(xs[K], seedlab, g->s, N, L, lp, U_out_dev);
    RW_LAUNCH_CHECK();
  }

  // ---- reverse ----
  RW_CHECK_CUDA(cudaMemsetAsync(cbar, 0, sizeof(float) * E, st));
  RW_CHECK_CUDA(cudaMemsetAsync(bbar, 0, sizeof(float) * Nl, st));
  k_fg_out_rev<<<rw_blocks(N, TB), TB, 0, st>>>(dloss_dU_dev, xs[K], seedlab, g->s, N, L, lp, xb0, sbar);
  RW_LAUNCH_CHECK();
  float* xb = xb0;
  float* xo = xb1;
  for (int t = K; t >= 1; --t) {
    k_fg_jacobi_rev<<<rw_blocks(N, TB), TB, 0, st>>>(G, xb, xs[t - 1], seedlab, g->cw, lp, om,
                                                      aa, xo, bbar, cbar);
    RW_LAUNCH_CHECK();
    std::swap(xb, xo);
  }
  RW_TRY(rw_gram(Q, ldq, xb, lp, N, m, lp, Cbar, lp, false, st));       // C-bar = Q_n^T x-bar_0
  k_fg_small1<<<rw_blocks(m, 128), 128, 0, st>>>(Cbar, C64, lam, gamma, m, lp, Ybar32, lgbar);
  RW_LAUNCH_CHECK();
  RW_TRY(rw_gemm_tall(Qs, ldx, Ybar32, lp, S, m, lp, 1.f, 0.f, Fsbar, lp, st));  // F_s-bar
  RW_TRY(rw_gram(X, ldx, Fsbar, lp, S, m, lp, t2, lp, false, st));       // X^T F_s-bar
  k_lu64_solve<<<1, 32, 0, st>>>(Km, m, piv, t2, lp, lp, 1);             // K^{-T}
  RW_LAUNCH_CHECK();
  k_f64_to_f32_n<<<rw_blocks((int64_t)m * lp, TB), TB, 0, st>>>(t2, v32, m * lp);
  RW_LAUNCH_CHECK();
  RW_CHECK_CUDA(cudaMemcpyAsync(rbar, Fsbar, sizeof(float) * S * lp, cudaMemcpyDeviceToDevice, st));
  RW_TRY(rw_gemm_tall(Qs, ldx, v32, lp, S, m, lp, 1.f, 1.f, rbar, lp, st));     // rhs-bar
  RW_TRY(rw_gram(X, ldx, rbar, lp, S, m, lp, t3, lp, false, st));        // X^T rhs-bar
  k_qn2<<<m, 256, 0, st>>>(Q, ldq, N, m, qn2);
  RW_LAUNCH_CHECK();
  k_fg_small2<<<rw_blocks(m, 128), 128, 0, st>>>(t3, t1, Z, Ybar32, lam, qn2, gamma, m, lp,
                                                 lgbar, Zbar32, coef);
  RW_LAUNCH_CHECK();
  RW_TRY(rw_gemm_tall(Q, ldq, Zbar32, lp, N, m, lp, 1.f, 0.f, QZbar, lp, st));  // Q Z-bar
  k_fg_sqbar_free<<<rw_blocks(N, TB), TB, 0, st>>>(QZbar, bbar, priors_dev, seedlab, N, L, lp, gf, sqbar);
  RW_LAUNCH_CHECK();
  k_fg_seed_rev<<<rw_blocks(S, TB), TB, 0, st>>>(G, seed_idx_dev, seedlab, pos, g->cw, rbar, bbar,
                                                 S, lp, gf, sqbar);
  RW_LAUNCH_CHECK();
  k_fg_cbar_seed<<<rw_blocks(N, TB), TB, 0, st>>>(G, seedlab, pos, g->sq, bbar, xs[0], rbar, lp, cbar);
  RW_LAUNCH_CHECK();
  k_fg_rayleigh_rev<<<rw_blocks(N * 32, TB), TB, 0, st>>>(G, Q, ldq, m, g->w, g->s, coef, sray, wray);
  RW_LAUNCH_CHECK();
  k_fg_node<<<rw_blocks(N, TB), TB, 0, st>>>(G, sbar, sray, sqbar, cbar, g->w, g->s, dbar);
  RW_LAUNCH_CHECK();
  k_fg_edge<<<kBetaBlocks, 256, 0, st>>>(G, wray, cbar, dbar, g->s, g->J, g->w, g->form,
                                         grad_w_dev, part);
  RW_LAUNCH_CHECK();
  k_sum_part<<<1, 256, 0, st>>>(part, kBetaBlocks, gbeta_dev);
  RW_LAUNCH_CHECK();
  int badh = 0;
  double gb = 0.0;
  RW_CHECK_CUDA(cudaMemcpyAsync(&badh, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
  RW_CHECK_CUDA(cudaMemcpyAsync(&gb, gbeta_dev, sizeof(double), cudaMemcpyDeviceToHost, st));
  RW_CHECK_CUDA(cudaStreamSynchronize(st));
  rw_status ds = rw_last_device_status(g, stream);
  if (ds != RW_OK) return ds;
  if (badh) return RW_ERR_SINGULAR;
  if (grad_beta_host) *grad_beta_host = gb;
  return RW_OK;
}
