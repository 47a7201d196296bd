// Aggregated image graphs (Sec. III-C): super-vertex basis and graph.
//
// A projection function eta (N x N-bar, rows sum to 1) and an aggregation function eta-bar
// (N x N-bar on eta's pattern, columns sum to 1; eta with normalized columns if absent) carry
// each stored column q to the super-vertices, naively, Eq. (q_agg_1), q-bar_y =
// sum_x eta-bar(x, y) q_x, or weighted by the local change of eta, Eq. (q_agg_2),
//   Delta(x) = sum_{x' ~ x, w > 0} sum_y |eta(x, y) - eta(x', y)|,
//   q-bar_y  = sum_x Delta(x) eta-bar(x, y) q_x.
// The aggregated columns are made orthonormal by classical Gram-Schmidt with one
// re-orthogonalization pass, in column order, in FP64; a column whose norm after projection is
// below 1e-10 of its norm before is dropped.  The aggregate graph is the Galerkin product
// L-bar = eta^T L eta (L-bar 1 = 0 because the rows of eta sum to 1), stored as a CSR weight
// matrix W-bar = -offdiag(L-bar), i.e. W-bar_yz = -sum_e w_e delta_e(y) delta_e(z) with
// delta_e = eta_a - eta_b for the edge e = (a, b); its degrees are the row sums.  The new values
// are the Rayleigh quotients (Eq. z_ray) of the new columns on the new graph.
//
// Every reduction has a fixed order (one thread or one block per output), so the result does
// not depend on scheduling.
#include "rw_internal.cuh"

#include <algorithm>
#include <vector>

rw_status rw_make_basis(const rw_graph* g, int m, const float* X, int64_t ldx,
                        const double* lam_h, cudaStream_t st, rw_basis** out);

namespace {

constexpr int kMaxAggNbrs = 64;        // distinct neighbouring super-vertices per super-vertex
constexpr int kMaxColLen = 1 << 16;    // voxels per super-vertex (column of eta)
constexpr double kDropTol = 1e-10;     // Gram-Schmidt: drop when |v_after| < tol |v_before|

enum { AGG_BAD_ETA = 1, AGG_TOO_MANY_NBRS = 2, AGG_COL_TOO_LONG = 4, AGG_ISOLATED = 8 };

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

// every neighbour x' of x joined by an edge of positive weight: fn(x', w)
template <class F>
__device__ __forceinline__ void for_each_live_nbr(const Grid3& G, const float* __restrict__ w,
                                                  int64_t x, F fn) {
  int c[3];
  G.coords(x, c);
  for (int a = 0; a < G.ndim; ++a) {
    const int64_t st = G.stride(a);
    if (c[a] > 0) {
      const float we = w[a * G.N + x - st];
      if (we > 0.f) fn(x - st, we);
    }
    if (c[a] + 1 < G.extent(a)) {
      const float we = w[a * G.N + x];
      if (we > 0.f) fn(x + st, we);
    }
  }
}

// eta(x, y) by binary search in the sorted row x; *stored tells whether (x, y) is an entry of
// eta's pattern (an explicitly stored 0 counts as stored)
__device__ __forceinline__ float eta_at(const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                                        const float* __restrict__ val, int64_t x, int y,
                                        bool* stored) {
  int lo = rp[x], hi = rp[x + 1];
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    const int c = col[mid];
    if (c == y) { *stored = true; return val[mid]; }
    if (c < y) lo = mid + 1; else hi = mid;
  }
  *stored = false;
  return 0.f;
}

// rows: non-decreasing row pointers, columns in range and strictly increasing, values finite
// and >= 0 (eta and eta-bar), row sums of eta within 1e-3 of 1
__global__ void k_eta_check(const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                            const float* __restrict__ val, const float* __restrict__ vbar,
                            int64_t N, int64_t nnz, int nbar, int* __restrict__ flag) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= N) return;
  const int p0 = rp[x], p1 = rp[x + 1];
  // every row pointer inside [0, nnz] before any entry is read
  if (p0 < 0 || p1 < p0 || p1 > nnz || (x == 0 && p0 != 0)) { atomicOr(flag, AGG_BAD_ETA); return; }
  double sum = 0.0;
  int prev = -1;
  for (int p = p0; p < p1; ++p) {
    const int c = col[p];
    const float v = val[p];
    if (c <= prev || c >= nbar || !(v >= 0.f) || !isfinite(v)) { atomicOr(flag, AGG_BAD_ETA); return; }
    if (vbar && (!(vbar[p] >= 0.f) || !isfinite(vbar[p]))) { atomicOr(flag, AGG_BAD_ETA); return; }
    prev = c;
    sum += v;
  }
  if (fabs(sum - 1.0) > 1e-3) atomicOr(flag, AGG_BAD_ETA);
}

__global__ void k_count_cols(const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                             int64_t N, int* __restrict__ cnt) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= N) return;
  for (int p = rp[x]; p < rp[x + 1]; ++p) atomicAdd(&cnt[col[p]], 1);
}

// exclusive prefix sum of n counts into out[0..n] by one CTA (chunks of 1024 with a carry)
__global__ void __launch_bounds__(1024) k_scan(const int* __restrict__ in, int64_t n,
                                               int* __restrict__ out) {
  __shared__ int buf[1024];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < n; base += 1024) {
    const int64_t i = base + threadIdx.x;
    const int v = i < n ? in[i] : 0;
    buf[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
      const int t = threadIdx.x >= o ? buf[threadIdx.x - o] : 0;
      __syncthreads();
      buf[threadIdx.x] += t;
      __syncthreads();
    }
    if (i < n) out[i] = carry + buf[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry += buf[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[n] = carry;
}

// scatter the CSR positions into columns (order within a column fixed afterwards)
__global__ void k_fill_cols(const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                            int64_t N, const int* __restrict__ cp, int* __restrict__ fill,
                            int* __restrict__ tpos) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= N) return;
  for (int p = rp[x]; p < rp[x + 1]; ++p) {
    const int y = col[p];
    tpos[cp[y] + atomicAdd(&fill[y], 1)] = p;
  }
}

// sort each column's CSR positions ascending (= ascending voxel index); insertion sort, the
// scatter leaves the runs nearly sorted.  Also the column sums of eta (FP64, fixed order).
__global__ void k_sort_cols(const int* __restrict__ cp, int nbar, int* __restrict__ tpos,
                            const float* __restrict__ val, double* __restrict__ colsum,
                            int* __restrict__ flag) {
  const int y = blockIdx.x * blockDim.x + threadIdx.x;
  if (y >= nbar) return;
  const int a = cp[y], b = cp[y + 1];
  if (b - a > kMaxColLen) { atomicOr(flag, AGG_COL_TOO_LONG); return; }
  for (int i = a + 1; i < b; ++i) {
    const int key = tpos[i];
    int j = i - 1;
    while (j >= a && tpos[j] > key) { tpos[j + 1] = tpos[j]; --j; }
    tpos[j + 1] = key;
  }
  double s = 0.0;
  for (int i = a; i < b; ++i) s += val[tpos[i]];
  colsum[y] = s;
}

// eta-bar values on eta's pattern: given, or eta / column sum
__global__ void k_etabar(const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                         const float* __restrict__ val, const float* __restrict__ vbar_in,
                         const double* __restrict__ colsum, int64_t N, double* __restrict__ vbar) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= N) return;
  for (int p = rp[x]; p < rp[x + 1]; ++p)
    vbar[p] = vbar_in ? (double)vbar_in[p] : (double)val[p] / colsum[col[p]];
}

// Delta(x) of Eq. (q_agg_2): L1 distance of the sorted rows x and x' over the live neighbours
__global__ void k_delta(Grid3 G, const float* __restrict__ w, const int32_t* __restrict__ rp,
                        const int32_t* __restrict__ col, const float* __restrict__ val,
                        double* __restrict__ delta) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= G.N) return;
  double acc = 0.0;
  for_each_live_nbr(G, w, x, [&](int64_t xp, float) {
    int p = rp[x], q = rp[xp];
    const int pe = rp[x + 1], qe = rp[xp + 1];
    while (p < pe || q < qe) {
      const int cp_ = p < pe ? col[p] : INT32_MAX, cq = q < qe ? col[q] : INT32_MAX;
      if (cp_ == cq) { acc += fabs((double)val[p] - (double)val[q]); ++p; ++q; }
      else if (cp_ < cq) { acc += fabs((double)val[p]); ++p; }
      else { acc += fabs((double)val[q]); ++q; }
    }
  });
  delta[x] = acc;
}

// one warp per super-vertex y: A[c * ldA + y] = sum_{x in column y} eta-bar(x, y) [Delta(x)] q_x[c]
__global__ void k_agg_cols(const int* __restrict__ cp, const int* __restrict__ tpos,
                           const double* __restrict__ vbar, const double* __restrict__ delta,
                           const int* __restrict__ rowof, const float* __restrict__ Q,
                           int64_t ldq, int m, int nbar, int64_t ldA, double* __restrict__ A) {
  const int y = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (y >= nbar) return;
  for (int c0 = 0; c0 < m; c0 += 32) {
    const int c = c0 + lane;
    double acc = 0.0;
    for (int t = cp[y]; t < cp[y + 1]; ++t) {
      const int p = tpos[t];
      const int64_t x = rowof[p];
      const double f = delta ? vbar[p] * delta[x] : vbar[p];
      if (c < m) acc += f * (double)Q[x * ldq + c];
    }
    if (c < m) A[(int64_t)c * ldA + y] = acc;
  }
}

// row index of every CSR position
__global__ void k_rowof(const int32_t* __restrict__ rp, int64_t N, int* __restrict__ rowof) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= N) return;
  for (int p = rp[x]; p < rp[x + 1]; ++p) rowof[p] = (int)x;
}

// ---- classical Gram-Schmidt with re-orthogonalization, FP64, column-major (ld = n) ----------
__device__ double block_sum(double v, double* red) {
  red[threadIdx.x] = v;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  const double r = red[0];
  __syncthreads();
  return r;
}

// out = ||v||
__global__ void __launch_bounds__(256) k_norm(const double* __restrict__ v, int64_t n,
                                              double* __restrict__ out) {
  __shared__ double red[256];
  double a = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) a += v[i] * v[i];
  a = block_sum(a, red);
  if (threadIdx.x == 0) *out = sqrt(a);
}

// block i < kept: c[i] = Qb[:, i] . v
__global__ void __launch_bounds__(256) k_cgs_dots(const double* __restrict__ Qb, int64_t n,
                                                  const double* __restrict__ v,
                                                  const int* __restrict__ kept,
                                                  double* __restrict__ c) {
  __shared__ double red[256];
  const int i = blockIdx.x;
  if (i >= *kept) return;
  const double* q = Qb + (int64_t)i * n;
  double a = 0.0;
  for (int64_t r = threadIdx.x; r < n; r += blockDim.x) a += q[r] * v[r];
  a = block_sum(a, red);
  if (threadIdx.x == 0) c[i] = a;
}

// v -= Qb[:, :kept] c
__global__ void k_cgs_axpy(const double* __restrict__ Qb, int64_t n, const double* __restrict__ c,
                           const int* __restrict__ kept, double* __restrict__ v) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const int k = *kept;
  double s = v[r];
  for (int i = 0; i < k; ++i) s -= Qb[(int64_t)i * n + r] * c[i];
  v[r] = s;
}

// keep the column if |v| >= tol |v before|: Qb[:, kept] = v / |v|
__global__ void k_cgs_store(const double* __restrict__ v, int64_t n, const double* __restrict__ nrm,
                            const int* __restrict__ kept, double* __restrict__ Qb) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const double n0 = nrm[0], nv = nrm[1];
  if (!(n0 > 0.0) || !(nv >= kDropTol * n0)) return;
  Qb[(int64_t)(*kept) * n + r] = v[r] / nv;
}

__global__ void k_cgs_commit(const double* __restrict__ nrm, int j, int* __restrict__ kept,
                             int* __restrict__ kept_idx) {
  const double n0 = nrm[0], nv = nrm[1];
  if (n0 > 0.0 && nv >= kDropTol * n0) {
    kept_idx[*kept] = j;
    *kept += 1;
  }
}

// ---- Galerkin graph W-bar_yz = -sum_e w_e delta_e(y) delta_e(z), y != z --------------------
struct Row {
  int n = 0;
  int z[kMaxAggNbrs];
  double v[kMaxAggNbrs];
  __device__ bool add(int zz, double vv) {
    int lo = 0, hi = n;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (z[mid] < zz) lo = mid + 1; else hi = mid;
    }
    if (lo < n && z[lo] == zz) { v[lo] += vv; return true; }
    if (n == kMaxAggNbrs) return false;
    for (int t = n; t > lo; --t) { z[t] = z[t - 1]; v[t] = v[t - 1]; }
    z[lo] = zz;
    v[lo] = vv;
    ++n;
    return true;
  }
};

// Every edge (x, x') with x in column y and delta(y) != 0, visited once (from the smaller end
// when both ends are in column y): the contributions -w delta(y) delta(z) for z != y.
__device__ bool wbar_row(const Grid3& G, const float* __restrict__ w, const int32_t* __restrict__ rp,
                         const int32_t* __restrict__ col, const float* __restrict__ val,
                         const int* __restrict__ cp, const int* __restrict__ tpos,
                         const int* __restrict__ rowof, int y, Row& row) {
  bool ok = true;
  for (int t = cp[y]; t < cp[y + 1] && ok; ++t) {
    const int p0 = tpos[t];
    const int64_t x = rowof[p0];
    const float exy = val[p0];
    for_each_live_nbr(G, w, x, [&](int64_t xp, float we) {
      if (!ok) return;
      bool in_y = false;
      const float epy = eta_at(rp, col, val, xp, y, &in_y);
      if (in_y && xp < x) return;  // counted from xp
      const double dy = (double)exy - (double)epy;
      if (dy == 0.0) return;
      int p = rp[x], q = rp[xp];
      const int pe = rp[x + 1], qe = rp[xp + 1];
      while (p < pe || q < qe) {
        const int cp_ = p < pe ? col[p] : INT32_MAX, cq = q < qe ? col[q] : INT32_MAX;
        int z;
        double dz;
        if (cp_ == cq) { z = cp_; dz = (double)val[p] - (double)val[q]; ++p; ++q; }
        else if (cp_ < cq) { z = cp_; dz = val[p]; ++p; }
        else { z = cq; dz = -(double)val[q]; ++q; }
        if (z != y && dz != 0.0 && !row.add(z, -(double)we * dy * dz)) { ok = false; return; }
      }
    });
  }
  return ok;
}

__global__ void k_wbar_count(Grid3 G, const float* __restrict__ w, const int32_t* __restrict__ rp,
                             const int32_t* __restrict__ col, const float* __restrict__ val,
                             const int* __restrict__ cp, const int* __restrict__ tpos,
                             const int* __restrict__ rowof, int nbar, int* __restrict__ cnt,
                             int* __restrict__ flag) {
  const int y = blockIdx.x * blockDim.x + threadIdx.x;
  if (y >= nbar) return;
  Row row;
  if (!wbar_row(G, w, rp, col, val, cp, tpos, rowof, y, row)) {
    atomicOr(flag, AGG_TOO_MANY_NBRS);
    cnt[y] = 0;
    return;
  }
  int k = 0;
  for (int t = 0; t < row.n; ++t) k += row.v[t] != 0.0;
  cnt[y] = k;
}

__global__ void k_wbar_fill(Grid3 G, const float* __restrict__ w, const int32_t* __restrict__ rp,
                            const int32_t* __restrict__ col, const float* __restrict__ val,
                            const int* __restrict__ cp, const int* __restrict__ tpos,
                            const int* __restrict__ rowof, int nbar, const int32_t* __restrict__ orp,
                            int32_t* __restrict__ ocol, float* __restrict__ ow,
                            float* __restrict__ od) {
  const int y = blockIdx.x * blockDim.x + threadIdx.x;
  if (y >= nbar) return;
  Row row;
  wbar_row(G, w, rp, col, val, cp, tpos, rowof, y, row);
  int o = orp[y];
  double dsum = 0.0;
  for (int t = 0; t < row.n; ++t) {
    if (row.v[t] == 0.0) continue;
    ocol[o] = row.z[t];
    ow[o] = (float)row.v[t];
    dsum += row.v[t];
    ++o;
  }
  od[y] = (float)dsum;
}

// scalings and operator coefficients of a CSR graph
__global__ void k_csr_scalings(const float* __restrict__ d, int64_t n, int normalized,
                               float* __restrict__ s, float* __restrict__ sq, int* __restrict__ flag) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (!normalized) { s[i] = 1.f; sq[i] = 1.f; return; }
  const float di = d[i];
  if (!(di > 0.f)) { atomicOr(flag, AGG_ISOLATED); s[i] = 0.f; sq[i] = 0.f; return; }
  const float r = sqrtf(di);
  sq[i] = r;
  s[i] = 1.f / r;
}

__global__ void k_csr_coeffs(const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                             const float* __restrict__ wv, const float* __restrict__ s, int64_t n,
                             int normalized, float* __restrict__ cv) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int p = rp[i]; p < rp[i + 1]; ++p) cv[p] = normalized ? wv[p] * s[i] * s[col[p]] : wv[p];
}

// FP64 column-major (ld = n) -> FP32 row-major (ld = k)
__global__ void k_colmajor_to_rows(const double* __restrict__ A, int64_t n, int k,
                                   float* __restrict__ X) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * k) return;
  const int64_t r = e / k;
  const int c = (int)(e % k);
  X[e] = (float)A[(int64_t)c * n + r];
}

struct Tmp {
  std::vector<void*> ptrs;
  ~Tmp() { for (void* p : ptrs) cudaFree(p); }
  template <class T> T* get(size_t n) {
    void* p = nullptr;
    if (cudaMalloc(&p, std::max<size_t>(sizeof(T) * n, 16)) != cudaSuccess) return nullptr;
    ptrs.push_back(p);
    return reinterpret_cast<T*>(p);
  }
};

rw_status agg_flag_status(int bits) {
  if (bits & AGG_BAD_ETA) {
    rw_set_error_message("aggregate: eta must have sorted in-range columns, finite values >= 0 "
                         "and rows summing to 1");
    return RW_ERR_INVALID_ARG;
  }
  if (bits & AGG_COL_TOO_LONG) {
    rw_set_error_message("aggregate: a super-vertex holds more than 65536 voxels");
    return RW_ERR_UNSUPPORTED;
  }
  if (bits & AGG_TOO_MANY_NBRS) {
    rw_set_error_message("aggregate: a super-vertex has more than 64 neighbouring super-vertices");
    return RW_ERR_UNSUPPORTED;
  }
  if (bits & AGG_ISOLATED) return RW_ERR_ISOLATED_NODE;
  return RW_OK;
}

}  // namespace

rw_status rw_aggregate(rw_graph* g, rw_basis* b, const rw_topology_update* u, cudaStream_t st,
                       rw_graph** gout, rw_basis** bout) {
  *gout = nullptr;
  *bout = nullptr;
  if (g->kind != RW_GRAPH_GRID) {
    rw_set_error_message("aggregate: the source graph must be an image grid");
    return RW_ERR_UNSUPPORTED;
  }
  if (b->N != g->N || u->n_bar < 1 || u->n_bar > g->N || !u->eta_rowptr_dev || !u->eta_col_dev ||
      !u->eta_val_dev)
    return RW_ERR_INVALID_ARG;
  const int64_t N = g->N;
  const int nbar = (int)u->n_bar;
  const int m = b->m;
  const int32_t* rp = u->eta_rowptr_dev;
  const int32_t* col = u->eta_col_dev;
  const float* val = u->eta_val_dev;
  const float* vbar_in = u->etabar_val_dev;
  Grid3 G{g->ndim, g->dims[0], g->dims[1], g->dims[2], N};
  const unsigned TB = 256;
  Tmp tmp;
  int* flag = tmp.get<int>(4);
  if (!flag) return RW_ERR_OOM;
  int32_t ends[2] = {0, 0};
  RW_CHECK_CUDA(cudaMemcpyAsync(&ends[0], rp, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  RW_CHECK_CUDA(cudaMemcpyAsync(&ends[1], rp + N, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  RW_CHECK_CUDA(cudaMemsetAsync(flag, 0, sizeof(int) * 4, st));
  RW_CHECK_CUDA(cudaStreamSynchronize(st));
  if (ends[0] != 0 || ends[1] < N) return RW_ERR_INVALID_ARG;  // every row has an entry
  const int64_t nnz = ends[1];
  k_eta_check<<<rw_blocks(N, TB), TB, 0, st>>>(rp, col, val, vbar_in, N, nnz, nbar, flag);
  RW_LAUNCH_CHECK();
  int bits = 0;
  RW_CHECK_CUDA(cudaMemcpyAsync(&bits, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  RW_CHECK_CUDA(cudaStreamSynchronize(st));
  RW_TRY(agg_flag_status(bits));

  // transpose of eta (column -> sorted CSR positions)
  int* cnt = tmp.get<int>(nbar + 1);
  int* cp = tmp.get<int>(nbar + 1);
  int* fill = tmp.get<int>(nbar + 1);
  int* tpos = tmp.get<int>(nnz);
  int* rowof = tmp.get<int>(nnz);
  double* colsum = tmp.get<double>(nbar);
  double* vbar = tmp.get<double>(nnz);
  double* delta = tmp.get<double>(N);
  if (!cnt || !cp || !fill || !tpos || !rowof || !colsum || !vbar || !delta) return RW_ERR_OOM;
  RW_CHECK_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * (nbar + 1), st));
  RW_CHECK_CUDA(cudaMemsetAsync(fill, 0, sizeof(int) * (nbar + 1), st));
  k_count_cols<<<rw_blocks(N, TB), TB, 0, st>>>(rp, col, N, cnt);
  RW_LAUNCH_CHECK();
  k_scan<<<1, 1024, 0, st>>>(cnt, nbar, cp);
  RW_LAUNCH_CHECK();
  k_fill_cols<<<rw_blocks(N, TB), TB, 0, st>>>(rp, col, N, cp, fill, tpos);
  RW_LAUNCH_CHECK();
  k_sort_cols<<<rw_blocks(nbar, TB), TB, 0, st>>>(cp, nbar, tpos, val, colsum, flag);
  RW_LAUNCH_CHECK();
  RW_CHECK_CUDA(cudaMemcpyAsync(&bits, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  RW_CHECK_CUDA(cudaStreamSynchronize(st));
  RW_TRY(agg_flag_status(bits));
  k_rowof<<<rw_blocks(N, TB), TB, 0, st>>>(rp, N, rowof);
  RW_LAUNCH_CHECK();
  k_etabar<<<rw_blocks(N, TB), TB, 0, st>>>(rp, col, val, vbar_in, colsum, N, vbar);
  RW_LAUNCH_CHECK();
  if (!u->naive) {
    k_delta<<<rw_blocks(N, TB), TB, 0, st>>>(G, g->w, rp, col, val, delta);
    RW_LAUNCH_CHECK();
  }
  // aggregated columns, FP64 column-major n-bar x m
  double* A = tmp.get<double>((size_t)nbar * m);
  double* Qb = tmp.get<double>((size_t)nbar * m);
  double* cf = tmp.get<double>(m + 2);
  double* nrm = tmp.get<double>(2);
  int* kept = tmp.get<int>(1);
  int* kept_idx = tmp.get<int>(m);
  if (!A || !Qb || !cf || !nrm || !kept || !kept_idx) return RW_ERR_OOM;
  k_agg_cols<<<rw_blocks((int64_t)nbar * 32, TB), TB, 0, st>>>(
      cp, tpos, vbar, u->naive ? nullptr : delta, rowof, b->Q32, b->ld32, m, nbar, nbar, A);
  RW_LAUNCH_CHECK();
  RW_CHECK_CUDA(cudaMemsetAsync(kept, 0, sizeof(int), st));
  for (int j = 0; j < m; ++j) {
    double* v = A + (int64_t)j * nbar;
    k_norm<<<1, 256, 0, st>>>(v, nbar, nrm);
    RW_LAUNCH_CHECK();
    for (int pass = 0; pass < 2 && j > 0; ++pass) {
      k_cgs_dots<<<j, 256, 0, st>>>(Qb, nbar, v, kept, cf);
      RW_LAUNCH_CHECK();
      k_cgs_axpy<<<rw_blocks(nbar, TB), TB, 0, st>>>(Qb, nbar, cf, kept, v);
      RW_LAUNCH_CHECK();
    }
    k_norm<<<1, 256, 0, st>>>(v, nbar, nrm + 1);
    RW_LAUNCH_CHECK();
    k_cgs_store<<<rw_blocks(nbar, TB), TB, 0, st>>>(v, nbar, nrm, kept, Qb);
    RW_LAUNCH_CHECK();
    k_cgs_commit<<<1, 1, 0, st>>>(nrm, j, kept, kept_idx);
    RW_LAUNCH_CHECK();
  }
  int k = 0;
  RW_CHECK_CUDA(cudaMemcpyAsync(&k, kept, sizeof(int), cudaMemcpyDeviceToHost, st));
  RW_CHECK_CUDA(cudaStreamSynchronize(st));
  if (k < 1) {
    rw_set_error_message("aggregate: every aggregated column vanished");
    return RW_ERR_SINGULAR;
  }

  // Galerkin graph
  int* wcnt = tmp.get<int>(nbar + 1);
  if (!wcnt) return RW_ERR_OOM;
  k_wbar_count<<<rw_blocks(nbar, 128), 128, 0, st>>>(G, g->w, rp, col, val, cp, tpos, rowof, nbar,
                                                     wcnt, flag);
  RW_LAUNCH_CHECK();
  RW_CHECK_CUDA(cudaMemcpyAsync(&bits, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  RW_CHECK_CUDA(cudaStreamSynchronize(st));
  RW_TRY(agg_flag_status(bits));
  rw_graph* gb = new (std::nothrow) rw_graph();
  if (!gb) return RW_ERR_OOM;
  auto fail = [&](rw_status s) { rw_graph_free(gb); return s; };
  gb->kind = RW_GRAPH_CSR;
  gb->device = g->device;
  gb->ndim = 1;
  gb->dims[0] = nbar; gb->dims[1] = 1; gb->dims[2] = 1;
  gb->N = nbar;
  gb->beta = g->beta;
  gb->form = g->form;
  gb->normalized = g->normalized;
  if (cudaMalloc(&gb->rowptr, sizeof(int32_t) * (nbar + 1)) != cudaSuccess) return fail(RW_ERR_OOM);
  k_scan<<<1, 1024, 0, st>>>(wcnt, nbar, gb->rowptr);
  RW_LAUNCH_CHECK();
  int32_t nnzb = 0;
  RW_CHECK_CUDA(cudaMemcpyAsync(&nnzb, gb->rowptr + nbar, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  RW_CHECK_CUDA(cudaStreamSynchronize(st));
  gb->nnz = nnzb;
  if (cudaMalloc(&gb->col, sizeof(int32_t) * std::max(nnzb, 1)) != cudaSuccess ||
      cudaMalloc(&gb->wcsr, sizeof(float) * std::max(nnzb, 1)) != cudaSuccess ||
      cudaMalloc(&gb->ccsr, sizeof(float) * std::max(nnzb, 1)) != cudaSuccess ||
      cudaMalloc(&gb->d, sizeof(float) * nbar) != cudaSuccess ||
      cudaMalloc(&gb->s, sizeof(float) * nbar) != cudaSuccess ||
      cudaMalloc(&gb->sq, sizeof(float) * nbar) != cudaSuccess ||
      cudaMalloc(&gb->status, sizeof(int)) != cudaSuccess)
    return fail(RW_ERR_OOM);
  if (cudaMemsetAsync(gb->status, 0, sizeof(int), st) != cudaSuccess) return fail(RW_ERR_CUDA);
  k_wbar_fill<<<rw_blocks(nbar, 128), 128, 0, st>>>(G, g->w, rp, col, val, cp, tpos, rowof, nbar,
                                                    gb->rowptr, gb->col, gb->wcsr, gb->d);
  if (cudaGetLastError() != cudaSuccess) return fail(RW_ERR_CUDA);
  rw_count_launch();
  k_csr_scalings<<<rw_blocks(nbar, TB), TB, 0, st>>>(gb->d, nbar, gb->normalized, gb->s, gb->sq, flag);
  k_csr_coeffs<<<rw_blocks(nbar, TB), TB, 0, st>>>(gb->rowptr, gb->col, gb->wcsr, gb->s, nbar,
                                                   gb->normalized, gb->ccsr);
  if (cudaGetLastError() != cudaSuccess) return fail(RW_ERR_CUDA);
  rw_count_launch();
  rw_count_launch();
  if (cudaMemcpyAsync(&bits, flag, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return fail(RW_ERR_CUDA);
  if (bits) return fail(agg_flag_status(bits));
  if (rw_graph_reserve_scratch(gb) != RW_OK) return fail(RW_ERR_OOM);
  if (rw_graph_degree_sum(gb, st) != RW_OK) return fail(RW_ERR_CUDA);

  // basis on the aggregate graph: the kept columns, values by Eq. (z_ray)
  float* X = tmp.get<float>((size_t)nbar * k);
  if (!X) return fail(RW_ERR_OOM);
  k_colmajor_to_rows<<<rw_blocks((int64_t)nbar * k, TB), TB, 0, st>>>(Qb, nbar, k, X);
  if (cudaGetLastError() != cudaSuccess) return fail(RW_ERR_CUDA);
  rw_count_launch();
  std::vector<double> zeros(k, 0.0);
  rw_basis* bb = nullptr;
  rw_status s = rw_make_basis(gb, k, X, k, zeros.data(), st, &bb);
  if (s != RW_OK) return fail(s);
  s = rw_basis_rayleigh(gb, bb, st);
  if (s != RW_OK) { rw_basis_free(bb); return fail(s); }
  *gout = gb;
  *bout = bb;
  return RW_OK;
}
