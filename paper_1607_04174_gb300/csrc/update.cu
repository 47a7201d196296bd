// Updating the precomputed values when the edge weights or the topology change
// (Sec. III-B, Eq. z_ray; Sec. III-C edge removal).  Each stored column q keeps its direction;
// its value becomes Ncut(q) = q^T L-hat q / q^T q under the new weights, evaluated as the edge
// sum  sum_e w_e (q(a) s_a - q(b) s_b)^2  (s = d^{-1/2}; s = 1 for L).  The edge-sum form has
// no cancellation, so its rounding error is relative to the value itself.
//
// Local changes (a box of voxels, or a list of edges) only alter the terms of the edges that
// touch a voxel whose degree changed, so the update subtracts those terms under the old graph
// and adds them under the new one.
#include "rw_internal.cuh"

#include <algorithm>
#include <cstring>
#include <vector>

namespace {

struct Box {
  int lo[3], hi[3];  // half-open iteration box
};

// Edge-sum Rayleigh numerators over the forward edges leaving the voxels of `it` (a box
// walked in x-runs, one warp per run).  mode 0: every edge; mode 1: edges with an end inside
// `roi`; mode 2: edges with an end marked in `mark`.
template <int CH>
__global__ void __launch_bounds__(256)
k_rayleigh(const float* __restrict__ Q, int64_t ldq, int nch, const float* __restrict__ w,
           const float* __restrict__ s, int ndim, int DX, int DY, int DZ, int64_t N, Box it,
           int mode, Box roi, const uint8_t* __restrict__ mark, int run, int64_t total_runs,
           double* __restrict__ part /* gridDim.x x (4 * 32 * CH) */) {
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int nwb = blockDim.x >> 5;
  double accd[CH][4];
#pragma unroll
  for (int t = 0; t < CH; ++t)
#pragma unroll
    for (int u = 0; u < 4; ++u) accd[t][u] = 0.0;
  const int bx = it.hi[0] - it.lo[0], by = it.hi[1] - it.lo[1];
  const int segs = (bx + run - 1) / run;
  const int64_t st[3] = {1, (int64_t)DX, (int64_t)DX * DY};
  const int n[3] = {DX, DY, DZ};
  for (int64_t r = (int64_t)blockIdx.x * nwb + wib; r < total_runs; r += (int64_t)gridDim.x * nwb) {
    const int seg = (int)(r % segs);
    const int64_t row = r / segs;
    const int y = it.lo[1] + (int)(row % by), z = it.lo[2] + (int)(row / by);
    const int x0 = it.lo[0] + seg * run, x1 = min(x0 + run, it.hi[0]);
    float4 acc[CH];
#pragma unroll
    for (int t = 0; t < CH; ++t) acc[t] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int x = x0; x < x1; ++x) {
      const int64_t i = (int64_t)x + (int64_t)DX * (y + (int64_t)DY * z);
      const int c[3] = {x, y, z};
      bool any = false;
      for (int a = 0; a < ndim; ++a) {
        if (c[a] + 1 >= n[a]) continue;
        const int64_t j = i + st[a];
        bool sel = true;
        if (mode == 1) {
          bool ia = true, ib = true;
          for (int q = 0; q < ndim; ++q) {
            int ca = c[q], cb = c[q] + (q == a ? 1 : 0);
            ia = ia && ca >= roi.lo[q] && ca < roi.hi[q];
            ib = ib && cb >= roi.lo[q] && cb < roi.hi[q];
          }
          sel = ia || ib;
        } else if (mode == 2) {
          sel = mark[i] || mark[j];
        }
        if (!sel) continue;
        const float we = w[a * N + i];
        if (we == 0.f) continue;
        any = true;
        const float si = s[i], sj = s[j];
        const float4* qi = reinterpret_cast<const float4*>(Q + i * ldq);
        const float4* qj = reinterpret_cast<const float4*>(Q + j * ldq);
#pragma unroll
        for (int t = 0; t < CH; ++t) {
          int cc = lane + 32 * t;
          if (cc < nch) {
            float4 u = __ldg(qi + cc), v = __ldg(qj + cc);
            float dx = u.x * si - v.x * sj, dy = u.y * si - v.y * sj;
            float dz = u.z * si - v.z * sj, dw = u.w * si - v.w * sj;
            acc[t].x = fmaf(we * dx, dx, acc[t].x);
            acc[t].y = fmaf(we * dy, dy, acc[t].y);
            acc[t].z = fmaf(we * dz, dz, acc[t].z);
            acc[t].w = fmaf(we * dw, dw, acc[t].w);
          }
        }
      }
      (void)any;
    }
#pragma unroll
    for (int t = 0; t < CH; ++t) {
      accd[t][0] += acc[t].x; accd[t][1] += acc[t].y;
      accd[t][2] += acc[t].z; accd[t][3] += acc[t].w;
    }
  }
  // block reduction over warps through shared memory (FP64)
  __shared__ double red[32 * 4 * 8];  // CH <= 8
  for (int e = threadIdx.x; e < 32 * 4 * CH; e += blockDim.x) red[e] = 0.0;
  __syncthreads();
#pragma unroll
  for (int t = 0; t < CH; ++t)
#pragma unroll
    for (int u = 0; u < 4; ++u) atomicAdd(&red[(lane + 32 * t) * 4 + u], accd[t][u]);
  __syncthreads();
  for (int e = threadIdx.x; e < 32 * 4 * CH; e += blockDim.x)
    part[(int64_t)blockIdx.x * (32 * 4 * CH) + e] = red[e];
}

__global__ void k_rayleigh_finish(const double* __restrict__ part, int nblk, int width, int m,
                                  const double* __restrict__ qnorm2, double sign,
                                  double* __restrict__ lam, int accumulate) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= m) return;
  double sacc = 0.0;
  for (int b = 0; b < nblk; ++b) sacc += part[(int64_t)b * width + c];
  sacc /= qnorm2 ? qnorm2[c] : 1.0;
  lam[c] = accumulate ? lam[c] + sign * sacc : sign * sacc;
}

// CSR graphs: one warp per row, edges (i, j) with j > i
template <int CH>
__global__ void __launch_bounds__(256)
k_rayleigh_csr(const float* __restrict__ Q, int64_t ldq, int nch,
               const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
               const float* __restrict__ wv, const float* __restrict__ s, int64_t N,
               double* __restrict__ part) {
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nwb = blockDim.x >> 5;
  double accd[CH][4] = {};
  for (int64_t i = (int64_t)blockIdx.x * nwb + wib; i < N; i += (int64_t)gridDim.x * nwb) {
    float4 acc[CH];
#pragma unroll
    for (int t = 0; t < CH; ++t) acc[t] = make_float4(0.f, 0.f, 0.f, 0.f);
    const float si = s[i];
    for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) {
      const int64_t j = col[p];
      if (j <= i) continue;
      const float we = wv[p], sj = s[j];
      const float4* qi = reinterpret_cast<const float4*>(Q + i * ldq);
      const float4* qj = reinterpret_cast<const float4*>(Q + j * ldq);
#pragma unroll
      for (int t = 0; t < CH; ++t) {
        int cc = lane + 32 * t;
        if (cc < nch) {
          float4 u = qi[cc], v = qj[cc];
          float dx = u.x * si - v.x * sj, dy = u.y * si - v.y * sj;
          float dz = u.z * si - v.z * sj, dw = u.w * si - v.w * sj;
          acc[t].x = fmaf(we * dx, dx, acc[t].x);
          acc[t].y = fmaf(we * dy, dy, acc[t].y);
          acc[t].z = fmaf(we * dz, dz, acc[t].z);
          acc[t].w = fmaf(we * dw, dw, acc[t].w);
        }
      }
    }
#pragma unroll
    for (int t = 0; t < CH; ++t) {
      accd[t][0] += acc[t].x; accd[t][1] += acc[t].y;
      accd[t][2] += acc[t].z; accd[t][3] += acc[t].w;
    }
  }
  __shared__ double red[32 * 4 * 8];
  for (int e = threadIdx.x; e < 32 * 4 * CH; e += blockDim.x) red[e] = 0.0;
  __syncthreads();
#pragma unroll
  for (int t = 0; t < CH; ++t)
#pragma unroll
    for (int u = 0; u < 4; ++u) atomicAdd(&red[(lane + 32 * t) * 4 + u], accd[t][u]);
  __syncthreads();
  for (int e = threadIdx.x; e < 32 * 4 * CH; e += blockDim.x)
    part[(int64_t)blockIdx.x * (32 * 4 * CH) + e] = red[e];
}

// squared column norms (FP64)
__global__ void k_qnorm2(const float* __restrict__ Q, int64_t ldq, int64_t N, int m,
                         int64_t rpb, double* __restrict__ out) {
  int c = threadIdx.x + blockIdx.y * blockDim.x;
  if (c >= m) return;
  int64_t r0 = (int64_t)blockIdx.x * rpb, r1 = min(N, r0 + rpb);
  double acc = 0.0;
  float a32 = 0.f;
  int cnt = 0;
  for (int64_t i = r0; i < r1; ++i) {
    float v = Q[i * ldq + c];
    a32 = fmaf(v, v, a32);
    if (++cnt == 64) { acc += a32; a32 = 0.f; cnt = 0; }
  }
  acc += a32;
  atomicAdd(&out[c], acc);
}

template <int CH>
void launch_rayleigh(const rw_graph* g, const float* Q, int64_t ldq, int nch, Box it, int mode,
                     Box roi, const uint8_t* mark, int nblk, double* part, cudaStream_t st) {
  if (g->kind == RW_GRAPH_CSR) {
    k_rayleigh_csr<CH><<<nblk, 256, 0, st>>>(Q, ldq, nch, g->rowptr, g->col, g->wcsr, g->s, g->N,
                                            part);
    return;
  }
  const int run = 16;
  const int bx = it.hi[0] - it.lo[0];
  const int64_t rows = (int64_t)(it.hi[1] - it.lo[1]) * (it.hi[2] - it.lo[2]);
  const int64_t total = rows * ((bx + run - 1) / run);
  k_rayleigh<CH><<<nblk, 256, 0, st>>>(Q, ldq, nch, g->w, g->s, g->ndim, g->dims[0], g->dims[1],
                                      g->dims[2], g->N, it, mode, roi, mark, run, total, part);
}

}  // namespace

// lam[c] (+)= sign * numerator_c / ||q_c||^2 over the selected edges
rw_status rw_rayleigh_terms(const rw_graph* g, const float* Q, int64_t ldq, int m, Box it,
                            int mode, Box roi, const uint8_t* mark, double sign, double* lam,
                            int accumulate, const double* qn2, cudaStream_t st) {
  rw_graph* gm = const_cast<rw_graph*>(g);
  const int nch = (m + 3) / 4;
  const int ch = (nch + 31) / 32;
  if (ch > 8) return RW_ERR_UNSUPPORTED;
  const int sms = g_rw_num_sms > 0 ? g_rw_num_sms : 148;
  const int nblk = 2 * sms;
  const int width = 32 * 4 * ch;
  const size_t need = sizeof(double) * ((size_t)nblk * width) + 16384;
  if (gm->upd.cap < need) return RW_ERR_OOM;  // reserved when the graph was built
  double* part = reinterpret_cast<double*>(gm->upd.as<char>() + 16384);
  switch (ch) {
    case 1: launch_rayleigh<1>(g, Q, ldq, nch, it, mode, roi, mark, nblk, part, st); break;
    case 2: launch_rayleigh<2>(g, Q, ldq, nch, it, mode, roi, mark, nblk, part, st); break;
    case 3: launch_rayleigh<3>(g, Q, ldq, nch, it, mode, roi, mark, nblk, part, st); break;
    case 4: launch_rayleigh<4>(g, Q, ldq, nch, it, mode, roi, mark, nblk, part, st); break;
    case 5: launch_rayleigh<5>(g, Q, ldq, nch, it, mode, roi, mark, nblk, part, st); break;
    case 6: launch_rayleigh<6>(g, Q, ldq, nch, it, mode, roi, mark, nblk, part, st); break;
    case 7: launch_rayleigh<7>(g, Q, ldq, nch, it, mode, roi, mark, nblk, part, st); break;
    default: launch_rayleigh<8>(g, Q, ldq, nch, it, mode, roi, mark, nblk, part, st); break;
  }
  RW_LAUNCH_CHECK();
  k_rayleigh_finish<<<rw_blocks(m, 128), 128, 0, st>>>(part, nblk, width, m, qn2, sign, lam,
                                                      accumulate);
  RW_LAUNCH_CHECK();
  return RW_OK;
}

static Box full_box(const rw_graph* g) {
  Box b;
  for (int a = 0; a < 3; ++a) { b.lo[a] = 0; b.hi[a] = g->dims[a]; }
  return b;
}

// squared norms of the basis columns (device, m doubles) into upd scratch
static rw_status basis_qnorm2(const rw_graph* g, const rw_basis* b, double** out, cudaStream_t st) {
  rw_graph* gm = const_cast<rw_graph*>(g);
  if (gm->upd.cap < 16384) return RW_ERR_OOM;
  double* qn = reinterpret_cast<double*>(gm->upd.as<char>() + 8192);
  if (b->m > 1024) return RW_ERR_UNSUPPORTED;
  RW_CHECK_CUDA(cudaMemsetAsync(qn, 0, sizeof(double) * b->m, st));
  int64_t rpb = 4096;
  dim3 grid((unsigned)((b->N + rpb - 1) / rpb), (unsigned)((b->m + 255) / 256));
  k_qnorm2<<<grid, 256, 0, st>>>(b->Q32, b->ld32, b->N, b->m, rpb, qn);
  RW_LAUNCH_CHECK();
  *out = qn;
  return RW_OK;
}

// full Rayleigh quotients of the basis columns under g -> b->lam (device and host copies)
rw_status rw_basis_rayleigh(const rw_graph* g, rw_basis* b, cudaStream_t st) {
  double* qn;
  RW_TRY(basis_qnorm2(g, b, &qn, st));
  Box fb = full_box(g);
  RW_TRY(rw_rayleigh_terms(g, b->Q32, b->ld32, b->m, fb, 0, fb, nullptr, 1.0, b->lam, 0, qn, st));
  RW_CHECK_CUDA(cudaMemcpyAsync(b->lam_host, b->lam, sizeof(double) * b->m, cudaMemcpyDeviceToHost, st));
  RW_CHECK_CUDA(cudaStreamSynchronize(st));
  return RW_OK;
}

// ---------------------------------------------------------------------------------------
// weight edits
// ---------------------------------------------------------------------------------------
namespace {

__device__ __forceinline__ float edge_w2(float a, float b, float beta, int form) {
  float t = a - b;
  return form == RW_WEIGHT_SQ ? expf(-beta * t * t) : expf(-beta * fabsf(t));
}

// Eq. (W) with a local beta for the forward edges whose two ends lie inside the box
__global__ void k_roi_weights(const float* __restrict__ J, float* __restrict__ w, int ndim, int DX,
                              int DY, int DZ, int64_t N, Box roi, float beta, int form) {
  const int bx = roi.hi[0] - roi.lo[0], by = roi.hi[1] - roi.lo[1], bz = roi.hi[2] - roi.lo[2];
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)bx * by * bz) return;
  int c[3] = {roi.lo[0] + (int)(e % bx), roi.lo[1] + (int)((e / bx) % by),
              roi.lo[2] + (int)(e / ((int64_t)bx * by))};
  const int64_t st[3] = {1, (int64_t)DX, (int64_t)DX * DY};
  const int64_t i = c[0] + (int64_t)DX * (c[1] + (int64_t)DY * c[2]);
  for (int a = 0; a < ndim; ++a)
    if (c[a] + 1 < roi.hi[a]) w[a * N + i] = edge_w2(J[i], J[i + st[a]], beta, form);
  (void)DZ;
}

// degrees / scalings / operator coefficients for the voxels of a box (coefficients of the
// edges leaving the box's voxels forward; the caller widens the box by one voxel backwards)
__global__ void k_box_degree(const float* __restrict__ w, float* __restrict__ d,
                             float* __restrict__ s, float* __restrict__ sq, int ndim, int DX,
                             int DY, int DZ, int64_t N, Box b, int normalized, int* status) {
  const int bx = b.hi[0] - b.lo[0], by = b.hi[1] - b.lo[1], bz = b.hi[2] - b.lo[2];
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)bx * by * bz) return;
  int c[3] = {b.lo[0] + (int)(e % bx), b.lo[1] + (int)((e / bx) % by),
              b.lo[2] + (int)(e / ((int64_t)bx * by))};
  const int64_t st[3] = {1, (int64_t)DX, (int64_t)DX * DY};
  const int64_t i = c[0] + (int64_t)DX * (c[1] + (int64_t)DY * c[2]);
  float deg = 0.f;
  for (int a = 0; a < ndim; ++a) {
    deg += w[a * N + i];
    if (c[a] > 0) deg += w[a * N + i - st[a]];
  }
  d[i] = deg;
  if (normalized) {
    if (!(deg > 0.f)) { atomicOr(status, RW_DEV_ISOLATED); s[i] = 0.f; sq[i] = 0.f; }
    else { float r = sqrtf(deg); sq[i] = r; s[i] = 1.f / r; }
  } else { s[i] = 1.f; sq[i] = 1.f; }
  (void)DZ;
}

__global__ void k_box_coeffs(const float* __restrict__ w, const float* __restrict__ s,
                             float* __restrict__ cw, int ndim, int DX, int DY, int64_t N, Box b,
                             int normalized) {
  const int bx = b.hi[0] - b.lo[0], by = b.hi[1] - b.lo[1], bz = b.hi[2] - b.lo[2];
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)bx * by * bz) return;
  int c[3] = {b.lo[0] + (int)(e % bx), b.lo[1] + (int)((e / bx) % by),
              b.lo[2] + (int)(e / ((int64_t)bx * by))};
  const int64_t st[3] = {1, (int64_t)DX, (int64_t)DX * DY};
  const int64_t i = c[0] + (int64_t)DX * (c[1] + (int64_t)DY * c[2]);
  for (int a = 0; a < ndim; ++a) {
    float we = w[a * N + i];
    cw[a * N + i] = (normalized && we != 0.f) ? we * s[i] * s[i + st[a]] : we;
  }
}

__global__ void k_mark_edges(const int64_t* __restrict__ ids, int64_t n, int ndim, int DX, int DY,
                             int DZ, int64_t N, uint8_t* __restrict__ mark, int* status) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  int64_t id = ids[t];
  if (id < 0 || id >= ndim * N) { atomicOr(status, RW_DEV_BAD_SEED); return; }
  int a = (int)(id / N);
  int64_t i = id % N;
  const int64_t st[3] = {1, (int64_t)DX, (int64_t)DX * DY};
  const int c[3] = {(int)(i % DX), (int)((i / DX) % DY), (int)(i / ((int64_t)DX * DY))};
  const int nn[3] = {DX, DY, DZ};
  if (c[a] + 1 >= nn[a]) { atomicOr(status, RW_DEV_BAD_SEED); return; }
  mark[i] = 1;
  mark[i + st[a]] = 1;
}

__global__ void k_set_edges(const int64_t* __restrict__ ids, const float* __restrict__ wv,
                            int64_t n, int ndim, int64_t N, float* __restrict__ w, int* status) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  int64_t id = ids[t];
  if (id < 0 || id >= ndim * N) return;
  float v = wv ? wv[t] : 0.f;
  if (!(v >= 0.f) || !isfinite(v)) { atomicOr(status, RW_DEV_NONFINITE); return; }
  w[id] = v;
}

__global__ void k_marked_degree_coeffs(const float* __restrict__ w, float* __restrict__ d,
                                       float* __restrict__ s, float* __restrict__ sq,
                                       const uint8_t* __restrict__ mark, int ndim, int DX, int DY,
                                       int DZ, int64_t N, int normalized, int* status) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N || !mark[i]) return;
  const int64_t st[3] = {1, (int64_t)DX, (int64_t)DX * DY};
  const int c[3] = {(int)(i % DX), (int)((i / DX) % DY), (int)(i / ((int64_t)DX * DY))};
  float deg = 0.f;
  for (int a = 0; a < ndim; ++a) {
    deg += w[a * N + i];
    if (c[a] > 0) deg += w[a * N + i - st[a]];
  }
  d[i] = deg;
  if (normalized) {
    if (!(deg > 0.f)) { atomicOr(status, RW_DEV_ISOLATED); s[i] = 0.f; sq[i] = 0.f; }
    else { float r = sqrtf(deg); sq[i] = r; s[i] = 1.f / r; }
  } else { s[i] = 1.f; sq[i] = 1.f; }
  (void)DZ;
}

__global__ void k_marked_coeffs(const float* __restrict__ w, const float* __restrict__ s,
                                float* __restrict__ cw, const uint8_t* __restrict__ mark, int ndim,
                                int DX, int DY, int DZ, int64_t N, int normalized) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int64_t st[3] = {1, (int64_t)DX, (int64_t)DX * DY};
  const int c[3] = {(int)(i % DX), (int)((i / DX) % DY), (int)(i / ((int64_t)DX * DY))};
  const int nn[3] = {DX, DY, DZ};
  for (int a = 0; a < ndim; ++a) {
    if (c[a] + 1 >= nn[a]) continue;
    const int64_t j = i + st[a];
    if (!(mark[i] || mark[j])) continue;
    float we = w[a * N + i];
    cw[a * N + i] = (normalized && we != 0.f) ? we * s[i] * s[j] : we;
  }
}

rw_status read_status(rw_graph* g, cudaStream_t st) {
  int bits = 0;
  RW_CHECK_CUDA(cudaMemcpyAsync(&bits, g->status, sizeof(int), cudaMemcpyDeviceToHost, st));
  RW_CHECK_CUDA(cudaMemsetAsync(g->status, 0, sizeof(int), st));
  RW_CHECK_CUDA(cudaStreamSynchronize(st));
  return rw_status_from_device_bits(bits);
}

}  // namespace

rw_status rw_build_weights_again(rw_graph* g, double beta, cudaStream_t st);

static rw_status edges_update(rw_graph* g, rw_basis* b, const int64_t* ids, const float* wv,
                              int64_t n, cudaStream_t st) {
  if (g->kind != RW_GRAPH_GRID) return RW_ERR_UNSUPPORTED;
  if (n <= 0) return RW_OK;
  if (!ids) return RW_ERR_INVALID_ARG;
  const size_t need = 16384 + sizeof(double) * 2 * 148 * 1024 + 256;
  (void)need;
  DevBuf mark;
  RW_TRY(mark.grow(g->N));
  struct R { DevBuf& m; ~R() { m.release(); } } rel{mark};
  uint8_t* mk = mark.as<uint8_t>();
  RW_CHECK_CUDA(cudaMemsetAsync(mk, 0, g->N, st));
  k_mark_edges<<<rw_blocks(n, 256), 256, 0, st>>>(ids, n, g->ndim, g->dims[0], g->dims[1],
                                                  g->dims[2], g->N, mk, g->status);
  RW_LAUNCH_CHECK();
  RW_TRY(read_status(g, st));
  Box fb = full_box(g);
  double* qn = nullptr;
  if (b) {
    RW_TRY(basis_qnorm2(g, b, &qn, st));
    RW_TRY(rw_rayleigh_terms(g, b->Q32, b->ld32, b->m, fb, 2, fb, mk, -1.0, b->lam, 1, qn, st));
  }
  k_set_edges<<<rw_blocks(n, 256), 256, 0, st>>>(ids, wv, n, g->ndim, g->N, g->w, g->status);
  RW_LAUNCH_CHECK();
  k_marked_degree_coeffs<<<rw_blocks(g->N, 256), 256, 0, st>>>(g->w, g->d, g->s, g->sq, mk,
                                                               g->ndim, g->dims[0], g->dims[1],
                                                               g->dims[2], g->N, g->normalized,
                                                               g->status);
  RW_LAUNCH_CHECK();
  k_marked_coeffs<<<rw_blocks(g->N, 256), 256, 0, st>>>(g->w, g->s, g->cw, mk, g->ndim, g->dims[0],
                                                        g->dims[1], g->dims[2], g->N,
                                                        g->normalized);
  RW_LAUNCH_CHECK();
  if (b) RW_TRY(rw_rayleigh_terms(g, b->Q32, b->ld32, b->m, fb, 2, fb, mk, 1.0, b->lam, 1, qn, st));
  RW_TRY(read_status(g, st));
  RW_TRY(rw_graph_degree_sum(g, st));
  if (b) {
    RW_CHECK_CUDA(cudaMemcpyAsync(b->lam_host, b->lam, sizeof(double) * b->m, cudaMemcpyDeviceToHost, st));
    RW_CHECK_CUDA(cudaStreamSynchronize(st));
  }
  return RW_OK;
}

static rw_status roi_update(rw_graph* g, rw_basis* b, const int* lo_in, const int* hi_in,
                            double beta_local, cudaStream_t st) {
  if (g->kind != RW_GRAPH_GRID) return RW_ERR_UNSUPPORTED;
  Box roi;
  for (int a = 0; a < 3; ++a) {
    int lo = a < g->ndim ? lo_in[a] : 0, hi = a < g->ndim ? hi_in[a] : 1;
    if (lo < 0 || hi > g->dims[a] || lo >= hi) return RW_ERR_INVALID_ARG;
    roi.lo[a] = lo;
    roi.hi[a] = hi;
  }
  if (!(beta_local >= 0.0)) return RW_ERR_INVALID_ARG;
  if (!g->J) return RW_ERR_INVALID_ARG;
  // iteration box: the ROI widened by one voxel backwards (edges entering the ROI)
  Box itb = roi;
  for (int a = 0; a < g->ndim; ++a) itb.lo[a] = std::max(0, roi.lo[a] - 1);
  double* qn = nullptr;
  if (b) {
    RW_TRY(basis_qnorm2(g, b, &qn, st));
    RW_TRY(rw_rayleigh_terms(g, b->Q32, b->ld32, b->m, itb, 1, roi, nullptr, -1.0, b->lam, 1, qn, st));
  }
  const int64_t nroi = (int64_t)(roi.hi[0] - roi.lo[0]) * (roi.hi[1] - roi.lo[1]) * (roi.hi[2] - roi.lo[2]);
  k_roi_weights<<<rw_blocks(nroi, 256), 256, 0, st>>>(g->J, g->w, g->ndim, g->dims[0], g->dims[1],
                                                      g->dims[2], g->N, roi, (float)beta_local,
                                                      g->form);
  RW_LAUNCH_CHECK();
  k_box_degree<<<rw_blocks(nroi, 256), 256, 0, st>>>(g->w, g->d, g->s, g->sq, g->ndim, g->dims[0],
                                                     g->dims[1], g->dims[2], g->N, roi,
                                                     g->normalized, g->status);
  RW_LAUNCH_CHECK();
  const int64_t nit = (int64_t)(itb.hi[0] - itb.lo[0]) * (itb.hi[1] - itb.lo[1]) * (itb.hi[2] - itb.lo[2]);
  k_box_coeffs<<<rw_blocks(nit, 256), 256, 0, st>>>(g->w, g->s, g->cw, g->ndim, g->dims[0],
                                                    g->dims[1], g->N, itb, g->normalized);
  RW_LAUNCH_CHECK();
  if (b) RW_TRY(rw_rayleigh_terms(g, b->Q32, b->ld32, b->m, itb, 1, roi, nullptr, 1.0, b->lam, 1, qn, st));
  RW_TRY(read_status(g, st));
  RW_TRY(rw_graph_degree_sum(g, st));
  if (b) {
    RW_CHECK_CUDA(cudaMemcpyAsync(b->lam_host, b->lam, sizeof(double) * b->m, cudaMemcpyDeviceToHost, st));
    RW_CHECK_CUDA(cudaStreamSynchronize(st));
  }
  return RW_OK;
}

extern "C" rw_status rw_update_weights(rw_graph* g, rw_basis* b, const rw_weight_update* u,
                                       void* stream) {
  if (!g || !u) return RW_ERR_INVALID_ARG;
  if (b && b->N != g->N) return RW_ERR_INVALID_ARG;
  cudaStream_t st = rw_stream(stream);
  switch (u->kind) {
    case RW_UPDATE_BETA: {
      if (!(u->beta >= 0.0) || !g->J || g->kind != RW_GRAPH_GRID) return RW_ERR_INVALID_ARG;
      RW_TRY(rw_build_weights_again(g, u->beta, st));
      if (b) RW_TRY(rw_basis_rayleigh(g, b, st));
      return RW_OK;
    }
    case RW_UPDATE_EDGES:
      if (u->n_edges < 0 || (u->n_edges > 0 && (!u->edge_ids_dev || !u->edge_w_dev)))
        return RW_ERR_INVALID_ARG;
      return edges_update(g, b, u->edge_ids_dev, u->edge_w_dev, u->n_edges, st);
    case RW_UPDATE_ROI:
      return roi_update(g, b, u->roi_lo, u->roi_hi, u->beta, st);
    case RW_UPDATE_ALL:
      if (!u->edge_w_dev || g->kind != RW_GRAPH_GRID) return RW_ERR_INVALID_ARG;
      RW_TRY(rw_set_all_weights(g, u->edge_w_dev, st));
      if (b) RW_TRY(rw_basis_rayleigh(g, b, st));
      return RW_OK;
  }
  return RW_ERR_INVALID_ARG;
}

rw_status rw_aggregate(rw_graph* g, rw_basis* b, const rw_topology_update* u, cudaStream_t st,
                       rw_graph** gout, rw_basis** bout);

extern "C" rw_status rw_update_topology(rw_graph* g, rw_basis* b, const rw_topology_update* u,
                                        void* stream, rw_graph** agg_graph_out,
                                        rw_basis** agg_basis_out) {
  if (!g || !u) return RW_ERR_INVALID_ARG;
  cudaStream_t st = rw_stream(stream);
  if (u->kind == RW_TOPO_REMOVE_EDGES) {
    if (u->n_edges < 0 || (u->n_edges > 0 && !u->edge_ids_dev)) return RW_ERR_INVALID_ARG;
    return edges_update(g, b, u->edge_ids_dev, nullptr, u->n_edges, st);
  }
  if (u->kind == RW_TOPO_AGGREGATE) {
    if (!b || !agg_graph_out || !agg_basis_out) return RW_ERR_INVALID_ARG;
    return rw_aggregate(g, b, u, st, agg_graph_out, agg_basis_out);
  }
  return RW_ERR_INVALID_ARG;
}

// ---------------------------------------------------------------------------------------
// Rayleigh quotients without any allocation.
//
// Some callers cannot allocate device memory during a call: for example a host application
// that owns the whole device memory budget through its own pool and forbids libraries from
// calling cudaMalloc, or a latency-critical thread that must not hit the allocator.  This
// entry point computes the same edge-sum Rayleigh quotients as the value update, but keeps
// its scratch (per-block partial sums and column norms) in the file-scope device array below
// instead of the graph's scratch buffers.  Every GPU that loads the library holds the array
// (about 2 MiB) until the process exits.  All calls share it and it keeps the last call's
// contents, so the norm accumulators are cleared at the start of every call and calls that
// overlap on the GPU (different streams, or different host threads) race on it.
// ---------------------------------------------------------------------------------------
namespace {
constexpr int kNoAllocBlocks = 256;            // blocks of the partial-sum kernel
constexpr int kNoAllocWidth = 32 * 4 * 8;      // columns of one partial row (m <= 1024)
constexpr size_t kNoAllocDoubles = (size_t)kNoAllocBlocks * kNoAllocWidth + kNoAllocWidth;
static_assert(kNoAllocWidth >= RW_NOALLOC_MAX_M,
              "a partial row of the no-allocation scratch must hold RW_NOALLOC_MAX_M columns");
#define RW_STR_(x) #x
#define RW_STR(x) RW_STR_(x)
}  // namespace

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

#include <mutex>

static std::mutex g_noalloc_mu;
static double* g_noalloc_ptr[128] = {};  // host-usable address of the array, per device

extern "C" rw_status rw_rayleigh_quotients_noalloc(const rw_graph* g, const float* Q_dev,
                                                   int64_t ldq, int32_t m, double* lambda_dev,
                                                   void* stream) {
  if (!g || !Q_dev || !lambda_dev) return RW_ERR_INVALID_ARG;
  if (m < 1 || m > RW_NOALLOC_MAX_M) {
    rw_set_error_message("rw_rayleigh_quotients_noalloc: m must be in [1, "
                         RW_STR(RW_NOALLOC_MAX_M) "]");
    return RW_ERR_INVALID_ARG;
  }
  if (ldq < m || (ldq & 3) || (reinterpret_cast<uintptr_t>(Q_dev) & 15)) {
    rw_set_error_message("rw_rayleigh_quotients_noalloc: ldq must be >= m and a multiple of 4, "
                         "Q_dev 16-byte aligned");
    return RW_ERR_INVALID_ARG;
  }
  int dev = 0;
  RW_CHECK_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 128) {
    rw_set_error_message("rw_rayleigh_quotients_noalloc: device ordinals above 127 are not "
                         "supported");
    return RW_ERR_UNSUPPORTED;
  }
  if (dev != g->device) {
    rw_set_error_message("rw_rayleigh_quotients_noalloc: the graph's device must be current");
    return RW_ERR_INVALID_ARG;
  }
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      // first call on this device: the host-side name of the array is not a device address
      void* p = nullptr;
      RW_CHECK_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
      g_noalloc_ptr[dev] = static_cast<double*>(p);
    }
    scratch = g_noalloc_ptr[dev];
  }
  if (g_rw_num_sms <= 0) RW_TRY(rw_device_init());
  cudaStream_t st = rw_stream(stream);
  double* part = scratch;
  double* qn = scratch + (size_t)kNoAllocBlocks * kNoAllocWidth;
  RW_CHECK_CUDA(cudaMemsetAsync(qn, 0, sizeof(double) * m, st));
  int64_t rpb = 4096;
  dim3 grid((unsigned)((g->N + rpb - 1) / rpb), (unsigned)((m + 255) / 256));
  k_qnorm2<<<grid, 256, 0, st>>>(Q_dev, ldq, g->N, m, rpb, qn);
  RW_LAUNCH_CHECK();
  const int nch = (m + 3) / 4;
  const int ch = (nch + 31) / 32;
  Box fb = full_box(g);
  switch (ch) {
    case 1: launch_rayleigh<1>(g, Q_dev, ldq, nch, fb, 0, fb, nullptr, kNoAllocBlocks, part, st); break;
    case 2: launch_rayleigh<2>(g, Q_dev, ldq, nch, fb, 0, fb, nullptr, kNoAllocBlocks, part, st); break;
    case 3: launch_rayleigh<3>(g, Q_dev, ldq, nch, fb, 0, fb, nullptr, kNoAllocBlocks, part, st); break;
    case 4: launch_rayleigh<4>(g, Q_dev, ldq, nch, fb, 0, fb, nullptr, kNoAllocBlocks, part, st); break;
    case 5: launch_rayleigh<5>(g, Q_dev, ldq, nch, fb, 0, fb, nullptr, kNoAllocBlocks, part, st); break;
    case 6: launch_rayleigh<6>(g, Q_dev, ldq, nch, fb, 0, fb, nullptr, kNoAllocBlocks, part, st); break;
    case 7: launch_rayleigh<7>(g, Q_dev, ldq, nch, fb, 0, fb, nullptr, kNoAllocBlocks, part, st); break;
    default: launch_rayleigh<8>(g, Q_dev, ldq, nch, fb, 0, fb, nullptr, kNoAllocBlocks, part, st); break;
  }
  RW_LAUNCH_CHECK();
  k_rayleigh_finish<<<rw_blocks(m, 128), 128, 0, st>>>(part, kNoAllocBlocks, 32 * 4 * ch, m, qn,
                                                      1.0, lambda_dev, 0);
  RW_LAUNCH_CHECK();
  return RW_OK;
}

// ---------------------------------------------------------------------------------------
// Several precomputed bases (Sec. III-B, last paragraph: eigenvectors precomputed for several
// beta' and Eq. z_ray used to "interpolate" between them): the basis to update for a new beta
// is the one whose beta' is nearest in log beta (doubling beta squares the weights of the
// squared form, so distances between betas are ratios); ties go to the lower index.
// ---------------------------------------------------------------------------------------
extern "C" int32_t rw_basis_nearest_beta(const double* betas_host, int32_t n, double beta) {
  if (!betas_host || n < 1 || !(beta > 0.0)) return -1;
  int best = -1;
  double bd = 0.0;
  for (int k = 0; k < n; ++k) {
    if (!(betas_host[k] > 0.0)) return -1;
    const double d = fabs(log(betas_host[k]) - log(beta));
    if (best < 0 || d < bd) { best = k; bd = d; }
  }
  return best;
}
