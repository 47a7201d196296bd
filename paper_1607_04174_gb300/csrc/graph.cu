// Image graph (Sec. II-A, Eq. W), degrees, the normalized Laplacian's coefficients
// (Sec. II-C) and the matrix-free Laplacian apply on node-major N x k blocks.
#include "rw_internal.cuh"

#include <algorithm>

#include <cstdio>
#include <cstring>
#include <new>

// ---------------------------------------------------------------------------------------
// Eq. (W): one thread per voxel computes its forward-edge weights (stored), recomputes its
// backward-edge weights (not stored) and sums all of them into the degree d_i = sum_j w_ij.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ float edge_w(float a, float b, float beta, int form) {
  float t = a - b;
  return form == RW_WEIGHT_SQ ? expf(-beta * t * t) : expf(-beta * fabsf(t));
}

__global__ void k_build_weights(const float* __restrict__ J, int64_t N, int ndim, int X, int Y,
                                int Z, float beta, int form, int normalized,
                                float* __restrict__ w, float* __restrict__ d,
                                float* __restrict__ s, float* __restrict__ sq, int* status) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int64_t st[3] = {1, (int64_t)X, (int64_t)X * Y};
  const int c[3] = {(int)(i % X), (int)((i / X) % Y), (int)(i / ((int64_t)X * Y))};
  const int n[3] = {X, Y, Z};
  float Ji = J[i];
  if (!isfinite(Ji)) atomicOr(status, RW_DEV_NONFINITE);
  float deg = 0.f;
  for (int a = 0; a < ndim; ++a) {
    float wf = 0.f;
    if (c[a] + 1 < n[a]) {
      wf = edge_w(Ji, J[i + st[a]], beta, form);
      deg += wf;
    }
    w[a * N + i] = wf;
    if (c[a] > 0) deg += edge_w(J[i - st[a]], Ji, beta, form);
  }
  d[i] = deg;
  if (normalized) {
    if (!(deg > 0.f)) {
      atomicOr(status, RW_DEV_ISOLATED);
      s[i] = 0.f;
      sq[i] = 0.f;
    } else {
      float r = sqrtf(deg);
      sq[i] = r;
      s[i] = 1.f / r;
    }
  } else {
    s[i] = 1.f;
    sq[i] = 1.f;
  }
}

// degrees (and scalings) from stored per-axis weights, for voxels flagged in `mark` (or all)
__global__ void k_degree_from_w(const float* __restrict__ w, int64_t N, int ndim, int X, int Y,
                                int Z, int normalized, const uint8_t* __restrict__ mark,
                                float* __restrict__ d, float* __restrict__ s,
                                float* __restrict__ sq, int* status) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  if (mark && !mark[i]) return;
  const int64_t st[3] = {1, (int64_t)X, (int64_t)X * Y};
  const int c[3] = {(int)(i % X), (int)((i / X) % Y), (int)(i / ((int64_t)X * Y))};
  float deg = 0.f;
  for (int a = 0; a < ndim; ++a) {
    deg += w[a * N + i];  // 0 at the border
    if (c[a] > 0) deg += w[a * N + i - st[a]];
  }
  d[i] = deg;
  if (normalized) {
    if (!(deg > 0.f)) {
      atomicOr(status, RW_DEV_ISOLATED);
      s[i] = 0.f;
      sq[i] = 0.f;
    } else {
      float r = sqrtf(deg);
      sq[i] = r;
      s[i] = 1.f / r;
    }
  } else {
    s[i] = 1.f;
    sq[i] = 1.f;
  }
  (void)Z;
}

// operator coefficient of each forward edge: w_e s_a s_b (L-hat) or w_e (L)
__global__ void k_coeffs(const float* __restrict__ w, const float* __restrict__ s, int64_t N,
                         int ndim, int X, int Y, int normalized, float* __restrict__ cw) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int64_t st[3] = {1, (int64_t)X, (int64_t)X * Y};
  for (int a = 0; a < ndim; ++a) {
    float we = w[a * N + i];
    float c = we;
    if (normalized && we != 0.f) c = we * s[i] * s[i + st[a]];
    cw[a * N + i] = c;
  }
}

rw_status rw_graph_coeffs(rw_graph* g, cudaStream_t st) {
  k_coeffs<<<rw_blocks(g->N, 256), 256, 0, st>>>(g->w, g->s, g->N, g->ndim, g->dims[0],
                                                  g->dims[1], g->normalized, g->cw);
  RW_LAUNCH_CHECK();
  return RW_OK;
}

// ---------------------------------------------------------------------------------------
// Stencil Y = alpha * (Op X) + beta * X + gamma * Zm on an N x k node-major block, where
// Op = L-hat (normalized: (Op x)_i = x_i - sum_j c_ij x_j, c_ij = w_ij s_i s_j) or
// Op = L ((Op x)_i = d_i x_i - sum_j w_ij x_j).  One warp walks a run of voxels along x with
// a register window (left, centre, right rows); the y/z neighbour rows come through L1/L2.
// Each lane owns float4 chunks lane, lane+32, ... of a row (CH chunks).
// ---------------------------------------------------------------------------------------
template <int CH>
__device__ __forceinline__ void ld_row(float4 (&r)[CH], const float* __restrict__ base,
                                       int nch, int lane) {
#pragma unroll
  for (int t = 0; t < CH; ++t) {
    int c = lane + 32 * t;
    r[t] = (c < nch) ? __ldg(reinterpret_cast<const float4*>(base) + c)
                     : make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

template <int CH>
__device__ __forceinline__ void fms_row(float4 (&acc)[CH], float c, const float4 (&r)[CH]) {
#pragma unroll
  for (int t = 0; t < CH; ++t) {
    acc[t].x = fmaf(-c, r[t].x, acc[t].x);
    acc[t].y = fmaf(-c, r[t].y, acc[t].y);
    acc[t].z = fmaf(-c, r[t].z, acc[t].z);
    acc[t].w = fmaf(-c, r[t].w, acc[t].w);
  }
}

template <int CH>
__global__ void __launch_bounds__(256)
k_stencil_wide(const float* __restrict__ X, int64_t ldx, float* __restrict__ Y, int64_t ldy,
               int nch, const float* __restrict__ cw, const float* __restrict__ dg,
               int normalized, int ndim, int DX, int DY, int DZ, int64_t N, int run,
               float alpha, float beta, const float* __restrict__ Zm, int64_t ldz,
               float gamma) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int segs = (DX + run - 1) / run;
  const int64_t total = (int64_t)DY * DZ * segs;
  if (warp >= total) return;
  const int64_t row = warp / segs;
  const int x0 = (int)(warp % segs) * run;
  const int x1 = min(x0 + run, DX);
  const int y = (int)(row % DY), z = (int)(row / DY);
  const int64_t base = row * DX;
  const int64_t sy = DX, sz = (int64_t)DX * DY;
  float4 prv[CH], cur[CH], nxt[CH];
  if (x0 > 0) ld_row<CH>(prv, X + (base + x0 - 1) * ldx, nch, lane);
  ld_row<CH>(cur, X + (base + x0) * ldx, nch, lane);
  for (int x = x0; x < x1; ++x) {
    const int64_t i = base + x;
    if (x + 1 < DX) ld_row<CH>(nxt, X + (i + 1) * ldx, nch, lane);
    float4 acc[CH];
    const float dd = normalized ? 1.f : __ldg(dg + i);
#pragma unroll
    for (int t = 0; t < CH; ++t)
      acc[t] = make_float4(dd * cur[t].x, dd * cur[t].y, dd * cur[t].z, dd * cur[t].w);
    if (x > 0) fms_row<CH>(acc, __ldg(cw + i - 1), prv);
    if (x + 1 < DX) fms_row<CH>(acc, __ldg(cw + i), nxt);
    {
      float4 r[CH];
      if (y > 0) {
        ld_row<CH>(r, X + (i - sy) * ldx, nch, lane);
        fms_row<CH>(acc, __ldg(cw + N + i - sy), r);
      }
      if (y + 1 < DY) {
        ld_row<CH>(r, X + (i + sy) * ldx, nch, lane);
        fms_row<CH>(acc, __ldg(cw + N + i), r);
      }
      if (ndim == 3) {
        if (z > 0) {
          ld_row<CH>(r, X + (i - sz) * ldx, nch, lane);
          fms_row<CH>(acc, __ldg(cw + 2 * N + i - sz), r);
        }
        if (z + 1 < DZ) {
          ld_row<CH>(r, X + (i + sz) * ldx, nch, lane);
          fms_row<CH>(acc, __ldg(cw + 2 * N + i), r);
        }
      }
    }
    float4* yo = reinterpret_cast<float4*>(Y + i * ldy);
    const float4* zi = Zm ? reinterpret_cast<const float4*>(Zm + i * ldz) : nullptr;
#pragma unroll
    for (int t = 0; t < CH; ++t) {
      int c = lane + 32 * t;
      if (c < nch) {
        float4 o;
        o.x = alpha * acc[t].x + beta * cur[t].x;
        o.y = alpha * acc[t].y + beta * cur[t].y;
        o.z = alpha * acc[t].z + beta * cur[t].z;
        o.w = alpha * acc[t].w + beta * cur[t].w;
        if (zi) {
          float4 zz = __ldg(zi + c);
          o.x += gamma * zz.x; o.y += gamma * zz.y; o.z += gamma * zz.z; o.w += gamma * zz.w;
        }
        yo[c] = o;
      }
    }
#pragma unroll
    for (int t = 0; t < CH; ++t) { prv[t] = cur[t]; cur[t] = nxt[t]; }
  }
}

// Grid graphs, the bandwidth-bound default: one thread per (x, float4 chunk) column of a
// segment of RY consecutive rows along y.  Threads of a row of voxels are consecutive (chunk
// fastest), so a warp reads 512 contiguous bytes of X per access.  The thread marches along y
// keeping rows y - 1, y, y + 1 in registers and loading two rows ahead, so per output it reads
// one new row (the first touch from DRAM) plus the x neighbours (L1: the neighbouring threads'
// rows) and the z neighbours (L2); the earlier one-output-per-thread form also read both y
// neighbours from L2 and was 11-33% slower.
template <int RY>
__global__ void __launch_bounds__(256)
k_stencil_yroll(const float* __restrict__ X, int64_t ldx, float* __restrict__ Y, int64_t ldy,
                int nch, const float* __restrict__ cw, const float* __restrict__ dg,
                int normalized, int ndim, int DX, int DY, int DZ, int64_t N, float alpha,
                float beta, const float* __restrict__ Zm, int64_t ldz, float gamma) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= DX * nch) return;
  const int x = t / nch, c = t - x * nch;
  const int y0 = blockIdx.y * RY, y1 = min(DY, y0 + RY), z = blockIdx.z;
  const int64_t sy = DX, sz = (int64_t)DX * DY;
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  auto ld = [&](int64_t j) { return __ldg(reinterpret_cast<const float4*>(X + j * ldx) + c); };
  const int64_t ib = x + sz * z;
  float4 prv = y0 > 0 ? ld(ib + sy * (y0 - 1)) : zero;
  float4 cur = ld(ib + sy * y0);
  float4 nx1 = y0 + 1 < DY ? ld(ib + sy * (y0 + 1)) : zero;
  float4 nx2 = y0 + 2 < DY ? ld(ib + sy * (y0 + 2)) : zero;
  const bool hx0 = x > 0, hx1 = x + 1 < DX;
  const bool hz0 = ndim == 3 && z > 0, hz1 = ndim == 3 && z + 1 < DZ;
  for (int y = y0; y < y1; ++y) {
    const int64_t i = ib + sy * y;
    const float4 vx0 = hx0 ? ld(i - 1) : zero, vx1 = hx1 ? ld(i + 1) : zero;
    const float4 vz0 = hz0 ? ld(i - sz) : zero, vz1 = hz1 ? ld(i + sz) : zero;
    // two rows ahead (the window's last row is y1, the segment's lower neighbour)
    const float4 nx3 = (y + 3 < DY && y + 3 <= y1) ? ld(i + 3 * sy) : zero;
    const float cx0 = hx0 ? __ldg(cw + i - 1) : 0.f, cx1 = hx1 ? __ldg(cw + i) : 0.f;
    const float cy0 = y > 0 ? __ldg(cw + N + i - sy) : 0.f;
    const float cy1 = y + 1 < DY ? __ldg(cw + N + i) : 0.f;
    const float cz0 = hz0 ? __ldg(cw + 2 * N + i - sz) : 0.f;
    const float cz1 = hz1 ? __ldg(cw + 2 * N + i) : 0.f;
    const float dd = normalized ? 1.f : __ldg(dg + i);
    auto lap = [&](float o, float a0, float a1, float b0, float b1, float e0, float e1) {
      float acc = dd * o;
      acc = fmaf(-cx0, a0, acc); acc = fmaf(-cx1, a1, acc);
      acc = fmaf(-cy0, b0, acc); acc = fmaf(-cy1, b1, acc);
      acc = fmaf(-cz0, e0, acc); acc = fmaf(-cz1, e1, acc);
      return alpha * acc + beta * o;
    };
    float4 out;
    out.x = lap(cur.x, vx0.x, vx1.x, prv.x, nx1.x, vz0.x, vz1.x);
    out.y = lap(cur.y, vx0.y, vx1.y, prv.y, nx1.y, vz0.y, vz1.y);
    out.z = lap(cur.z, vx0.z, vx1.z, prv.z, nx1.z, vz0.z, vz1.z);
    out.w = lap(cur.w, vx0.w, vx1.w, prv.w, nx1.w, vz0.w, vz1.w);
    if (Zm) {
      const float4 zz = __ldg(reinterpret_cast<const float4*>(Zm + i * ldz) + c);
      out.x = fmaf(gamma, zz.x, out.x); out.y = fmaf(gamma, zz.y, out.y);
      out.z = fmaf(gamma, zz.z, out.z); out.w = fmaf(gamma, zz.w, out.w);
    }
    reinterpret_cast<float4*>(Y + i * ldy)[c] = out;
    prv = cur; cur = nx1; nx1 = nx2; nx2 = nx3;
  }
}

// general (CSR) graph: one warp per row
template <int CH>
__global__ void __launch_bounds__(256)
k_stencil_csr(const float* __restrict__ X, int64_t ldx, float* __restrict__ Y, int64_t ldy,
              int nch, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
              const float* __restrict__ cc, const float* __restrict__ dg, int normalized,
              int64_t N, float alpha, float beta, const float* __restrict__ Zm, int64_t ldz,
              float gamma) {
  const int lane = threadIdx.x & 31;
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (i >= N) return;
  float4 cur[CH], acc[CH];
  ld_row<CH>(cur, X + i * ldx, nch, lane);
  const float dd = normalized ? 1.f : dg[i];
#pragma unroll
  for (int t = 0; t < CH; ++t)
    acc[t] = make_float4(dd * cur[t].x, dd * cur[t].y, dd * cur[t].z, dd * cur[t].w);
  for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) {
    float4 r[CH];
    ld_row<CH>(r, X + (int64_t)col[p] * ldx, nch, lane);
    fms_row<CH>(acc, cc[p], r);
  }
  float4* yo = reinterpret_cast<float4*>(Y + i * ldy);
  const float4* zi = Zm ? reinterpret_cast<const float4*>(Zm + i * ldz) : nullptr;
#pragma unroll
  for (int t = 0; t < CH; ++t) {
    int c = lane + 32 * t;
    if (c < nch) {
      float4 o;
      o.x = alpha * acc[t].x + beta * cur[t].x;
      o.y = alpha * acc[t].y + beta * cur[t].y;
      o.z = alpha * acc[t].z + beta * cur[t].z;
      o.w = alpha * acc[t].w + beta * cur[t].w;
      if (zi) {
        float4 zz = zi[c];
        o.x += gamma * zz.x; o.y += gamma * zz.y; o.z += gamma * zz.z; o.w += gamma * zz.w;
      }
      yo[c] = o;
    }
  }
}

template <int CH>
static void launch_wide(const rw_graph* g, const float* X, int64_t ldx, float* Y, int64_t ldy,
                        int nch, float alpha, float beta, const float* Z, int64_t ldz,
                        float gamma, cudaStream_t st) {
  if (g->kind == RW_GRAPH_CSR) {
    k_stencil_csr<CH><<<rw_blocks(g->N * 32, 256), 256, 0, st>>>(
        X, ldx, Y, ldy, nch, g->rowptr, g->col, g->ccsr, g->d, g->normalized, g->N, alpha,
        beta, Z, ldz, gamma);
    return;
  }
  const int run = 16;
  const int segs = (g->dims[0] + run - 1) / run;
  const int64_t warps = (int64_t)g->dims[1] * g->dims[2] * segs;
  k_stencil_wide<CH><<<rw_blocks(warps * 32, 256), 256, 0, st>>>(
      X, ldx, Y, ldy, nch, g->cw, g->d, g->normalized, g->ndim, g->dims[0], g->dims[1],
      g->dims[2], g->N, run, alpha, beta, Z, ldz, gamma);
}

rw_status rw_stencil_apply(const rw_graph* g, const float* X, int64_t ldx, float* Y,
                           int64_t ldy, int k, float alpha, float beta, const float* Z,
                           int64_t ldz, float gamma, cudaStream_t st) {
  if (k <= 0 || k > 1024) return RW_ERR_INVALID_ARG;
  const int nch = (k + 3) / 4;
  if (g->kind == RW_GRAPH_GRID && (int64_t)g->dims[0] * nch < ((int64_t)1 << 31) &&
      g->dims[2] <= 65535) {
    // segments of 8 rows (2-D) / 16 rows (3-D): the fastest in a sweep on GB300
    const int ry = g->ndim == 3 ? 16 : 8;
    const dim3 grid(rw_blocks((int64_t)g->dims[0] * nch, 256),
                    (unsigned)((g->dims[1] + ry - 1) / ry), (unsigned)g->dims[2]);
    if (ry == 16)
      k_stencil_yroll<16><<<grid, 256, 0, st>>>(X, ldx, Y, ldy, nch, g->cw, g->d, g->normalized,
                                                 g->ndim, g->dims[0], g->dims[1], g->dims[2],
                                                 g->N, alpha, beta, Z, ldz, gamma);
    else
      k_stencil_yroll<8><<<grid, 256, 0, st>>>(X, ldx, Y, ldy, nch, g->cw, g->d, g->normalized,
                                                g->ndim, g->dims[0], g->dims[1], g->dims[2],
                                                g->N, alpha, beta, Z, ldz, gamma);
    RW_LAUNCH_CHECK();
    return RW_OK;
  }
  const int ch = (nch + 31) / 32;
  switch (ch) {
    case 1: launch_wide<1>(g, X, ldx, Y, ldy, nch, alpha, beta, Z, ldz, gamma, st); break;
    case 2: launch_wide<2>(g, X, ldx, Y, ldy, nch, alpha, beta, Z, ldz, gamma, st); break;
    case 3: launch_wide<3>(g, X, ldx, Y, ldy, nch, alpha, beta, Z, ldz, gamma, st); break;
    case 4: launch_wide<4>(g, X, ldx, Y, ldy, nch, alpha, beta, Z, ldz, gamma, st); break;
    case 5: launch_wide<5>(g, X, ldx, Y, ldy, nch, alpha, beta, Z, ldz, gamma, st); break;
    case 6: launch_wide<6>(g, X, ldx, Y, ldy, nch, alpha, beta, Z, ldz, gamma, st); break;
    case 7: launch_wide<7>(g, X, ldx, Y, ldy, nch, alpha, beta, Z, ldz, gamma, st); break;
    default: launch_wide<8>(g, X, ldx, Y, ldy, nch, alpha, beta, Z, ldz, gamma, st); break;
  }
  RW_LAUNCH_CHECK();
  return RW_OK;
}

// The update scratch (`upd`) holds small per-call arrays at fixed offsets (priors fit at 0,
// PCG iteration count at 4096, degree sum at 6144, column norms at 8192) and per-block
// partial sums from 16384 on.  It is sized once here so no call ever reallocates it while
// holding a pointer into it.
rw_status rw_graph_reserve_scratch(rw_graph* g) {
  const int sms = g_rw_num_sms > 0 ? g_rw_num_sms : 148;
  return g->upd.grow(16384 + sizeof(double) * (size_t)2 * sms * 1024 + 4096);
}

// ---------------------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------------------
static void graph_release(rw_graph* g) {
  if (!g) return;
  cudaFree(g->J); cudaFree(g->w); cudaFree(g->cw); cudaFree(g->d); cudaFree(g->s);
  cudaFree(g->sq); cudaFree(g->status); cudaFree(g->rowptr); cudaFree(g->col);
  cudaFree(g->wcsr); cudaFree(g->ccsr);
  g->ws.seedlab.release(); g->ws.seedpart.release(); g->ws.small.release(); g->ws.xhat[0].release();
  g->ws.xhat[1].release(); g->ws.phat.release(); g->ws.pcg.release(); g->ws.stage.release(); g->ws.grad.release(); g->ws.reg.release(); g->ws.host.release();
  for (auto& e : g->ws.ev) if (e) cudaEventDestroy(e);
  g->upd.release();
  delete g;
}

extern "C" void rw_graph_free(rw_graph* g) { graph_release(g); }

extern "C" int64_t rw_graph_num_nodes(const rw_graph* g) { return g ? g->N : 0; }

extern "C" rw_status rw_build_graph(const rw_graph_desc* desc, const float* J_dev, void* stream,
                                    rw_graph** out) {
  if (!desc || !J_dev || !out) return RW_ERR_INVALID_ARG;
  *out = nullptr;
  if (desc->ndim != 2 && desc->ndim != 3) return RW_ERR_INVALID_ARG;
  if (!(desc->beta >= 0.0)) return RW_ERR_INVALID_ARG;
  if (desc->weight_form != RW_WEIGHT_SQ && desc->weight_form != RW_WEIGHT_ABS)
    return RW_ERR_INVALID_ARG;
  int dz = desc->ndim == 3 ? desc->dims[2] : 1;
  if (desc->dims[0] < 1 || desc->dims[1] < 1 || dz < 1) return RW_ERR_INVALID_ARG;
  int64_t N = (int64_t)desc->dims[0] * desc->dims[1] * dz;
  if (N > 0x7fffffffLL) return RW_ERR_INVALID_ARG;
  RW_TRY(rw_device_init());
  cudaStream_t st = rw_stream(stream);
  rw_graph* g = new (std::nothrow) rw_graph();
  if (!g) return RW_ERR_OOM;
  if (cudaGetDevice(&g->device) != cudaSuccess) g->device = 0;
  g->kind = RW_GRAPH_GRID;
  g->ndim = desc->ndim;
  g->dims[0] = desc->dims[0]; g->dims[1] = desc->dims[1]; g->dims[2] = dz;
  g->N = N;
  g->stride[0] = 1; g->stride[1] = g->dims[0]; g->stride[2] = (int64_t)g->dims[0] * g->dims[1];
  g->beta = desc->beta;
  g->form = desc->weight_form;
  g->normalized = desc->normalized ? 1 : 0;
  auto fail = [&](rw_status s) { graph_release(g); return s; };
  if (cudaMalloc(&g->J, N * 4) != cudaSuccess || cudaMalloc(&g->w, g->ndim * N * 4) != cudaSuccess ||
      cudaMalloc(&g->cw, g->ndim * N * 4) != cudaSuccess || cudaMalloc(&g->d, N * 4) != cudaSuccess ||
      cudaMalloc(&g->s, N * 4) != cudaSuccess || cudaMalloc(&g->sq, N * 4) != cudaSuccess ||
      cudaMalloc(&g->status, sizeof(int)) != cudaSuccess)
    return fail(RW_ERR_OOM);
  if (cudaMemcpyAsync(g->J, J_dev, N * 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
      cudaMemsetAsync(g->status, 0, sizeof(int), st) != cudaSuccess)
    return fail(RW_ERR_CUDA);
  k_build_weights<<<rw_blocks(N, 256), 256, 0, st>>>(g->J, N, g->ndim, g->dims[0], g->dims[1],
                                                     g->dims[2], (float)g->beta, g->form,
                                                     g->normalized, g->w, g->d, g->s, g->sq,
                                                     g->status);
  if (cudaGetLastError() != cudaSuccess) return fail(RW_ERR_CUDA);
  if (rw_graph_coeffs(g, st) != RW_OK) return fail(RW_ERR_CUDA);
  int bits = 0;
  if (cudaMemcpyAsync(&bits, g->status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return fail(RW_ERR_CUDA);
  if (bits) {
    rw_status s = rw_status_from_device_bits(bits);
    return fail(s);
  }
  if (rw_graph_reserve_scratch(g) != RW_OK) return fail(RW_ERR_OOM);
  if (rw_graph_degree_sum(g, st) != RW_OK) return fail(RW_ERR_CUDA);
  *out = g;
  return RW_OK;
}

extern "C" rw_status rw_graph_weights(const rw_graph* g, float* w_dev, float* d_dev,
                                      void* stream) {
  if (!g) return RW_ERR_INVALID_ARG;
  cudaStream_t st = rw_stream(stream);
  if (w_dev) {
    if (g->kind != RW_GRAPH_GRID) return RW_ERR_UNSUPPORTED;
    RW_CHECK_CUDA(cudaMemcpyAsync(w_dev, g->w, g->ndim * g->N * 4, cudaMemcpyDeviceToDevice, st));
  }
  if (d_dev) RW_CHECK_CUDA(cudaMemcpyAsync(d_dev, g->d, g->N * 4, cudaMemcpyDeviceToDevice, st));
  return RW_OK;
}

extern "C" rw_status rw_apply_laplacian(const rw_graph* g, const float* X_dev, int64_t ldx,
                                        float* Y_dev, int64_t ldy, int32_t k, void* stream) {
  if (!g || !X_dev || !Y_dev || k < 1 || k > 1024) return RW_ERR_INVALID_ARG;
  if (ldx < k || ldy < k || (ldx & 3) || (ldy & 3)) return RW_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(X_dev) & 15) || (reinterpret_cast<uintptr_t>(Y_dev) & 15))
    return RW_ERR_INVALID_ARG;
  if (rw_round_up(k, 4) > ldx || rw_round_up(k, 4) > ldy) return RW_ERR_INVALID_ARG;
  return rw_stencil_apply(g, X_dev, ldx, Y_dev, ldy, k, 1.f, 0.f, nullptr, 0, 0.f,
                          rw_stream(stream));
}

// every weight from a caller array in edge-id layout (slots without an edge are ignored and
// stored as 0); a negative or non-finite weight sets RW_DEV_NONFINITE
__global__ void k_set_all_weights(const float* __restrict__ src, int64_t N, int ndim, int X,
                                  int Y, int Z, float* __restrict__ w, int* status) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ndim * N) return;
  const int a = (int)(e / N);
  const int64_t i = e % N;
  const int c = a == 0 ? (int)(i % X) : (a == 1 ? (int)((i / X) % Y) : (int)(i / ((int64_t)X * Y)));
  const int n = a == 0 ? X : (a == 1 ? Y : Z);
  float v = 0.f;
  if (c + 1 < n) {
    v = src[e];
    if (!(v >= 0.f) || !isfinite(v)) { atomicOr(status, RW_DEV_NONFINITE); v = 0.f; }
  }
  w[e] = v;
}

rw_status rw_set_all_weights(rw_graph* g, const float* w_dev, cudaStream_t st) {
  if (g->kind != RW_GRAPH_GRID || !w_dev) return RW_ERR_INVALID_ARG;
  k_set_all_weights<<<rw_blocks(g->ndim * g->N, 256), 256, 0, st>>>(
      w_dev, g->N, g->ndim, g->dims[0], g->dims[1], g->dims[2], g->w, g->status);
  RW_LAUNCH_CHECK();
  k_degree_from_w<<<rw_blocks(g->N, 256), 256, 0, st>>>(g->w, g->N, g->ndim, g->dims[0],
                                                        g->dims[1], g->dims[2], g->normalized,
                                                        nullptr, g->d, g->s, g->sq, g->status);
  RW_LAUNCH_CHECK();
  RW_TRY(rw_graph_coeffs(g, st));
  int bits = 0;
  RW_CHECK_CUDA(cudaMemcpyAsync(&bits, g->status, sizeof(int), cudaMemcpyDeviceToHost, st));
  RW_CHECK_CUDA(cudaMemsetAsync(g->status, 0, sizeof(int), st));
  RW_CHECK_CUDA(cudaStreamSynchronize(st));
  if (bits) return rw_status_from_device_bits(bits);
  return rw_graph_degree_sum(g, st);
}

// new beta for every edge: weights, degrees, scalings, coefficients, degree sum
rw_status rw_build_weights_again(rw_graph* g, double beta, cudaStream_t st) {
  if (g->kind != RW_GRAPH_GRID || !g->J) return RW_ERR_INVALID_ARG;
  g->beta = beta;
  k_build_weights<<<rw_blocks(g->N, 256), 256, 0, st>>>(g->J, g->N, g->ndim, g->dims[0],
                                                        g->dims[1], g->dims[2], (float)beta,
                                                        g->form, g->normalized, g->w, g->d,
                                                        g->s, g->sq, g->status);
  RW_LAUNCH_CHECK();
  RW_TRY(rw_graph_coeffs(g, st));
  int bits = 0;
  RW_CHECK_CUDA(cudaMemcpyAsync(&bits, g->status, sizeof(int), cudaMemcpyDeviceToHost, st));
  RW_CHECK_CUDA(cudaMemsetAsync(g->status, 0, sizeof(int), st));
  RW_CHECK_CUDA(cudaStreamSynchronize(st));
  if (bits) return rw_status_from_device_bits(bits);
  return rw_graph_degree_sum(g, st);
}
