// Basic random walker on the GPU: Eq. (rw_eq) in the normalized form of Sec. II-C,
//   (L-hat_n + gamma I) U-hat_n = gamma P-hat_n - B-hat^T U-hat_s,
// solved by Jacobi-preconditioned CG, every label column with its own recurrence, all columns
// in one persistent cooperative kernel.  An iteration is two passes over the voxels separated
// by grid-wide barriers:
//   pass A: p <- z + beta p (z = r / a_ii, recomputed for the neighbours from r and the previous
//           p, so no separate p pass is needed; p is double-buffered), q = A p, partial p.q;
//   pass B: x += alpha p, r -= alpha q, partial r.z and r.r.
// Seeded rows keep r = p = q = 0, so pass B needs no seed test and neighbours need none.
// Dot products: FP32 per thread, FP64 per block in a fixed order, block partials written to
// global memory and summed by every block in the same fixed order after the barrier (no
// atomics; every block holds bit-identical step lengths).
// Grid graphs walk row tiles (one division per tile); the 2-D working set stays in L2.
#include "rw_internal.cuh"

#include <cooperative_groups.h>

#include <algorithm>

namespace cg = cooperative_groups;

namespace {

constexpr int kPcgThreads = 512;
constexpr int kPcgWarps = kPcgThreads / 32;

struct PcgArgs {
  // graph
  int kind, ndim, DX, DY, DZ, normalized;
  int64_t N;
  const float* cw;
  const float* d;
  const float* s;
  const float* sq;
  const int32_t* rowptr;
  const int32_t* col;
  const float* ccsr;
  // problem
  const float* phat;    // N x lp (hat priors), used when bexp == nullptr
  const float* bexp;    // N x lp explicit right-hand side (hat space), or nullptr
  const int* seedlab;   // N
  int L;
  float gamma;
  // state (N x lp each; p double-buffered)
  float *x, *r, *p0, *p1, *q;
  double* part;              // [gridDim][3 * lp] block partials
  int iters;
  double tol;
  int start_zero;
  int* iters_done;
  float* U;                  // output N x L (or nullptr: leave x in hat space)
  uint8_t* labels;
  int unscale_out;           // 1: U = s * x; 0: U = x
};

template <int LP>
struct V {
  float4 v[LP / 4];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int t = 0; t < LP / 4; ++t) v[t] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  __device__ __forceinline__ void load(const float* base, int64_t i) {
    const float4* b = reinterpret_cast<const float4*>(base) + i * (LP / 4);
#pragma unroll
    for (int t = 0; t < LP / 4; ++t) v[t] = b[t];
  }
  __device__ __forceinline__ void store(float* base, int64_t i) const {
    float4* b = reinterpret_cast<float4*>(base) + i * (LP / 4);
#pragma unroll
    for (int t = 0; t < LP / 4; ++t) b[t] = v[t];
  }
  __device__ __forceinline__ float& operator[](int k) { return reinterpret_cast<float*>(v)[k]; }
  __device__ __forceinline__ float operator[](int k) const {
    return reinterpret_cast<const float*>(v)[k];
  }
};

// Visits every voxel once over the whole grid.  Grid graphs: a tile is a segment of one row
// (rows wider than the block) or R = blockDim / DX whole rows (narrower rows), so no more than
// DX - 1 threads of a block idle; y and z come from one division per tile.  CSR graphs:
// grid-stride over i.  f(i, x, y, z, valid); every thread of a block takes the same trips.
__host__ __device__ __forceinline__ int64_t pcg_grid_tiles(int DX, int64_t rows, int threads) {
  if (DX >= threads) return rows * ((DX + threads - 1) / threads);
  const int R = threads / DX;
  return (rows + R - 1) / R;
}

template <typename F>
__device__ __forceinline__ void for_nodes(const PcgArgs& a, F&& f) {
  if (a.kind == RW_GRAPH_GRID) {
    // 32-bit tile arithmetic (rows = DY * DZ < 2^31, checked at launch)
    const int B = blockDim.x;
    const int rows = a.DY * a.DZ;
    const int tiles = (int)pcg_grid_tiles(a.DX, rows, B);
    const bool wide = a.DX >= B;
    const int chunks = wide ? (a.DX + B - 1) / B : 1;   // tiles per row (wide rows)
    const int R = wide ? 1 : B / a.DX;                  // rows per tile (narrow rows)
    const int ry = wide ? 0 : (int)threadIdx.x / a.DX;
    const int xoff = (int)threadIdx.x - ry * a.DX;
    for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
      const int tr = t / chunks;
      const int row = tr * R + ry;
      const int x = (t - tr * chunks) * B + xoff;
      const bool ok = ry < R && row < rows && x < a.DX;
      const int rr = ok ? row : 0;
      const int z = rr / a.DY, y = rr - z * a.DY;
      f(ok ? x + (int64_t)a.DX * rr : 0, x, y, z, ok);
    }
  } else {
    const int64_t nth = (int64_t)gridDim.x * blockDim.x;
    const int64_t span = (a.N + nth - 1) / nth * nth;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < span; i += nth)
      f(i, 0, 0, 0, i < a.N);
  }
}

// acc += sum over the neighbours j of i of c_ij * v(j), v(j) an N x LP row functor
template <int LP, typename G>
__device__ __forceinline__ void nbr_acc(const PcgArgs& a, int64_t i, int x, int y, int z,
                                        G&& vrow, V<LP>& acc) {
  auto add = [&](int64_t j, float c) {
    const V<LP> v = vrow(j);
#pragma unroll
    for (int k = 0; k < LP; ++k) acc[k] = fmaf(c, v[k], acc[k]);
  };
  if (a.kind == RW_GRAPH_GRID) {
    const int64_t N = a.N, sy = a.DX, sz = (int64_t)a.DX * a.DY;
    if (x > 0) add(i - 1, a.cw[i - 1]);
    if (x + 1 < a.DX) add(i + 1, a.cw[i]);
    if (y > 0) add(i - sy, a.cw[N + i - sy]);
    if (y + 1 < a.DY) add(i + sy, a.cw[N + i]);
    if (a.ndim == 3) {
      if (z > 0) add(i - sz, a.cw[2 * N + i - sz]);
      if (z + 1 < a.DZ) add(i + sz, a.cw[2 * N + i]);
    }
  } else {
    for (int e = a.rowptr[i]; e < a.rowptr[i + 1]; ++e) add(a.col[e], a.ccsr[e]);
  }
}

__device__ __forceinline__ float aii(const PcgArgs& a, int64_t i) {
  return (a.normalized ? 1.f : a.d[i]) + a.gamma;
}

// Block sum of NQ per-thread FP32 values in a fixed order, FP64 from the warp level up;
// quantity k goes to part[blockIdx.x * stride + off + k].
template <int NQ>
__device__ __forceinline__ void block_partials(const float (&v)[NQ], double* part, int stride,
                                               int off, double* sh) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NQ; ++k) {
    float t = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) sh[w * NQ + k] = (double)t;
  }
  __syncthreads();
  if (threadIdx.x < NQ) {
    double acc = 0.0;
    for (int ww = 0; ww < kPcgWarps; ++ww) acc += sh[ww * NQ + threadIdx.x];
    part[(size_t)blockIdx.x * stride + off + threadIdx.x] = acc;
  }
  __syncthreads();
}

// Totals of nq quantities over all block partials, in the same order in every block:
// warp k % warps sums quantity k (lane l takes blocks l, l + 32, ...), then a fixed xor tree.
__device__ __forceinline__ void grid_totals(const double* part, int stride, int off, int nq,
                                            double* out) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int k = w; k < nq; k += kPcgWarps) {
    double acc = 0.0;
    for (int b = lane; b < (int)gridDim.x; b += 32) acc += part[(size_t)b * stride + off + k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) out[k] = acc;
  }
  __syncthreads();
}

template <int LP>
__global__ void __launch_bounds__(kPcgThreads) k_pcg(PcgArgs a) {
  cg::grid_group grid = cg::this_grid();
  __shared__ double sh[kPcgWarps * 2 * LP];
  __shared__ double tot[2 * LP];
  // partial row of a block: [p.q | r.z | r.r] (the init writes r.z and b.b into the last two).
  // Pass A and pass B write disjoint parts, so a block may write its next partials while a
  // slower block still reads the previous pass's totals.
  const int stride = 3 * LP;
  const float g = a.gamma;

  // ---- init: seeded rows x = one-hot * d^{1/2}, r = p = q = 0; free rows x = 0 (zero start)
  for_nodes(a, [&](int64_t i, int, int, int, bool ok) {
    if (!ok) return;
    const int sl = a.seedlab[i];
    if (sl >= 0) {
      V<LP> xv, z;
      z.zero();
#pragma unroll
      for (int k = 0; k < LP; ++k) xv[k] = (k == sl) ? a.sq[i] : 0.f;
      xv.store(a.x, i);
      z.store(a.r, i); z.store(a.p0, i); z.store(a.p1, i); z.store(a.q, i);
    } else if (a.start_zero) {
      V<LP> z;
      z.zero();
      z.store(a.x, i);
    }
  });
  grid.sync();
  // r = b - A_n x_n, b = gamma p-hat + (coupling to the seeds) or the given right-hand side;
  // partial r.z and b.b
  {
    float pr[2 * LP];
#pragma unroll
    for (int k = 0; k < 2 * LP; ++k) pr[k] = 0.f;
    for_nodes(a, [&](int64_t i, int x, int y, int z, bool ok) {
      if (!ok || a.seedlab[i] >= 0) return;
      V<LP> nb, sn;
      nb.zero(); sn.zero();
      nbr_acc<LP>(a, i, x, y, z, [&](int64_t j) { V<LP> v; v.load(a.x, j); return v; }, nb);
      nbr_acc<LP>(a, i, x, y, z, [&](int64_t j) {
        V<LP> v;
        if (a.seedlab[j] >= 0) v.load(a.x, j); else v.zero();
        return v;
      }, sn);
      V<LP> xv, bv, pv;
      xv.load(a.x, i);
      if (a.bexp) bv.load(a.bexp, i);
      else {
        pv.load(a.phat, i);
#pragma unroll
        for (int k = 0; k < LP; ++k) bv[k] = fmaf(g, pv[k], sn[k]);
      }
      const float di = aii(a, i), inv = 1.f / di;
      V<LP> rv;
#pragma unroll
      for (int k = 0; k < LP; ++k) {
        rv[k] = bv[k] - di * xv[k] + (nb[k] - sn[k]);
        pr[k] = fmaf(rv[k] * inv, rv[k], pr[k]);
        pr[LP + k] = fmaf(bv[k], bv[k], pr[LP + k]);
      }
      rv.store(a.r, i);
    });
    block_partials<2 * LP>(pr, a.part, stride, LP, sh);
  }
  grid.sync();
  // every block holds the same totals: r.z and b.b per column, and the step lengths
  __shared__ double srz[LP], sbb[LP];
  __shared__ float salpha[LP], sbeta[LP];
  grid_totals(a.part, stride, LP, 2 * LP, tot);
  if (threadIdx.x < LP) {
    srz[threadIdx.x] = tot[threadIdx.x];
    sbb[threadIdx.x] = tot[LP + threadIdx.x];
    sbeta[threadIdx.x] = 0.f;
  }
  __syncthreads();

  int t = 0;
  for (; t < a.iters; ++t) {
    const float* pold = (t & 1) ? a.p1 : a.p0;
    float* pnew = (t & 1) ? a.p0 : a.p1;
    const bool first = (t == 0);
    // ---- pass A: p = z + beta p_old, q = A p, partial p.q
    {
      float beta[LP], ppq[LP];
#pragma unroll
      for (int k = 0; k < LP; ++k) { beta[k] = sbeta[k]; ppq[k] = 0.f; }
      auto prow = [&](int64_t j) {
        V<LP> rv, pv;
        rv.load(a.r, j);
        const float inv = 1.f / aii(a, j);
        if (first) {
#pragma unroll
          for (int k = 0; k < LP; ++k) pv[k] = rv[k] * inv;
        } else {
          pv.load(pold, j);
#pragma unroll
          for (int k = 0; k < LP; ++k) pv[k] = fmaf(beta[k], pv[k], rv[k] * inv);
        }
        return pv;
      };
      for_nodes(a, [&](int64_t i, int x, int y, int z, bool ok) {
        if (!ok || a.seedlab[i] >= 0) return;
        const V<LP> pv = prow(i);
        V<LP> nb;
        nb.zero();
        nbr_acc<LP>(a, i, x, y, z, prow, nb);
        const float di = aii(a, i);
        V<LP> qv;
#pragma unroll
        for (int k = 0; k < LP; ++k) {
          qv[k] = di * pv[k] - nb[k];
          ppq[k] = fmaf(pv[k], qv[k], ppq[k]);
        }
        pv.store(pnew, i);
        qv.store(a.q, i);
      });
      block_partials<LP>(ppq, a.part, stride, 0, sh);
    }
    grid.sync();
    grid_totals(a.part, stride, 0, LP, tot);
    if (threadIdx.x < LP) {
      const int k = threadIdx.x;
      salpha[k] = tot[k] > 0.0 ? (float)(srz[k] / tot[k]) : 0.f;
    }
    __syncthreads();
    // ---- pass B: x += alpha p, r -= alpha q, partial r.z and r.r
    {
      float alpha[LP], pr[2 * LP];
#pragma unroll
      for (int k = 0; k < LP; ++k) { alpha[k] = salpha[k]; pr[k] = 0.f; pr[LP + k] = 0.f; }
      for_nodes(a, [&](int64_t i, int, int, int, bool ok) {
        if (!ok) return;
        V<LP> xv, rv, pv, qv;
        xv.load(a.x, i); rv.load(a.r, i); pv.load(pnew, i); qv.load(a.q, i);
        const float inv = 1.f / aii(a, i);
#pragma unroll
        for (int k = 0; k < LP; ++k) {
          xv[k] = fmaf(alpha[k], pv[k], xv[k]);
          rv[k] = fmaf(-alpha[k], qv[k], rv[k]);
          pr[k] = fmaf(rv[k] * inv, rv[k], pr[k]);
          pr[LP + k] = fmaf(rv[k], rv[k], pr[LP + k]);
        }
        xv.store(a.x, i);
        rv.store(a.r, i);
      });
      block_partials<2 * LP>(pr, a.part, stride, LP, sh);
    }
    grid.sync();
    grid_totals(a.part, stride, LP, 2 * LP, tot);
    bool done = a.tol > 0.0;
    if (done)
      for (int k = 0; k < a.L; ++k)
        if (sbb[k] > 0.0 && tot[LP + k] > a.tol * a.tol * sbb[k]) done = false;
    __syncthreads();   // every thread has read sbb / tot before they change
    if (threadIdx.x < LP) {
      const int k = threadIdx.x;
      sbeta[k] = srz[k] > 0.0 ? (float)(tot[k] / srz[k]) : 0.f;
      srz[k] = tot[k];
    }
    __syncthreads();
    if (done) { ++t; break; }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && a.iters_done) *a.iters_done = t;
  if (a.U) {
    for_nodes(a, [&](int64_t i, int, int, int, bool ok) {
      if (!ok) return;
      const int sl = a.seedlab[i];
      V<LP> xv;
      xv.load(a.x, i);
      const float si = a.unscale_out ? a.s[i] : 1.f;
      int best = 0;
      float bv = -INFINITY;
      for (int k = 0; k < a.L; ++k) {
        const float u = (sl >= 0) ? (k == sl ? 1.f : 0.f) : xv[k] * si;
        a.U[i * a.L + k] = u;
        if (u > bv) { bv = u; best = k; }
      }
      if (a.labels) a.labels[i] = (uint8_t)best;
    });
  }
}

template <int LP>
rw_status launch_pcg(PcgArgs& a, const rw_graph* g, cudaStream_t st) {
  int per_sm = 0;
  RW_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg<LP>, kPcgThreads, 0));
  const int sms = g_rw_num_sms > 0 ? g_rw_num_sms : 148;
  const int64_t resident = (int64_t)sms * std::min(std::max(per_sm, 1), 2);
  // work items: row tiles (grid graphs) or thread-sized node groups (CSR); the block count is
  // the fewest that keeps the same number of trips per block
  if (g->kind == RW_GRAPH_GRID && (int64_t)g->dims[1] * g->dims[2] >= (int64_t)1 << 31)
    return RW_ERR_UNSUPPORTED;
  int64_t items = g->kind == RW_GRAPH_GRID
      ? pcg_grid_tiles(g->dims[0], (int64_t)g->dims[1] * g->dims[2], kPcgThreads)
      : (g->N + kPcgThreads - 1) / kPcgThreads;
  items = std::max<int64_t>(items, 1);
  const int64_t trips = (items + resident - 1) / resident;
  const int blocks = (int)std::max<int64_t>(1, (items + trips - 1) / trips);
  void* kargs[] = {&a};
  RW_CHECK_CUDA(cudaLaunchCooperativeKernel((void*)k_pcg<LP>, dim3(blocks), dim3(kPcgThreads),
                                            kargs, 0, st));
  rw_count_launch();
  return RW_OK;
}

}  // namespace

// Runs the cooperative PCG.  xhat0: N x lp start (hat space) or nullptr for a zero start.
rw_status rw_pcg_run(const rw_graph* g, const float* phat, const float* bexp, const int* seedlab,
                     int L, int lp, double gamma, const float* xhat0, int iters, double tol,
                     float* U, uint8_t* labels, int unscale_out, int* iters_done_dev,
                     float** x_out, cudaStream_t st) {
  if (lp != 4 && lp != 8 && lp != 16) return RW_ERR_INVALID_ARG;
  rw_graph* gm = const_cast<rw_graph*>(g);
  const size_t vec = sizeof(float) * (size_t)g->N * lp;
  const size_t stride = (vec + 255) & ~size_t(255);
  const int sms = g_rw_num_sms > 0 ? g_rw_num_sms : 148;
  const size_t part_bytes = sizeof(double) * 3 * 16 * (size_t)sms * 2;
  const size_t need = 5 * stride + part_bytes;
  RW_TRY(gm->ws.pcg.grow(std::max(gm->ws.pcg.cap, need)));
  char* base = gm->ws.pcg.as<char>();
  PcgArgs a{};
  a.kind = g->kind; a.ndim = g->ndim; a.DX = g->dims[0]; a.DY = g->dims[1]; a.DZ = g->dims[2];
  a.normalized = g->normalized; a.N = g->N; a.cw = g->cw; a.d = g->d; a.s = g->s; a.sq = g->sq;
  a.rowptr = g->rowptr; a.col = g->col; a.ccsr = g->ccsr;
  a.phat = phat; a.bexp = bexp; a.seedlab = seedlab; a.L = L; a.gamma = (float)gamma;
  a.x = reinterpret_cast<float*>(base);
  a.r = reinterpret_cast<float*>(base + stride);
  a.p0 = reinterpret_cast<float*>(base + 2 * stride);
  a.p1 = reinterpret_cast<float*>(base + 3 * stride);
  a.q = reinterpret_cast<float*>(base + 4 * stride);
  a.part = reinterpret_cast<double*>(base + 5 * stride);
  a.iters = iters; a.tol = tol; a.iters_done = iters_done_dev;
  a.U = U; a.labels = labels; a.unscale_out = unscale_out;
  a.start_zero = xhat0 ? 0 : 1;
  if (xhat0) RW_CHECK_CUDA(cudaMemcpyAsync(a.x, xhat0, vec, cudaMemcpyDeviceToDevice, st));
  switch (lp) {
    case 4: RW_TRY(launch_pcg<4>(a, g, st)); break;
    case 8: RW_TRY(launch_pcg<8>(a, g, st)); break;
    default: RW_TRY(launch_pcg<16>(a, g, st)); break;
  }
  if (x_out) *x_out = a.x;
  return RW_OK;
}

rw_status rw_pcg_from(const rw_graph* g, const float* phat, const int* seedlab, int L, int lp,
                      double gamma, float* xhat0, int iters, double tol, float* U,
                      uint8_t* labels, int* iters_done, cudaStream_t st) {
  (void)iters_done;
  return rw_pcg_run(g, phat, nullptr, seedlab, L, lp, gamma, xhat0, iters, tol, U, labels, 1,
                    nullptr, nullptr, st);
}


extern "C" rw_status rw_solve_pcg(const rw_graph* g, const int32_t* seed_idx_dev,
                                  const int32_t* seed_lab_dev, int32_t S, int32_t n_labels,
                                  const float* priors_dev, double gamma, int32_t prior_mode,
                                  int32_t iters, double tol, float* prob_dev,
                                  uint8_t* labels_dev, int32_t* iters_done, void* stream) {
  if (!g || !prob_dev) return RW_ERR_INVALID_ARG;
  if (S < 0 || S > 65536 || n_labels < 1 || n_labels > RW_MAX_LABELS) return RW_ERR_INVALID_ARG;
  if (S > 0 && (!seed_idx_dev || !seed_lab_dev)) return RW_ERR_INVALID_ARG;
  if (S == 0 && prior_mode != 1) return RW_ERR_INVALID_ARG;   // no seeds: priors are given
  if (!(gamma >= 0.0) || (gamma == 0.0 && S == 0)) return RW_ERR_INVALID_ARG;  // singular
  if (iters < 0) return RW_ERR_INVALID_ARG;
  if (gamma > 0.0 && ((prior_mode == 1 && !priors_dev) || (prior_mode == 0 && !g->J)))
    return RW_ERR_INVALID_ARG;
  cudaStream_t st = rw_stream(stream);
  const int lp = n_labels <= 4 ? 4 : (n_labels <= 8 ? 8 : 16);
  float* phat;
  int* seedlab;
  // gamma = 0: no priors (the P-hat term is gamma P-hat = 0; P-hat is zeroed so it is finite)
  RW_TRY(rw_solve_priors_internal(g, seed_idx_dev, seed_lab_dev, S, n_labels, prior_mode,
                                  priors_dev, lp, st, &phat, &seedlab, nullptr, gamma == 0.0));
  if (gamma == 0.0)
    RW_CHECK_CUDA(cudaMemsetAsync(phat, 0, sizeof(float) * g->N * lp, st));
  rw_graph* gm = const_cast<rw_graph*>(g);
  if (gm->upd.cap < 8192) return RW_ERR_OOM;
  int* it_dev = reinterpret_cast<int*>(gm->upd.as<char>() + 4096);
  RW_TRY(rw_pcg_run(g, phat, nullptr, seedlab, n_labels, lp, gamma, nullptr, iters, tol, prob_dev,
                    labels_dev, 1, it_dev, nullptr, st));
  if (iters_done) {
    int h = 0;
    RW_CHECK_CUDA(cudaMemcpyAsync(&h, it_dev, sizeof(int), cudaMemcpyDeviceToHost, st));
    RW_CHECK_CUDA(cudaStreamSynchronize(st));
    *iters_done = h;
    return rw_last_device_status(g, stream);
  }
  return RW_OK;
}

// P = P-hat / d^{1/2}, compacting the lp-padded rows to n_labels
__global__ void k_unhat(const float* __restrict__ phat, const float* __restrict__ s, int64_t N,
                        int lp, int L, float* __restrict__ P) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * L) return;
  int64_t i = e / L;
  int k = (int)(e % L);
  P[e] = phat[i * lp + k] * s[i];
}

rw_status rw_unhat_priors(const rw_graph* g, const float* phat, int lp, int L, float* P,
                          cudaStream_t st) {
  k_unhat<<<rw_blocks(g->N * L, 256), 256, 0, st>>>(phat, g->s, g->N, lp, L, P);
  RW_LAUNCH_CHECK();
  return RW_OK;
}

// sum of degrees (rho^2 of Sec. III-A-1 with the normalized Laplacian)
__global__ void k_sum(const float* __restrict__ v, int64_t n, double* out) {
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    acc += (double)v[i];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffff, acc, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, acc);
}

rw_status rw_graph_degree_sum(rw_graph* g, cudaStream_t st) {
  if (g->upd.cap < 8192) return RW_ERR_OOM;
  double* dd = reinterpret_cast<double*>(g->upd.as<char>() + 6144);
  RW_CHECK_CUDA(cudaMemsetAsync(dd, 0, sizeof(double), st));
  k_sum<<<256, 256, 0, st>>>(g->d, g->N, dd);
  RW_LAUNCH_CHECK();
  double h = 0.0;
  RW_CHECK_CUDA(cudaMemcpyAsync(&h, dd, sizeof(double), cudaMemcpyDeviceToHost, st));
  RW_CHECK_CUDA(cudaStreamSynchronize(st));
  g->dsum = h;
  return RW_OK;
}
