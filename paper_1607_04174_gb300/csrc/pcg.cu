// Basic random walker on the GPU: Eq. (rw_eq) in the normalized form of Sec. II-C,
//   (L-hat_n + gamma I) U-hat_n = gamma P-hat_n - B-hat^T U-hat_s,
// solved by Jacobi-preconditioned CG, every label column with its own recurrence, all
// columns in one persistent cooperative kernel (grid-wide barriers between the phases of an
// iteration; the working set stays in L2 for 2-D images).
#include "rw_internal.cuh"

#include <cooperative_groups.h>

#include <algorithm>

namespace cg = cooperative_groups;

namespace {

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
  int L, lp;
  float gamma;
  // state
  float *x, *r, *z, *p, *q;  // N x lp
  double* dots;              // [pq 2][rz 2][rr 2][bb 1] x 16
  int iters;
  double tol;
  int start_zero;
  int* iters_done;
  float* U;                  // output N x L (or nullptr: leave x in hat space)
  uint8_t* labels;
  int unscale_out;           // 1: U = s * x; 0: U = x
};

__device__ __forceinline__ float aii(const PcgArgs& a, int64_t i, float gamma) {
  return (a.normalized ? 1.f : a.d[i]) + gamma;
}

// y = sum_j c_ij v_j over the neighbours of i (all of them; the caller zeroes seeded rows)
__device__ __forceinline__ void nbr_sum(const PcgArgs& a, const float* __restrict__ v, int64_t i,
                                        float* acc) {
  const int lp = a.lp;
  auto add = [&](int64_t j, float c) {
    const float* vj = v + j * lp;
    for (int k = 0; k < lp; ++k) acc[k] = fmaf(c, vj[k], acc[k]);
  };
  if (a.kind == RW_GRAPH_GRID) {
    const int64_t st[3] = {1, (int64_t)a.DX, (int64_t)a.DX * a.DY};
    const int cc[3] = {(int)(i % a.DX), (int)((i / a.DX) % a.DY), (int)(i / ((int64_t)a.DX * a.DY))};
    const int n[3] = {a.DX, a.DY, a.DZ};
    for (int ax = 0; ax < a.ndim; ++ax) {
      if (cc[ax] > 0) add(i - st[ax], a.cw[ax * a.N + i - st[ax]]);
      if (cc[ax] + 1 < n[ax]) add(i + st[ax], a.cw[ax * a.N + i]);
    }
  } else {
    for (int p = a.rowptr[i]; p < a.rowptr[i + 1]; ++p) add(a.col[p], a.ccsr[p]);
  }
}

__device__ void block_accum(double* dst, float* vals, int lp) {
  // vals: per-thread lp partial sums -> warp reduce -> one atomic per warp per column
  for (int k = 0; k < lp; ++k) {
    float v = vals[k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffff, v, o);
    if ((threadIdx.x & 31) == 0 && v != 0.f) atomicAdd(&dst[k], (double)v);
  }
}

__global__ void __launch_bounds__(256) k_pcg(PcgArgs a) {
  cg::grid_group grid = cg::this_grid();
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  const int lp = a.lp;
  double* pq = a.dots;          // [2][16]
  double* rz = a.dots + 32;     // [2][16]
  double* rr = a.dots + 64;     // [2][16]
  double* bb = a.dots + 96;     // [16]
  const float g = a.gamma;
  // init: r = b - A x, z = r / a_ii, p = z
  {
    float prz[16] = {}, pbb[16] = {};
    for (int64_t i0 = tid; i0 < ((a.N + 31) / 32) * 32; i0 += nth) {
      const int64_t i = i0;
      if (i < a.N) {
        float* xi = a.x + i * lp;
        float* ri = a.r + i * lp;
        float* zi = a.z + i * lp;
        float* pi = a.p + i * lp;
        const int sl = a.seedlab[i];
        if (sl >= 0) {
          for (int k = 0; k < lp; ++k) {
            xi[k] = (k == sl) ? a.sq[i] : 0.f;
            ri[k] = zi[k] = pi[k] = 0.f;
          }
        } else if (a.start_zero) {
          for (int k = 0; k < lp; ++k) xi[k] = 0.f;
        }
      }
    }
    grid.sync();
    for (int64_t i0 = tid; i0 < ((a.N + 31) / 32) * 32; i0 += nth) {
      const int64_t i = i0;
      float lr[16], lz[16], lb[16];
      for (int k = 0; k < lp; ++k) lr[k] = lz[k] = lb[k] = 0.f;
      if (i < a.N && a.seedlab[i] < 0) {
        // nb = sum_j c_ij x_j over all neighbours (seeded x_j = U-hat_j), sn = the seeded part.
        // b = gamma p-hat_i + sn (Eq. rw_eq in hat variables) unless given explicitly;
        // r = b - A_n x_n = b - a_ii x_i + (nb - sn).
        float nb[16], sn[16];
        for (int k = 0; k < lp; ++k) { nb[k] = 0.f; sn[k] = 0.f; }
        nbr_sum(a, a.x, i, nb);
        auto addseed = [&](int64_t j, float c) {
          if (a.seedlab[j] >= 0)
            for (int k = 0; k < lp; ++k) sn[k] = fmaf(c, a.x[j * lp + k], sn[k]);
        };
        if (a.kind == RW_GRAPH_GRID) {
          const int64_t st[3] = {1, (int64_t)a.DX, (int64_t)a.DX * a.DY};
          const int cc[3] = {(int)(i % a.DX), (int)((i / a.DX) % a.DY), (int)(i / ((int64_t)a.DX * a.DY))};
          const int n[3] = {a.DX, a.DY, a.DZ};
          for (int ax = 0; ax < a.ndim; ++ax) {
            if (cc[ax] > 0) addseed(i - st[ax], a.cw[ax * a.N + i - st[ax]]);
            if (cc[ax] + 1 < n[ax]) addseed(i + st[ax], a.cw[ax * a.N + i]);
          }
        } else {
          for (int p = a.rowptr[i]; p < a.rowptr[i + 1]; ++p) addseed(a.col[p], a.ccsr[p]);
        }
        const float* xi = a.x + i * lp;
        const float di = aii(a, i, g);
        for (int k = 0; k < lp; ++k) {
          float b = a.bexp ? a.bexp[i * lp + k] : fmaf(g, a.phat[i * lp + k], sn[k]);
          lb[k] = b;
          lr[k] = b - di * xi[k] + (nb[k] - sn[k]);
        }
        float* ri = a.r + i * lp;
        float* zi = a.z + i * lp;
        float* pi = a.p + i * lp;
        for (int k = 0; k < lp; ++k) {
          ri[k] = lr[k];
          zi[k] = lr[k] / di;
          pi[k] = zi[k];
          lz[k] = lr[k] * zi[k];
          lb[k] = lb[k] * lb[k];
        }
      }
      for (int k = 0; k < lp; ++k) { prz[k] += lz[k]; pbb[k] += lb[k]; }
    }
    block_accum(&rz[16], prz, lp);
    block_accum(bb, pbb, lp);
  }
  grid.sync();
  int t = 0;
  for (; t < a.iters; ++t) {
    const int sI = t & 1, oI = sI ^ 1;
    // phase 1: q = A p (unseeded rows; seeded p = 0), pq = p . q
    if (tid == 0) for (int k = 0; k < 16; ++k) rz[16 * sI + k] = 0.0;
    {
      float ppq[16];
      for (int k = 0; k < lp; ++k) ppq[k] = 0.f;
      for (int64_t i0 = tid; i0 < ((a.N + 31) / 32) * 32; i0 += nth) {
        const int64_t i = i0;
        if (i < a.N) {
          float* qi = a.q + i * lp;
          if (a.seedlab[i] >= 0) {
            for (int k = 0; k < lp; ++k) qi[k] = 0.f;
          } else {
            float nb[16];
            for (int k = 0; k < lp; ++k) nb[k] = 0.f;
            nbr_sum(a, a.p, i, nb);
            const float di = aii(a, i, g);
            const float* pi = a.p + i * lp;
            for (int k = 0; k < lp; ++k) {
              float v = di * pi[k] - nb[k];
              qi[k] = v;
              ppq[k] = fmaf(pi[k], v, ppq[k]);
            }
          }
        }
      }
      block_accum(&pq[16 * sI], ppq, lp);
    }
    grid.sync();
    // phase 2: x += alpha p, r -= alpha q, z = r / a_ii, rz, rr
    {
      float alpha[16], prz[16], prr[16];
      for (int k = 0; k < lp; ++k) {
        double den = pq[16 * sI + k];
        alpha[k] = den > 0.0 ? (float)(rz[16 * oI + k] / den) : 0.f;
        prz[k] = prr[k] = 0.f;
      }
      if (tid == 0) for (int k = 0; k < 16; ++k) { pq[16 * oI + k] = 0.0; rr[16 * oI + k] = 0.0; }
      for (int64_t i0 = tid; i0 < ((a.N + 31) / 32) * 32; i0 += nth) {
        const int64_t i = i0;
        if (i < a.N && a.seedlab[i] < 0) {
          float* xi = a.x + i * lp;
          float* ri = a.r + i * lp;
          float* zi = a.z + i * lp;
          const float* pi = a.p + i * lp;
          const float* qi = a.q + i * lp;
          const float di = aii(a, i, g);
          for (int k = 0; k < lp; ++k) {
            xi[k] = fmaf(alpha[k], pi[k], xi[k]);
            float rv = fmaf(-alpha[k], qi[k], ri[k]);
            ri[k] = rv;
            float zv = rv / di;
            zi[k] = zv;
            prz[k] = fmaf(rv, zv, prz[k]);
            prr[k] = fmaf(rv, rv, prr[k]);
          }
        }
      }
      block_accum(&rz[16 * sI], prz, lp);
      block_accum(&rr[16 * sI], prr, lp);
    }
    grid.sync();
    if (a.tol > 0.0) {
      bool done = true;
      for (int k = 0; k < a.L; ++k) {
        double b2 = bb[k];
        if (b2 > 0.0 && rr[16 * sI + k] > a.tol * a.tol * b2) done = false;
      }
      if (done) { ++t; break; }
    }
    // phase 3: p = z + beta p
    {
      float beta[16];
      for (int k = 0; k < lp; ++k) {
        double den = rz[16 * oI + k];
        beta[k] = den > 0.0 ? (float)(rz[16 * sI + k] / den) : 0.f;
      }
      for (int64_t i = tid; i < a.N; i += nth) {
        if (a.seedlab[i] >= 0) continue;
        float* pi = a.p + i * lp;
        const float* zi = a.z + i * lp;
        for (int k = 0; k < lp; ++k) pi[k] = fmaf(beta[k], pi[k], zi[k]);
      }
    }
    grid.sync();
  }
  if (tid == 0 && a.iters_done) *a.iters_done = t;
  if (a.U) {
    for (int64_t i = tid; i < a.N; i += nth) {
      const int sl = a.seedlab[i];
      const float* xi = a.x + i * lp;
      const float si = a.unscale_out ? a.s[i] : 1.f;
      int best = 0;
      float bv = -INFINITY;
      for (int k = 0; k < a.L; ++k) {
        float u = (sl >= 0) ? (k == sl ? 1.f : 0.f) : xi[k] * si;
        a.U[i * a.L + k] = u;
        if (u > bv) { bv = u; best = k; }
      }
      if (a.labels) a.labels[i] = (uint8_t)best;
    }
  }
}

}  // namespace

// Runs the cooperative PCG.  xhat0: N x lp start (hat space) or nullptr for a zero start.
rw_status rw_pcg_run(const rw_graph* g, const float* phat, const float* bexp, const int* seedlab,
                     int L, int lp, double gamma, const float* xhat0, int iters, double tol,
                     float* U, uint8_t* labels, int unscale_out, int* iters_done_dev,
                     float** x_out, cudaStream_t st) {
  rw_graph* gm = const_cast<rw_graph*>(g);
  const size_t vec = sizeof(float) * (size_t)g->N * lp;
  const size_t dots_off = 5 * ((vec + 255) & ~size_t(255));
  RW_TRY(gm->ws.pcg.grow(std::max(gm->ws.pcg.cap, dots_off + 4096)));
  char* base = gm->ws.pcg.as<char>();
  const size_t stride = (vec + 255) & ~size_t(255);
  PcgArgs a{};
  a.kind = g->kind; a.ndim = g->ndim; a.DX = g->dims[0]; a.DY = g->dims[1]; a.DZ = g->dims[2];
  a.normalized = g->normalized; a.N = g->N; a.cw = g->cw; a.d = g->d; a.s = g->s; a.sq = g->sq;
  a.rowptr = g->rowptr; a.col = g->col; a.ccsr = g->ccsr;
  a.phat = phat; a.bexp = bexp; a.seedlab = seedlab; a.L = L; a.lp = lp; a.gamma = (float)gamma;
  a.x = reinterpret_cast<float*>(base);
  a.r = reinterpret_cast<float*>(base + stride);
  a.z = reinterpret_cast<float*>(base + 2 * stride);
  a.p = reinterpret_cast<float*>(base + 3 * stride);
  a.q = reinterpret_cast<float*>(base + 4 * stride);
  a.dots = reinterpret_cast<double*>(base + dots_off);
  a.iters = iters; a.tol = tol; a.iters_done = iters_done_dev;
  a.U = U; a.labels = labels; a.unscale_out = unscale_out;
  a.start_zero = xhat0 ? 0 : 1;
  if (xhat0) RW_CHECK_CUDA(cudaMemcpyAsync(a.x, xhat0, vec, cudaMemcpyDeviceToDevice, st));
  RW_CHECK_CUDA(cudaMemsetAsync(a.dots, 0, sizeof(double) * 7 * 16, st));
  int per_sm = 0;
  RW_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg, 256, 0));
  const int sms = g_rw_num_sms > 0 ? g_rw_num_sms : 148;
  int64_t want = (g->N + 255) / 256;
  int blocks = (int)std::min<int64_t>((int64_t)sms * std::max(per_sm, 1), std::max<int64_t>(want, 1));
  void* kargs[] = {&a};
  RW_CHECK_CUDA(cudaLaunchCooperativeKernel((void*)k_pcg, dim3(blocks), dim3(256), kargs, 0, st));
  rw_count_launch();
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
  if (!g || !seed_idx_dev || !seed_lab_dev || !prob_dev) return RW_ERR_INVALID_ARG;
  if (S < 1 || S > 65536 || n_labels < 1 || n_labels > RW_MAX_LABELS) return RW_ERR_INVALID_ARG;
  if (!(gamma > 0.0)) return gamma == 0.0 ? RW_ERR_UNSUPPORTED : RW_ERR_INVALID_ARG;
  if (iters < 0 || (prior_mode == 1 && !priors_dev) || (prior_mode == 0 && !g->J))
    return RW_ERR_INVALID_ARG;
  cudaStream_t st = rw_stream(stream);
  const int lp = n_labels <= 4 ? 4 : (n_labels <= 8 ? 8 : 16);
  float* phat;
  int* seedlab;
  RW_TRY(rw_solve_priors_internal(g, seed_idx_dev, seed_lab_dev, S, n_labels, prior_mode,
                                  priors_dev, lp, st, &phat, &seedlab, nullptr));
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
