// Gradients of a loss on the label probabilities with respect to the edge weights and beta,
// through the exact random-walker system Eq. (rw_eq) (normalized form of Sec. II-C).
//
// The paper has no gradients; they differentiate its equations.  U_n solves
//   r(U_n, w) = [(L + gamma D~) U - gamma D~ P]_n = 0,   D~ = D (normalized) or I,
// with U_s fixed.  For G = d loss / d U_n the adjoint A lambda = G (A = L_n + gamma D~_n,
// symmetric) gives d loss / d w_e = -lambda-bar^T (d r / d w_e), lambda-bar = lambda padded with
// zeros on the seeds.  For the edge e = (a, b), d L / d w_e = (e_a - e_b)(e_a - e_b)^T and
// d D / d w_e = e_a e_a^T + e_b e_b^T, hence
//   d loss / d w_e = -sum_k [(lam_a - lam_b)(u_a - u_b)
//                            + c gamma (lam_a (u_a - p_a) + lam_b (u_b - p_b))],  c = [normalized],
//   d loss / d beta = sum_e (d loss / d w_e) (d w_e / d beta),  d w_e / d beta from Eq. (W).
//
// The adjoint is solved in the hat variables of the PCG kernel: with s = d^{-1/2} (normalized;
// 1 otherwise), s A s = L-hat_n + gamma I (normalized) or A itself, so lambda = s x where
// (s A s) x = s G.
#include "rw_internal.cuh"

rw_status rw_pcg_run(const rw_graph* g, const float* phat, const float* bexp, const int* seedlab,
                     int L, int lp, double gamma, const float* xhat0, int iters, double tol,
                     float* U, uint8_t* labels, int unscale_out, int* iters_done_dev,
                     float** x_out, cudaStream_t st);

namespace {

constexpr int kGradBlocks = 1024;  // partial sums of d loss / d beta (fixed order)

// right-hand side of the adjoint in hat variables: b_i = s_i G_i (N x lp, seeded rows 0)
__global__ void k_adj_rhs(const float* __restrict__ G, int L, int lp, const float* __restrict__ s,
                          const int* __restrict__ seedlab, int64_t N, float* __restrict__ b) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * lp) return;
  const int64_t i = e / lp;
  const int k = (int)(e % lp);
  b[e] = (k < L && seedlab[i] < 0) ? s[i] * G[i * L + k] : 0.f;
}

// One thread per voxel i and its ndim forward edges e = axis * N + i (to j = i + stride):
// d loss / d w_e, and the block's share of d loss / d beta in FP64.
__global__ void __launch_bounds__(256)
k_edge_grad(const float* __restrict__ xhat, int lp, const float* __restrict__ s,
            const int* __restrict__ seedlab, const float* __restrict__ U,
            const float* __restrict__ P, int L, float cgamma, const float* __restrict__ J,
            const float* __restrict__ w, int form, int ndim, int DX, int DY, int DZ, int64_t N,
            float* __restrict__ gw, double* __restrict__ part) {
  const int64_t st[3] = {1, (int64_t)DX, (int64_t)DX * DY};
  const int n[3] = {DX, DY, DZ};
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int c[3] = {(int)(i % DX), (int)((i / DX) % DY), (int)(i / ((int64_t)DX * DY))};
    const bool free_i = seedlab[i] < 0;
    const float si = s[i];
    for (int a = 0; a < ndim; ++a) {
      const int64_t e = a * N + i;
      if (c[a] + 1 >= n[a]) { gw[e] = 0.f; continue; }
      const int64_t j = i + st[a];
      const bool free_j = seedlab[j] < 0;
      const float sj = s[j];
      float gsum = 0.f;
      for (int k = 0; k < L; ++k) {
        const float li = free_i ? si * xhat[i * lp + k] : 0.f;
        const float lj = free_j ? sj * xhat[j * lp + k] : 0.f;
        const float ui = U[i * L + k], uj = U[j * L + k];
        float t = (li - lj) * (ui - uj);
        if (cgamma != 0.f) t = fmaf(cgamma, li * (ui - P[i * L + k]) + lj * (uj - P[j * L + k]), t);
        gsum -= t;
      }
      gw[e] = gsum;
      const float dJ = J[i] - J[j];
      const float we = w[e];
      const float dwdb = form == RW_WEIGHT_SQ ? -(dJ * dJ) * we : -fabsf(dJ) * we;
      acc += (double)gsum * (double)dwdb;
    }
  }
  __shared__ double red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void k_sum_fixed(const double* __restrict__ part, int n, double* __restrict__ out) {
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

}  // namespace

extern "C" rw_status rw_grad_exact(const rw_graph* g, const int32_t* seed_idx_dev,
                                   const int32_t* seed_lab_dev, int32_t S, int32_t n_labels,
                                   const float* priors_dev, double gamma, const float* U_dev,
                                   const float* dloss_dU_dev, double rel_tol, int32_t max_iter,
                                   float* grad_w_dev, double* grad_beta_host, void* stream) {
  if (!g || !priors_dev || !U_dev || !dloss_dU_dev || !grad_w_dev) return RW_ERR_INVALID_ARG;
  if (S < 0 || S > 65536 || n_labels < 1 || n_labels > RW_MAX_LABELS) return RW_ERR_INVALID_ARG;
  if (S > 0 && (!seed_idx_dev || !seed_lab_dev)) return RW_ERR_INVALID_ARG;
  if (!(gamma > 0.0)) return gamma == 0.0 ? RW_ERR_UNSUPPORTED : RW_ERR_INVALID_ARG;
  if (!(rel_tol > 0.0) || max_iter < 1) return RW_ERR_INVALID_ARG;
  if (g->kind != RW_GRAPH_GRID) {
    rw_set_error_message("rw_grad_exact: edge gradients are defined for grid graphs only");
    return RW_ERR_UNSUPPORTED;
  }
  if (grad_beta_host && !g->J) return RW_ERR_INVALID_ARG;
  cudaStream_t st = rw_stream(stream);
  rw_graph* gm = const_cast<rw_graph*>(g);
  const int L = n_labels;
  const int lp = L <= 4 ? 4 : (L <= 8 ? 8 : 16);
  float* phat;
  int* seedlab;
  RW_TRY(rw_solve_priors_internal(g, seed_idx_dev, seed_lab_dev, S, L, 1, priors_dev, lp, st,
                                  &phat, &seedlab, nullptr));
  RW_TRY(gm->ws.xhat[0].grow(sizeof(float) * (size_t)g->N * lp));
  float* b = gm->ws.xhat[0].as<float>();
  k_adj_rhs<<<rw_blocks(g->N * lp, 256), 256, 0, st>>>(dloss_dU_dev, L, lp, g->s, seedlab, g->N, b);
  RW_LAUNCH_CHECK();
  const size_t need = 16384 + sizeof(double) * (kGradBlocks + 8);
  if (gm->upd.cap < need) return RW_ERR_OOM;  // reserved when the graph was built
  char* ub = gm->upd.as<char>();
  int* it_dev = reinterpret_cast<int*>(ub + 4096);
  double* gbeta_dev = reinterpret_cast<double*>(ub + 6144 + 64);
  double* part = reinterpret_cast<double*>(ub + 16384);
  float* x = nullptr;
  RW_TRY(rw_pcg_run(g, phat, b, seedlab, L, lp, gamma, nullptr, max_iter, rel_tol, nullptr,
                    nullptr, 0, it_dev, &x, st));
  k_edge_grad<<<kGradBlocks, 256, 0, st>>>(
      x, lp, g->s, seedlab, U_dev, priors_dev, L, g->normalized ? (float)gamma : 0.f,
      g->J ? g->J : g->d, g->w, g->form, g->ndim, g->dims[0], g->dims[1], g->dims[2], g->N,
      grad_w_dev, part);
  RW_LAUNCH_CHECK();
  k_sum_fixed<<<1, 256, 0, st>>>(part, kGradBlocks, gbeta_dev);
  RW_LAUNCH_CHECK();
  int iters = 0;
  double gb = 0.0;
  RW_CHECK_CUDA(cudaMemcpyAsync(&iters, it_dev, sizeof(int), cudaMemcpyDeviceToHost, st));
  RW_CHECK_CUDA(cudaMemcpyAsync(&gb, gbeta_dev, sizeof(double), cudaMemcpyDeviceToHost, st));
  RW_CHECK_CUDA(cudaStreamSynchronize(st));
  rw_status ds = rw_last_device_status(g, stream);
  if (ds != RW_OK) return ds;
  if (grad_beta_host) *grad_beta_host = g->J ? gb : 0.0;
  return iters >= max_iter ? RW_WARN_NOT_CONVERGED : RW_OK;
}
