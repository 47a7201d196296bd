// Gradients of a loss on the label probabilities with respect to the edge weights and beta,
// through the exact random-walker system Eq. (rw_eq) (normalized form of Sec. II-C).
#include "rw_internal.cuh"

extern "C" rw_status rw_grad_exact(const rw_graph* g, const int32_t* seed_idx_dev,
                                   const int32_t* seed_lab_dev, int32_t S, int32_t n_labels,
                                   const float* priors_dev, double gamma, const float* U_dev,
                                   const float* dloss_dU_dev, double rel_tol, int32_t max_iter,
                                   float* grad_w_dev, double* grad_beta_host, void* stream) {
  (void)g; (void)seed_idx_dev; (void)seed_lab_dev; (void)S; (void)n_labels; (void)priors_dev;
  (void)gamma; (void)U_dev; (void)dloss_dU_dev; (void)rel_tol; (void)max_iter; (void)grad_w_dev;
  (void)grad_beta_host; (void)stream;
  return RW_ERR_UNSUPPORTED;
}
