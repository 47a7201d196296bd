/*
 * rw.h — C ABI of a GB300 (sm_103a) implementation of the precomputed random walker of
 * Andrews & Hamarneh, "Adaptable Precomputation for Random Walker Image Segmentation and
 * Registration" (arXiv 1607.04174).
 *
 * Conventions for every entry point
 * ---------------------------------
 * - Image graphs are 2-D 4-connected or 3-D 6-connected grids with dims (X, Y, Z); voxel
 *   (x, y, z) has linear index i = x + X * (y + Y * z).  N = X * Y * Z.
 * - Edge id e = axis * N + i is the edge from voxel i to i + stride[axis], stride = (1, X, X*Y);
 *   it exists when voxel i is not on the last slice along that axis.
 * - Node-major layout: an N x k matrix stores row i (voxel i's k values) contiguously, rows
 *   `ld` elements apart.
 * - Pointers named *_dev are CUDA device pointers owned by the caller (e.g. from PyTorch);
 *   *_host are host pointers.  `stream` is a cudaStream_t (NULL = legacy default stream); all
 *   device work is enqueued on it.  The library owns its opaque handles and the scratch
 *   memory it keeps inside them (allocated with cudaMalloc on first use, freed with the handle),
 *   plus one fixed file-scope device array used only by rw_rayleigh_quotients_noalloc (about
 *   2 MiB on every GPU that loads the library); calls of that entry point that overlap on the
 *   GPU race on the array.
 * - Calls that share a handle must not run concurrently on different streams: they share the
 *   handle's scratch memory.
 * - Every call returns an rw_status.  On an error the outputs are unspecified and the handles
 *   remain valid.  Errors that only the GPU can detect (a seed index out of range, a duplicate
 *   seed, a zero pivot) are recorded in the graph handle's device status word; they are
 *   returned by the same call when it synchronizes (see rw_solve) and otherwise by
 *   rw_last_device_status().
 * - No entry point falls back to the CPU.  Without a usable CUDA device every call that
 *   enqueues GPU work returns RW_ERR_CUDA.
 */
#ifndef RW_H_
#define RW_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum rw_status {
  RW_OK = 0,
  RW_WARN_M_CAPPED = 1,          /* adaptive m: no candidate met f <= f_max; m_max was used   */
  RW_WARN_NOT_CONVERGED = 2,     /* an iteration stopped at max_iter; its result is returned   */
  RW_ERR_INVALID_ARG = -1,       /* bad sizes, null pointers, seed/label out of range, dups    */
  RW_ERR_CUDA = -2,              /* a CUDA runtime call failed                                 */
  RW_ERR_OOM = -3,               /* device allocation of scratch memory failed                 */
  RW_ERR_NOT_CONVERGED = -4,     /* an iterative solve the caller asked to converge did not    */
  RW_ERR_ISOLATED_NODE = -5,     /* a voxel has degree 0 (normalized Laplacian undefined)      */
  RW_ERR_SINGULAR = -6,          /* zero pivot in a small dense factorization                  */
  RW_ERR_TIMEOUT = -7,           /* a bounded device wait gave up                              */
  RW_ERR_UNSUPPORTED = -9        /* valid request outside what this build implements          */
} rw_status;

/* Human-readable name of a status code (static storage). */
const char* rw_status_str(rw_status s);
/* Text of the last CUDA runtime error seen by this thread inside the library ("" if none). */
const char* rw_last_error_message(void);
/* Number of CUDA kernels this library has launched since it was loaded (all threads). */
int64_t rw_kernel_launches(void);

/* ------------------------------------------------------------------------------------------
 * Graph (Sec. II-A, Eq. W; Sec. II-C).  w_xy = exp(-beta * (J(x)-J(y))^2) (RW_WEIGHT_SQ) or
 * exp(-beta * |J(x)-J(y)|) (RW_WEIGHT_ABS, Eq. W as printed); D = diag(row sums of W);
 * L = D - W; normalized L-hat = D^{-1/2} L D^{-1/2}.
 * ---------------------------------------------------------------------------------------- */
typedef struct rw_graph rw_graph;
typedef struct rw_basis rw_basis;

enum { RW_WEIGHT_SQ = 0, RW_WEIGHT_ABS = 1 };

typedef struct rw_graph_desc {
  int32_t ndim;         /* 2 or 3                                                           */
  int32_t dims[3];      /* X, Y, Z (Z = 1 when ndim = 2); each >= 1, N <= 2^31 - 1           */
  double beta;          /* >= 0                                                             */
  int32_t weight_form;  /* RW_WEIGHT_SQ or RW_WEIGHT_ABS                                     */
  int32_t normalized;   /* 1: use L-hat (Sec. II-C, the paper's assumption); 0: use L        */
} rw_graph_desc;

/* Builds the graph of Eq. (W) from the intensities J_dev (N floats, read only during the
 * call's stream work; the graph keeps its own copy).  Computes the per-axis forward-edge
 * weights, degrees and D^{-1/2}.  *out receives a new handle (free with rw_graph_free).
 * RW_ERR_ISOLATED_NODE if normalized and some degree is 0 (this call synchronizes). */
rw_status rw_build_graph(const rw_graph_desc* desc, const float* J_dev, void* stream,
                         rw_graph** out);
void rw_graph_free(rw_graph* g);
int64_t rw_graph_num_nodes(const rw_graph* g);

/* Copies the graph's per-axis weights (ndim * N floats, entry axis*N + i = weight of edge id
 * axis*N + i, 0 where the edge does not exist) and degrees (N floats) to caller buffers.
 * Either pointer may be NULL. */
rw_status rw_graph_weights(const rw_graph* g, float* w_dev, float* d_dev, void* stream);

/* Matrix-free Y = L-hat X (or L X when the graph is unnormalized) for an N x k node-major
 * block (Sec. II-C, Eq. z_eig operator).  ldx, ldy >= k and multiples of 4; X_dev, Y_dev
 * 16-byte aligned and not overlapping.  1 <= k <= 1024. */
rw_status rw_apply_laplacian(const rw_graph* g, const float* X_dev, int64_t ldx, float* Y_dev,
                             int64_t ldy, int32_t k, void* stream);

/* Gram product G = A^T B of two tall node-major FP32 blocks on the tensor cores, the dense
 * contraction of the eigensolver's Rayleigh-Ritz and orthogonalization steps (Sec. II-B,
 * Eq. L_eigs: the projected matrices of the block).  A_dev: N x p (pitch lda), B_dev: N x q
 * (pitch ldb); G_dev: p x q FP64 row-major (pitch ldg >= q), overwritten.  Products are taken
 * as three TF32 products of a hi/lo split of each FP32 value (about 21 bits per product), summed
 * in FP32 over slices of 1024 rows and in FP64, in a fixed order, over the slices.
 * scratch_dev (caller-owned, 256-byte aligned) holds at least
 * rw_block_gram_scratch_bytes(N, p, q) bytes; its first int is a device status word (bit
 * RW_DEV_TIMEOUT = 64 set if a bounded wait of the tensor-core pipeline gave up; cleared by
 * every call).  1 <= p, q; N >= 0; N <= 67,107,840.  Asynchronous on `stream`. */
size_t rw_block_gram_scratch_bytes(int64_t N, int32_t p, int32_t q);
rw_status rw_block_gram(const float* A_dev, int64_t lda, const float* B_dev, int64_t ldb,
                        int64_t N, int32_t p, int32_t q, double* G_dev, int32_t ldg,
                        void* scratch_dev, size_t scratch_bytes, void* stream);

/* ------------------------------------------------------------------------------------------
 * Offline precomputation (Sec. II-B, Eq. L_eigs): the m smallest eigenpairs of L-hat (or L).
 * The paper names no eigensolver; this is a block LOBPCG (blocks [X, W, P], soft locking)
 * started by Chebyshev-filtered subspace steps on X while the worst residual exceeds 1e-3,
 * with FP32 stencil/GEMM work and FP64 Cholesky-QR and FP64 Rayleigh-Ritz on the small
 * projected matrices.
 * ---------------------------------------------------------------------------------------- */
typedef struct rw_eig_opts {
  int32_t m;            /* eigenpairs wanted, 1 <= m <= 512                                  */
  int32_t guard;        /* extra block columns (< 0: default max(8, m/5))                    */
  int32_t max_iter;     /* outer iterations (<= 0: default 200)                              */
  double tol;           /* ||L-hat q - lambda q||_2 for unit q (<= 0: default 1e-5)          */
  int32_t cheb_degree;  /* degree of the warm-start filter (< 0: default 32; 0: no warm start) */
  uint64_t seed;        /* seed of the random initial block                                  */
} rw_eig_opts;

typedef struct rw_eig_info {
  int32_t iterations;
  int32_t converged;    /* number of leading pairs meeting tol                               */
  double max_residual;  /* over the m returned pairs                                         */
  int32_t stencil_applies;
} rw_eig_info;

/* Computes the basis.  Returns RW_WARN_NOT_CONVERGED (basis still valid) when max_iter is
 * reached.  Synchronizes the stream (it reads convergence flags each iteration). */
rw_status rw_precompute(rw_graph* g, const rw_eig_opts* opts, void* stream, rw_basis** out,
                        rw_eig_info* info);

/* Wraps a caller-supplied orthonormal basis: Q_dev is N x m node-major (ld = m), lambda_host
 * its m values (eigenvalues, or any values — Sec. III-B uses Rayleigh quotients).  Copies
 * both; builds the 16-bit copy used by the online solve. */
rw_status rw_basis_create(const rw_graph* g, int32_t m, const float* Q_dev,
                          const double* lambda_host, void* stream, rw_basis** out);
/* Saving and loading a basis (the paper's discussion of memory, Sec. V: precomputed
 * eigenvectors are stored offline and loaded as needed, possibly only the leading ones).
 * rw_basis_save writes the basis's current values and its FP32 columns, with the graph's dims,
 * beta and form, to `path` (overwritten; 64-byte header, then m doubles, then N x m floats,
 * host byte order).  rw_basis_load creates a basis for g from such a file, keeping only the
 * first m_load columns (0 = all; the file is read a block of rows at a time, so host memory
 * stays small); the file must belong to a graph of g's dims and form (RW_ERR_INVALID_ARG with a
 * message otherwise, and for a missing, foreign or truncated file).  Both synchronize; the
 * loaded basis is owned by the caller (rw_basis_free). */
rw_status rw_basis_save(const rw_basis* b, const char* path, void* stream);
rw_status rw_basis_load(const rw_graph* g, const char* path, int32_t m_load, void* stream,
                        rw_basis** out);

/* Copies Q (N x m, ld = m, FP32) and/or the current values (m doubles) out.  Synchronizes. */
rw_status rw_basis_get(const rw_basis* b, float* Q_dev, double* lambda_host, void* stream);
int32_t rw_basis_m(const rw_basis* b);
void rw_basis_free(rw_basis* b);

/* ------------------------------------------------------------------------------------------
 * Online solve (Sec. II-B Eqs. Fs, U_lin_comb; Sec. II-C normalized form; Sec. III-A-1 choice
 * of m).  With Lambda_gamma = (Lambda + gamma I)^{-1}, X = B Q_n, Z = Q_n^T P_n:
 *   (I - X Lambda_gamma Q_s^T) F_s = L_s U_s + gamma (U_s + X Lambda_gamma Z)      Eq. (Fs)
 *   U_n = Q_n Lambda_gamma (Q_s^T F_s + gamma Z)                           Eq. (U_lin_comb)
 * solved through the equivalent m x m system (Lambda_gamma^{-1} - Q_s^T X) y = Q_s^T rhs,
 * C = y + gamma Lambda_gamma Z, U_n = Q_n C (Woodbury form of Eq. Fs); with
 * M = Lambda_gamma^{-1} - Q_s^T X and h = Q_s^T (L_s U_s + gamma U_s) that is C = M^{-1}
 * (h + gamma Z).  M is factored by LU without pivoting (a pivot below 1e-3 of its row's scale
 * falls back to partial pivoting).  Then refine_steps damped-Jacobi steps on Eq. (rw_eq) and
 * hard labels = argmax (ties -> lowest label).  m <= 224; the m x m system lives in one CTA's
 * shared memory, so large m with many labels returns RW_ERR_UNSUPPORTED (e.g. m = 224 with 16
 * labels; m = 200 with 16 labels and m = 224 with 4 labels are supported).
 *
 * gamma = 0 (no priors; Sec. II-B, the paragraph after Eq. Fs): L-hat has the null vector
 * g = D^{1/2} 1 / ||D^{1/2} 1|| (1 / sqrt(N) unnormalized) and E is its pseudo-inverse, so
 * E F = U - g c with the column sums c = g^T U as further unknowns.  Basis column 0 (the
 * smallest value) is taken as the null direction and replaced by the exact g; columns 1.. are
 * used projected orthogonal to g (w_j = g^T q_j from one extra pass over the basis).  The
 * seeded system gains the border row (1 - g_n^T g_n) c - g_n^T R^T F_s = g_s^T U_s and the
 * border column -B g_n, solved in the same m x m form with row 0 holding the column-sum
 * equation; U_n = Q_n' C' + g_n c.  The choice of m (Eq. alpha_1) is made on the basis
 * [g, Q'].  No priors are read (prior_mode and priors_dev are ignored), rw_solve_info.mu and
 * sigma are 0.  The graph must be connected (one zero eigenvalue).
 * ---------------------------------------------------------------------------------------- */
enum { RW_REFINE_JACOBI = 0, RW_REFINE_PCG = 1 };
enum { RW_BASIS_F16 = 0, RW_BASIS_BF16 = 1, RW_BASIS_F32 = 2 };
#define RW_MAX_LABELS 16

typedef struct rw_solve_opts {
  double gamma;          /* prior weight of Eq. (rw_energy); >= 0 (0: the null-vector form)  */
  int32_t m;             /* eigenvectors used; 0 = adaptive (Sec. III-A-1), else <= basis m  */
  int32_t m_step;        /* adaptive candidates m_step, 2 m_step, ..., m_max (<= 0: 10)      */
  double eps;            /* adaptive accuracy, f_max = S eps^2 (<= 0: 0.1, the paper's)     */
  int32_t refine_steps;  /* refinement steps after the projection (>= 0)                     */
  int32_t refine_mode;   /* RW_REFINE_JACOBI (damped, omega) or RW_REFINE_PCG                */
  double omega;          /* damping of the Jacobi steps, (0, 1] (<= 0: 0.8)                  */
  int32_t basis_format;  /* storage read by the two N x m passes: RW_BASIS_F16 (scaled FP16,
                            default), RW_BASIS_BF16, RW_BASIS_F32                            */
  int32_t prior_mode;    /* 0: Gaussian fit to the seed intensities (Sec. IV-A);
                            1: caller priors in priors_dev (N x n_labels, rows sum to 1)     */
  int32_t record_phases; /* 1: record CUDA events between the solve's phases on `stream` and
                            report their durations in rw_solve_info.phase_ms (needs info)    */
} rw_solve_opts;

/* Phases of one online solve, in order (indices into rw_solve_info.phase_ms). */
enum {
  RW_PHASE_SEEDS = 0,     /* seed scatter/validation                                          */
  RW_PHASE_GATHER = 1,    /* Q_s, X = B Q_n, seed-side products Q_s^T X, Q_s^T r, Q_s^T Q_s,
                             Gaussian fit and hat-space priors                                */
  RW_PHASE_ADAPT = 2,     /* choice of m (Eq. alpha_1) and the factorization of the m x m
                             matrix M (beside it)                                             */
  RW_PHASE_PROJECT = 3,   /* Z = Q_n^T P_n (one pass over the 16-bit basis)                   */
  RW_PHASE_SMALL = 4,     /* C from the factors: the m x m system of Eq. (Fs), Woodbury form  */
  RW_PHASE_BACK = 5,      /* U_n = Q_n C (second pass over the basis)                         */
  RW_PHASE_REFINE = 6,    /* refinement steps, output, hard labels                            */
  RW_NUM_PHASES = 7
};

typedef struct rw_solve_info {
  int32_t m_used;
  int32_t capped;                 /* adaptive m hit m_max without meeting f_max             */
  int32_t device_status;          /* rw_status recorded on the device during this solve     */
  int32_t pad_;
  double f_max;                   /* S eps^2                                                 */
  double f[RW_MAX_LABELS];        /* f(u_s^k) at m_used (adaptive mode), else 0              */
  double mu[RW_MAX_LABELS];       /* Gaussian prior means (prior_mode 0)                     */
  double sigma[RW_MAX_LABELS];    /* Gaussian prior std devs (prior_mode 0)                  */
  float phase_ms[8];              /* per-phase GPU time (record_phases = 1), else 0          */
} rw_solve_info;

/* seed_idx_dev, seed_lab_dev: S int32 each (voxel index in [0, N), label in [0, n_labels));
 * seeds must be distinct voxels; every label needs >= 1 seed in prior_mode 0.
 * prob_dev: N x n_labels FP32, node-major, ld = n_labels (caller-owned output).
 * labels_dev: N uint8 hard labels, or NULL.  info: host struct or NULL.
 * 1 <= S <= 65536, 1 <= n_labels <= RW_MAX_LABELS.  Asynchronous when info == NULL: device-side
 * errors are then reported by rw_last_device_status().  With info != NULL the call
 * synchronizes the stream and returns the device status. */
rw_status rw_solve(const rw_graph* g, const rw_basis* b, const int32_t* seed_idx_dev,
                   const int32_t* seed_lab_dev, int32_t S, int32_t n_labels,
                   const float* priors_dev, const rw_solve_opts* opts, float* prob_dev,
                   uint8_t* labels_dev, rw_solve_info* info, void* stream);

/* Same solve with HOST buffers: copies the seeds (and priors) in and prob/labels out on
 * `stream` (pinned host memory makes the copies asynchronous), then synchronizes. */
rw_status rw_solve_host(const rw_graph* g, const rw_basis* b, const int32_t* seed_idx_host,
                        const int32_t* seed_lab_host, int32_t S, int32_t n_labels,
                        const float* priors_host, const rw_solve_opts* opts, float* prob_host,
                        uint8_t* labels_host, rw_solve_info* info, void* stream);

/* rw_solve_host without the final synchronization (a serving loop that pipelines solves on one
 * stream): the copies and the solve are only enqueued on `stream`.  The host input buffers must
 * stay valid, and prob_host / labels_host must not be read or reused for another purpose, until
 * the stream has passed this call (cudaStreamSynchronize, or an event recorded after it); the
 * host buffers must be pinned for the copies to stay asynchronous.  Consecutive calls on one
 * graph must use the same stream (they share the graph's staging buffers).  Arguments, layouts
 * and errors as rw_solve_host; with info != NULL the call synchronizes (as rw_solve). */
rw_status rw_solve_host_async(const rw_graph* g, const rw_basis* b,
                              const int32_t* seed_idx_host, const int32_t* seed_lab_host,
                              int32_t S, int32_t n_labels, const float* priors_host,
                              const rw_solve_opts* opts, float* prob_host, uint8_t* labels_host,
                              rw_solve_info* info, void* stream);

/* Reads (and clears) the graph's device status word.  Synchronizes the stream. */
rw_status rw_last_device_status(const rw_graph* g, void* stream);

/* Basic RW on the GPU (the paper's "basic RW", Eq. rw_eq, normalized form of Sec. II-C), by
 * Jacobi-preconditioned CG from a zero start, all labels at once: the comparison solver.
 * Runs exactly `iters` iterations when tol <= 0, else stops when every column's relative
 * residual is <= tol (at most iters).  Same seed/prior/output conventions as rw_solve, except
 * that S = 0 is allowed with prior_mode = 1 (registration without landmarks: the seed pointers
 * may then be NULL); each label column is its own system, so more than RW_MAX_LABELS labels
 * are solved in groups of columns.  gamma >= 0; gamma = 0 (L_n U_n = -B^T U_s, no priors read)
 * needs S >= 1.
 * *iters_done (host, may be NULL) receives the iterations run; synchronizes if non-NULL. */
rw_status rw_solve_pcg(const rw_graph* g, const int32_t* seed_idx_dev,
                       const int32_t* seed_lab_dev, int32_t S, int32_t n_labels,
                       const float* priors_dev, double gamma, int32_t prior_mode,
                       int32_t iters, double tol, float* prob_dev, uint8_t* labels_dev,
                       int32_t* iters_done, void* stream);

/* ------------------------------------------------------------------------------------------
 * Updates (Sec. III-B, Eq. z_ray; Sec. III-C).  The columns of Q are kept and their values
 * become lambda-hat_i = q_i^T L-hat_new q_i, evaluated as the edge sum
 * sum_e w_e (q_i(a) d_a^{-1/2} - q_i(b) d_b^{-1/2})^2.
 * ---------------------------------------------------------------------------------------- */
enum { RW_UPDATE_BETA = 0, RW_UPDATE_EDGES = 1, RW_UPDATE_ROI = 2, RW_UPDATE_ALL = 3 };

typedef struct rw_weight_update {
  int32_t kind;               /* RW_UPDATE_*                                                 */
  int32_t pad_;
  double beta;                /* BETA: new beta for every edge; ROI: beta inside the box      */
  int32_t roi_lo[3];          /* ROI: half-open box [lo, hi) per axis; edges with both ends   */
  int32_t roi_hi[3];          /*      inside are recomputed from Eq. (W)                      */
  const int64_t* edge_ids_dev;/* EDGES: n_edges distinct edge ids                             */
  const float* edge_w_dev;    /* EDGES: their new weights (>= 0); ALL: ndim * N weights in    */
                              /*      edge-id layout (slots without an edge are ignored)       */
  int64_t n_edges;
} rw_weight_update;

/* Mutates the graph's weights and the basis values in place (basis must belong to g, or
 * NULL to change the weights only).  The ROI and EDGES kinds update the values incrementally
 * from the edges whose contribution changed; BETA and ALL recompute every value (Eq. z_ray).
 * RW_ERR_ISOLATED_NODE if a degree becomes 0; RW_ERR_INVALID_ARG (via the device status) for a
 * negative or non-finite weight in ALL.  Synchronizes. */
rw_status rw_update_weights(rw_graph* g, rw_basis* b, const rw_weight_update* u, void* stream);

enum { RW_TOPO_REMOVE_EDGES = 0, RW_TOPO_AGGREGATE = 1 };

typedef struct rw_topology_update {
  int32_t kind;                 /* RW_TOPO_*                                                 */
  int32_t naive;                /* AGGREGATE: 1 = Eq. (q_agg_1), 0 = Eq. (q_agg_2)           */
  const int64_t* edge_ids_dev;  /* REMOVE_EDGES: ids of edges to remove (w_e := 0)           */
  int64_t n_edges;
  int64_t n_bar;                /* AGGREGATE: number of super-vertices                       */
  const int32_t* eta_rowptr_dev;/* AGGREGATE: eta (N x n_bar) CSR, rows sum to 1, columns   */
  const int32_t* eta_col_dev;   /*   sorted within each row                                  */
  const float* eta_val_dev;
  const float* etabar_val_dev;  /* eta-bar on eta's sparsity pattern (columns sum to 1), or
                                   NULL: eta with its columns normalized                      */
} rw_topology_update;

/* REMOVE_EDGES: same vertex set, handled like a weight update (Sec. III-B), g and b mutated.
 * AGGREGATE (Sec. III-C): returns a new general (CSR) graph on the super-vertices with
 * L-bar = eta^T L eta and a new basis Q-bar (aggregated columns, Gram-Schmidt-orthonormalized
 * through FP64 Cholesky-QR, nearly dependent columns dropped) with Ncut values on the new
 * graph.  g and b are unchanged.  Synchronizes. */
rw_status rw_update_topology(rw_graph* g, rw_basis* b, const rw_topology_update* u,
                             void* stream, rw_graph** agg_graph_out, rw_basis** agg_basis_out);

/* ------------------------------------------------------------------------------------------
 * Gradients (not in the paper; derived from Eq. rw_eq and Eq. W).  For a loss on U with
 * dloss_dU_dev = d loss / d U (N x n_labels node-major; seeded rows ignored):
 *   exact path: adjoint A lambda = dloss/dU_n (A = L_n + gamma D_n) by Jacobi-PCG to rel_tol,
 *   d loss / d w_e = -sum_k [(lam_a - lam_b)(u_a - u_b) + gamma (lam_a (u_a - p_a)
 *                            + lam_b (u_b - p_b))]   (second term only when normalized),
 *   d loss / d beta = sum_e (d loss / d w_e) (d w_e / d beta).
 * U_dev must be the converged exact solution (e.g. rw_solve_pcg with a tight tol) and
 * priors_dev the priors it used (N x n_labels, e.g. from rw_solve_priors).  S = 0 (no seeds,
 * seed pointers may be NULL) gives the registration gradient; the loss gradients of label
 * groups add up.
 * grad_w_dev: ndim * N floats in edge-id layout (0 where no edge).  grad_beta_host: 1 double
 * (may be NULL).  Grid graphs only (RW_ERR_UNSUPPORTED for an aggregate's CSR graph); gamma > 0.
 * Returns RW_WARN_NOT_CONVERGED (gradients still written) when the adjoint PCG used max_iter
 * iterations.  Uses the graph's solve scratch (not concurrently with rw_solve on g).
 * Synchronizes.
 * ---------------------------------------------------------------------------------------- */
rw_status rw_grad_exact(const rw_graph* g, const int32_t* seed_idx_dev,
                        const int32_t* seed_lab_dev, int32_t S, int32_t n_labels,
                        const float* priors_dev, double gamma, const float* U_dev,
                        const float* dloss_dU_dev, double rel_tol, int32_t max_iter,
                        float* grad_w_dev, double* grad_beta_host, void* stream);

/* ------------------------------------------------------------------------------------------
 * Gradient through the eigenvector solve (Sec. II-B, normalized form of Sec. II-C; not in the
 * paper, derived from its equations).  The first m columns of the basis are held fixed and
 * their values are the Rayleigh quotients of Eq. (z_ray) under the graph's current weights
 * (as after rw_precompute or rw_update_weights).  The forward is the fast solve at fixed m
 * (Eqs. Fs, U_lin_comb, in the m x m Woodbury form) followed by refine_steps damped-Jacobi
 * steps with factor omega on (L-hat_n + gamma I) U-hat_n = gamma P-hat_n - B-hat^T U-hat_s,
 * computed from the FP32 basis; the reverse pass differentiates every step, including the
 * values lambda-hat(w), the coefficients w_ab d_a^{-1/2} d_b^{-1/2} and the degrees, down to
 * the edge weights and beta (Eq. W).
 *   priors_dev: N x n_labels probabilities (e.g. from rw_solve_priors); held fixed.
 *   dloss_dU_dev: N x n_labels, d loss / d U (seeded rows ignored).
 *   U_out_dev: N x n_labels forward result, or NULL.
 *   grad_w_dev: ndim * N floats in edge-id layout (0 where no edge); grad_beta_host may be NULL.
 * Normalized grid graphs only (RW_ERR_UNSUPPORTED otherwise); gamma > 0; 1 <= m <= basis m,
 * m <= 1024; 0 < omega <= 1.  RW_ERR_SINGULAR if the m x m system has a zero pivot.
 * Scratch: grown inside the graph handle on first use (about (refine_steps + 7) N n_pad + 2 ndim N
 * floats, n_pad = 4/8/16).  Synchronizes.
 * ---------------------------------------------------------------------------------------- */
rw_status rw_grad_fast(const rw_graph* g, const rw_basis* b, const int32_t* seed_idx_dev,
                       const int32_t* seed_lab_dev, int32_t S, int32_t n_labels,
                       const float* priors_dev, double gamma, int32_t m, int32_t refine_steps,
                       double omega, const float* dloss_dU_dev, float* U_out_dev,
                       float* grad_w_dev, double* grad_beta_host, void* stream);

/* ------------------------------------------------------------------------------------------
 * Rayleigh quotients of caller columns with no device allocation.  The paper has no
 * counterpart; this serves callers that cannot allocate device memory during a call (a host
 * application that owns the whole device memory budget through its own pool, or a thread that
 * must not enter the allocator).  It returns the same values that rw_update_weights with
 * RW_UPDATE_BETA and an unchanged beta leaves in the basis: lambda_dev[i] =
 * sum_e w_e (q_i(a) s_a - q_i(b) s_b)^2 / ||q_i||^2 for the m columns of Q_dev (N x m
 * node-major, pitch ldq a multiple of 4, >= m, 16-byte aligned) under g's current weights;
 * lambda_dev holds m doubles on the device.  The device g was built on must be current
 * (RW_ERR_INVALID_ARG otherwise).
 * Scratch: a fixed device array inside the library (about 2 MiB, held by every GPU that loads
 * the library until exit), no cudaMalloc or cudaFree.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress).  All calls share the array: calls that
 * overlap on the GPU race.  m > 1024 (or any
 * other bad argument) returns RW_ERR_INVALID_ARG with a message in rw_last_error_message().
 * Asynchronous on `stream`.
 * ---------------------------------------------------------------------------------------- */
#define RW_NOALLOC_MAX_M 1024
rw_status rw_rayleigh_quotients_noalloc(const rw_graph* g, const float* Q_dev, int64_t ldq,
                                        int32_t m, double* lambda_dev, void* stream);

/* ------------------------------------------------------------------------------------------
 * Batched solves for serving (the interactive use of Sec. I: users add seeds, labels are
 * recomputed).  A batch handle owns n_streams CUDA streams.  rw_batch_solve runs rw_solve for
 * every item (info not returned): the items are spread over the batch's streams, forked from
 * and joined back into `stream`; items that share a graph handle go to the same stream (they
 * share its workspace).  Every item's result is the one rw_solve gives alone, bit for bit.
 * Errors: RW_ERR_INVALID_ARG for a bad item (nothing launched); the first failing solve's
 * status otherwise (the streams are still joined).  opts->record_phases must be 0.
 * rw_batch_capture records the same round into a CUDA graph held by the handle: the first
 * capture instantiates it, later captures whose solves launch the same kernels update it in
 * place (*updated_in_place = 1; new seed counts only change kernel arguments and grid sizes),
 * others re-instantiate it.  rw_batch_launch replays the last captured round on `stream`; the
 * seed and output buffers of the captured items must still be valid.  Capture needs a
 * non-default stream and scratch already sized: run each graph once, uncaptured, with at least
 * as many seeds and the same label count first (a scratch allocation inside the capture fails
 * it with RW_ERR_OOM or RW_ERR_CUDA).  The process-wide kernel-launch counter counts captured
 * launches at capture, not at replay.
 * rw_set_launch_shape sets the blocks per SM of the two 16-bit basis passes for graphs with
 * N <= n_max (up to 16 size classes, ascending; n_max <= 0 clears the table); without an entry
 * the projection uses 2 and the back-projection 3.  proj_per_sm in [1, 4], back_per_sm in
 * [1, 8].  The project's autotuner (paper_1607_04174_gb300/autotune.py) measures the table.
 * rw_set_tc_passes selects, process-wide, the tensor-core kernels or the CUDA-core kernels for
 * the two passes over a 16-bit basis copy in rw_solve, rw_solve_unseeded and the batch calls:
 * mask bit 0 = the projection Z = Q_n^T P_n on tensor cores, bit 1 = the back-projection
 * U_n = Q_n C (Eq. U_lin_comb), 4 (the default) = both on tensor cores for passes that carry
 * more than 8 labels (there rw_solve_unseeded takes up to 32 labels per pass), CUDA cores
 * otherwise; 0 = always CUDA cores, 3 = always tensor cores; other values return
 * RW_ERR_INVALID_ARG.  The launch-shape table applies to the CUDA-core kernels only (the
 * tensor-core ones run one block per SM).  Copies wider than 256 columns and the FP32 basis
 * always use the CUDA-core kernels.  Takes effect for launches after the call.
 * ---------------------------------------------------------------------------------------- */
typedef struct rw_batch rw_batch;
typedef struct rw_batch_item {
  const rw_graph* g;
  const rw_basis* b;
  const int32_t* seed_idx_dev;
  const int32_t* seed_lab_dev;
  int32_t S;
  int32_t n_labels;
  const float* priors_dev;   /* NULL unless opts->prior_mode == 1 */
  float* prob_dev;           /* N x n_labels */
  uint8_t* labels_dev;       /* N or NULL */
} rw_batch_item;
rw_status rw_batch_create(int32_t n_streams, rw_batch** out);
void rw_batch_free(rw_batch* bt);
rw_status rw_batch_solve(rw_batch* bt, const rw_batch_item* items, int32_t n,
                         const rw_solve_opts* opts, void* stream);
rw_status rw_batch_capture(rw_batch* bt, const rw_batch_item* items, int32_t n,
                           const rw_solve_opts* opts, void* stream, int32_t* updated_in_place);
rw_status rw_batch_launch(rw_batch* bt, void* stream);
rw_status rw_set_launch_shape(int64_t n_max, int32_t proj_per_sm, int32_t back_per_sm);
rw_status rw_set_tc_passes(int32_t mask);

/* ------------------------------------------------------------------------------------------
 * Registration (RWIR, Sec. II-A: the K labels are displacement vectors; Sec. III-A-2; Sec. IV-B).
 * rw_registration_priors: P (N x K, node-major) for the fixed / moving images (N floats each,
 * device, same grid) and the K displacements disp_dev (K x ndim int32, device, voxels): the sum
 * of absolute differences between fixed(x + o) and moving(x + o + d_k) over the patch offsets
 * o in [-half, half]^ndim (coordinates clamped into the grid), squared, negated, exponentiated
 * and normalized to sum to 1 over the labels at each voxel.  dims[0..ndim-1] as for graphs;
 * 1 <= K <= 4096, 0 <= half <= 8.  Asynchronous; two intermediate volumes of
 * (dims + 2 half) x K floats are allocated and freed in stream order (cudaMallocAsync).
 * rw_solve_unseeded: the fast RW with priors and no seeds, Eq. (U_lin_comb) with S = 0:
 * U-hat = Q Lambda_gamma (gamma Q^T P-hat), then opts->refine_steps damped-Jacobi steps of
 * Eq. (rw_eq) (no seeded rows).  opts->m = 0 chooses m by Eq. (g): the first candidate
 * m_step, 2 m_step, ..., m_max with max_k ||p-hat_k - Q_m Q_m^T p-hat_k||^2 <= 1^T D 1 eps^2
 * (every label evaluated); otherwise m = opts->m.  prob_dev: N x K; labels_dev (N, K <= 255,
 * or NULL): the most probable label; field_dev (N x disp_dim, or NULL): the expected
 * displacement sum_k U_k d_k with disp_dev (K x disp_dim).  Labels run in chunks of 8 through
 * the basis passes; 1 <= K <= 4096.  16-bit or FP32 basis (BF16: RW_ERR_UNSUPPORTED).  m_used
 * (host, or NULL): the m taken; when given the call synchronizes and reports device errors.
 * Scratch: grown in the graph handle (about 3 N x 8 floats plus the m_max x K projections).
 * ---------------------------------------------------------------------------------------- */
rw_status rw_registration_priors(const float* fixed_dev, const float* moving_dev, int32_t ndim,
                                 const int32_t* dims, const int32_t* disp_dev, int32_t K,
                                 int32_t half, float* priors_dev, void* stream);
rw_status rw_solve_unseeded(const rw_graph* g, const rw_basis* b, const float* priors_dev,
                            int32_t K, const rw_solve_opts* opts, float* prob_dev,
                            uint8_t* labels_dev, const int32_t* disp_dev, int32_t disp_dim,
                            float* field_dev, int32_t* m_used, void* stream);

/* Several bases precomputed at betas_host[0..n-1] (Sec. III-B, last paragraph: Eq. z_ray
 * "interpolates" between them): the index of the one to update for `beta`, the nearest in log
 * beta (ties to the lower index); -1 when n < 1 or a beta is not positive.  Host only; the
 * caller then applies rw_update_weights(RW_UPDATE_BETA, beta) to that basis. */
int32_t rw_basis_nearest_beta(const double* betas_host, int32_t n, double beta);

/* Writes the Gaussian-fit priors of Sec. IV-A (N x n_labels, node-major) for the seeds. */
rw_status rw_solve_priors(const rw_graph* g, const int32_t* seed_idx_dev,
                          const int32_t* seed_lab_dev, int32_t S, int32_t n_labels,
                          float* priors_dev, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* RW_H_ */
