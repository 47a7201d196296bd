// Batched online solves for serving: many images (graphs with their bases), each with its own
// seeds, labels and outputs, solved in one call (the interactive setting of Sec. I: a user adds
// seeds, the labels are recomputed).  The items of a batch are spread over the batch's streams,
// forked from and joined back into the caller's stream; items that share a graph share its
// workspace and therefore a stream.  A round can be captured into a CUDA graph once and, for
// later rounds whose solves launch the same kernels (new seed counts change only the kernels'
// arguments and grid sizes), the instantiated graph is updated in place and replayed.
#include "rw_internal.cuh"

#include <new>
#include <unordered_map>
#include <vector>

struct rw_batch {
  int device = 0;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> join;
  cudaEvent_t fork = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

void batch_release(rw_batch* bt) {
  if (!bt) return;
  if (bt->exec) cudaGraphExecDestroy(bt->exec);
  if (bt->graph) cudaGraphDestroy(bt->graph);
  for (auto s : bt->streams) if (s) cudaStreamDestroy(s);
  for (auto e : bt->join) if (e) cudaEventDestroy(e);
  if (bt->fork) cudaEventDestroy(bt->fork);
  delete bt;
}

rw_status check_items(const rw_batch_item* items, int32_t n) {
  if (!items || n < 1) return RW_ERR_INVALID_ARG;
  for (int k = 0; k < n; ++k) {
    const rw_batch_item& it = items[k];
    if (!it.g || !it.b || !it.seed_idx_dev || !it.seed_lab_dev || !it.prob_dev)
      return RW_ERR_INVALID_ARG;
    if (it.S < 1 || it.n_labels < 1 || it.n_labels > RW_MAX_LABELS) return RW_ERR_INVALID_ARG;
  }
  return RW_OK;
}

}  // namespace

extern "C" rw_status rw_batch_create(int32_t n_streams, rw_batch** out) {
  if (!out || n_streams < 1 || n_streams > 64) return RW_ERR_INVALID_ARG;
  *out = nullptr;
  rw_batch* bt = new (std::nothrow) rw_batch();
  if (!bt) return RW_ERR_OOM;
  auto fail = [&](cudaError_t e, const char* what) {
    rw_set_last_cuda_error(e, what, __FILE__, __LINE__);
    batch_release(bt);
    return RW_ERR_CUDA;
  };
  cudaError_t e = cudaGetDevice(&bt->device);
  if (e != cudaSuccess) return fail(e, "cudaGetDevice");
  e = cudaEventCreateWithFlags(&bt->fork, cudaEventDisableTiming);
  if (e != cudaSuccess) return fail(e, "cudaEventCreateWithFlags");
  bt->streams.assign(n_streams, nullptr);
  bt->join.assign(n_streams, nullptr);
  for (int k = 0; k < n_streams; ++k) {
    e = cudaStreamCreateWithFlags(&bt->streams[k], cudaStreamNonBlocking);
    if (e != cudaSuccess) return fail(e, "cudaStreamCreateWithFlags");
    e = cudaEventCreateWithFlags(&bt->join[k], cudaEventDisableTiming);
    if (e != cudaSuccess) return fail(e, "cudaEventCreateWithFlags");
  }
  *out = bt;
  return RW_OK;
}

extern "C" void rw_batch_free(rw_batch* bt) { batch_release(bt); }

extern "C" rw_status rw_batch_solve(rw_batch* bt, const rw_batch_item* items, int32_t n,
                                    const rw_solve_opts* opts, void* stream) {
  if (!bt || !opts) return RW_ERR_INVALID_ARG;
  RW_TRY(check_items(items, n));
  if (opts->record_phases) return RW_ERR_INVALID_ARG;   // phase events are per graph handle
  cudaStream_t st = rw_stream(stream);
  const int ns = (int)bt->streams.size();
  // a graph handle keeps its stream (its workspace is shared by its solves)
  std::unordered_map<const rw_graph*, int> owner;
  std::vector<int> which(n);
  std::vector<char> used(ns, 0);
  int next = 0;
  for (int k = 0; k < n; ++k) {
    auto f = owner.find(items[k].g);
    if (f == owner.end()) {
      f = owner.emplace(items[k].g, next).first;
      next = (next + 1) % ns;
    }
    which[k] = f->second;
    used[f->second] = 1;
  }
  RW_CHECK_CUDA(cudaEventRecord(bt->fork, st));
  for (int s = 0; s < ns; ++s)
    if (used[s]) RW_CHECK_CUDA(cudaStreamWaitEvent(bt->streams[s], bt->fork, 0));
  rw_status first_error = RW_OK;
  for (int k = 0; k < n && first_error == RW_OK; ++k) {
    const rw_batch_item& it = items[k];
    rw_status s = rw_solve(it.g, it.b, it.seed_idx_dev, it.seed_lab_dev, it.S, it.n_labels,
                           it.priors_dev, opts, it.prob_dev, it.labels_dev, nullptr,
                           bt->streams[which[k]]);
    if (s < 0) first_error = s;
  }
  // join every forked stream even after an error, so the caller's stream stays ordered
  for (int s = 0; s < ns; ++s)
    if (used[s]) {
      RW_CHECK_CUDA(cudaEventRecord(bt->join[s], bt->streams[s]));
      RW_CHECK_CUDA(cudaStreamWaitEvent(st, bt->join[s], 0));
    }
  return first_error;
}

extern "C" rw_status rw_batch_capture(rw_batch* bt, const rw_batch_item* items, int32_t n,
                                      const rw_solve_opts* opts, void* stream,
                                      int32_t* updated_in_place) {
  if (!bt || !opts) return RW_ERR_INVALID_ARG;
  RW_TRY(check_items(items, n));
  cudaStream_t st = rw_stream(stream);
  if (!st) return RW_ERR_INVALID_ARG;   // the legacy default stream cannot be captured
  RW_CHECK_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  rw_status s = rw_batch_solve(bt, items, n, opts, stream);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(st, &g);
  if (s < 0) {
    if (g) cudaGraphDestroy(g);
    return s;
  }
  if (e != cudaSuccess) {
    rw_set_last_cuda_error(e, "cudaStreamEndCapture", __FILE__, __LINE__);
    if (g) cudaGraphDestroy(g);
    return RW_ERR_CUDA;
  }
  int in_place = 0;
  if (bt->exec) {
    cudaGraphExecUpdateResultInfo info;
    if (cudaGraphExecUpdate(bt->exec, g, &info) == cudaSuccess) {
      in_place = 1;
    } else {
      (void)cudaGetLastError();   // the update's failure is not sticky: instantiate anew
      cudaGraphExecDestroy(bt->exec);
      bt->exec = nullptr;
    }
  }
  if (!bt->exec) {
    e = cudaGraphInstantiate(&bt->exec, g, 0);
    if (e != cudaSuccess) {
      rw_set_last_cuda_error(e, "cudaGraphInstantiate", __FILE__, __LINE__);
      cudaGraphDestroy(g);
      bt->exec = nullptr;
      return RW_ERR_CUDA;
    }
  }
  if (bt->graph) cudaGraphDestroy(bt->graph);
  bt->graph = g;
  if (updated_in_place) *updated_in_place = in_place;
  return RW_OK;
}

extern "C" rw_status rw_batch_launch(rw_batch* bt, void* stream) {
  if (!bt || !bt->exec) return RW_ERR_INVALID_ARG;
  RW_CHECK_CUDA(cudaGraphLaunch(bt->exec, rw_stream(stream)));
  return RW_OK;
}
