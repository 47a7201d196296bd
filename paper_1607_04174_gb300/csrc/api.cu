// Status codes, device set-up and the scratch-buffer helpers shared by every entry point.
#include "rw_internal.cuh"

#include <cstdio>

#include <atomic>

int g_rw_num_sms = 0;
static std::atomic<int64_t> g_launches{0};

void rw_count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

extern "C" int64_t rw_kernel_launches(void) { return g_launches.load(); }

static thread_local char g_last_err[256];

void rw_set_last_cuda_error(cudaError_t e, const char* what, const char* file, int line) {
  snprintf(g_last_err, sizeof(g_last_err), "%s: %s (%s:%d)", cudaGetErrorString(e), what, file,
           line);
}

void rw_set_error_message(const char* msg) { snprintf(g_last_err, sizeof(g_last_err), "%s", msg); }

extern "C" const char* rw_last_error_message(void) { return g_last_err; }

rw_status rw_device_init() {
  int dev = 0;
  RW_CHECK_CUDA(cudaGetDevice(&dev));
  int sms = 0;
  RW_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  g_rw_num_sms = sms;
  return RW_OK;
}

rw_status rw_status_from_device_bits(int bits) {
  if (bits & RW_DEV_BAD_SEED) return RW_ERR_INVALID_ARG;
  if (bits & RW_DEV_DUP_SEED) return RW_ERR_INVALID_ARG;
  if (bits & RW_DEV_EMPTY_LABEL) return RW_ERR_INVALID_ARG;
  if (bits & RW_DEV_NONFINITE) return RW_ERR_INVALID_ARG;
  if (bits & RW_DEV_ISOLATED) return RW_ERR_ISOLATED_NODE;
  if (bits & RW_DEV_SINGULAR) return RW_ERR_SINGULAR;
  if (bits & RW_DEV_TIMEOUT) return RW_ERR_TIMEOUT;
  return RW_OK;
}

rw_status DevBuf::grow(size_t bytes) {
  if (bytes <= cap) return RW_OK;
  if (p) cudaFree(p);
  p = nullptr;
  cap = 0;
  size_t b = (bytes + 255) & ~size_t(255);
  cudaError_t e = cudaMalloc(&p, b);
  if (e != cudaSuccess) {
    rw_set_last_cuda_error(e, "cudaMalloc(scratch)", __FILE__, __LINE__);
    p = nullptr;
    return RW_ERR_OOM;
  }
  cap = b;
  return RW_OK;
}

void DevBuf::release() {
  if (p) cudaFree(p);
  p = nullptr;
  cap = 0;
}

rw_status PinnedBuf::grow(size_t bytes) {
  if (bytes <= cap) return RW_OK;
  if (p) cudaFreeHost(p);
  p = nullptr;
  cap = 0;
  cudaError_t e = cudaMallocHost(&p, bytes);
  if (e != cudaSuccess) {
    rw_set_last_cuda_error(e, "cudaMallocHost", __FILE__, __LINE__);
    p = nullptr;
    return RW_ERR_OOM;
  }
  cap = bytes;
  return RW_OK;
}

void PinnedBuf::release() {
  if (p) cudaFreeHost(p);
  p = nullptr;
  cap = 0;
}

extern "C" const char* rw_status_str(rw_status s) {
  switch (s) {
    case RW_OK: return "RW_OK";
    case RW_WARN_M_CAPPED: return "RW_WARN_M_CAPPED";
    case RW_WARN_NOT_CONVERGED: return "RW_WARN_NOT_CONVERGED";
    case RW_ERR_INVALID_ARG: return "RW_ERR_INVALID_ARG";
    case RW_ERR_CUDA: return "RW_ERR_CUDA";
    case RW_ERR_OOM: return "RW_ERR_OOM";
    case RW_ERR_NOT_CONVERGED: return "RW_ERR_NOT_CONVERGED";
    case RW_ERR_ISOLATED_NODE: return "RW_ERR_ISOLATED_NODE";
    case RW_ERR_SINGULAR: return "RW_ERR_SINGULAR";
    case RW_ERR_TIMEOUT: return "RW_ERR_TIMEOUT";
    case RW_ERR_UNSUPPORTED: return "RW_ERR_UNSUPPORTED";
  }
  return "RW_UNKNOWN_STATUS";
}

extern "C" rw_status rw_last_device_status(const rw_graph* g, void* stream) {
  if (!g) return RW_ERR_INVALID_ARG;
  cudaStream_t st = rw_stream(stream);
  int bits = 0;
  RW_CHECK_CUDA(cudaMemcpyAsync(&bits, g->status, sizeof(int), cudaMemcpyDeviceToHost, st));
  RW_CHECK_CUDA(cudaMemsetAsync(g->status, 0, sizeof(int), st));
  RW_CHECK_CUDA(cudaStreamSynchronize(st));
  return rw_status_from_device_bits(bits);
}
