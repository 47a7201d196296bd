// Saving and loading a precomputed basis (the offline eigenvectors of Sec. II-B and their
// current values), and loading only its leading columns.  The paper's discussion of memory
// (Sec. V) notes that the eigenvectors can be loaded sequentially, so that a machine holds only
// as many as the online solve needs; rw_basis_load takes the first m_load columns of a saved
// basis, streaming the file through a pinned host buffer a block of rows at a time.
//
// File layout (host byte order): a 64-byte header
//   char magic[8] = "RWBASIS1", uint32 version = 1, uint32 header bytes = 64, int64 N, int32 m,
//   int32 dims[3], double beta, uint32 normalized, uint32 weight form, 8 bytes zero
// then the m values (double) and the N x m columns, node-major float32 without padding.
#include "rw_internal.cuh"

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

namespace {

struct BasisHeader {
  char magic[8];
  uint32_t version;
  uint32_t header_bytes;
  int64_t N;
  int32_t m;
  int32_t dims[3];
  double beta;
  uint32_t normalized;
  uint32_t form;
  uint64_t zero;
};
static_assert(sizeof(BasisHeader) == 64, "basis file header is 64 bytes");

constexpr char kMagic[8] = {'R', 'W', 'B', 'A', 'S', 'I', 'S', '1'};
constexpr int64_t kRowsPerBlock = 1 << 14;

struct File {
  FILE* f = nullptr;
  ~File() { if (f) fclose(f); }
};

struct PinnedTmp {
  void* p = nullptr;
  ~PinnedTmp() { if (p) cudaFreeHost(p); }
};

struct DevTmp {
  void* p = nullptr;
  ~DevTmp() { if (p) cudaFree(p); }
};

}  // namespace

extern "C" rw_status rw_basis_save(const rw_basis* b, const char* path, void* stream) {
  if (!b || !path || !b->owner) return RW_ERR_INVALID_ARG;
  cudaStream_t st = rw_stream(stream);
  const rw_graph* g = b->owner;
  BasisHeader h{};
  memcpy(h.magic, kMagic, 8);
  h.version = 1;
  h.header_bytes = sizeof(BasisHeader);
  h.N = b->N;
  h.m = b->m;
  for (int k = 0; k < 3; ++k) h.dims[k] = g->dims[k];
  h.beta = g->beta;
  h.normalized = (uint32_t)g->normalized;
  h.form = (uint32_t)g->form;
  std::vector<double> lam(b->m);
  RW_CHECK_CUDA(cudaMemcpyAsync(lam.data(), b->lam, sizeof(double) * b->m,
                                cudaMemcpyDeviceToHost, st));
  RW_CHECK_CUDA(cudaStreamSynchronize(st));
  File out;
  out.f = fopen(path, "wb");
  if (!out.f) {
    rw_set_error_message("rw_basis_save: cannot open the file for writing");
    return RW_ERR_INVALID_ARG;
  }
  auto fail_io = [&]() {
    rw_set_error_message("rw_basis_save: write failed");
    return RW_ERR_INVALID_ARG;
  };
  if (fwrite(&h, sizeof(h), 1, out.f) != 1) return fail_io();
  if (fwrite(lam.data(), sizeof(double), b->m, out.f) != (size_t)b->m) return fail_io();
  const size_t row_bytes = sizeof(float) * (size_t)b->m;
  PinnedTmp buf;
  RW_CHECK_CUDA(cudaMallocHost(&buf.p, row_bytes * kRowsPerBlock));
  for (int64_t r0 = 0; r0 < b->N; r0 += kRowsPerBlock) {
    const int64_t nr = std::min<int64_t>(kRowsPerBlock, b->N - r0);
    RW_CHECK_CUDA(cudaMemcpy2DAsync(buf.p, row_bytes, b->Q32 + r0 * b->ld32,
                                    sizeof(float) * b->ld32, row_bytes, nr,
                                    cudaMemcpyDeviceToHost, st));
    RW_CHECK_CUDA(cudaStreamSynchronize(st));
    if (fwrite(buf.p, row_bytes, nr, out.f) != (size_t)nr) return fail_io();
  }
  if (fflush(out.f) != 0) return fail_io();
  return RW_OK;
}

extern "C" rw_status rw_basis_load(const rw_graph* g, const char* path, int32_t m_load,
                                   void* stream, rw_basis** out) {
  if (!g || !path || !out || m_load < 0) return RW_ERR_INVALID_ARG;
  *out = nullptr;
  cudaStream_t st = rw_stream(stream);
  File in;
  in.f = fopen(path, "rb");
  if (!in.f) {
    rw_set_error_message("rw_basis_load: cannot open the file");
    return RW_ERR_INVALID_ARG;
  }
  BasisHeader h{};
  if (fread(&h, sizeof(h), 1, in.f) != 1 || memcmp(h.magic, kMagic, 8) != 0 || h.version != 1 ||
      h.header_bytes != sizeof(BasisHeader) || h.m < 1 || h.N < 1) {
    rw_set_error_message("rw_basis_load: not a basis file");
    return RW_ERR_INVALID_ARG;
  }
  if (h.N != g->N || h.dims[0] != g->dims[0] || h.dims[1] != g->dims[1] ||
      h.dims[2] != g->dims[2] || (int)h.normalized != g->normalized) {
    rw_set_error_message("rw_basis_load: the basis belongs to a graph of another shape or form");
    return RW_ERR_INVALID_ARG;
  }
  const int m = m_load == 0 ? h.m : m_load;
  if (m > h.m || m > 4096) {
    rw_set_error_message("rw_basis_load: m_load exceeds the columns in the file");
    return RW_ERR_INVALID_ARG;
  }
  std::vector<double> lam(h.m);
  if (fread(lam.data(), sizeof(double), h.m, in.f) != (size_t)h.m) {
    rw_set_error_message("rw_basis_load: file truncated");
    return RW_ERR_INVALID_ARG;
  }
  // the first m columns of every row, a block of rows at a time
  const size_t file_row = sizeof(float) * (size_t)h.m;
  const size_t dev_row = sizeof(float) * (size_t)m;
  PinnedTmp buf;
  DevTmp X;
  RW_CHECK_CUDA(cudaMallocHost(&buf.p, file_row * kRowsPerBlock));
  RW_CHECK_CUDA(cudaMalloc(&X.p, dev_row * (size_t)h.N));
  for (int64_t r0 = 0; r0 < h.N; r0 += kRowsPerBlock) {
    const int64_t nr = std::min<int64_t>(kRowsPerBlock, h.N - r0);
    if (fread(buf.p, file_row, nr, in.f) != (size_t)nr) {
      rw_set_error_message("rw_basis_load: file truncated");
      return RW_ERR_INVALID_ARG;
    }
    RW_CHECK_CUDA(cudaMemcpy2DAsync(static_cast<char*>(X.p) + dev_row * r0, dev_row, buf.p,
                                    file_row, dev_row, nr, cudaMemcpyHostToDevice, st));
    RW_CHECK_CUDA(cudaStreamSynchronize(st));  // the pinned block is reused
  }
  return rw_make_basis(g, m, static_cast<const float*>(X.p), m, lam.data(), st, out);
}
