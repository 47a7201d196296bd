// Gram products G = A^T B of tall node-major FP32 blocks on the 5th-generation tensor cores
// (tcgen05, TF32 with FP32 accumulation in tensor memory), for the block eigensolver's
// Rayleigh-Ritz and Cholesky-QR matrices (Sec. II-B, Eq. L_eigs).
//
// Precision.  A TF32 operand keeps 10 mantissa bits.  Each FP32 value is split as
// a = a_hi + a_lo with a_hi = a truncated to TF32 and a_lo = a - a_hi (exact in FP32); the
// product is taken as a_hi b_hi + a_hi b_lo + a_lo b_hi (the dropped a_lo b_lo is below 2^-20
// of |a b|), all three accumulated into the same FP32 tensor-memory accumulator.  Sums in
// tensor memory drift (measured: a 1024-row sum of squares of a unit column came out 2e-5 low),
// so an accumulator only ever sums 64 rows (24 MMA steps): two accumulators alternate, and the
// finished one is added into FP32 registers with round-to-nearest while the other fills.  A CTA
// covers 1024 rows; the per-CTA partial tiles are added in FP64, in a fixed order, by a second
// kernel (no atomics).
//
// Tiling.  One CTA (256 threads) owns a 128 x 256 output tile and a slice of 1024 rows; the
// rows stream through shared memory 32 at a time, double-buffered.  The operands of the MMA are
// K-major (the node index is the contraction index), while the blocks are node-major, so the
// threads transpose while splitting: a thread reads one column for a run of consecutive rows
// and stores each four hi and four lo values as one 16-byte chunk of the 128-byte-swizzled
// K-major tile.  One elected thread issues the 12 MMAs of a stage (3 products x 4 K-steps of 8)
// and commits them to the stage's mbarrier (and, at the end of a 64-row group, to the
// accumulator's); the threads wait on those mbarriers (bounded) before refilling a buffer or
// reading an accumulator.  Warp w reads accumulator lanes 32 (w % 4) .. + 31 with tcgen05.ld,
// columns 128 (w / 4) .. + 127.
#include "rw_internal.cuh"
#include "tc_common.cuh"

#include <algorithm>

using namespace rwtc;

namespace {

constexpr int kTM = 128;        // output rows per CTA (columns of A), MMA M
constexpr int kTN = 256;        // output columns per CTA (columns of B), MMA N
constexpr int kKB = 32;         // rows (nodes) per stage: one 128-byte TF32 row of K
constexpr int kSlice = 1024;    // rows per CTA
constexpr int kGroup = 2;       // stages per tensor-memory accumulation group (64 rows)
constexpr int kThreads = 256;
constexpr int kATile = kTM * 128;            // bytes of one K-major A tile (hi or lo)
constexpr int kBTile = kTN * 128;            // bytes of one K-major B tile
constexpr int kStage = 2 * kATile + 2 * kBTile;
constexpr int kSmem = 2 * kStage + 1024 + 64;  // two stages, alignment slack, barriers

// Instruction descriptor: dense, D = F32, A = B = TF32, both K-major, N = 256, M = 128.
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTN >> 3) << 17) |
                            ((uint32_t)(kTM >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ float tf32_hi(float a) {
  return __uint_as_float(__float_as_uint(a) & 0xFFFFE000u);
}

// Loads rows k0 + 4 j0 .. k0 + 4 (j0 + NJ) - 1 of column `col` (zero outside N x ncols),
// splits them and stores the hi and lo values as chunks j0 .. j0 + NJ - 1 of row `r` of the
// two tiles.
template <int NJ>
__device__ __forceinline__ void stage_column(const float* __restrict__ M, int64_t ld, int64_t N,
                                             int ncols, int col, int64_t k0, int j0,
                                             char* hi_tile, char* lo_tile, int r) {
  const bool cin = col < ncols;
  float v[4 * NJ];
#pragma unroll
  for (int k = 0; k < 4 * NJ; ++k) {
    const int64_t row = k0 + 4 * j0 + k;
    v[k] = (cin && row < N) ? __ldg(M + row * ld + col) : 0.f;
  }
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    float4 h, l;
    h.x = tf32_hi(v[4 * j + 0]); l.x = v[4 * j + 0] - h.x;
    h.y = tf32_hi(v[4 * j + 1]); l.y = v[4 * j + 1] - h.y;
    h.z = tf32_hi(v[4 * j + 2]); l.z = v[4 * j + 2] - h.z;
    h.w = tf32_hi(v[4 * j + 3]); l.w = v[4 * j + 3] - h.w;
    const int off = sw128_chunk(r, j0 + j);
    *reinterpret_cast<float4*>(hi_tile + off) = h;
    *reinterpret_cast<float4*>(lo_tile + off) = l;
  }
}

// 32 consecutive accumulator columns of this warp's 32 lanes (thread = lane)
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
        "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
        "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]),
        "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
        "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
        "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
}

__global__ void __launch_bounds__(kThreads, 1)
k_gram_tc(const float* __restrict__ A, int64_t lda, const float* __restrict__ B, int64_t ldb,
          int64_t N, int p, int q, float* __restrict__ part, int64_t ldp, int64_t slice_stride,
          int* status) {
  extern __shared__ __align__(1024) char smem_raw[];
  char* smem = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                       ~uintptr_t(1023));
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + 2 * kStage);   // [0,1]: stage buffers
  uint64_t* accbar = bar + 2;                                          // [0,1]: accumulators
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 4);
  __shared__ int wait_ok;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int i0 = blockIdx.x * kTM, j0 = blockIdx.y * kTN;
  const int64_t r0 = (int64_t)blockIdx.z * kSlice;
  const int64_t r1 = min(N, r0 + kSlice);
  const int nst = (int)((r1 - r0 + kKB - 1) / kKB);
  const int ng = (nst + kGroup - 1) / kGroup;

  if (tid == 0) {
    for (int k = 0; k < 4; ++k) mbar_init1(&bar[k]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {   // two accumulators of 256 columns: all 512 columns of tensor memory
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(tmem_slot)),
                 "r"(2 * kTN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  // Waits are taken by thread 0 and broadcast, so every thread leaves together on a timeout.
  auto wait_all = [&](uint64_t* b, unsigned parity) -> bool {
    if (tid == 0) wait_ok = mbar_wait_limited(b, parity, status) ? 1 : 0;
    __syncthreads();
    return wait_ok != 0;
  };
  // Every 64 rows the finished accumulator is added into FP32 registers (round to nearest), so
  // no tensor-memory sum runs over more than 24 MMA steps.  Warp w owns accumulator lanes
  // 32 (w % 4) .. + 31 and columns 128 (w / 4) .. + 127.
  float acc[kTN / 2];
#pragma unroll
  for (int c = 0; c < kTN / 2; ++c) acc[c] = 0.f;
  const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
  const uint32_t col_half = (uint32_t)((warp >> 2) * (kTN / 2));
  auto flush = [&](int gg) -> bool {
    if (!wait_all(&accbar[gg & 1], (gg >> 1) & 1)) return false;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t base = tmem + lane_base + (uint32_t)((gg & 1) * kTN) + col_half;
#pragma unroll
    for (int c0 = 0; c0 < kTN / 2; c0 += 32) {
      uint32_t v[32];
      tmem_ld32(base + (uint32_t)c0, v);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int u = 0; u < 32; ++u) acc[c0 + u] += __uint_as_float(v[u]);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    return true;
  };

  bool ok = true;
  for (int s = 0; s < nst && ok; ++s) {
    const int b = s & 1, g = s / kGroup;
    char* st = smem + b * kStage;
    if (s >= 2 && !wait_all(&bar[b], ((s - 2) >> 1) & 1)) { ok = false; break; }
    const int64_t k0 = r0 + (int64_t)s * kKB;
    const int64_t kend = min(r1, k0 + kKB);   // rows of the next slice are zeroed
    // A: threads t and t + 128 take column t, rows 0-15 and 16-31; B: thread t column t
    stage_column<kKB / 8>(A, lda, kend, p, i0 + (tid & 127), k0, (tid >> 7) * (kKB / 8), st,
                          st + kATile, tid & 127);
    stage_column<kKB / 4>(B, ldb, kend, q, j0 + tid, k0, 0, st + 2 * kATile,
                          st + 2 * kATile + kBTile, tid);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // visible to the MMA
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t d = tmem + (uint32_t)((g & 1) * kTN);
      const unsigned ahi = smem_addr(st), alo = ahi + kATile;
      const unsigned bhi = ahi + 2 * kATile, blo = bhi + kBTile;
      const bool first = (s % kGroup) == 0;
#pragma unroll
      for (int kk = 0; kk < kKB / 8; ++kk) {   // 8 TF32 values = 32 bytes per K-step
        const unsigned o = kk * 32;
        const uint32_t acc0 = (!first || kk > 0) ? 1u : 0u;
        mma_tf32(d, kmajor_desc(ahi + o), kmajor_desc(bhi + o), acc0);
        mma_tf32(d, kmajor_desc(ahi + o), kmajor_desc(blo + o), 1u);
        mma_tf32(d, kmajor_desc(alo + o), kmajor_desc(bhi + o), 1u);
      }
      mma_commit(&bar[b]);
      if ((s % kGroup) == kGroup - 1 || s == nst - 1) mma_commit(&accbar[g & 1]);
    }
    // the previous group finished issuing one stage ago: add it up while this one runs
    if ((s % kGroup) == 0 && g >= 1) ok = flush(g - 1);
  }
  if (ok && ng > 0) ok = flush(ng - 1);
  if (ok) {
    const int row = i0 + (warp & 3) * 32 + lane;
    if (row < p) {
      float* prow = part + (int64_t)blockIdx.z * slice_stride + (int64_t)row * ldp + j0 + col_half;
#pragma unroll
      for (int u = 0; u < kTN / 2; u += 4)
        *reinterpret_cast<float4*>(prow + u) = make_float4(acc[u], acc[u + 1], acc[u + 2],
                                                           acc[u + 3]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(2 * kTN)
                 : "memory");
}

// G[i][j] (+)= sum over slices of part[s][i][j], FP64, slices in order.
__global__ void k_gram_reduce(const float* __restrict__ part, int64_t ldp, int64_t slice_stride,
                              int nslices, int p, int q, double* __restrict__ G, int ldg,
                              int accumulate) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  if (j >= q) return;
  double acc = accumulate ? G[(int64_t)i * ldg + j] : 0.0;
  const float* pp = part + (int64_t)i * ldp + j;
  for (int s = 0; s < nslices; ++s) acc += (double)pp[(int64_t)s * slice_stride];
  G[(int64_t)i * ldg + j] = acc;
}

}  // namespace

size_t rw_gram_tc_scratch_bytes(int64_t N, int p, int q) {
  const int64_t ti = (p + kTM - 1) / kTM, tj = (q + kTN - 1) / kTN;
  const int64_t ns = (N + kSlice - 1) / kSlice;
  return sizeof(float) * (size_t)(ti * kTM) * (size_t)(tj * kTN) * (size_t)ns;
}

// G (p x q, row-major FP64, ldg) = (accumulate ? G : 0) + A^T B on the tensor cores.
// A: N x p (lda), B: N x q (ldb), node-major FP32; `scratch` holds at least
// rw_gram_tc_scratch_bytes(N, p, q) bytes; `status` is a device status word.
rw_status rw_gram_tc(const float* A, int64_t lda, const float* B, int64_t ldb, int64_t N, int p,
                     int q, double* G, int ldg, bool accumulate, void* scratch, int* status,
                     cudaStream_t st) {
  if (p <= 0 || q <= 0) return RW_OK;
  if (N <= 0) {
    if (!accumulate) RW_CHECK_CUDA(cudaMemset2DAsync(G, sizeof(double) * ldg, 0,
                                                     sizeof(double) * q, p, st));
    return RW_OK;
  }
  const int ti = (p + kTM - 1) / kTM, tj = (q + kTN - 1) / kTN;
  const int64_t ns = (N + kSlice - 1) / kSlice;
  if (ns > 65535) return RW_ERR_UNSUPPORTED;
  const int64_t ldp = (int64_t)tj * kTN;
  const int64_t slice_stride = (int64_t)ti * kTM * ldp;
  static int configured_dev = -1;
  int dev = 0;
  RW_CHECK_CUDA(cudaGetDevice(&dev));
  if (configured_dev != dev) {
    RW_CHECK_CUDA(cudaFuncSetAttribute(k_gram_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kSmem));
    configured_dev = dev;
  }
  float* part = static_cast<float*>(scratch);
  k_gram_tc<<<dim3(ti, tj, (unsigned)ns), kThreads, kSmem, st>>>(A, lda, B, ldb, N, p, q, part,
                                                                 ldp, slice_stride, status);
  RW_LAUNCH_CHECK();
  k_gram_reduce<<<dim3((q + 127) / 128, p), 128, 0, st>>>(part, ldp, slice_stride, (int)ns, p,
                                                          q, G, ldg, accumulate ? 1 : 0);
  RW_LAUNCH_CHECK();
  return RW_OK;
}

extern "C" size_t rw_block_gram_scratch_bytes(int64_t N, int32_t p, int32_t q) {
  if (N < 0 || p < 1 || q < 1) return 0;
  return 256 + rw_gram_tc_scratch_bytes(N, p, q);
}

extern "C" rw_status rw_block_gram(const float* A_dev, int64_t lda, const float* B_dev,
                                   int64_t ldb, int64_t N, int32_t p, int32_t q, double* G_dev,
                                   int32_t ldg, void* scratch_dev, size_t scratch_bytes,
                                   void* stream) {
  if (!A_dev || !B_dev || !G_dev || !scratch_dev) return RW_ERR_INVALID_ARG;
  if (N < 0 || p < 1 || q < 1 || lda < p || ldb < q || ldg < q) return RW_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(scratch_dev) & 255) != 0) return RW_ERR_INVALID_ARG;
  if (scratch_bytes < rw_block_gram_scratch_bytes(N, p, q)) {
    rw_set_error_message("rw_block_gram: scratch smaller than rw_block_gram_scratch_bytes()");
    return RW_ERR_INVALID_ARG;
  }
  if ((N + kSlice - 1) / kSlice > 65535) return RW_ERR_UNSUPPORTED;
  if (g_rw_num_sms <= 0) RW_TRY(rw_device_init());
  cudaStream_t st = rw_stream(stream);
  int* status = static_cast<int*>(scratch_dev);
  RW_CHECK_CUDA(cudaMemsetAsync(status, 0, sizeof(int), st));
  return rw_gram_tc(A_dev, lda, B_dev, ldb, N, p, q, G_dev, ldg, false,
                    static_cast<char*>(scratch_dev) + 256, status, st);
}
