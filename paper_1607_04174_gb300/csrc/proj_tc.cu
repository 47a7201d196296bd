// The two N-sized passes of the online solve over the 16-bit basis copy on the tensor cores
// (tcgen05, kind::f16, FP32 accumulation in tensor memory):
//   projection       Z = Q_n^T P-hat_n       (Eq. U_lin_comb: the m x l right-hand side)
//   back-projection  U-hat_n = Q_n C         (Eq. U_lin_comb: the solution from C, m x l)
// Both are dense contractions with l right-hand sides (l = 2..32 labels, the MMA's N padded to
// 16 or 32).  They read the basis once, 128 voxels per tile.  In the panel-major copy the 128
// consecutive voxels of one 8-column panel are 2048 contiguous bytes, so a tile arrives as one
// bulk copy per panel (completion counted in bytes on an mbarrier) into a tile made of 8-voxel x
// 16-byte core matrices without swizzle: it is the K-major A operand of the back-projection
// (M = voxels, K = columns) and the MN-major A operand of the projection (M = columns,
// K = voxels).  Tiles stream through a ring of stages (as many as the shared memory holds for
// the m of the call, at most kMaxStages).
//
// Warp roles.  Warps 0-3 are the epilogue (tensor-memory lane = voxel or column); one thread
// issues the bulk copies of each free stage; one thread issues the MMAs of each ready stage into
// a free accumulator (two alternate) and commits them to the stage's "empty" and the
// accumulator's "full" barrier; in the projection warps 4-7 turn each landed stage's P-hat rows
// into the B operand.  Every wait is bounded; a wait that gives up raises a block-wide abort
// that ends the others, and a block that aborts still lets its copies and MMAs finish before it
// frees its tensor memory.
//
// Precision.  The basis copy is exact as stored.  The other operand is FP32 (C, P-hat); it is
// split as v = hi + lo in the 16-bit type (after a power-of-two scale that keeps |v| below
// 2^14), and both halves are multiplied, so the products keep about 22 bits.  An accumulator
// sums one tile and is then added into FP32 registers (projection) or written out
// (back-projection).
#include "rw_internal.cuh"
#include "tc_common.cuh"

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

using namespace rwtc;

namespace {

constexpr int kTile = 128;                 // voxels per tile
constexpr int kChunkBytes = kTile * 16;    // one 8-column panel of a tile
constexpr int kEpi = 128;                  // epilogue threads (warps 0-3)
constexpr int kMaxStages = 8;
constexpr int kSmemBudget = 220 * 1024;    // dynamic shared memory of both kernels

template <typename T> struct TcType;
template <> struct TcType<__half> {
  static constexpr int fmt = 0;
  static __device__ __forceinline__ __half from(float v) { return __float2half_rn(v); }
  static __device__ __forceinline__ float to(__half v) { return __half2float(v); }
};
template <> struct TcType<__nv_bfloat16> {
  static constexpr int fmt = 1;
  static __device__ __forceinline__ __nv_bfloat16 from(float v) { return __float2bfloat16_rn(v); }
  static __device__ __forceinline__ float to(__nv_bfloat16 v) { return __bfloat162float(v); }
};

__device__ __forceinline__ char* align1024(char* p) {
  return reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(p) + 1023) & ~uintptr_t(1023));
}

// power of two that brings max |v| to [2^13, 2^14): v * scale and its 16-bit split stay normal
__device__ __forceinline__ float split_scale(float maxabs) {
  if (!(maxabs > 0.f) || !isfinite(maxabs)) return 1.f;
  int e;
  frexpf(maxabs, &e);   // maxabs = f 2^e, f in [0.5, 1)
  return ldexpf(1.f, 14 - e);
}

__device__ __forceinline__ float block_max(float v, float* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffff, v, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  float m = 0.f;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, red[w]);
  __syncthreads();
  return m;
}

__device__ __forceinline__ void zero_bytes(char* p, int bytes, int t0, int nthreads) {
  for (int e = t0; e < bytes / 16; e += nthreads)
    reinterpret_cast<float4*>(p)[e] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// one thread: bulk copies of the panels c < nch of voxels [i0, i0 + rows) into slots of 2048
// bytes, plus (extra, extra_bytes) when given, all counted on bar
template <typename T>
__device__ __forceinline__ void issue_tile(char* slot0, const T* __restrict__ Qp, int64_t N,
                                           int64_t i0, int rows, int nch, uint64_t* bar,
                                           char* extra = nullptr, const void* extra_src = nullptr,
                                           unsigned extra_bytes = 0) {
  const unsigned bytes = (unsigned)rows * 16u;
  mbar_expect_tx(bar, (unsigned)nch * bytes + extra_bytes);
  for (int c = 0; c < nch; ++c)
    bulk_g2s(slot0 + c * kChunkBytes, Qp + ((int64_t)c * N + i0) * 8, bytes, bar);
  if (extra_bytes) bulk_g2s(extra, extra_src, extra_bytes, bar);
}

// ---------------------------------------------------------------------------------------
// Back-projection, 192 threads (warps 0-3 epilogue, warp 4 copies, warp 5 MMAs):
// D (128 voxels x NL labels) = A (voxels x columns: the tile, K-major, core matrices 128 bytes
// apart along the voxels and 2048 along the columns) x B (columns x labels: C^T split hi / lo,
// K-major 128-byte-swizzled, row = label).  The epilogue writes either the refinement start
// (hat space, seeds = d^{1/2} one-hot) or U = d^{-1/2} U-hat with the labels, adding g_i c_eff
// when `nul` is given (gamma = 0); its per-voxel reads are issued one tile ahead.
// ---------------------------------------------------------------------------------------
constexpr int kBackThreads = 192;

template <typename T, int NL>
__global__ void __launch_bounds__(kBackThreads, 1)
k_backproject_tc(const T* __restrict__ Qp, int64_t N, int nchunk_max,
                 const float* __restrict__ Cg, int lp, float cscale,
                 const int* __restrict__ seedlab, const float* __restrict__ sq,
                 const float* __restrict__ s, int L, const int* __restrict__ mdev,
                 float* __restrict__ xhat, float* __restrict__ U, uint8_t* __restrict__ labels,
                 int* __restrict__ clear_seedlab, const float* __restrict__ nul,
                 int* __restrict__ status) {
  rw_grid_wait();
  rw_grid_trigger();
  extern __shared__ __align__(1024) char smem_raw[];
  char* sm = align1024(smem_raw);
  __shared__ uint64_t full[kMaxStages], empty[kMaxStages], accf[2], acce[2];
  __shared__ uint32_t tslot[1];
  __shared__ float red[kBackThreads / 32];
  __shared__ float nuls[NL];
  __shared__ int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int kchk_max = 2 * ((nchunk_max + 1) / 2);
  const int nblk_max = (kchk_max + 7) / 8;   // 64-column blocks of B
  const int BB = (NL / 8) * 1024;
  char* Bhi = sm;
  char* Blo = Bhi + nblk_max * BB;
  char* ring = Blo + nblk_max * BB;
  const int m = min(mdev[0], 8 * nchunk_max);
  const int nch = (m + 7) / 8, nk = (m + 15) / 16, nchk = 2 * nk;
  const int SB = nchk * kChunkBytes;
  const int nst = min(kMaxStages, (int)((smem_raw + kSmemBudget - ring) / SB));
  const int64_t ntile = (N + kTile - 1) / kTile;
  const int nt = (int64_t)blockIdx.x < ntile ? (int)((ntile - 1 - blockIdx.x) / gridDim.x + 1) : 0;
  auto tile_row = [&](int j) { return ((int64_t)blockIdx.x + (int64_t)j * gridDim.x) * kTile; };
  constexpr uint32_t kTcols = NL * 2 < 32 ? 32 : NL * 2;
  constexpr uint32_t kIdesc = f16_idesc(kTile, NL, TcType<T>::fmt, 0, 0);

  // B = (C scale)^T split into hi + lo, K-major (row = label, K = column)
  float mx = 0.f;
  for (int e = tid; e < m * L; e += blockDim.x) mx = fmaxf(mx, fabsf(Cg[(int64_t)(e / L) * lp + e % L]));
  const float scale = split_scale(block_max(mx, red));
  for (int e = tid; e < NL * nchk * 8; e += blockDim.x) {
    const int n = e / (nchk * 8), k = e % (nchk * 8);
    const float v = (n < L && k < m) ? Cg[(int64_t)k * lp + n] * scale : 0.f;
    const T h = TcType<T>::from(v);
    const T l = TcType<T>::from(v - TcType<T>::to(h));
    const int off = (k >> 6) * BB + sw128_chunk(n, (k & 63) >> 3) + (k & 7) * 2;
    *reinterpret_cast<T*>(Bhi + off) = h;
    *reinterpret_cast<T*>(Blo + off) = l;
  }
  // the padding panel of an odd panel count is zero in every stage (the copies never write it)
  if (nch < nchk)
    for (int st = 0; st < nst; ++st)
      zero_bytes(ring + st * SB + nch * kChunkBytes, kChunkBytes, tid, blockDim.x);
  if (tid < NL) nuls[tid] = (nul && tid < L) ? nul[tid] : 0.f;
  if (tid == 0) {
    for (int k = 0; k < kMaxStages; ++k) { mbar_init(&full[k], 1); mbar_init(&empty[k], 1); }
    for (int k = 0; k < 2; ++k) { mbar_init(&accf[k], 1); mbar_init(&acce[k], kEpi); }
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(tslot, kTcols);
  fence_async_smem();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tslot;
  volatile int* abort = &abort_flag;

  if (warp == 4) {   // copies
    if (lane == 0) {
      int issued = 0;
      for (int j = 0; j < nt; ++j) {
        const int st = j % nst;
        if (j >= nst &&
            !mbar_wait_limited(&empty[st], (unsigned)((j / nst) - 1) & 1u, status, abort))
          break;
        const int64_t i0 = tile_row(j);
        const int rows = (int)(N - i0 < kTile ? N - i0 : kTile);
        issue_tile(ring + st * SB, Qp, N, i0, rows, nch, &full[st]);
        issued = j + 1;
      }
      if (*abort)   // copies in flight land before the block exits
        for (int j = max(0, issued - nst); j < issued; ++j)
          mbar_wait_limited(&full[j % nst], (unsigned)(j / nst) & 1u, status);
    }
    __syncwarp();
  } else if (warp == 5) {   // MMAs
    if (lane == 0) {
      int issued = 0;
      for (int j = 0; j < nt; ++j) {
        const int st = j % nst, a = j & 1;
        if (!mbar_wait_limited(&full[st], (unsigned)(j / nst) & 1u, status, abort)) break;
        if (j >= 2 && !mbar_wait_limited(&acce[a], (unsigned)((j >> 1) - 1) & 1u, status, abort))
          break;
        fence_after_sync();
        const uint32_t d = tmem + (uint32_t)(a * NL);
        const unsigned a0 = smem_addr(ring + st * SB);
        const unsigned bh = smem_addr(Bhi), bl = smem_addr(Blo);
        for (int kk = 0; kk < nk; ++kk) {
          const uint64_t ad = plain_desc(a0 + (unsigned)(kk * 2 * kChunkBytes), kChunkBytes, 128);
          const unsigned kb = (unsigned)((kk >> 2) * BB + (kk & 3) * 32);
          mma_f16(d, ad, kmajor_desc(bh + kb), kIdesc, kk > 0 ? 1u : 0u);
          mma_f16(d, ad, kmajor_desc(bl + kb), kIdesc, 1u);
        }
        mma_commit(&empty[st]);
        mma_commit(&accf[a]);
        issued = j + 1;
      }
      if (*abort && issued > 0)   // the last MMAs finish before the tensor memory is freed
        mbar_wait_limited(&accf[(issued - 1) & 1], (unsigned)((issued - 1) >> 1) & 1u, status);
    }
    __syncwarp();
  } else {   // epilogue, warps 0-3: lane = voxel of the tile
    const float osc = cscale / scale;
    const bool hat_out = xhat != nullptr;
    int nsl = -1;
    float nsq = 0.f, ns = 0.f;
    auto prefetch = [&](int j) {
      const int64_t i = tile_row(j) + tid;
      if (j < nt && i < N) {
        nsl = __ldg(seedlab + i);
        if (hat_out || nul) nsq = __ldg(sq + i);
        if (!hat_out) ns = __ldg(s + i);
      }
    };
    prefetch(0);
    for (int j = 0; j < nt; ++j) {
      const int a = j & 1;
      const int sl = nsl;
      const float sqi = nsq, si = ns;
      prefetch(j + 1);
      if (!mbar_wait_limited(&accf[a], (unsigned)(j >> 1) & 1u, status, abort)) break;
      fence_after_sync();
      float v[NL];
#pragma unroll
      for (int c0 = 0; c0 < NL; c0 += 16) {
        float f[16];
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(a * NL + c0), f);
#pragma unroll
        for (int u = 0; u < 16; ++u) v[c0 + u] = f[u];
      }
      fence_before_sync();
      mbar_arrive(&acce[a]);
      const int64_t i = tile_row(j) + tid;
      if (i >= N) continue;
#pragma unroll
      for (int k = 0; k < NL; ++k) {
        v[k] *= osc;
        if (nul && sl < 0) v[k] = fmaf(sqi, nuls[k], v[k]);
      }
      if (hat_out) {
        float* xo = xhat + i * lp;
#pragma unroll
        for (int k4 = 0; k4 < NL; k4 += 4) {
          if (k4 < lp) {
            float o[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
              const int k = k4 + t;
              o[t] = (k >= L) ? 0.f : ((sl >= 0) ? (k == sl ? sqi : 0.f) : v[k]);
            }
            *reinterpret_cast<float4*>(xo + k4) = make_float4(o[0], o[1], o[2], o[3]);
          }
        }
      } else {
        int best = 0;
        float bv = -INFINITY;
#pragma unroll
        for (int k = 0; k < NL; ++k) {
          if (k < L) {
            const float u = (sl >= 0) ? (k == sl ? 1.f : 0.f) : v[k] * si;
            U[i * L + k] = u;
            if (u > bv) { bv = u; best = k; }
          }
        }
        if (labels) labels[i] = (uint8_t)best;
        if (clear_seedlab && sl >= 0) clear_seedlab[i] = -1;
      }
    }
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kTcols);
}

// ---------------------------------------------------------------------------------------
// Projection, 320 threads (warps 0-3 epilogue, warps 4-7 convert, warp 8 copies, warp 9 MMAs):
// D (128 columns x NL labels) += A (columns x voxels: the tile, MN-major, core matrices 2048
// bytes apart along the columns and 128 along the voxels) x B (voxels x labels: P-hat split
// hi / lo, K-major 128-byte-swizzled, row = label), for one or two 128-column halves.  A block
// owns a contiguous range of voxels.  Stage = [B hi | B lo | basis tile | P-hat rows (FP32)];
// the copy thread fills the tile and the P-hat rows, then converter thread pt turns row pt into
// B (zero for a seeded voxel or a row past the range, whose stale tile row it also clears) and
// marks the stage ready.  The seed labels come by cp.async, kLabAhead tiles ahead, into a small
// per-thread ring.  Each tile's products go to a fresh accumulator that the epilogue threads add
// into FP32 registers (thread = column 32 warp + lane of each half).  Partials as the CUDA-core
// projection writes them: part[block][column][label], lp labels, columns [0, 8 nchunk_max),
// scaled by kTcProjScale (P-hat below 2.5 stays normal in FP16 after it).
// ---------------------------------------------------------------------------------------
constexpr int kProjThreads = 320;
constexpr int kLabAhead = 4, kLabRing = 8;

template <typename T, int NL>
__global__ void __launch_bounds__(kProjThreads, 1)
k_project_tc(const T* __restrict__ Qp, int64_t N, int nchunk_max,
             const float* __restrict__ phat, int lp, const int* __restrict__ seedlab,
             const int* __restrict__ mdev, int64_t rows_per_block, float* __restrict__ part,
             int* __restrict__ status) {
  rw_grid_wait();
  rw_grid_trigger();
  extern __shared__ __align__(1024) char smem_raw[];
  char* sm = align1024(smem_raw);
  __shared__ uint64_t full[kMaxStages], ready[kMaxStages], empty[kMaxStages], accf[2], acce[2];
  __shared__ uint32_t tslot[1];
  __shared__ int labring[kLabRing][kTile];
  __shared__ int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m = min(mdev[0], 8 * nchunk_max);
  const int nch = (m + 7) / 8, nmt = (nch + 15) / 16, nchk = nmt * 16;   // 128-column halves
  const int BB = (NL / 8) * 1024;                // B: 64 voxels of one operand half
  const int offQ = 4 * BB;                       // [B hi | B lo] then the tile
  const int offP = offQ + nchk * kChunkBytes;    // then the P-hat rows
  const int SB = (offP + kTile * lp * 4 + 1023) & ~1023;
  const int nst = min(kMaxStages, (kSmemBudget - 1024) / SB);
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
  const int64_t r1 = min(N, r0 + rows_per_block);
  const int nt = r1 > r0 ? (int)((r1 - r0 + kTile - 1) / kTile) : 0;
  auto rows_of = [&](int j) {
    const int64_t left = r1 - (r0 + (int64_t)j * kTile);
    return (int)(left < kTile ? left : kTile);
  };
  constexpr uint32_t kTcols = 4 * NL < 32 ? 32 : 4 * NL;
  constexpr uint32_t kIdesc = f16_idesc(kTile, NL, TcType<T>::fmt, 1, 0);

  // the padding panels past the used columns are zero in every stage
  for (int st = 0; st < nst; ++st)
    zero_bytes(sm + st * SB + offQ + nch * kChunkBytes, (nchk - nch) * kChunkBytes, tid,
               blockDim.x);
  if (tid == 0) {
    for (int k = 0; k < kMaxStages; ++k) {
      mbar_init(&full[k], 1);
      mbar_init(&ready[k], kTile);
      mbar_init(&empty[k], 1);
    }
    for (int k = 0; k < 2; ++k) { mbar_init(&accf[k], 1); mbar_init(&acce[k], kEpi); }
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(tslot, kTcols);
  fence_async_smem();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tslot;
  volatile int* abort = &abort_flag;

  if (warp == 8) {   // copies
    if (lane == 0) {
      int issued = 0;
      for (int j = 0; j < nt; ++j) {
        const int st = j % nst;
        if (j >= nst &&
            !mbar_wait_limited(&empty[st], (unsigned)((j / nst) - 1) & 1u, status, abort))
          break;
        const int64_t i0 = r0 + (int64_t)j * kTile;
        const int rows = rows_of(j);
        char* stg = sm + st * SB;
        issue_tile(stg + offQ, Qp, N, i0, rows, nch, &full[st], stg + offP, phat + i0 * lp,
                   (unsigned)(rows * lp * 4));
        issued = j + 1;
      }
      if (*abort)
        for (int j = max(0, issued - nst); j < issued; ++j)
          mbar_wait_limited(&full[j % nst], (unsigned)(j / nst) & 1u, status);
    }
    __syncwarp();
  } else if (warp >= 4 && warp < 8) {   // convert: thread pt owns row pt of every tile
    const int pt = tid - 4 * 32;
    auto fetch_label = [&](int j) {
      if (j >= nt) return;
      int* dst = &labring[j % kLabRing][pt];
      const int64_t i = r0 + (int64_t)j * kTile + pt;
      const bool in = pt < rows_of(j);
      if (seedlab) cp_async4_zfill(dst, in ? seedlab + i : seedlab, in);
      else *dst = in ? -1 : 0;   // rows past the range read as seeded
    };
    for (int j = 0; j < kLabAhead; ++j) { fetch_label(j); cp_async_commit(); }
    for (int j = 0; j < nt; ++j) {
      const int st = j % nst;
      fetch_label(j + kLabAhead);
      cp_async_commit();
      if (!mbar_wait_limited(&full[st], (unsigned)(j / nst) & 1u, status, abort)) break;
      cp_async_wait<kLabAhead>();   // this tile's label (kLabAhead groups after it)
      char* stg = sm + st * SB;
      const bool in = pt < rows_of(j);
      const int lab = labring[j % kLabRing][pt];
      if (!in)   // a row past the range: its stale basis values must not be NaN
        for (int c = 0; c < nch; ++c)
          *reinterpret_cast<float4*>(stg + offQ + c * kChunkBytes + pt * 16) =
              make_float4(0.f, 0.f, 0.f, 0.f);
      const float* prow = reinterpret_cast<const float*>(stg + offP) + pt * lp;
      char* bh = stg;
      char* bl = stg + 2 * BB;
      const int base = (pt >> 6) * BB + (pt & 7) * 2;
#pragma unroll
      for (int n = 0; n < NL; ++n) {
        const float v = (in && lab < 0 && n < lp) ? prow[n] * kTcProjScale : 0.f;
        const T h = TcType<T>::from(v);
        const T l = TcType<T>::from(v - TcType<T>::to(h));
        const int off = base + sw128_chunk(n, (pt & 63) >> 3);
        *reinterpret_cast<T*>(bh + off) = h;
        *reinterpret_cast<T*>(bl + off) = l;
      }
      fence_async_smem();
      mbar_arrive(&ready[st]);
    }
    cp_async_wait_all();
  } else if (warp == 9) {   // MMAs
    if (lane == 0) {
      int issued = 0;
      for (int j = 0; j < nt; ++j) {
        const int st = j % nst, a = j & 1;
        if (!mbar_wait_limited(&ready[st], (unsigned)(j / nst) & 1u, status, abort)) break;
        if (j >= 2 && !mbar_wait_limited(&acce[a], (unsigned)((j >> 1) - 1) & 1u, status, abort))
          break;
        fence_after_sync();
        const unsigned s0 = smem_addr(sm + st * SB);
        const unsigned bhs = s0, bls = s0 + 2u * (unsigned)BB, q0 = s0 + (unsigned)offQ;
        for (int mt = 0; mt < nmt; ++mt) {
          const uint32_t d = tmem + (uint32_t)((a * 2 + mt) * NL);
          for (int kk = 0; kk < kTile / 16; ++kk) {
            const uint64_t ad = plain_desc(q0 + (unsigned)(16 * mt * kChunkBytes + kk * 256), 128,
                                           kChunkBytes);
            const unsigned kb = (unsigned)((kk >> 2) * BB + (kk & 3) * 32);
            mma_f16(d, ad, kmajor_desc(bhs + kb), kIdesc, kk > 0 ? 1u : 0u);
            mma_f16(d, ad, kmajor_desc(bls + kb), kIdesc, 1u);
          }
        }
        mma_commit(&empty[st]);
        mma_commit(&accf[a]);
        issued = j + 1;
      }
      if (*abort && issued > 0)
        mbar_wait_limited(&accf[(issued - 1) & 1], (unsigned)((issued - 1) >> 1) & 1u, status);
    }
    __syncwarp();
  } else {   // epilogue, warps 0-3: thread = column 32 warp + lane of each half
    float acc0[NL], acc1[NL];
#pragma unroll
    for (int k = 0; k < NL; ++k) { acc0[k] = 0.f; acc1[k] = 0.f; }
    bool done = true;
    for (int j = 0; j < nt; ++j) {
      const int a = j & 1;
      if (!mbar_wait_limited(&accf[a], (unsigned)(j >> 1) & 1u, status, abort)) { done = false; break; }
      fence_after_sync();
      const uint32_t lanes = (uint32_t)(warp * 32) << 16;
#pragma unroll
      for (int c0 = 0; c0 < NL; c0 += 16) {
        float f[16];
        tmem_ld16(tmem + lanes + (uint32_t)(a * 2 * NL + c0), f);
#pragma unroll
        for (int u = 0; u < 16; ++u) acc0[c0 + u] += f[u];
      }
      if (nmt > 1) {
#pragma unroll
        for (int c0 = 0; c0 < NL; c0 += 16) {
          float f[16];
          tmem_ld16(tmem + lanes + (uint32_t)((a * 2 + 1) * NL + c0), f);
#pragma unroll
          for (int u = 0; u < 16; ++u) acc1[c0 + u] += f[u];
        }
      }
      fence_before_sync();
      mbar_arrive(&acce[a]);
    }
    if (done) {
      const int ldq = 8 * nchunk_max;
      float* pb = part + (int64_t)blockIdx.x * ldq * lp;
      const int c0 = tid, c1 = 128 + tid;
      if (c0 < ldq) {
#pragma unroll
        for (int k = 0; k < NL; ++k)
          if (k < lp) pb[(int64_t)c0 * lp + k] = acc0[k];
      }
      if (c1 < ldq) {
#pragma unroll
        for (int k = 0; k < NL; ++k)
          if (k < lp) pb[(int64_t)c1 * lp + k] = nmt > 1 ? acc1[k] : 0.f;
      }
    }
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kTcols);
}

// whether two stages of the widest tile (m = 8 nchunk_max) fit beside the fixed parts
template <int NL>
bool back_fits(int nchunk_max) {
  const size_t kchk_max = 2 * ((nchunk_max + 1) / 2);
  const size_t nblk_max = (kchk_max + 7) / 8;
  return 1024 + 2 * nblk_max * (NL / 8) * 1024 + 2 * kchk_max * kChunkBytes <=
         (size_t)kSmemBudget;
}

template <int NL>
bool proj_fits(int nchunk_max, int lp) {
  const size_t nchk = 16 * (size_t)((nchunk_max + 15) / 16);
  const size_t SB = (4 * (size_t)(NL / 8) * 1024 + nchk * kChunkBytes + (size_t)kTile * lp * 4 +
                     1023) & ~(size_t)1023;
  return 1024 + 2 * SB <= (size_t)kSmemBudget;
}

template <typename F>
cudaError_t set_smem(F* f, size_t bytes) {
  return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename T, int NL>
rw_status back_launch(const T* Qp, int64_t N, int nchunk_max, const float* C, int lp,
                      float cscale, const int* seedlab, const float* sq, const float* s, int L,
                      const int* mdev, float* xhat, float* U, uint8_t* labels, int* clear,
                      const float* nul, int* status, int nblk, cudaStream_t st) {
  if (!back_fits<NL>(nchunk_max)) return RW_ERR_UNSUPPORTED;
  RW_CHECK_CUDA(set_smem(k_backproject_tc<T, NL>, kSmemBudget));
  RW_LAUNCH((k_backproject_tc<T, NL>), nblk, kBackThreads, kSmemBudget, st, Qp, N, nchunk_max, C,
            lp, cscale, seedlab, sq, s, L, mdev, xhat, U, labels, clear, nul, status);
  return RW_OK;
}

template <typename T, int NL>
rw_status proj_launch(const T* Qp, int64_t N, int nchunk_max, const float* phat, int lp,
                      const int* seedlab, const int* mdev, float* part, int nblk, int* status,
                      cudaStream_t st) {
  if (!proj_fits<NL>(nchunk_max, lp)) return RW_ERR_UNSUPPORTED;
  const int64_t rpb = (N + nblk - 1) / nblk;
  RW_CHECK_CUDA(set_smem(k_project_tc<T, NL>, kSmemBudget));
  RW_LAUNCH((k_project_tc<T, NL>), nblk, kProjThreads, kSmemBudget, st, Qp, N, nchunk_max, phat,
            lp, seedlab, mdev, rpb, part, status);
  return RW_OK;
}

}  // namespace

// Tensor-core projection: partials of Z = Q_n^T P-hat_n (scaled by kTcProjScale) for nblk
// blocks of voxels, in the CUDA-core projection's layout (k_reduce_partials adds them).
// lp <= 32, a multiple of 4; nchunk_max <= 32 (basis copies of at most 256 columns).
template <typename T>
rw_status rw_project_tc(const T* Qp, int64_t N, int nchunk_max, const float* phat, int lp,
                        const int* seedlab, const int* mdev, float* part, int nblk, int* status,
                        cudaStream_t st) {
  if (nchunk_max < 1 || nchunk_max > 32 || lp < 4 || lp > 32 || (lp & 3)) return RW_ERR_UNSUPPORTED;
  return lp <= 16 ? proj_launch<T, 16>(Qp, N, nchunk_max, phat, lp, seedlab, mdev, part, nblk, status, st)
                  : proj_launch<T, 32>(Qp, N, nchunk_max, phat, lp, seedlab, mdev, part, nblk, status, st);
}

// Tensor-core back-projection U-hat_n = Q_n C (C: m x lp FP32, rows >= m ignored) with the
// outputs of the CUDA-core back-projection.
template <typename T>
rw_status rw_backproject_tc(const T* Qp, int64_t N, int nchunk_max, const float* C, int lp,
                            float cscale, const int* seedlab, const float* sq, const float* s,
                            int L, const int* mdev, float* xhat, float* U, uint8_t* labels,
                            int* clear, const float* nul, int* status, int nblk, cudaStream_t st) {
  if (nchunk_max < 1 || nchunk_max > 32 || lp < 4 || lp > 32 || (lp & 3) || L > lp)
    return RW_ERR_UNSUPPORTED;
  return lp <= 16 ? back_launch<T, 16>(Qp, N, nchunk_max, C, lp, cscale, seedlab, sq, s, L, mdev,
                                       xhat, U, labels, clear, nul, status, nblk, st)
                  : back_launch<T, 32>(Qp, N, nchunk_max, C, lp, cscale, seedlab, sq, s, L, mdev,
                                       xhat, U, labels, clear, nul, status, nblk, st);
}

template rw_status rw_project_tc<__half>(const __half*, int64_t, int, const float*, int,
                                         const int*, const int*, float*, int, int*, cudaStream_t);
template rw_status rw_project_tc<__nv_bfloat16>(const __nv_bfloat16*, int64_t, int, const float*,
                                                int, const int*, const int*, float*, int, int*,
                                                cudaStream_t);
template rw_status rw_backproject_tc<__half>(const __half*, int64_t, int, const float*, int, float,
                                             const int*, const float*, const float*, int,
                                             const int*, float*, float*, uint8_t*, int*,
                                             const float*, int*, int, cudaStream_t);
template rw_status rw_backproject_tc<__nv_bfloat16>(const __nv_bfloat16*, int64_t, int,
                                                    const float*, int, float, const int*,
                                                    const float*, const float*, int, const int*,
                                                    float*, float*, uint8_t*, int*, const float*,
                                                    int*, int, cudaStream_t);
