// The two N-sized passes of the online solve over the 16-bit basis copy on the tensor cores
// (tcgen05, kind::f16, FP32 accumulation in tensor memory):
//   projection       Z = Q_n^T P-hat_n       (Eq. U_lin_comb: the m x l right-hand side)
//   back-projection  U-hat_n = Q_n C         (Eq. U_lin_comb: the solution from C, m x l)
// Both are dense contractions with l right-hand sides (l = 2..32 labels, the MMA's N padded to
// 16 or 32).  They read the basis once, 128 voxels per tile: the tile's 16-byte rows of each
// 8-column panel are copied by cp.async into a 128-byte-swizzled shared tile (row = voxel,
// 128 bytes = 64 columns), which serves as the K-major A operand of the back-projection
// (M = voxels, K = columns) and as the MN-major A operand of the projection (M = columns,
// K = voxels).  Tiles stream through NS stages; one elected thread issues the MMAs and commits
// them to an mbarrier; the waits are bounded (RW_DEV_TIMEOUT) and a kernel that gives up still
// drains its copies and frees its tensor memory.
//
// Precision.  The basis copy is exact as stored.  The other operand is FP32 (C, P-hat); it is
// split as v = hi + lo in the 16-bit type (after a power-of-two scale that keeps |v| below
// 2^14), and both halves are multiplied, so the products keep about 22 bits.  An accumulator
// sums one tile (at most 2 x 14 MMAs) and is then added into FP32 registers (projection) or
// written out (back-projection).
#include "rw_internal.cuh"
#include "tc_common.cuh"

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

using namespace rwtc;

namespace {

constexpr int kTile = 128;                 // voxels per tile (MMA M of the back-projection)
constexpr int kBlockBytes = kTile * 128;   // one 64-column block of a basis tile

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

// Rows [i0, i0 + 128) of the panel-major basis (panel c = columns 8c..8c+7, element (i, 8c + v)
// at ((c N + i) 8 + v)), chunks [0, nchk), into the swizzled tile: chunk c of row r at
// (c / 8) * kBlockBytes + sw128_chunk(r, c % 8).  Chunks >= nch and rows >= i1 are zeros.
template <typename T>
__device__ __forceinline__ void stage_basis(char* tile, const T* __restrict__ Qp, int64_t N,
                                            int64_t i0, int64_t i1, int nch, int nchk) {
  for (int e = threadIdx.x; e < nchk * kTile; e += blockDim.x) {
    const int r = e & (kTile - 1), c = e / kTile;
    const int64_t i = i0 + r;
    const bool valid = c < nch && i < i1;
    const T* src = valid ? Qp + ((int64_t)c * N + i) * 8 : Qp;
    cp_async16_zfill(tile + (c >> 3) * kBlockBytes + sw128_chunk(r, c & 7), src, valid);
  }
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

// ---------------------------------------------------------------------------------------
// Back-projection: D (128 voxels x NL labels) = A (voxels x columns, K-major basis tile)
// x B (columns x labels, C^T split hi / lo, K-major: row = label).  Two accumulators alternate
// between tiles, so the epilogue of one tile (warps 0-3: lane = voxel) overlaps the MMAs of
// the next.  The epilogue writes either the refinement start (hat space, seeds = d^{1/2}
// one-hot) or U = d^{-1/2} U-hat with the labels, adding g_i c_eff when `nul` is given
// (gamma = 0).
// ---------------------------------------------------------------------------------------
template <typename T, int NL, int NS>
__global__ void __launch_bounds__(256, 1)
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
  const int kchk_max = 2 * ((nchunk_max + 1) / 2);
  const int nblk_max = (kchk_max + 7) / 8;
  const int SB = nblk_max * kBlockBytes;
  const int BB = (NL / 8) * 1024;            // one 64-column block of B
  char* Bhi = sm + NS * SB;
  char* Blo = Bhi + nblk_max * BB;
  uint64_t* bar = reinterpret_cast<uint64_t*>(Blo + nblk_max * BB);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 2);
  __shared__ float red[8];
  __shared__ float nuls[NL];
  __shared__ int wait_ok;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m = min(mdev[0], 8 * nchunk_max);
  const int nch = (m + 7) / 8, nk = (m + 15) / 16, nchk = 2 * nk;
  const int64_t ntile = (N + kTile - 1) / kTile;
  const int nt = (int64_t)blockIdx.x < ntile ? (int)((ntile - 1 - blockIdx.x) / gridDim.x + 1) : 0;
  auto tile_row = [&](int j) { return ((int64_t)blockIdx.x + (int64_t)j * gridDim.x) * kTile; };
  constexpr uint32_t kTcols = NL * 2 < 32 ? 32 : NL * 2;
  constexpr uint32_t kIdesc = f16_idesc(kTile, NL, TcType<T>::fmt, 0, 0);

  // the first stages' basis tiles are requested before B is built
#pragma unroll
  for (int j = 0; j < NS; ++j) {
    if (j < nt) stage_basis(sm + j * SB, Qp, N, tile_row(j), N, nch, nchk);
    cp_async_commit();
  }
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
  if (tid < NL) nuls[tid] = (nul && tid < L) ? nul[tid] : 0.f;
  if (tid == 0) {
    mbar_init1(&bar[0]);
    mbar_init1(&bar[1]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(tslot, kTcols);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tslot;
  const float osc = cscale / scale;
  const bool hat_out = xhat != nullptr;

  auto epilogue = [&](int j) {
    const int r = warp * 32 + lane;
    const int64_t i = tile_row(j) + r;
    float v[NL];
#pragma unroll
    for (int c0 = 0; c0 < NL; c0 += 16) {
      float f[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)((j & 1) * NL + c0), f);
#pragma unroll
      for (int u = 0; u < 16; ++u) v[c0 + u] = f[u];
    }
    if (i >= N) return;
    const int sl = seedlab[i];
    const float sqi = (hat_out || nul) ? sq[i] : 0.f;
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
      const float si = s[i];
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
  };

  bool ok = true;
  int issued = 0;   // tiles whose MMAs were issued
  for (int j = 0; j <= nt; ++j) {
    if (j < nt) {
      // this tile's group: the groups after it are tiles j + 1 .. j + NS - 1 (j = 0) or
      // j + 1 .. j + NS - 2 (the refill of tile j + NS - 1 is committed after this point)
      if (j == 0) cp_async_wait<NS - 1>(); else cp_async_wait<NS - 2>();
      fence_async_smem();
      __syncthreads();
      if (tid == 0) {
        fence_after_sync();
        const uint32_t d = tmem + (uint32_t)((j & 1) * NL);
        const unsigned a0 = smem_addr(sm + (j % NS) * SB);
        const unsigned bh = smem_addr(Bhi), bl = smem_addr(Blo);
        for (int kk = 0; kk < nk; ++kk) {
          const unsigned ko = (unsigned)((kk >> 2) * kBlockBytes + (kk & 3) * 32);
          const unsigned kb = (unsigned)((kk >> 2) * BB + (kk & 3) * 32);
          const uint64_t ad = kmajor_desc(a0 + ko);
          mma_f16(d, ad, kmajor_desc(bh + kb), kIdesc, kk > 0 ? 1u : 0u);
          mma_f16(d, ad, kmajor_desc(bl + kb), kIdesc, 1u);
        }
        mma_commit(&bar[j & 1]);
      }
      issued = j + 1;
    }
    if (j >= 1) {
      const int jp = j - 1;
      if (tid == 0) wait_ok = mbar_wait_limited(&bar[jp & 1], (jp >> 1) & 1, status) ? 1 : 0;
      __syncthreads();
      if (!wait_ok) { ok = false; break; }
      fence_after_sync();
      if (warp < 4) epilogue(jp);
      fence_before_sync();
      // the stage of tile jp is free: refill it with tile jp + NS
      if (jp + NS < nt) stage_basis(sm + (jp % NS) * SB, Qp, N, tile_row(jp + NS), N, nch, nchk);
      cp_async_commit();
    }
  }
  if (!ok && issued > 0 && tid == 0) {   // let the last issued MMAs finish before freeing
    const int jl = issued - 1;
    mbar_wait_limited(&bar[jl & 1], (jl >> 1) & 1, status);
  }
  cp_async_wait_all();
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kTcols);
}

// ---------------------------------------------------------------------------------------
// Projection: D (128 columns x NL labels) += A (columns x voxels: the basis tile, MN-major)
// x B (voxels x labels: P-hat split hi / lo, K-major: row = label, K = voxel), for one or two
// 128-column halves.  A CTA owns a contiguous range of voxels; each tile's products go to a
// fresh accumulator (two alternate) that the threads then add into FP32 registers (warp w:
// column half w / 4, lanes 32 (w % 4)..).  Seeded voxels and voxels outside the range are zero
// rows of B.  Partials as the CUDA-core projection writes them: part[block][column][label], lp
// labels, columns [0, 8 nchunk_max), scaled by 2^12 (P-hat below 2.5 stays normal in FP16).
// ---------------------------------------------------------------------------------------
template <typename T, int NL, int NS>
__global__ void __launch_bounds__(256, 1)
k_project_tc(const T* __restrict__ Qp, int64_t N, int nchunk_max,
             const float* __restrict__ phat, int lp, const int* __restrict__ seedlab,
             const int* __restrict__ mdev, int64_t rows_per_block, float* __restrict__ part,
             int* __restrict__ status) {
  rw_grid_wait();
  rw_grid_trigger();
  extern __shared__ __align__(1024) char smem_raw[];
  char* sm = align1024(smem_raw);
  const int nmt_max = (nchunk_max + 15) / 16;   // 128-column halves
  const int SBq = nmt_max * 2 * kBlockBytes;     // basis tile
  const int SBp = kTile * lp * 4;                // P-hat rows (FP32)
  // + seed labels; stages (and B after them) start on 1024-byte boundaries, as the swizzle of
  // the MMA operands is taken from the shared-memory address
  const int SB = (SBq + SBp + kTile * 4 + 1023) & ~1023;
  const int BB = (NL / 8) * 1024;                // B: 64 voxels of one operand half
  char* Bbuf = sm + NS * SB;                     // [2 parities][hi, lo][2 voxel blocks] x BB
  uint64_t* bar = reinterpret_cast<uint64_t*>(Bbuf + 2 * 2 * 2 * BB);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 2);
  __shared__ int wait_ok;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m = min(mdev[0], 8 * nchunk_max);
  const int nch = (m + 7) / 8, nmt = (nch + 15) / 16, nchk = nmt * 16;
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
  const int64_t r1 = min(N, r0 + rows_per_block);
  const int nt = r1 > r0 ? (int)((r1 - r0 + kTile - 1) / kTile) : 0;
  constexpr uint32_t kTcols = 4 * NL < 32 ? 32 : 4 * NL;
  constexpr uint32_t kIdesc = f16_idesc(kTile, NL, TcType<T>::fmt, 1, 0);

  auto issue = [&](int j) {
    char* st = sm + (j % NS) * SB;
    const int64_t i0 = r0 + (int64_t)j * kTile;
    stage_basis(st, Qp, N, i0, r1, nch, nchk);
    float* praw = reinterpret_cast<float*>(st + SBq);
    int* lraw = reinterpret_cast<int*>(st + SBq + SBp);
    const int q4 = lp / 4;
    for (int e = tid; e < kTile * q4; e += blockDim.x) {
      const int r = e / q4, c = e % q4;
      const int64_t i = i0 + r;
      const bool valid = i < r1;
      cp_async16_zfill(praw + r * lp + 4 * c, valid ? phat + i * lp + 4 * c : phat, valid);
    }
    for (int r = tid; r < kTile; r += blockDim.x) {   // padding rows read as seeded (0)
      const int64_t i = i0 + r;
      if (seedlab) cp_async4_zfill(lraw + r, i < r1 ? seedlab + i : seedlab, i < r1);
      else lraw[r] = i < r1 ? -1 : 0;
    }
  };
#pragma unroll
  for (int j = 0; j < NS; ++j) {
    if (j < nt) issue(j);
    cp_async_commit();
  }
  if (tid == 0) {
    mbar_init1(&bar[0]);
    mbar_init1(&bar[1]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(tslot, kTcols);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tslot;
  const int half = warp >> 2;              // column half owned by this warp
  const int col = half * 128 + (warp & 3) * 32 + lane;
  float acc[NL];
#pragma unroll
  for (int k = 0; k < NL; ++k) acc[k] = 0.f;

  bool ok = true;
  int issued = 0;
  for (int j = 0; j <= nt; ++j) {
    if (j < nt) {
      if (j == 0) cp_async_wait<NS - 1>(); else cp_async_wait<NS - 2>();
      __syncthreads();
      // B of this tile from the staged rows: K-major (row = label), voxel pairs as adjacent
      // 16-bit stores; seeded voxels (label >= 0) and padding rows are zero
      const char* st = sm + (j % NS) * SB;
      const float* praw = reinterpret_cast<const float*>(st + SBq);
      const int* lraw = reinterpret_cast<const int*>(st + SBq + SBp);
      char* bh = Bbuf + (j & 1) * 4 * BB;
      char* bl = bh + 2 * BB;
      for (int e = tid; e < (kTile / 2) * NL; e += blockDim.x) {
        const int p = e % (kTile / 2), n = e / (kTile / 2);
        const int r = 2 * p;
        const bool u0 = n < lp && lraw[r] < 0, u1 = n < lp && lraw[r + 1] < 0;
        const float v0 = u0 ? praw[r * lp + n] * kTcProjScale : 0.f;
        const float v1 = u1 ? praw[(r + 1) * lp + n] * kTcProjScale : 0.f;
        const T h0 = TcType<T>::from(v0), h1 = TcType<T>::from(v1);
        const T l0 = TcType<T>::from(v0 - TcType<T>::to(h0));
        const T l1 = TcType<T>::from(v1 - TcType<T>::to(h1));
        const int off = (r >> 6) * BB + sw128_chunk(n, (r & 63) >> 3) + (r & 7) * 2;
        T* ph = reinterpret_cast<T*>(bh + off);
        T* pl = reinterpret_cast<T*>(bl + off);
        ph[0] = h0; ph[1] = h1;
        pl[0] = l0; pl[1] = l1;
      }
      fence_async_smem();
      __syncthreads();
      if (tid == 0) {
        fence_after_sync();
        const unsigned a0 = smem_addr(st);
        const unsigned bhs = smem_addr(bh), bls = smem_addr(bl);
        for (int mt = 0; mt < nmt; ++mt) {
          const uint32_t d = tmem + (uint32_t)(((j & 1) * 2 + mt) * NL);
          for (int kk = 0; kk < kTile / 16; ++kk) {
            const uint64_t ad = sw128_desc(a0 + (unsigned)(2 * mt * kBlockBytes + kk * 2048),
                                           kBlockBytes, 1024);
            const unsigned kb = (unsigned)((kk >> 2) * BB + (kk & 3) * 32);
            mma_f16(d, ad, kmajor_desc(bhs + kb), kIdesc, kk > 0 ? 1u : 0u);
            mma_f16(d, ad, kmajor_desc(bls + kb), kIdesc, 1u);
          }
        }
        mma_commit(&bar[j & 1]);
      }
      issued = j + 1;
    }
    if (j >= 1) {
      const int jp = j - 1;
      if (tid == 0) wait_ok = mbar_wait_limited(&bar[jp & 1], (jp >> 1) & 1, status) ? 1 : 0;
      __syncthreads();
      if (!wait_ok) { ok = false; break; }
      fence_after_sync();
      if (half < nmt) {
#pragma unroll
        for (int c0 = 0; c0 < NL; c0 += 16) {
          float f[16];
          tmem_ld16(tmem + ((uint32_t)((warp & 3) * 32) << 16) +
                        (uint32_t)(((jp & 1) * 2 + half) * NL + c0), f);
#pragma unroll
          for (int u = 0; u < 16; ++u) acc[c0 + u] += f[u];
        }
      }
      fence_before_sync();
      if (jp + NS < nt) issue(jp + NS);
      cp_async_commit();
    }
  }
  if (!ok && issued > 0 && tid == 0) {
    const int jl = issued - 1;
    mbar_wait_limited(&bar[jl & 1], (jl >> 1) & 1, status);
  }
  cp_async_wait_all();
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kTcols);
  if (!ok) return;
  const int ldq = 8 * nchunk_max;
  float* pb = part + (int64_t)blockIdx.x * ldq * lp;
  if (col < ldq) {
#pragma unroll
    for (int k = 0; k < NL; ++k)
      if (k < lp) pb[(int64_t)col * lp + k] = half < nmt ? acc[k] : 0.f;
  }
}

template <int NL, int NS>
size_t back_smem(int nchunk_max) {
  const int kchk_max = 2 * ((nchunk_max + 1) / 2);
  const int nblk_max = (kchk_max + 7) / 8;
  return 1024 + (size_t)NS * nblk_max * kBlockBytes + 2 * (size_t)nblk_max * (NL / 8) * 1024 + 64;
}

template <int NL, int NS>
size_t proj_smem(int nchunk_max, int lp) {
  const int nmt_max = (nchunk_max + 15) / 16;
  const size_t SB = ((size_t)nmt_max * 2 * kBlockBytes + (size_t)kTile * lp * 4 + kTile * 4 + 1023) &
                    ~(size_t)1023;
  return 1024 + NS * SB + 2 * 2 * 2 * (size_t)(NL / 8) * 1024 + 64;
}

constexpr size_t kSmemBudget = 220 * 1024;

template <typename F>
cudaError_t set_smem(F* f, size_t bytes) {
  return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename T, int NL, int NS>
rw_status back_launch_ns(const T* Qp, int64_t N, int nchunk_max, const float* C, int lp,
                         float cscale, const int* seedlab, const float* sq, const float* s,
                         int L, const int* mdev, float* xhat, float* U, uint8_t* labels,
                         int* clear, const float* nul, int* status, int nblk, cudaStream_t st) {
  const size_t shm = back_smem<NL, NS>(nchunk_max);
  RW_CHECK_CUDA(set_smem(k_backproject_tc<T, NL, NS>, shm));
  RW_LAUNCH((k_backproject_tc<T, NL, NS>), nblk, 256, shm, st, Qp, N, nchunk_max, C, lp, cscale,
            seedlab, sq, s, L, mdev, xhat, U, labels, clear, nul, status);
  return RW_OK;
}

template <typename T, int NL>
rw_status back_launch(const T* Qp, int64_t N, int nchunk_max, const float* C, int lp,
                      float cscale, const int* seedlab, const float* sq, const float* s, int L,
                      const int* mdev, float* xhat, float* U, uint8_t* labels, int* clear,
                      const float* nul, int* status, int nblk, cudaStream_t st) {
  if (back_smem<NL, 4>(nchunk_max) <= kSmemBudget)
    return back_launch_ns<T, NL, 4>(Qp, N, nchunk_max, C, lp, cscale, seedlab, sq, s, L, mdev,
                                    xhat, U, labels, clear, nul, status, nblk, st);
  if (back_smem<NL, 3>(nchunk_max) <= kSmemBudget)
    return back_launch_ns<T, NL, 3>(Qp, N, nchunk_max, C, lp, cscale, seedlab, sq, s, L, mdev,
                                    xhat, U, labels, clear, nul, status, nblk, st);
  if (back_smem<NL, 2>(nchunk_max) <= kSmemBudget)
    return back_launch_ns<T, NL, 2>(Qp, N, nchunk_max, C, lp, cscale, seedlab, sq, s, L, mdev,
                                    xhat, U, labels, clear, nul, status, nblk, st);
  return RW_ERR_UNSUPPORTED;
}

template <typename T, int NL, int NS>
rw_status proj_launch_ns(const T* Qp, int64_t N, int nchunk_max, const float* phat, int lp,
                         const int* seedlab, const int* mdev, float* part, int nblk, int* status,
                         cudaStream_t st) {
  const int64_t rpb = (N + nblk - 1) / nblk;
  const size_t shm = proj_smem<NL, NS>(nchunk_max, lp);
  RW_CHECK_CUDA(set_smem(k_project_tc<T, NL, NS>, shm));
  RW_LAUNCH((k_project_tc<T, NL, NS>), nblk, 256, shm, st, Qp, N, nchunk_max, phat, lp, seedlab,
            mdev, rpb, part, status);
  return RW_OK;
}

template <typename T, int NL>
rw_status proj_launch(const T* Qp, int64_t N, int nchunk_max, const float* phat, int lp,
                      const int* seedlab, const int* mdev, float* part, int nblk, int* status,
                      cudaStream_t st) {
  if (proj_smem<NL, 4>(nchunk_max, lp) <= kSmemBudget)
    return proj_launch_ns<T, NL, 4>(Qp, N, nchunk_max, phat, lp, seedlab, mdev, part, nblk, status, st);
  if (proj_smem<NL, 3>(nchunk_max, lp) <= kSmemBudget)
    return proj_launch_ns<T, NL, 3>(Qp, N, nchunk_max, phat, lp, seedlab, mdev, part, nblk, status, st);
  if (proj_smem<NL, 2>(nchunk_max, lp) <= kSmemBudget)
    return proj_launch_ns<T, NL, 2>(Qp, N, nchunk_max, phat, lp, seedlab, mdev, part, nblk, status, st);
  return RW_ERR_UNSUPPORTED;
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
