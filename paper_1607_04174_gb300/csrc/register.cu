// Random-walker registration priors (Sec. IV-B): for every voxel x of the fixed image and every
// displacement label d_k, the local dissimilarity is the sum of absolute intensity differences
// between the fixed image at x and the moving image at x + d_k over a (2 h + 1)^d patch
// (patch voxels outside the volume take the nearest voxel inside); the prior is the negative
// exponential of its square, normalized to sum to 1 at each voxel.
//
// The patch sum is a box filter of A_k(y) = |F(clamp(y)) - M(clamp(y + d_k))| taken over the
// grid extended by h voxels on every side (so the clamping of each patch voxel is exactly the
// definition's), computed as one pass per axis of 2 h + 1 taps.  Every buffer is voxel-major
// with the K labels interleaved (label fastest), so each pass reads and writes coalesced:
//   k_reg_absdiff_x: A summed along x, computed from F and M on the fly (the extended grid
//                    shrunk back to the image along x; k_reg_absdiff_x_win for K <= 32 labels
//                    forms each difference once, in a sliding register window);
//   k_reg_box:       the sum along the middle axis (3-D: y);
//   k_reg_box_norm:  the sum along the last axis and the normalization, 32 voxels per block:
//                    the sums go through shared memory and one thread per voxel takes the
//                    log-sum-exp shift by the smallest squared sum.
// The sums are taken in the same order as the definition's passes (A, then x, y, z).
#include "rw_internal.cuh"

namespace {

__device__ __forceinline__ int clampi(int v, int n) { return v < 0 ? 0 : (v >= n ? n - 1 : v); }

// B[((ze * EY + ye) * DX + x) * K + k] = sum over t in [0, 2h] of A_k at extended (x + t, ye, ze),
// i.e. of |F - M(. + d_k)| at image coordinates (x + t - h, ye - h, ze - h), clamped.
// Grid: (row of DX K entries in blocks, ye, ze).
__global__ void __launch_bounds__(256)
k_reg_absdiff_x(const float* __restrict__ F, const float* __restrict__ M, int ndim, int DX,
                int DY, int DZ, const int32_t* __restrict__ disp, int K, int h, int EY, int EZ,
                float* __restrict__ B) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;   // entry of the row: x K + k
  if (r >= DX * K) return;
  const int x0 = r / K, k = r - x0 * K;
  const int ye = blockIdx.y, ze = blockIdx.z;
  const int64_t e = ((int64_t)ze * EY + ye) * DX * K + r;
  const int y = ye - (EY > DY ? h : 0), z = ze - (EZ > DZ ? h : 0);
  const int dx = disp[k * ndim + 0], dy = disp[k * ndim + 1];
  const int dz = ndim == 3 ? disp[k * ndim + 2] : 0;
  const float* Fr = F + ((int64_t)clampi(z, DZ) * DY + clampi(y, DY)) * DX;
  const float* Mr = M + ((int64_t)clampi(z + dz, DZ) * DY + clampi(y + dy, DY)) * DX;
  float sum = 0.f;
  for (int t = 0; t <= 2 * h; ++t) {
    const int x = x0 + t - h;
    sum += fabsf(__ldg(Fr + clampi(x, DX)) - __ldg(Mr + clampi(x + dx, DX)));
  }
  B[e] = sum;
}

// out[(z, y, x) in the output box][k] = sum over t in [0, 2h] of in[(z, y, x) + t along axis][k],
// in has extent (IX, IY, IZ), out (OX, OY, OZ) with the summed axis shorter by 2 h.
// Grid: (row of OX K entries in blocks, y, z).
__global__ void __launch_bounds__(256)
k_reg_box(const float* __restrict__ in, int IX, int IY, int axis, int h, int OX, int OY, int OZ,
          int K, float* __restrict__ out) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;   // x K + k
  if (r >= OX * K) return;
  const int y = blockIdx.y, z = blockIdx.z;
  const int64_t step = (axis == 0 ? 1 : (axis == 1 ? (int64_t)IX : (int64_t)IX * IY)) * K;
  const int64_t base = ((int64_t)z * IY + y) * IX * K + r;
  float s = 0.f;
  for (int t = 0; t <= 2 * h; ++t) s += __ldg(in + base + t * step);
  out[((int64_t)z * OY + y) * OX * K + r] = s;
}

// The same x pass for K <= 32 labels and half-width H: a warp takes 32 consecutive x of one
// row, lane = label; each difference is formed once and kept in a register window of 2 H + 1
// values, summed in the same order as above (same results).  Grid: (x segments of 128, ye, ze).
template <int H>
__global__ void __launch_bounds__(128)
k_reg_absdiff_x_win(const float* __restrict__ F, const float* __restrict__ M, int ndim, int DX,
                    int DY, int DZ, const int32_t* __restrict__ disp, int K, int EY, int EZ,
                    float* __restrict__ B) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int x0 = (blockIdx.x * 4 + warp) * 32;
  if (x0 >= DX) return;
  const int ye = blockIdx.y, ze = blockIdx.z;
  const int y = ye - (EY > DY ? H : 0), z = ze - (EZ > DZ ? H : 0);
  const bool act = lane < K;
  const int k = act ? lane : 0;
  const int dx = disp[k * ndim + 0], dy = disp[k * ndim + 1];
  const int dz = ndim == 3 ? disp[k * ndim + 2] : 0;
  const float* Fr = F + ((int64_t)clampi(z, DZ) * DY + clampi(y, DY)) * DX;
  const float* Mr = M + ((int64_t)clampi(z + dz, DZ) * DY + clampi(y + dy, DY)) * DX;
  auto diff = [&](int x) { return fabsf(__ldg(Fr + clampi(x, DX)) - __ldg(Mr + clampi(x + dx, DX))); };
  float win[2 * H + 1];
#pragma unroll
  for (int t = 0; t < 2 * H; ++t) win[t] = diff(x0 - H + t);
  const int x1 = min(DX, x0 + 32);
  float* out = B + ((int64_t)ze * EY + ye) * DX * K + k;
  for (int x = x0; x < x1; ++x) {
    win[2 * H] = diff(x + H);
    float sum = win[0];
#pragma unroll
    for (int t = 1; t <= 2 * H; ++t) sum += win[t];
    if (act) out[(int64_t)x * K] = sum;
#pragma unroll
    for (int t = 0; t < 2 * H; ++t) win[t] = win[t + 1];
  }
}

// the box sum along `axis` (as k_reg_box, output extent (OX, OY, OZ) = the image) and the
// priors: for the 32 voxels of a block, P_k = exp(lo - s_k^2) / sum_j exp(lo - s_j^2) with
// lo = min_k s_k^2; the block's sums and priors are contiguous, read and written coalesced
constexpr int kNormVox = 32;

// Grid: (32-voxel segments of a row, y, z).
__global__ void __launch_bounds__(256)
k_reg_box_norm(const float* __restrict__ in, int IX, int IY, int axis, int h, int OX, int OY,
               int K, float* __restrict__ P) {
  extern __shared__ float sbuf[];   // kNormVox x K sums
  const int x0 = blockIdx.x * kNormVox, y = blockIdx.y, z = blockIdx.z;
  const int nv = OX - x0 < kNormVox ? OX - x0 : kNormVox;
  const int64_t step = (axis == 0 ? 1 : (axis == 1 ? (int64_t)IX : (int64_t)IX * IY)) * K;
  const int64_t base = (((int64_t)z * IY + y) * IX + x0) * K;
  const int64_t v0 = ((int64_t)z * OY + y) * OX + x0;
  for (int e = threadIdx.x; e < nv * K; e += blockDim.x) {
    float s = 0.f;
    for (int t = 0; t <= 2 * h; ++t) s += __ldg(in + base + e + t * step);
    sbuf[e] = s;
  }
  __syncthreads();
  if (threadIdx.x < nv) {
    float* p = sbuf + threadIdx.x * K;
    float lo = INFINITY;
    for (int k = 0; k < K; ++k) lo = fminf(lo, p[k] * p[k]);
    float sum = 0.f;
    for (int k = 0; k < K; ++k) {
      const float v = expf(lo - p[k] * p[k]);
      p[k] = v;
      sum += v;
    }
    const float inv = 1.f / sum;
    for (int k = 0; k < K; ++k) p[k] *= inv;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nv * K; e += blockDim.x) P[v0 * K + e] = sbuf[e];
}

}  // namespace

extern "C" rw_status rw_registration_priors(const float* fixed_dev, const float* moving_dev,
                                            int32_t ndim, const int32_t* dims,
                                            const int32_t* disp_dev, int32_t K, int32_t half,
                                            float* priors_dev, void* stream) {
  if (!fixed_dev || !moving_dev || !dims || !disp_dev || !priors_dev) return RW_ERR_INVALID_ARG;
  if ((ndim != 2 && ndim != 3) || K < 1 || K > 4096 || half < 0 || half > 8)
    return RW_ERR_INVALID_ARG;
  const int DX = dims[0], DY = dims[1], DZ = ndim == 3 ? dims[2] : 1;
  if (DX < 1 || DY < 1 || DZ < 1) return RW_ERR_INVALID_ARG;
  const int64_t N = (int64_t)DX * DY * DZ;
  if (N * K > ((int64_t)1 << 40)) return RW_ERR_INVALID_ARG;
  cudaStream_t st = rw_stream(stream);
  const int EY = DY + 2 * half, EZ = ndim == 3 ? DZ + 2 * half : 1;
  const size_t norm_shm = sizeof(float) * kNormVox * (size_t)K;
  if (norm_shm > 200 * 1024) return RW_ERR_UNSUPPORTED;
  // the intermediate volumes: stream-ordered allocation, freed behind the last pass
  const int64_t nb = (int64_t)DX * EY * EZ * K, nc = ndim == 3 ? (int64_t)DX * DY * EZ * K : 0;
  void* scratch = nullptr;
  RW_CHECK_CUDA(cudaMallocAsync(&scratch, sizeof(float) * (size_t)(nb + nc), st));
  float* B = static_cast<float*>(scratch);
  float* C = B + nb;
  // x (fused with the differences): -> (DX, EY, EZ); 3-D y: -> (DX, DY, EZ); last axis with the
  // normalization: -> (DX, DY, DZ)
  if (DX * K > (1 << 30) || EY > 65535 || EZ > 65535) return RW_ERR_UNSUPPORTED;
  const unsigned rowblk = (unsigned)((DX * K + 255) / 256);
  const dim3 wgrid((unsigned)((DX + 127) / 128), EY, EZ);
  if (K <= 32 && half == 1)
    k_reg_absdiff_x_win<1><<<wgrid, 128, 0, st>>>(fixed_dev, moving_dev, ndim, DX, DY, DZ,
                                                 disp_dev, K, EY, EZ, B);
  else if (K <= 32 && half == 2)
    k_reg_absdiff_x_win<2><<<wgrid, 128, 0, st>>>(fixed_dev, moving_dev, ndim, DX, DY, DZ,
                                                 disp_dev, K, EY, EZ, B);
  else if (K <= 32 && half == 3)
    k_reg_absdiff_x_win<3><<<wgrid, 128, 0, st>>>(fixed_dev, moving_dev, ndim, DX, DY, DZ,
                                                 disp_dev, K, EY, EZ, B);
  else
    k_reg_absdiff_x<<<dim3(rowblk, EY, EZ), 256, 0, st>>>(fixed_dev, moving_dev, ndim, DX, DY,
                                                          DZ, disp_dev, K, half, EY, EZ, B);
  RW_LAUNCH_CHECK();
  if (norm_shm > 48 * 1024)
    RW_CHECK_CUDA(cudaFuncSetAttribute(k_reg_box_norm, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)norm_shm));
  const dim3 ngrid((unsigned)((DX + kNormVox - 1) / kNormVox), DY, DZ);
  if (ndim == 3) {
    k_reg_box<<<dim3(rowblk, DY, EZ), 256, 0, st>>>(B, DX, EY, 1, half, DX, DY, EZ, K, C);
    RW_LAUNCH_CHECK();
    k_reg_box_norm<<<ngrid, 256, norm_shm, st>>>(C, DX, DY, 2, half, DX, DY, K, priors_dev);
  } else {
    k_reg_box_norm<<<ngrid, 256, norm_shm, st>>>(B, DX, EY, 1, half, DX, DY, K, priors_dev);
  }
  RW_LAUNCH_CHECK();
  RW_CHECK_CUDA(cudaFreeAsync(scratch, st));
  return RW_OK;
}
