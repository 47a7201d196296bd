// Random-walker registration priors (Sec. IV-B): for every voxel x of the fixed image and every
// displacement label d_k, the local dissimilarity is the sum of absolute intensity differences
// between the fixed image at x and the moving image at x + d_k over a (2 h + 1)^d patch
// (patch voxels outside the volume take the nearest voxel inside); the prior is the negative
// exponential of its square, normalized to sum to 1 at each voxel.
//
// k_reg_sad: one thread per (voxel, label), label fastest, so a warp's threads share a voxel's
// fixed-image patch through L1.  k_reg_normalize: one thread per voxel, the log-sum-exp shift
// by the smallest squared dissimilarity.
#include "rw_internal.cuh"

namespace {

__device__ __forceinline__ int clampi(int v, int n) { return v < 0 ? 0 : (v >= n ? n - 1 : v); }

__global__ void __launch_bounds__(256)
k_reg_sad(const float* __restrict__ F, const float* __restrict__ M, int ndim, int DX, int DY,
          int DZ, const int32_t* __restrict__ disp, int K, int h, int64_t N,
          float* __restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * K) return;
  const int64_t i = e / K;
  const int k = (int)(e - i * K);
  const int x = (int)(i % DX), y = (int)((i / DX) % DY), z = (int)(i / ((int64_t)DX * DY));
  const int dx = disp[k * ndim + 0], dy = disp[k * ndim + 1];
  const int dz = ndim == 3 ? disp[k * ndim + 2] : 0;
  const int hz = ndim == 3 ? h : 0;
  float s = 0.f;
  for (int oz = -hz; oz <= hz; ++oz) {
    const int fz = clampi(z + oz, DZ), mz = clampi(z + oz + dz, DZ);
    for (int oy = -h; oy <= h; ++oy) {
      const int fy = clampi(y + oy, DY), my = clampi(y + oy + dy, DY);
      const int64_t frow = ((int64_t)fz * DY + fy) * DX, mrow = ((int64_t)mz * DY + my) * DX;
      for (int ox = -h; ox <= h; ++ox) {
        const float fv = __ldg(F + frow + clampi(x + ox, DX));
        const float mv = __ldg(M + mrow + clampi(x + ox + dx, DX));
        s += fabsf(fv - mv);
      }
    }
  }
  out[e] = s;
}

__global__ void __launch_bounds__(256)
k_reg_normalize(float* __restrict__ P, int K, int64_t N) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  float* p = P + i * K;
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
  k_reg_sad<<<rw_blocks(N * K, 256), 256, 0, st>>>(fixed_dev, moving_dev, ndim, DX, DY, DZ,
                                                   disp_dev, K, half, N, priors_dev);
  RW_LAUNCH_CHECK();
  k_reg_normalize<<<rw_blocks(N, 256), 256, 0, st>>>(priors_dev, K, N);
  RW_LAUNCH_CHECK();
  return RW_OK;
}
