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
//   k_reg_absdiff: A on the extended grid;
//   k_reg_box:     the sum along one axis, shrinking that axis back to the image;
//   k_reg_normalize: one thread per voxel, log-sum-exp shift by the smallest squared sum.
#include "rw_internal.cuh"

namespace {

__device__ __forceinline__ int clampi(int v, int n) { return v < 0 ? 0 : (v >= n ? n - 1 : v); }

// A[((ze * EY + ye) * EX + xe) * K + k], extended coordinates xe = x + h, ...
__global__ void __launch_bounds__(256)
k_reg_absdiff(const float* __restrict__ F, const float* __restrict__ M, int ndim, int DX, int DY,
              int DZ, const int32_t* __restrict__ disp, int K, int h, int EX, int EY, int EZ,
              float* __restrict__ A) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t total = (int64_t)EX * EY * EZ * K;
  if (e >= total) return;
  const int64_t v = e / K;
  const int k = (int)(e - v * K);
  const int xe = (int)(v % EX), ye = (int)((v / EX) % EY), ze = (int)(v / ((int64_t)EX * EY));
  const int x = xe - h, y = ye - (EY > DY ? h : 0), z = ze - (EZ > DZ ? h : 0);
  const int dx = disp[k * ndim + 0], dy = disp[k * ndim + 1];
  const int dz = ndim == 3 ? disp[k * ndim + 2] : 0;
  const float fv = __ldg(F + ((int64_t)clampi(z, DZ) * DY + clampi(y, DY)) * DX + clampi(x, DX));
  const float mv = __ldg(M + ((int64_t)clampi(z + dz, DZ) * DY + clampi(y + dy, DY)) * DX +
                         clampi(x + dx, DX));
  A[e] = fabsf(fv - mv);
}

// out[(z, y, x) in the output box][k] = sum over t in [0, 2h] of in[(z, y, x) + t along axis][k],
// in has extent (IX, IY, IZ), out (OX, OY, OZ) with the summed axis shorter by 2 h
__global__ void __launch_bounds__(256)
k_reg_box(const float* __restrict__ in, int IX, int IY, int axis, int h, int OX, int OY, int OZ,
          int K, float* __restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t total = (int64_t)OX * OY * OZ * K;
  if (e >= total) return;
  const int64_t v = e / K;
  const int k = (int)(e - v * K);
  const int x = (int)(v % OX), y = (int)((v / OX) % OY), z = (int)(v / ((int64_t)OX * OY));
  const int64_t step = axis == 0 ? 1 : (axis == 1 ? (int64_t)IX : (int64_t)IX * IY);
  const int64_t base = (((int64_t)z * IY + y) * IX + x) * K + k;
  float s = 0.f;
  for (int t = 0; t <= 2 * h; ++t) s += __ldg(in + base + t * step * K);
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
  const int EX = DX + 2 * half, EY = DY + 2 * half, EZ = ndim == 3 ? DZ + 2 * half : 1;
  const int64_t ext = (int64_t)EX * EY * EZ * K;
  // the two intermediate volumes: stream-ordered allocation, freed behind the last pass
  void* scratch = nullptr;
  RW_CHECK_CUDA(cudaMallocAsync(&scratch, 2 * sizeof(float) * (size_t)ext, st));
  float* A = static_cast<float*>(scratch);
  float* B = A + ext;
  k_reg_absdiff<<<rw_blocks(ext, 256), 256, 0, st>>>(fixed_dev, moving_dev, ndim, DX, DY, DZ,
                                                     disp_dev, K, half, EX, EY, EZ, A);
  RW_LAUNCH_CHECK();
  // x: (EX, EY, EZ) -> (DX, EY, EZ); y: -> (DX, DY, EZ); z (3-D): -> (DX, DY, DZ)
  k_reg_box<<<rw_blocks((int64_t)DX * EY * EZ * K, 256), 256, 0, st>>>(A, EX, EY, 0, half, DX, EY,
                                                                       EZ, K, B);
  RW_LAUNCH_CHECK();
  float* ylast = ndim == 3 ? A : priors_dev;
  k_reg_box<<<rw_blocks((int64_t)DX * DY * EZ * K, 256), 256, 0, st>>>(B, DX, EY, 1, half, DX, DY,
                                                                       EZ, K, ylast);
  RW_LAUNCH_CHECK();
  if (ndim == 3) {
    k_reg_box<<<rw_blocks((int64_t)DX * DY * DZ * K, 256), 256, 0, st>>>(A, DX, DY, 2, half, DX,
                                                                         DY, DZ, K, priors_dev);
    RW_LAUNCH_CHECK();
  }
  RW_CHECK_CUDA(cudaFreeAsync(scratch, st));
  k_reg_normalize<<<rw_blocks(N, 256), 256, 0, st>>>(priors_dev, K, N);
  RW_LAUNCH_CHECK();
  return RW_OK;
}
