// evr_peaks.cu -- measured bandwidth of the memory levels the solvers keep their state
// in, as denominators of a roofline (the paper has no counterpart; it is measurement
// support for the benchmark).
//
//   level 0 (L2): a copy between two device buffers of 16 MiB each, which together stay
//     resident in L2 (126 MB on GB300) after the first pass; bytes = read + written.
//   level 1 (shared memory): every SM's CTA reads 16-byte words of a 32 KiB shared array,
//     conflict-free (consecutive lanes read consecutive words); bytes = read.  Aggregate
//     over all SMs; a kernel that uses k of the SMs is bounded by k / SMs of it.
// Each is timed with CUDA events on the caller's stream after a warm-up launch; the best
// of a few repetitions is returned.
#include <cuda_runtime.h>

#include "../../include/evr.h"

namespace {

constexpr size_t kL2Bytes = 16u << 20;  // per buffer
constexpr int kL2Reps = 20;             // copies per timed launch
constexpr int kSmemWords = 2048;        // float4 words: 32 KiB
constexpr int kSmemIters = 4096;        // reads per thread per launch

__global__ void __launch_bounds__(512) k_l2_copy(const float4* __restrict__ a,
                                                 float4* __restrict__ b, size_t n, int reps) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (int r = 0; r < reps; ++r) {
    const float4* src = (r & 1) ? b : a;
    float4* dst = (r & 1) ? (float4*)a : b;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
      float4 v = __ldcg(src + i);
      __stcg(dst + i, v);
    }
    __syncthreads();  // keeps the copies of a CTA in order; CTAs overlap freely
  }
}

__global__ void __launch_bounds__(1024) k_smem_read(float* out, int iters) {
  __shared__ float4 s[kSmemWords];
  for (int i = threadIdx.x; i < kSmemWords; i += blockDim.x)
    s[i] = make_float4((float)i, 1.0f, 2.0f, 3.0f);
  __syncthreads();
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  int idx = threadIdx.x;
#pragma unroll 8
  for (int k = 0; k < iters; ++k) {
    const float4 v = s[idx];
    acc.x += v.x;
    acc.y += v.y;
    acc.z += v.z;
    acc.w += v.w;
    idx = (idx + 32) & (kSmemWords - 1);  // the warp moves on by one 512-byte row
  }
  if (acc.x + acc.y + acc.z + acc.w == -1.0f) out[blockIdx.x] = acc.x;  // keeps the loop
}

}  // namespace

extern "C" int evr_measure_peak(int level, double* gbs, void* cuda_stream) {
  if (!gbs || (level != 0 && level != 1)) return EVR_ERR_INVALID_ARG;
  *gbs = 0.0;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return EVR_ERR_CUDA;
  void* buf = nullptr;
  const size_t bytes = level == 0 ? 2 * kL2Bytes : sizeof(float) * sms;
  if (cudaMalloc(&buf, bytes) != cudaSuccess) return EVR_ERR_OOM;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = EVR_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = EVR_ERR_CUDA;
  if (!rc && level == 0 && cudaMemsetAsync(buf, 0, bytes, st) != cudaSuccess) rc = EVR_ERR_CUDA;
  double best = 0.0;
  for (int rep = 0; rep < 6 && !rc; ++rep) {  // the first launch warms up
    if (cudaEventRecord(e0, st) != cudaSuccess) rc = EVR_ERR_CUDA;
    double moved = 0.0;
    if (level == 0) {
      const size_t n = kL2Bytes / sizeof(float4);
      float4* a = (float4*)buf;
      k_l2_copy<<<sms * 4, 512, 0, st>>>(a, a + n, n, kL2Reps);
      moved = 2.0 * (double)kL2Bytes * kL2Reps;
    } else {
      k_smem_read<<<sms, 1024, 0, st>>>((float*)buf, kSmemIters);
      moved = 16.0 * kSmemIters * 1024.0 * sms;
    }
    if (!rc && cudaGetLastError() != cudaSuccess) rc = EVR_ERR_CUDA;
    if (!rc && cudaEventRecord(e1, st) != cudaSuccess) rc = EVR_ERR_CUDA;
    float ms = 0.f;
    if (!rc && (cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
      rc = EVR_ERR_CUDA;
    if (!rc && rep > 0 && ms > 0.f) {
      const double g = moved / (ms * 1e-3) / 1e9;
      if (g > best) best = g;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(buf);
  *gbs = best;
  return rc;
}
