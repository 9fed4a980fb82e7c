// evr_tma.cuh -- tensor-memory-access (TMA) copies into shared memory and the mbarriers
// that count their bytes, shared by the staged solver passes (evr_staged.cu) and the
// differentiation's reverse pass (evr_grad.cu).  All copies read this GPU's own memory;
// none is multicast.
#pragma once
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace evr {
namespace tma {

#ifdef __CUDACC__
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
// an mbarrier with one arrival per phase
__device__ __forceinline__ void mbar_init1(uint32_t mb) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// the phase's one arrival, raising its transaction count by `bytes`
__device__ __forceinline__ void mbar_arm(uint32_t mb, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(mb),
               "r"(bytes)
               : "memory");
}
// non-blocking test of the phase with the given parity
__device__ __forceinline__ bool mbar_done(uint32_t mb, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(mb), "r"(parity)
      : "memory");
  return ok != 0;
}
// orders this thread's earlier generic-proxy accesses to shared memory before later
// tensor copies into it (a stage is refilled after the threads have read it)
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// 2-D / 3-D tensor copy of the box at the given coordinates of `map` into shared memory
// at `dst` (128-byte aligned), completing its bytes on the mbarrier `mb`.  The innermost
// coordinate x times the element size must be a multiple of 16 bytes.
__device__ __forceinline__ void load_2d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                        uint32_t mb) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"((unsigned long long)map), "r"(x), "r"(y), "r"(mb)
      : "memory");
}
__device__ __forceinline__ void load_3d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                        int z, uint32_t mb) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"((unsigned long long)map), "r"(x), "r"(y), "r"(z), "r"(mb)
      : "memory");
}
#endif

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link to libcuda);
// null when the driver does not provide it.
inline PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    else
      cudaGetLastError();
  }
  return fn;
}

// A tensor map over FP32 planes: dims[0] elements per row (x, innermost), rows of
// row_stride bytes, and for rank 3 `dims[2]` planes of plane_stride bytes; box[] elements.
// Outside the tensor a copy reads zeros.
inline bool encode_f32(CUtensorMap* m, const float* base, int rank, const uint64_t* dims,
                       uint64_t row_stride, uint64_t plane_stride, const uint32_t* box) {
  auto fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t d[3] = {dims[0], dims[1], rank > 2 ? dims[2] : 1};
  const cuuint64_t strides[2] = {row_stride, plane_stride};
  const cuuint32_t b[3] = {box[0], box[1], rank > 2 ? box[2] : 1};
  const cuuint32_t es[3] = {1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (cuuint32_t)rank, (void*)base, d, strides, b, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace tma
}  // namespace evr
