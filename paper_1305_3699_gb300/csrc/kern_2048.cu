// Kernels of the 2048-bit size class (k = 72 channels per base).
#include "kernels.cuh"
#include "kernels_api.h"

namespace mr {

using C2048 = Cfg<72, 64, 66, 8, 128, 4>;

static cudaError_t launch_modexp_2048(const LaunchArgs& a, unsigned grid, cudaStream_t s) {
  static const cudaError_t attr =
      cudaFuncSetAttribute(modexp_kernel<C2048>, cudaFuncAttributeMaxDynamicSharedMemorySize, C2048::SMEM_BYTES);
  if (attr != cudaSuccess) return attr;
  modexp_kernel<C2048><<<grid, C2048::THREADS, C2048::SMEM_BYTES, s>>>(a);
  return cudaGetLastError();
}

static cudaError_t launch_crt_2048(const LaunchArgs& a, unsigned grid, cudaStream_t s) {
  static const cudaError_t attr =
      cudaFuncSetAttribute(crt_kernel<C2048>, cudaFuncAttributeMaxDynamicSharedMemorySize, C2048::SMEM_BYTES);
  if (attr != cudaSuccess) return attr;
  crt_kernel<C2048><<<grid, C2048::THREADS, C2048::SMEM_BYTES, s>>>(a);
  return cudaGetLastError();
}

extern const ClassKernels kClass2048 = {
    2048, C2048::K, C2048::W, C2048::WX, C2048::TPI, C2048::THREADS, C2048::IPB, C2048::NPT, C2048::SMEM_BYTES,
    launch_modexp_2048, launch_crt_2048};

}  // namespace mr
