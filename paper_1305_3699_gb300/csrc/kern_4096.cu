// Kernels of the 4096-bit size class (k = 145 channels per base).
#include "kernels.cuh"
#include "kernels_api.h"

namespace mr {

using C4096 = Cfg<145, 128, 129, 16, 384, 2>;

static cudaError_t launch_modexp_4096(const LaunchArgs& a, unsigned grid, cudaStream_t s) {
  static const cudaError_t attr =
      cudaFuncSetAttribute(modexp_kernel<C4096>, cudaFuncAttributeMaxDynamicSharedMemorySize, C4096::SMEM_BYTES);
  if (attr != cudaSuccess) return attr;
  modexp_kernel<C4096><<<grid, C4096::THREADS, C4096::SMEM_BYTES, s>>>(a);
  return cudaGetLastError();
}

static cudaError_t launch_crt_4096(const LaunchArgs& a, unsigned grid, cudaStream_t s) {
  static const cudaError_t attr =
      cudaFuncSetAttribute(crt_kernel<C4096>, cudaFuncAttributeMaxDynamicSharedMemorySize, C4096::SMEM_BYTES);
  if (attr != cudaSuccess) return attr;
  crt_kernel<C4096><<<grid, C4096::THREADS, C4096::SMEM_BYTES, s>>>(a);
  return cudaGetLastError();
}

extern const ClassKernels kClass4096 = {
    4096, C4096::K, C4096::W, C4096::WX, C4096::TPI, C4096::THREADS, C4096::IPB, C4096::NPT, C4096::SMEM_BYTES,
    launch_modexp_4096, launch_crt_4096};

}  // namespace mr
