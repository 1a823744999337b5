// Kernels of the 1536-bit size class (k = 54 channels per base). Generated by gen_kernels.py.
#include "kernels.cuh"
#include "kernels_api.h"
#include "mr_kernel.cuh"

namespace mr {

using C1536v0 = Cfg<54, 48, 50, 8, 128, 4>;
static cudaError_t launch_modexp_1536_0(const LaunchArgs& a, unsigned grid, cudaStream_t s) {
  static const cudaError_t attr =
      cudaFuncSetAttribute(modexp_kernel<C1536v0>, cudaFuncAttributeMaxDynamicSharedMemorySize, C1536v0::SMEM_BYTES);
  if (attr != cudaSuccess) return attr;
  modexp_kernel<C1536v0><<<grid, C1536v0::THREADS, C1536v0::SMEM_BYTES, s>>>(a);
  return cudaGetLastError();
}

static cudaError_t launch_crt_1536_0(const LaunchArgs& a, unsigned grid, cudaStream_t s) {
  static const cudaError_t attr =
      cudaFuncSetAttribute(crt_kernel<C1536v0>, cudaFuncAttributeMaxDynamicSharedMemorySize, C1536v0::SMEM_BYTES);
  if (attr != cudaSuccess) return attr;
  crt_kernel<C1536v0><<<grid, C1536v0::THREADS, C1536v0::SMEM_BYTES, s>>>(a);
  return cudaGetLastError();
}

static cudaError_t launch_mr_1536_0(const MRArgs& a, unsigned grid, cudaStream_t s) {
  static const cudaError_t attr =
      cudaFuncSetAttribute(mr_kernel<C1536v0>, cudaFuncAttributeMaxDynamicSharedMemorySize, C1536v0::SMEM_BYTES);
  if (attr != cudaSuccess) return attr;
  mr_kernel<C1536v0><<<grid, C1536v0::THREADS, C1536v0::SMEM_BYTES, s>>>(a);
  return cudaGetLastError();
}

extern const ClassKernels kClass1536 = {
    1536, 54, 48, 50, 1,
    {
     {C1536v0::TPI, C1536v0::THREADS, C1536v0::IPB, C1536v0::NPT, C1536v0::SMEM_BYTES, launch_modexp_1536_0, launch_crt_1536_0, launch_mr_1536_0}}};

}  // namespace mr
