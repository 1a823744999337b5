// Kernels of the 4096-bit size class (k = 145 channels per base). Generated by gen_kernels.py.
#include "kernels.cuh"
#include "kernels_api.h"
#include "mr_kernel.cuh"

namespace mr {

using C4096v0 = Cfg<145, 128, 129, 16, 384, 2, 0, 0>;
static cudaError_t launch_modexp_4096_0(const LaunchArgs& a, unsigned grid, cudaStream_t s) {
  modexp_kernel<C4096v0><<<grid, C4096v0::THREADS, C4096v0::SMEM_MODEXP_BYTES, s>>>(a);
  return cudaGetLastError();
}

static cudaError_t launch_crt_4096_0(const LaunchArgs& a, unsigned grid, cudaStream_t s) {
  crt_kernel<C4096v0><<<grid, C4096v0::THREADS, C4096v0::SMEM_BYTES, s>>>(a);
  return cudaGetLastError();
}

static cudaError_t launch_mr_4096_0(const MRArgs& a, unsigned grid, cudaStream_t s) {
  mr_kernel<C4096v0><<<grid, C4096v0::THREADS, C4096v0::SMEM_BYTES, s>>>(a);
  return cudaGetLastError();
}

static cudaError_t prepare_4096_0() {
  cudaError_t e = cudaSuccess, r;
  if ((r = cudaFuncSetAttribute(modexp_kernel<C4096v0>, cudaFuncAttributeMaxDynamicSharedMemorySize, C4096v0::SMEM_MODEXP_BYTES)) != cudaSuccess) e = r;
  if ((r = cudaFuncSetAttribute(crt_kernel<C4096v0>, cudaFuncAttributeMaxDynamicSharedMemorySize, C4096v0::SMEM_BYTES)) != cudaSuccess) e = r;
  if ((r = cudaFuncSetAttribute(mr_kernel<C4096v0>, cudaFuncAttributeMaxDynamicSharedMemorySize, C4096v0::SMEM_BYTES)) != cudaSuccess) e = r;
  return e;
}

static int occupancy_4096_0() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, modexp_kernel<C4096v0>, C4096v0::THREADS, C4096v0::SMEM_MODEXP_BYTES) != cudaSuccess) n = 1;
  return n > 0 ? n : 1;
}

extern const ClassKernels kClass4096 = {
    4096, 145, 128, 129, 1,
    {
     {C4096v0::TPI, C4096v0::THREADS, C4096v0::IPB, C4096v0::NPT, C4096v0::SMEM_MODEXP_BYTES, C4096v0::TC, launch_modexp_4096_0, launch_crt_4096_0, launch_mr_4096_0, prepare_4096_0, occupancy_4096_0}},
    nullptr, 0};

}  // namespace mr
