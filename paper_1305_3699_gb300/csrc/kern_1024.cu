// Kernels of the 1024-bit size class (k = 36 channels per base). Generated by gen_kernels.py.
#include "kernels.cuh"
#include "kernels_api.h"
#include "mr_kernel.cuh"

namespace mr {

using C1024v0 = Cfg<36, 32, 34, 4, 128, 4, 2, 1>;
static cudaError_t launch_modexp_1024_0(const LaunchArgs& a, unsigned grid, cudaStream_t s) {
  modexp_kernel<C1024v0><<<grid, C1024v0::THREADS, C1024v0::SMEM_MODEXP_BYTES, s>>>(a);
  return cudaGetLastError();
}

static cudaError_t launch_crt_1024_0(const LaunchArgs& a, unsigned grid, cudaStream_t s) {
  crt_kernel<C1024v0><<<grid, C1024v0::THREADS, C1024v0::SMEM_BYTES, s>>>(a);
  return cudaGetLastError();
}

static cudaError_t launch_mr_1024_0(const MRArgs& a, unsigned grid, cudaStream_t s) {
  mr_kernel<C1024v0><<<grid, C1024v0::THREADS, C1024v0::SMEM_BYTES, s>>>(a);
  return cudaGetLastError();
}

static cudaError_t prepare_1024_0() {
  cudaError_t e = cudaSuccess, r;
  if ((r = cudaFuncSetAttribute(modexp_kernel<C1024v0>, cudaFuncAttributeMaxDynamicSharedMemorySize, C1024v0::SMEM_MODEXP_BYTES)) != cudaSuccess) e = r;
  if ((r = cudaFuncSetAttribute(crt_kernel<C1024v0>, cudaFuncAttributeMaxDynamicSharedMemorySize, C1024v0::SMEM_BYTES)) != cudaSuccess) e = r;
  if ((r = cudaFuncSetAttribute(mr_kernel<C1024v0>, cudaFuncAttributeMaxDynamicSharedMemorySize, C1024v0::SMEM_BYTES)) != cudaSuccess) e = r;
  return e;
}

static int occupancy_1024_0() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, modexp_kernel<C1024v0>, C1024v0::THREADS, C1024v0::SMEM_MODEXP_BYTES) != cudaSuccess) n = 1;
  return n > 0 ? n : 1;
}

using C1024v1 = Cfg<36, 32, 34, 4, 128, 4, 3, 0>;
static cudaError_t launch_modexp_1024_1(const LaunchArgs& a, unsigned grid, cudaStream_t s) {
  modexp_kernel<C1024v1><<<grid, C1024v1::THREADS, C1024v1::SMEM_MODEXP_BYTES, s>>>(a);
  return cudaGetLastError();
}

static cudaError_t launch_crt_1024_1(const LaunchArgs& a, unsigned grid, cudaStream_t s) {
  crt_kernel<C1024v1><<<grid, C1024v1::THREADS, C1024v1::SMEM_BYTES, s>>>(a);
  return cudaGetLastError();
}

static cudaError_t launch_mr_1024_1(const MRArgs& a, unsigned grid, cudaStream_t s) {
  mr_kernel<C1024v1><<<grid, C1024v1::THREADS, C1024v1::SMEM_BYTES, s>>>(a);
  return cudaGetLastError();
}

static cudaError_t prepare_1024_1() {
  cudaError_t e = cudaSuccess, r;
  if ((r = cudaFuncSetAttribute(modexp_kernel<C1024v1>, cudaFuncAttributeMaxDynamicSharedMemorySize, C1024v1::SMEM_MODEXP_BYTES)) != cudaSuccess) e = r;
  if ((r = cudaFuncSetAttribute(crt_kernel<C1024v1>, cudaFuncAttributeMaxDynamicSharedMemorySize, C1024v1::SMEM_BYTES)) != cudaSuccess) e = r;
  if ((r = cudaFuncSetAttribute(mr_kernel<C1024v1>, cudaFuncAttributeMaxDynamicSharedMemorySize, C1024v1::SMEM_BYTES)) != cudaSuccess) e = r;
  return e;
}

static int occupancy_1024_1() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, modexp_kernel<C1024v1>, C1024v1::THREADS, C1024v1::SMEM_MODEXP_BYTES) != cudaSuccess) n = 1;
  return n > 0 ? n : 1;
}

using C1024v2 = Cfg<36, 32, 34, 8, 128, 4, 4, 0>;
static cudaError_t launch_modexp_1024_2(const LaunchArgs& a, unsigned grid, cudaStream_t s) {
  modexp_kernel<C1024v2><<<grid, C1024v2::THREADS, C1024v2::SMEM_MODEXP_BYTES, s>>>(a);
  return cudaGetLastError();
}

static cudaError_t launch_crt_1024_2(const LaunchArgs& a, unsigned grid, cudaStream_t s) {
  crt_kernel<C1024v2><<<grid, C1024v2::THREADS, C1024v2::SMEM_BYTES, s>>>(a);
  return cudaGetLastError();
}

static cudaError_t launch_mr_1024_2(const MRArgs& a, unsigned grid, cudaStream_t s) {
  mr_kernel<C1024v2><<<grid, C1024v2::THREADS, C1024v2::SMEM_BYTES, s>>>(a);
  return cudaGetLastError();
}

static cudaError_t prepare_1024_2() {
  cudaError_t e = cudaSuccess, r;
  if ((r = cudaFuncSetAttribute(modexp_kernel<C1024v2>, cudaFuncAttributeMaxDynamicSharedMemorySize, C1024v2::SMEM_MODEXP_BYTES)) != cudaSuccess) e = r;
  if ((r = cudaFuncSetAttribute(crt_kernel<C1024v2>, cudaFuncAttributeMaxDynamicSharedMemorySize, C1024v2::SMEM_BYTES)) != cudaSuccess) e = r;
  if ((r = cudaFuncSetAttribute(mr_kernel<C1024v2>, cudaFuncAttributeMaxDynamicSharedMemorySize, C1024v2::SMEM_BYTES)) != cudaSuccess) e = r;
  return e;
}

static int occupancy_1024_2() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, modexp_kernel<C1024v2>, C1024v2::THREADS, C1024v2::SMEM_MODEXP_BYTES) != cudaSuccess) n = 1;
  return n > 0 ? n : 1;
}

extern const ClassKernels kClass1024 = {
    1024, 36, 32, 34, 3,
    {
     {C1024v0::TPI, C1024v0::THREADS, C1024v0::IPB, C1024v0::NPT, C1024v0::SMEM_MODEXP_BYTES, C1024v0::TC, launch_modexp_1024_0, launch_crt_1024_0, launch_mr_1024_0, prepare_1024_0, occupancy_1024_0},
     {C1024v1::TPI, C1024v1::THREADS, C1024v1::IPB, C1024v1::NPT, C1024v1::SMEM_MODEXP_BYTES, C1024v1::TC, launch_modexp_1024_1, launch_crt_1024_1, launch_mr_1024_1, prepare_1024_1, occupancy_1024_1},
     {C1024v2::TPI, C1024v2::THREADS, C1024v2::IPB, C1024v2::NPT, C1024v2::SMEM_MODEXP_BYTES, C1024v2::TC, launch_modexp_1024_2, launch_crt_1024_2, launch_mr_1024_2, prepare_1024_2, occupancy_1024_2}},
    nullptr, 0};

}  // namespace mr
