// Kernels of the 512-bit size class (k = 18 channels per base). Generated by gen_kernels.py.
#include "kernels.cuh"
#include "kernels_api.h"
#include "mr_kernel.cuh"

namespace mr {

using C512v0 = Cfg<18, 16, 17, 2, 128, 4, 2, 0>;
static cudaError_t launch_modexp_512_0(const LaunchArgs& a, unsigned grid, cudaStream_t s) {
  modexp_kernel<C512v0><<<grid, C512v0::THREADS, C512v0::SMEM_MODEXP_BYTES, s>>>(a);
  return cudaGetLastError();
}

static cudaError_t launch_crt_512_0(const LaunchArgs& a, unsigned grid, cudaStream_t s) {
  crt_kernel<C512v0><<<grid, C512v0::THREADS, C512v0::SMEM_BYTES, s>>>(a);
  return cudaGetLastError();
}

static cudaError_t launch_mr_512_0(const MRArgs& a, unsigned grid, cudaStream_t s) {
  mr_kernel<C512v0><<<grid, C512v0::THREADS, C512v0::SMEM_BYTES, s>>>(a);
  return cudaGetLastError();
}

static cudaError_t prepare_512_0() {
  cudaError_t e = cudaSuccess, r;
  if ((r = cudaFuncSetAttribute(modexp_kernel<C512v0>, cudaFuncAttributeMaxDynamicSharedMemorySize, C512v0::SMEM_MODEXP_BYTES)) != cudaSuccess) e = r;
  if ((r = cudaFuncSetAttribute(crt_kernel<C512v0>, cudaFuncAttributeMaxDynamicSharedMemorySize, C512v0::SMEM_BYTES)) != cudaSuccess) e = r;
  if ((r = cudaFuncSetAttribute(mr_kernel<C512v0>, cudaFuncAttributeMaxDynamicSharedMemorySize, C512v0::SMEM_BYTES)) != cudaSuccess) e = r;
  return e;
}

static int occupancy_512_0() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, modexp_kernel<C512v0>, C512v0::THREADS, C512v0::SMEM_MODEXP_BYTES) != cudaSuccess) n = 1;
  return n > 0 ? n : 1;
}

using C512v1 = Cfg<18, 16, 17, 4, 128, 4, 4, 0>;
static cudaError_t launch_modexp_512_1(const LaunchArgs& a, unsigned grid, cudaStream_t s) {
  modexp_kernel<C512v1><<<grid, C512v1::THREADS, C512v1::SMEM_MODEXP_BYTES, s>>>(a);
  return cudaGetLastError();
}

static cudaError_t launch_crt_512_1(const LaunchArgs& a, unsigned grid, cudaStream_t s) {
  crt_kernel<C512v1><<<grid, C512v1::THREADS, C512v1::SMEM_BYTES, s>>>(a);
  return cudaGetLastError();
}

static cudaError_t launch_mr_512_1(const MRArgs& a, unsigned grid, cudaStream_t s) {
  mr_kernel<C512v1><<<grid, C512v1::THREADS, C512v1::SMEM_BYTES, s>>>(a);
  return cudaGetLastError();
}

static cudaError_t prepare_512_1() {
  cudaError_t e = cudaSuccess, r;
  if ((r = cudaFuncSetAttribute(modexp_kernel<C512v1>, cudaFuncAttributeMaxDynamicSharedMemorySize, C512v1::SMEM_MODEXP_BYTES)) != cudaSuccess) e = r;
  if ((r = cudaFuncSetAttribute(crt_kernel<C512v1>, cudaFuncAttributeMaxDynamicSharedMemorySize, C512v1::SMEM_BYTES)) != cudaSuccess) e = r;
  if ((r = cudaFuncSetAttribute(mr_kernel<C512v1>, cudaFuncAttributeMaxDynamicSharedMemorySize, C512v1::SMEM_BYTES)) != cudaSuccess) e = r;
  return e;
}

static int occupancy_512_1() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, modexp_kernel<C512v1>, C512v1::THREADS, C512v1::SMEM_MODEXP_BYTES) != cudaSuccess) n = 1;
  return n > 0 ? n : 1;
}

using C512v2 = Cfg<18, 16, 17, 4, 128, 4, 4, 1>;
static cudaError_t launch_modexp_512_2(const LaunchArgs& a, unsigned grid, cudaStream_t s) {
  modexp_kernel<C512v2><<<grid, C512v2::THREADS, C512v2::SMEM_MODEXP_BYTES, s>>>(a);
  return cudaGetLastError();
}

static cudaError_t launch_crt_512_2(const LaunchArgs& a, unsigned grid, cudaStream_t s) {
  crt_kernel<C512v2><<<grid, C512v2::THREADS, C512v2::SMEM_BYTES, s>>>(a);
  return cudaGetLastError();
}

static cudaError_t launch_mr_512_2(const MRArgs& a, unsigned grid, cudaStream_t s) {
  mr_kernel<C512v2><<<grid, C512v2::THREADS, C512v2::SMEM_BYTES, s>>>(a);
  return cudaGetLastError();
}

static cudaError_t prepare_512_2() {
  cudaError_t e = cudaSuccess, r;
  if ((r = cudaFuncSetAttribute(modexp_kernel<C512v2>, cudaFuncAttributeMaxDynamicSharedMemorySize, C512v2::SMEM_MODEXP_BYTES)) != cudaSuccess) e = r;
  if ((r = cudaFuncSetAttribute(crt_kernel<C512v2>, cudaFuncAttributeMaxDynamicSharedMemorySize, C512v2::SMEM_BYTES)) != cudaSuccess) e = r;
  if ((r = cudaFuncSetAttribute(mr_kernel<C512v2>, cudaFuncAttributeMaxDynamicSharedMemorySize, C512v2::SMEM_BYTES)) != cudaSuccess) e = r;
  return e;
}

static int occupancy_512_2() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, modexp_kernel<C512v2>, C512v2::THREADS, C512v2::SMEM_MODEXP_BYTES) != cudaSuccess) n = 1;
  return n > 0 ? n : 1;
}

extern const ClassKernels kClass512 = {
    512, 18, 16, 17, 3,
    {
     {C512v0::TPI, C512v0::THREADS, C512v0::IPB, C512v0::NPT, C512v0::SMEM_MODEXP_BYTES, C512v0::TC, launch_modexp_512_0, launch_crt_512_0, launch_mr_512_0, prepare_512_0, occupancy_512_0},
     {C512v1::TPI, C512v1::THREADS, C512v1::IPB, C512v1::NPT, C512v1::SMEM_MODEXP_BYTES, C512v1::TC, launch_modexp_512_1, launch_crt_512_1, launch_mr_512_1, prepare_512_1, occupancy_512_1},
     {C512v2::TPI, C512v2::THREADS, C512v2::IPB, C512v2::NPT, C512v2::SMEM_MODEXP_BYTES, C512v2::TC, launch_modexp_512_2, launch_crt_512_2, launch_mr_512_2, prepare_512_2, occupancy_512_2}},
    nullptr, 0};

}  // namespace mr
