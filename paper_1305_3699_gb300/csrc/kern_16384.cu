// Kernel of the 16384-bit size class (k = 599 channels per base). Generated by gen_kernels.py.
#include "big_kernel.cuh"
#include "kernels_api.h"

namespace mr {

using CB16384v0 = BigCfg<599, 512, 513, 4, 8>;
static size_t slot_words_16384_0(uint32_t wbits) { return CB16384v0::slot_words(wbits); }

static cudaError_t launch_big_16384_0(const BigArgs& a, cudaStream_t s) {
  void* args[] = {const_cast<BigArgs*>(&a)};
  return cudaLaunchCooperativeKernel((const void*)big_modexp_kernel<CB16384v0>, dim3(a.slots * CB16384v0::SLICES),
                                     dim3(CB16384v0::THREADS), args, CB16384v0::SMEM_BYTES, s);
}

static cudaError_t prepare_big_16384_0() {
  return cudaFuncSetAttribute(big_modexp_kernel<CB16384v0>, cudaFuncAttributeMaxDynamicSharedMemorySize, CB16384v0::SMEM_BYTES);
}

static int occupancy_big_16384_0() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, big_modexp_kernel<CB16384v0>, CB16384v0::THREADS, CB16384v0::SMEM_BYTES) != cudaSuccess) n = 0;
  return n;
}

using CB16384v1 = BigTcCfg<599, 512, 513>;
static size_t slot_words_16384_1(uint32_t wbits) { return CB16384v1::slot_words(wbits); }

static cudaError_t launch_big_16384_1(const BigArgs& a, cudaStream_t s) {
  void* args[] = {const_cast<BigArgs*>(&a)};
  return cudaLaunchCooperativeKernel((const void*)big_modexp_kernel<CB16384v1>, dim3(a.slots * CB16384v1::SLICES),
                                     dim3(CB16384v1::THREADS), args, CB16384v1::SMEM_BYTES, s);
}

static cudaError_t prepare_big_16384_1() {
  return cudaFuncSetAttribute(big_modexp_kernel<CB16384v1>, cudaFuncAttributeMaxDynamicSharedMemorySize, CB16384v1::SMEM_BYTES);
}

static int occupancy_big_16384_1() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, big_modexp_kernel<CB16384v1>, CB16384v1::THREADS, CB16384v1::SMEM_BYTES) != cudaSuccess) n = 0;
  return n;
}

static const BigKernel kBig16384[2] = {
    {CB16384v0::SC, CB16384v0::SLICES, CB16384v0::THREADS, CB16384v0::SMEM_BYTES, 0, 1.000f, slot_words_16384_0, launch_big_16384_0, prepare_big_16384_0, occupancy_big_16384_0},
    {CB16384v1::SC, CB16384v1::SLICES, CB16384v1::THREADS, CB16384v1::SMEM_BYTES, 1, 0.434f, slot_words_16384_1, launch_big_16384_1, prepare_big_16384_1, occupancy_big_16384_1}};
extern const ClassKernels kClass16384 = {16384, 599, 512, 513, 0, {}, kBig16384, 2};

}  // namespace mr
