// Kernel of the 16384-bit size class (k = 599 channels per base). Generated by gen_kernels.py.
#include "big_kernel.cuh"
#include "kernels_api.h"

namespace mr {

using CB16384 = BigCfg<599, 512, 513, 4, 8>;
static size_t slot_words_16384(uint32_t wbits) { return CB16384::slot_words(wbits); }

static cudaError_t launch_big_16384(const BigArgs& a, cudaStream_t s) {
  void* args[] = {const_cast<BigArgs*>(&a)};
  return cudaLaunchCooperativeKernel((const void*)big_modexp_kernel<CB16384>, dim3(a.slots * CB16384::SLICES),
                                     dim3(CB16384::THREADS), args, CB16384::SMEM_BYTES, s);
}

static cudaError_t prepare_big_16384() {
  return cudaFuncSetAttribute(big_modexp_kernel<CB16384>, cudaFuncAttributeMaxDynamicSharedMemorySize, CB16384::SMEM_BYTES);
}

static int occupancy_big_16384() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, big_modexp_kernel<CB16384>, CB16384::THREADS, CB16384::SMEM_BYTES) != cudaSuccess) n = 0;
  return n;
}

static const BigKernel kBig16384 = {CB16384::SC, CB16384::SLICES, CB16384::THREADS, CB16384::SMEM_BYTES, slot_words_16384,
                                 launch_big_16384, prepare_big_16384, occupancy_big_16384};
extern const ClassKernels kClass16384 = {16384, 599, 512, 513, 0, {}, &kBig16384};

}  // namespace mr
