// Host-visible description of the compiled kernels of each size class.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "layout.h"

namespace mr {

struct LaunchArgs {
  const uint32_t* cls;   // class table block (device)
  const void* items;     // MxItem[] or CrtItem[] (device)
  uint32_t n_items;
  uint32_t wbits;        // window width (modexp), 1..6
  uint32_t* scratch;     // window tables (modexp): per warp (1 << wbits) x 2 NPT x 32 words
  uint8_t* status;       // per-item status bytes or nullptr
};

struct ClassKernels {
  uint32_t L, k, W, WX, tpi, threads, ipb, npt, smem_bytes;
  cudaError_t (*modexp)(const LaunchArgs&, unsigned grid, cudaStream_t);
  cudaError_t (*crt)(const LaunchArgs&, unsigned grid, cudaStream_t);
};

// nullptr when no kernel is compiled for class L
const ClassKernels* class_kernels(uint32_t L);

// scratch words one modexp launch of n items needs
inline size_t modexp_scratch_words(const ClassKernels& kc, uint32_t n, uint32_t wbits) {
  size_t grid = (n + kc.ipb - 1) / kc.ipb;
  size_t warps = grid * (kc.threads / 32);
  return warps * ((size_t)1 << wbits) * 2 * kc.npt * 32;
}

}  // namespace mr
