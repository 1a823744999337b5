// Integer-multiply throughput probe behind mr_imad_peak: a stream of 32x32
// multiply-adds, the instructions the RNS channel arithmetic and the
// base-extension dot products (Sec. 3.1) are made of (mad.wide.u32, mad.lo.u32,
// the carry-pair form of a 64-bit accumulation, mad.hi.u32).  Each thread keeps 12
// independent accumulators; every step feeds an accumulator's own low word
// back as a multiplicand (acc = lo(acc) * t + acc, or acc = acc * acc + t), so
// the recurrence is not linear in any loop-invariant value and the compiler
// cannot fold the steps into fewer multiplies.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/mr.h"
#include "peak.h"

namespace mr {

constexpr int PEAK_ACC = 12;
constexpr int PEAK_THREADS = 256;

template <int KIND>
__global__ void __launch_bounds__(PEAK_THREADS) imad_stream_kernel(uint64_t* sink, uint32_t seed, int iters) {
  uint64_t acc[PEAK_ACC];
  uint32_t t[PEAK_ACC];
  uint32_t x = seed ^ (blockIdx.x * PEAK_THREADS + threadIdx.x);
#pragma unroll
  for (int s = 0; s < PEAK_ACC; s++) {
    acc[s] = x + 31u * s;
    t[s] = ((x + 977u * s) * 2654435761u) | 1u;
  }
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int s = 0; s < PEAK_ACC; s++) {
      if (KIND == 0) {
        uint64_t r;
        asm volatile("mad.wide.u32 %0, %1, %2, %3;" : "=l"(r) : "r"((uint32_t)acc[s]), "r"(t[s]), "l"(acc[s]));
        acc[s] = r;
      } else if (KIND == 1) {
        uint32_t r, v = (uint32_t)acc[s];
        asm volatile("mad.lo.u32 %0, %1, %1, %2;" : "=r"(r) : "r"(v), "r"(t[s]));
        acc[s] = r;
      } else if (KIND == 2) {
        // 64-bit accumulation of a 32x32 product as a carry pair: low word with carry out,
        // high word with carry in (the sum of a dot product of k terms with k m^2 < 2^64 never
        // carries out of the high word)
        uint32_t lo = (uint32_t)acc[s], hi = (uint32_t)(acc[s] >> 32);
        asm volatile("mad.lo.cc.u32 %0, %2, %3, %0;\n\tmadc.hi.u32 %1, %2, %3, %1;"
                     : "+r"(lo), "+r"(hi)
                     : "r"(lo), "r"(t[s]));
        acc[s] = ((uint64_t)hi << 32) | lo;
      } else {
        uint32_t r, v = (uint32_t)acc[s];
        asm volatile("mad.hi.u32 %0, %1, %2, %1;" : "=r"(r) : "r"(v), "r"(t[s]));
        acc[s] = r;
      }
    }
  }
  uint64_t r = 0;
#pragma unroll
  for (int s = 0; s < PEAK_ACC; s++) r ^= acc[s];
  if ((uint32_t)(r ^ (r >> 32)) == 0x7f4a7c15u) sink[0] = r;  // keeps the stream live; rarely taken
}

cudaError_t imad_stream_rate(int device, cudaStream_t stream, int kind, double* per_second) {
  int sms = 0;
  cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess) return e;
  uint64_t* sink = nullptr;
  if ((e = cudaMallocAsync(&sink, sizeof(uint64_t), stream)) != cudaSuccess) return e;
  const unsigned grid = (unsigned)sms * 6;  // 6 blocks of 8 warps: 12 warps per scheduler
  const int iters = 4096;
  cudaEvent_t a = nullptr, b = nullptr;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  auto launch = [&]() {
    if (kind == 0) imad_stream_kernel<0><<<grid, PEAK_THREADS, 0, stream>>>(sink, 12345u, iters);
    else if (kind == 1) imad_stream_kernel<1><<<grid, PEAK_THREADS, 0, stream>>>(sink, 12345u, iters);
    else if (kind == 2) imad_stream_kernel<2><<<grid, PEAK_THREADS, 0, stream>>>(sink, 12345u, iters);
    else imad_stream_kernel<3><<<grid, PEAK_THREADS, 0, stream>>>(sink, 12345u, iters);
  };
  launch();  // warm-up
  cudaEventRecord(a, stream);
  const int reps = 5;
  for (int r = 0; r < reps; r++) launch();
  cudaEventRecord(b, stream);
  e = cudaEventSynchronize(b);
  float ms = 0;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFreeAsync(sink, stream);
  if (e == cudaSuccess)
    *per_second = (double)grid * PEAK_THREADS * iters * PEAK_ACC * reps / (ms * 1e-3);
  return e;
}

}  // namespace mr
