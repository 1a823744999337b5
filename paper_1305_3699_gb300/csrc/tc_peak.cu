// Tensor-core throughput probes behind mr_tensor_peak, and the layout check
// behind mr_debug_tc_mma.
//
// The base extensions of the RNS Montgomery multiplication (Sec. 3.1) are
// products with constant matrices, so they may run on the tensor cores as
// exact products of small-integer slices.  Which tensor instruction pays on
// this GPU is measured here, not assumed:
//   kind 0  tcgen05.mma kind::f16 (fp16 operands from shared memory, fp32
//           accumulator in tensor memory), M = 128, N = 256, K = 16, one
//           thread issuing back-to-back accumulating products, one CTA per SM;
//   kind 1  mma.sync m16n8k32 s8 x s8 -> s32 (the legacy warp-level integer
//           path; tcgen05 kind::i8 does not exist for sm_103a: ptxas rejects it);
//   kind 2  mma.sync m16n8k16 f16 x f16 -> f32 (legacy warp-level path).
// Each reports multiply-add operations x 2 per second.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "peak.h"
#include "tc_device.cuh"

namespace mr {

namespace {

constexpr uint32_t TC_M = 128, TC_N = 256, TC_K = 16;
constexpr int TC_THREADS = 128;
constexpr uint64_t TC_WAIT_NS = 2000000000ull;  // 2 s: far beyond any legitimate completion

// shared memory: A tile 4 KB, B tile 8 KB, then the mbarrier and the tensor-memory address
constexpr uint32_t TCP_A = 0, TCP_B = TC_M * TC_K * 2, TCP_MBAR = TCP_B + TC_N * TC_K * 2, TCP_TADDR = TCP_MBAR + 8;
constexpr uint32_t TCP_BYTES = TCP_TADDR + 8;

__global__ void __launch_bounds__(TC_THREADS, 1) tc_f16_rate_kernel(int iters, uint32_t* err) {
  extern __shared__ __align__(1024) uint8_t sm[];
  uint16_t* a = reinterpret_cast<uint16_t*>(sm + TCP_A);
  uint16_t* b = reinterpret_cast<uint16_t*>(sm + TCP_B);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + TCP_MBAR);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + TCP_TADDR);
  // operands: small integers (exact in fp16); their values do not matter for the rate
  for (uint32_t i = threadIdx.x; i < TC_M * TC_K; i += TC_THREADS) a[i] = __half_as_ushort(__float2half((float)(i % 7)));
  for (uint32_t i = threadIdx.x; i < TC_N * TC_K; i += TC_THREADS) b[i] = __half_as_ushort(__float2half((float)(i % 5)));
  tc::fence_smem_async();
  if (threadIdx.x < 32) {
    tc::tmem_alloc(tslot, TC_N);
    tc::tmem_relinquish();
  }
  if (threadIdx.x == 0) {
    tc::mbar_init(mbar, 1);
    tc::fence_smem_async();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = *tslot;
  if (threadIdx.x == 0) {
    const uint64_t ad = tc::sdesc(tc::saddr(a), 16 * TC_M, 128);
    const uint64_t bd = tc::sdesc(tc::saddr(b), 16 * TC_N, 128);
    const uint32_t id = tc::idesc_f16_f32(TC_M, TC_N);
    for (int i = 0; i < iters; i++) tc::mma_f16(taddr, ad, bd, id, i > 0 ? 1u : 0u);
    tc::mma_commit(mbar);
    if (!tc::mbar_wait_ns(mbar, 0, TC_WAIT_NS)) atomicExch(err, 1u);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (threadIdx.x < 32) tc::tmem_dealloc(taddr, TC_N);
}

constexpr int MMA_ACC = 8;  // independent accumulators per warp

__global__ void __launch_bounds__(256) mma_s8_rate_kernel(int iters, uint32_t seed, int* sink) {
  uint32_t av[4], bv[2];
#pragma unroll
  for (int i = 0; i < 4; i++) av[i] = (seed + threadIdx.x * 7u + i) * 0x01010101u;
  bv[0] = (seed ^ threadIdx.x) * 0x00010101u;
  bv[1] = bv[0] + 0x01000001u;
  int d[MMA_ACC][4];
#pragma unroll
  for (int j = 0; j < MMA_ACC; j++)
#pragma unroll
    for (int i = 0; i < 4; i++) d[j][i] = j + i;
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int j = 0; j < MMA_ACC; j++)
      asm volatile(
          "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
          "{%0, %1, %2, %3};"
          : "+r"(d[j][0]), "+r"(d[j][1]), "+r"(d[j][2]), "+r"(d[j][3])
          : "r"(av[0]), "r"(av[1]), "r"(av[2]), "r"(av[3]), "r"(bv[0]), "r"(bv[1]));
  }
  int r = 0;
#pragma unroll
  for (int j = 0; j < MMA_ACC; j++) r ^= d[j][0] ^ d[j][1] ^ d[j][2] ^ d[j][3];
  if (r == 0x5bd1e995) sink[0] = r;  // keeps the products live; rarely taken
}

__global__ void __launch_bounds__(256) mma_f16_rate_kernel(int iters, uint32_t seed, float* sink) {
  uint32_t av[4], bv[2];
#pragma unroll
  for (int i = 0; i < 4; i++) av[i] = 0x3C003C00u ^ ((seed + threadIdx.x + i) & 0x00030003u);
  bv[0] = 0x3C003C00u ^ (seed & 0x00010001u);
  bv[1] = 0x3C003C00u;
  float d[MMA_ACC][4];
#pragma unroll
  for (int j = 0; j < MMA_ACC; j++)
#pragma unroll
    for (int i = 0; i < 4; i++) d[j][i] = (float)(j + i);
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int j = 0; j < MMA_ACC; j++)
      asm volatile(
          "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
          "{%0, %1, %2, %3};"
          : "+f"(d[j][0]), "+f"(d[j][1]), "+f"(d[j][2]), "+f"(d[j][3])
          : "r"(av[0]), "r"(av[1]), "r"(av[2]), "r"(av[3]), "r"(bv[0]), "r"(bv[1]));
  }
  float r = 0;
#pragma unroll
  for (int j = 0; j < MMA_ACC; j++) r += d[j][0] + d[j][1] + d[j][2] + d[j][3];
  if (r == -1.0f) sink[0] = r;
}

// One CTA: D (128 x n, fp32) = A (128 x kdim, fp16, row-major in global) * B^T (B: n x kdim,
// row-major), with both tiles staged in the K-major layout of tc_device.cuh.  swap_strides
// exchanges the two descriptor offsets (layout diagnosis only; the reads stay inside the
// 32 KB regions reserved per operand for n <= 256, kdim <= 64).
constexpr uint32_t DBG_REGION = 32768;
constexpr uint32_t DBG_BYTES = 2 * DBG_REGION + 16;

__global__ void __launch_bounds__(TC_THREADS, 1) tc_debug_mma_kernel(const uint16_t* A, const uint16_t* B, float* D,
                                                                     uint32_t n, uint32_t kdim, uint32_t swap_strides,
                                                                     uint32_t* err) {
  extern __shared__ __align__(1024) uint8_t sm[];
  uint8_t* as = sm;
  uint8_t* bs = sm + DBG_REGION;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + 2 * DBG_REGION);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + 2 * DBG_REGION + 8);
  for (uint32_t i = threadIdx.x; i < 2 * DBG_REGION / 4; i += TC_THREADS) reinterpret_cast<uint32_t*>(sm)[i] = 0u;
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < TC_M * kdim; i += TC_THREADS) {
    const uint32_t r = i / kdim, k = i % kdim;
    *reinterpret_cast<uint16_t*>(as + tc::tile_off(TC_M, r, k)) = A[i];
  }
  for (uint32_t i = threadIdx.x; i < n * kdim; i += TC_THREADS) {
    const uint32_t r = i / kdim, k = i % kdim;
    *reinterpret_cast<uint16_t*>(bs + tc::tile_off(n, r, k)) = B[i];
  }
  tc::fence_smem_async();
  if (threadIdx.x < 32) {
    tc::tmem_alloc(tslot, 256);
    tc::tmem_relinquish();
  }
  if (threadIdx.x == 0) {
    tc::mbar_init(mbar, 1);
    tc::fence_smem_async();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = *tslot;
  const bool a_tmem = swap_strides == 2;  // A from tensor memory, columns n .. n + kdim/2 - 1
  // (swap_strides 3: the product as for 0, read back with the 16x256b load shape)
  if (a_tmem) {
    // row 32 w + lane of A into lane 32 w + lane: two fp16 values of K per column, lower index low
    const uint32_t w = threadIdx.x >> 5, lane = threadIdx.x & 31, row = 32 * w + lane;
    for (uint32_t k0 = 0; k0 < kdim; k0 += 8) {
      uint32_t p[4];
#pragma unroll
      for (int j = 0; j < 4; j++) p[j] = (uint32_t)A[row * kdim + k0 + 2 * j] | ((uint32_t)A[row * kdim + k0 + 2 * j + 1] << 16);
      tc::tmem_st4(taddr + ((32 * w) << 16) + n + k0 / 2, make_uint4(p[0], p[1], p[2], p[3]));
    }
    tc::tmem_st_wait();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
  }
  if (threadIdx.x == 0) {
    const uint32_t id = tc::idesc_f16_f32(TC_M, n);
    for (uint32_t s = 0; s < kdim / 16; s++) {
      // K step s: column groups 2s, 2s+1
      const uint32_t a0 = tc::saddr(as) + 2 * s * 16 * TC_M, b0 = tc::saddr(bs) + 2 * s * 16 * n;
      const bool sw = swap_strides == 1;  // (3 reads D differently, the product is that of 0)
      const uint64_t ad = sw ? tc::sdesc(a0, 128, 16 * TC_M) : tc::sdesc(a0, 16 * TC_M, 128);
      const uint64_t bd = sw ? tc::sdesc(b0, 128, 16 * n) : tc::sdesc(b0, 16 * n, 128);
      if (a_tmem)
        tc::mma_f16_ts(taddr, taddr + n + 8 * s, bd, id, s > 0 ? 1u : 0u);
      else
        tc::mma_f16(taddr, ad, bd, id, s > 0 ? 1u : 0u);
    }
    tc::mma_commit(mbar);
  }
  bool ok = true;
  if (threadIdx.x == 0) ok = tc::mbar_wait_ns(mbar, 0, TC_WAIT_NS);
  if (!__syncthreads_and(ok)) {
    if (threadIdx.x == 0) atomicExch(err, 1u);
  } else if (swap_strides == 3) {
    // D read back with the 16x256b shape (two 16-lane halves of each warp's quarter, 16 columns per
    // load) and stored by the register layout tc_device.cuh states for it
    tc::fence_after_sync();
    const uint32_t w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (uint32_t half = 0; half < 2; half++)
      for (uint32_t c0 = 0; c0 < n; c0 += 16) {
        uint32_t v[8];
        tc::tmem_ld16x256b_x2(taddr + ((32 * w + 16 * half) << 16) + c0, v);
        tc::tmem_ld_wait();
        const uint32_t r0 = 32 * w + 16 * half + lane / 4, col = c0 + 2 * (lane % 4);
#pragma unroll
        for (uint32_t p = 0; p < 2; p++) {
          D[r0 * n + col + 8 * p] = __uint_as_float(v[4 * p]);
          D[r0 * n + col + 8 * p + 1] = __uint_as_float(v[4 * p + 1]);
          D[(r0 + 8) * n + col + 8 * p] = __uint_as_float(v[4 * p + 2]);
          D[(r0 + 8) * n + col + 8 * p + 1] = __uint_as_float(v[4 * p + 3]);
        }
      }
  } else {
    tc::fence_after_sync();
    const uint32_t w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t row = 32 * w + lane;
    for (uint32_t c0 = 0; c0 < n; c0 += 8) {
      uint32_t v[8];
      tc::tmem_ld8(taddr + ((32 * w) << 16) + c0, v);
      tc::tmem_ld_wait();
#pragma unroll
      for (int j = 0; j < 8; j++) D[row * n + c0 + j] = __uint_as_float(v[j]);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (threadIdx.x < 32) tc::tmem_dealloc(taddr, 256);
}

}  // namespace

cudaError_t tensor_rate(int device, cudaStream_t stream, int kind, double* per_second) {
  int sms = 0;
  cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess) return e;
  uint32_t* scratch = nullptr;
  if ((e = cudaMallocAsync(&scratch, 64, stream)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(scratch, 0, 64, stream)) != cudaSuccess) return e;
  if (kind == 0 &&
      (e = cudaFuncSetAttribute(tc_f16_rate_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TCP_BYTES)) != cudaSuccess)
    return e;
  const int iters = kind == 0 ? 4096 : 2048;
  double ops_per_launch = 0;
  auto launch = [&]() {
    if (kind == 0) {
      tc_f16_rate_kernel<<<sms, TC_THREADS, TCP_BYTES, stream>>>(iters, scratch);
      ops_per_launch = (double)sms * iters * 2.0 * TC_M * TC_N * TC_K;
    } else if (kind == 1) {
      mma_s8_rate_kernel<<<sms * 4, 256, 0, stream>>>(iters, 17u, reinterpret_cast<int*>(scratch) + 4);
      ops_per_launch = (double)sms * 4 * 8 * iters * MMA_ACC * 2.0 * 16 * 8 * 32;
    } else {
      mma_f16_rate_kernel<<<sms * 4, 256, 0, stream>>>(iters, 17u, reinterpret_cast<float*>(scratch) + 4);
      ops_per_launch = (double)sms * 4 * 8 * iters * MMA_ACC * 2.0 * 16 * 8 * 16;
    }
  };
  cudaEvent_t a = nullptr, b = nullptr;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  launch();  // warm-up
  cudaEventRecord(a, stream);
  const int reps = 5;
  for (int r = 0; r < reps; r++) launch();
  cudaEventRecord(b, stream);
  e = cudaEventSynchronize(b);
  float ms = 0;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
  if (e == cudaSuccess) e = cudaGetLastError();
  uint32_t err = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&err, scratch, 4, cudaMemcpyDeviceToHost);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFreeAsync(scratch, stream);
  if (e == cudaSuccess && err) return cudaErrorLaunchTimeout;
  if (e == cudaSuccess) *per_second = ops_per_launch * reps / (ms * 1e-3);
  return e;
}

cudaError_t tensor_debug_mma(const uint16_t* a_host, const uint16_t* b_host, uint32_t n, uint32_t kdim,
                             uint32_t swap_strides, float* d_host, cudaStream_t stream) {
  const size_t abytes = (size_t)TC_M * kdim * 2, bbytes = (size_t)n * kdim * 2, dbytes = (size_t)TC_M * n * 4;
  uint8_t* buf = nullptr;
  cudaError_t e = cudaMallocAsync(&buf, abytes + bbytes + dbytes + 16, stream);
  if (e != cudaSuccess) return e;
  uint16_t* A = reinterpret_cast<uint16_t*>(buf);
  uint16_t* B = reinterpret_cast<uint16_t*>(buf + abytes);
  float* D = reinterpret_cast<float*>(buf + abytes + bbytes);
  uint32_t* err = reinterpret_cast<uint32_t*>(buf + abytes + bbytes + dbytes);
  uint32_t herr = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(A, a_host, abytes, cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(B, b_host, bbytes, cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, 16, stream);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(tc_debug_mma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, DBG_BYTES);
  if (e == cudaSuccess) {
    tc_debug_mma_kernel<<<1, TC_THREADS, DBG_BYTES, stream>>>(A, B, D, n, kdim, swap_strides, err);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_host, D, dbytes, cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  cudaFreeAsync(buf, stream);
  if (e == cudaSuccess && herr) return cudaErrorLaunchTimeout;
  return e;
}

}  // namespace mr
