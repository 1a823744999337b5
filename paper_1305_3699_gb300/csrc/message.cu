// Message-level RSA (Sec. 3.3: messages are split into blocks of the key's length and all blocks
// are encrypted or decrypted in one pass).  A byte string becomes rows of limbs, one block of
// B = (bits(N) - 1) / 8 bytes per row (the last one shorter), each block read little-endian so that
// it lies below N; the rows go through the batched encryption / CRT decryption; decryption writes
// the bytes back.  These two kernels only move bytes.
#include <cstdint>

#include "kernels_api.h"

namespace mr {
namespace {

// rows[i][w] = bytes [4w, 4w + 4) of block i (little-endian; bytes past the block or the message are 0)
__global__ void pack_kernel(const uint8_t* msg, size_t len, uint32_t B, uint32_t W, size_t n_blocks, uint32_t* rows) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n_blocks * W) return;
  const size_t i = idx / W;
  const uint32_t w = (uint32_t)(idx % W);
  uint32_t v = 0;
  for (uint32_t b = 0; b < 4; b++) {
    const uint32_t byte = 4 * w + b;
    const size_t pos = i * B + byte;
    if (byte < B && pos < len) v |= (uint32_t)msg[pos] << (8 * b);
  }
  rows[idx] = v;
}

// msg[pos] = byte (pos mod B) of row pos / B
__global__ void unpack_kernel(const uint32_t* rows, uint32_t B, uint32_t W, size_t len, uint8_t* msg) {
  const size_t pos = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (pos >= len) return;
  const size_t i = pos / B;
  const uint32_t byte = (uint32_t)(pos % B);
  msg[pos] = (uint8_t)(rows[i * W + byte / 4] >> (8 * (byte % 4)));
}

}  // namespace

cudaError_t launch_pack_message(const uint8_t* msg, size_t len, uint32_t B, uint32_t W, size_t n_blocks, uint32_t* rows,
                                cudaStream_t s) {
  const size_t n = n_blocks * W;
  if (n == 0) return cudaSuccess;
  pack_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(msg, len, B, W, n_blocks, rows);
  return cudaGetLastError();
}

cudaError_t launch_unpack_message(const uint32_t* rows, uint32_t B, uint32_t W, size_t len, uint8_t* msg, cudaStream_t s) {
  if (len == 0) return cudaSuccess;
  unpack_kernel<<<(unsigned)((len + 255) / 256), 256, 0, s>>>(rows, B, W, len, msg);
  return cudaGetLastError();
}

}  // namespace mr
