// Garner recombination of RSA CRT decryptions whose halves are in a large size class
// (8192-bit primes, 16384-bit keys).  Sec. 3.3 decrypts through the CRT:
// m_p = c^dp mod p, m_q = c^dq mod q, h = qinv (m_p - m_q) mod p, m = m_q + h q.  The two
// exponentiations run in the large-class kernel; this kernel forms h and m in binary.
//
// One warp per decryption.  The product d * qr and the reduction of h by p are kept in
// carry-save form: one 64-bit accumulator per 32-bit column in shared memory, each lane adding
// its own columns (disjoint addresses within a pass, __syncwarp between passes), so no column
// overflows (each receives fewer than 2^11 words below 2^32).  Carries are resolved once, by
// lane 0, in the serial passes, which are a few hundred steps per number: the recombination is a
// small fraction of one 8192-bit exponentiation.
//
//   d  = m_p + P2 - m_q              W+1 limbs, 0 < d < 3 * 2^(32W), d = m_p - m_q (mod p)
//   h' = d * qr * 2^(-32(W+1)) mod p  Montgomery product with qr = qinv 2^(32(W+1)) mod p:
//                                     below 2p, so one conditional subtraction gives h in [0, p)
//   m  = m_q + h q                   2W limbs, m < p q = N
#include <cstdint>

#include "kernels_api.h"
#include "layout.h"
#include "rns_device.cuh"

namespace mr {
namespace {

constexpr int MAXJ = CRT_BIN_MAX_W / 32;  // limbs of p per lane

inline size_t crt_bin_smem_bytes(uint32_t W) {
  return (size_t)(2 * W + 4) * 8 + (size_t)(W + 4 + 4 * W + 2 * W) * 4;
}

// acc[c] += the 96-bit column sums (s2:s1:s0) of this lane's columns (3 passes, disjoint within each)
__device__ __forceinline__ void add_column(uint64_t* acc, uint32_t c, bool on, uint32_t s0, uint32_t s1,
                                           uint32_t s2, uint32_t extra) {
  if (on) acc[c] += (uint64_t)s0 + extra;
  __syncwarp();
  if (on) acc[c + 1] += s1;
  __syncwarp();
  if (on) acc[c + 2] += s2;
  __syncwarp();
}

__global__ void __launch_bounds__(32) crt_bin_kernel(const CrtItem* items, uint32_t W, uint32_t n_off) {
  extern __shared__ uint64_t acc[];                                // 2W + 4 columns
  uint32_t* d = reinterpret_cast<uint32_t*>(acc + 2 * W + 4);     // W + 1 limbs (d, then h)
  uint32_t* pm = d + W + 4;                                        // p
  uint32_t* qr = pm + W;                                           // qinv 2^(32(W+1)) mod p
  uint32_t* qv = qr + W;                                           // q
  uint32_t* mq = qv + W;                                           // m_q
  uint32_t* res = mq + W;                                          // 2W limbs of m
  const uint32_t lane = threadIdx.x;
  const CrtItem it = items[blockIdx.x];
  const CrtBinOff o = crt_bin_offsets(W);
  const uint32_t* p = it.keyp + n_off;
  for (uint32_t w = lane; w < W; w += 32) {
    pm[w] = __ldg(p + w);
    qr[w] = __ldg(it.crt + o.qr + w);
    qv[w] = __ldg(it.crt + o.q + w);
    mq[w] = it.mq[w];
  }
  for (uint32_t c = lane; c < 2 * W + 4; c += 32) acc[c] = 0;
  const uint32_t pinv = __ldg(it.crt + o.pinv);
  __syncwarp();

  // d = m_p + P2 - m_q
  if (lane == 0) {
    uint32_t cy = 0, br = 0;
    for (uint32_t w = 0; w <= W; w++) {
      const uint64_t a = (uint64_t)__ldg(it.crt + o.p2 + w) + (w < W ? it.mp[w] : 0u) + cy;
      cy = hi32(a);
      const uint64_t b = (uint64_t)lo32(a) - (w < W ? mq[w] : 0u) - br;
      d[w] = lo32(b);
      br = hi32(b) ? 1u : 0u;
    }
  }
  __syncwarp();

  // T = d * qr: columns 0 .. 2W-1, lane = column mod 32
  for (uint32_t c0 = 0; c0 < 2 * W; c0 += 32) {
    const uint32_t c = c0 + lane;
    uint32_t s0 = 0, s1 = 0, s2 = 0;
    const uint32_t ilo = c + 1 > W ? c + 1 - W : 0u, ihi = c < W ? c : W;
    for (uint32_t i = ilo; i <= ihi; i++) mac96(s0, s1, s2, d[i], qr[c - i]);
    add_column(acc, c, c < 2 * W, s0, s1, s2, 0u);
  }

  // Montgomery reduction by p over W+1 words: column i is cleared by u_i p 2^(32i)
  uint64_t carry = 0;  // lane 0: carry out of the cleared column
  for (uint32_t i = 0; i <= W; i++) {
    uint64_t v = 0;
    uint32_t u = 0;
    if (lane == 0) {
      v = acc[i] + carry;
      u = lo32(v) * pinv;
    }
    u = __shfl_sync(0xffffffffu, u, 0);
    uint64_t pr[MAXJ];
#pragma unroll
    for (int r = 0; r < MAXJ; r++) {
      const uint32_t j = lane + 32u * r;
      pr[r] = j < W ? mulw(u, pm[j]) : 0ull;
    }
#pragma unroll
    for (int r = 0; r < MAXJ; r++) {
      const uint32_t j = lane + 32u * r;
      if (j == 0) carry = (v + lo32(pr[r])) >> 32;  // the low word of column i is now zero
      else if (j < W) acc[i + j] += lo32(pr[r]);
    }
    __syncwarp();
#pragma unroll
    for (int r = 0; r < MAXJ; r++) {
      const uint32_t j = lane + 32u * r;
      if (j < W) acc[i + j + 1] += hi32(pr[r]);
    }
    __syncwarp();
  }

  // h' = columns W+1 .. 2W+1 with the carries resolved; h = h' - p when h' >= p
  if (lane == 0) {
    for (uint32_t c = W + 1; c <= 2 * W + 1; c++) {
      const uint64_t v = acc[c] + carry;
      d[c - W - 1] = lo32(v);
      carry = v >> 32;
    }
    bool ge = d[W] != 0;
    if (!ge) {
      ge = true;
      for (int w = (int)W - 1; w >= 0; w--)
        if (d[w] != pm[w]) {
          ge = d[w] > pm[w];
          break;
        }
    }
    if (ge) {
      uint32_t br = 0;
      for (uint32_t w = 0; w < W; w++) {
        const uint64_t b = (uint64_t)d[w] - pm[w] - br;
        d[w] = lo32(b);
        br = hi32(b) ? 1u : 0u;
      }
    }
  }
  __syncwarp();  // lane 0 has read the columns and written h
  for (uint32_t c = lane; c < 2 * W + 4; c += 32) acc[c] = 0;
  __syncwarp();

  // m = m_q + h q: columns 0 .. 2W-1
  for (uint32_t c0 = 0; c0 < 2 * W; c0 += 32) {
    const uint32_t c = c0 + lane;
    uint32_t s0 = 0, s1 = 0, s2 = 0;
    const uint32_t ilo = c + 1 > W ? c + 1 - W : 0u, ihi = c < W ? c : W - 1;
    for (uint32_t i = ilo; i <= ihi; i++) mac96(s0, s1, s2, d[i], qv[c - i]);
    add_column(acc, c, c < 2 * W, s0, s1, s2, c < W ? mq[c] : 0u);
  }
  if (lane == 0) {
    uint64_t cy = 0;
    for (uint32_t c = 0; c < 2 * W; c++) {
      const uint64_t v = acc[c] + cy;
      res[c] = lo32(v);
      cy = v >> 32;
    }
  }
  __syncwarp();
  for (uint32_t w = lane; w < it.out_limbs; w += 32) it.out[w] = w < 2 * W ? res[w] : 0u;
}

}  // namespace

cudaError_t launch_crt_bin(const CrtItem* items, uint32_t n_items, uint32_t W, uint32_t n_off, cudaStream_t s) {
  if (n_items == 0) return cudaSuccess;
  if (W == 0 || W > CRT_BIN_MAX_W) return cudaErrorInvalidValue;
  crt_bin_kernel<<<n_items, 32, crt_bin_smem_bytes(W), s>>>(items, W, n_off);
  return cudaGetLastError();
}

}  // namespace mr
