// Trial division of primality candidates by the first primes, the sieve that key generation runs
// ahead of the Miller-Rabin rounds (Sec. 4.3: candidates are tested against the first 10,000
// primes before any exponentiation; Sec. 3.2: the survivors go to the Miller-Rabin kernel).
//
// A candidate N passes when N >= 2 and no listed prime other than N itself divides N.  For each
// listed prime p the residue N mod p is formed as sum_w N_w * (2^(32w) mod p), one 64-bit
// multiply-add per limb (the table of 2^(32w) mod p is shared by every candidate and stays in
// L2), and reduced once by Barrett's method with mu = floor((2^64 - 1) / p).  One warp per
// candidate, lanes over the primes, 32 primes per step; the warp stops at the first step that
// finds a divisor (most random candidates have a small factor).  Survivors are appended to a
// device list (index and slot) for the Miller-Rabin launch.
#include <cstdint>
#include <vector>

#include "kernels_api.h"
#include "rns_device.cuh"

namespace mr {
namespace {

constexpr uint32_t TRIAL_WARPS = 8;  // candidates per block

__global__ void __launch_bounds__(TRIAL_WARPS * 32)
    trial_kernel(const uint32_t* cand, uint32_t nl, uint32_t n, const uint32_t* tab, uint32_t np, uint32_t* sel,
                 uint32_t* slot, uint32_t* count) {
  __shared__ uint32_t limbs[TRIAL_WARPS][TRIAL_MAX_LIMBS];
  const uint32_t w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t c = blockIdx.x * TRIAL_WARPS + w;
  if (c >= n) return;  // whole warps only: c is uniform across the warp
  const uint32_t* N = cand + (size_t)c * nl;
  uint32_t* L = limbs[w];
  for (uint32_t i = lane; i < nl; i += 32) L[i] = N[i];
  __syncwarp();
  // significant limbs, and the value when it fits 32 bits (to recognise N equal to a listed prime)
  uint32_t nn = nl;
  while (nn > 0 && L[nn - 1] == 0) nn--;
  const bool small = nn <= 1;
  const uint32_t v0 = nn ? L[0] : 0u;
  const uint32_t* C = tab;                                                    // [limb][prime]
  const uint32_t* P = tab + (size_t)TRIAL_MAX_LIMBS * TRIAL_STRIDE;           // primes
  const uint64_t* MU = reinterpret_cast<const uint64_t*>(P + TRIAL_STRIDE);   // Barrett factors
  bool divisible = small && v0 < 2u;
  for (uint32_t j0 = 0; j0 < np && !divisible; j0 += 32) {
    const uint32_t j = j0 + lane;
    bool hit = false;
    if (j < np) {
      uint64_t acc = 0;
      for (uint32_t i = 0; i < nn; i++) acc = madw(L[i], __ldg(C + (size_t)i * TRIAL_STRIDE + j), acc);
      const uint32_t p = __ldg(P + j);
      const uint64_t q = __umul64hi(acc, __ldg(MU + j));
      uint64_t r = acc - q * p;  // in [0, 2p)
      if (r >= p) r -= p;
      if (r >= p) r -= p;
      hit = r == 0 && !(small && v0 == p);
    }
    divisible = __any_sync(0xffffffffu, hit);
  }
  if (lane == 0) {
    if (divisible) {
      slot[c] = TRIAL_NONE;
    } else {
      const uint32_t pos = atomicAdd(count, 1u);
      sel[pos] = c;
      slot[c] = pos;
    }
  }
}

// verdict[c] = 0 (failed trial division), 1 (a round failed), 2 (every round passed)
__global__ void prime_combine_kernel(const uint8_t* item_pass, const uint32_t* slot, uint32_t n, uint32_t per,
                                     uint8_t* verdict) {
  const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const uint32_t s = slot[c];
  if (s == TRIAL_NONE) {
    verdict[c] = 0;
    return;
  }
  uint8_t all = 1;
  for (uint32_t r = 0; r < per; r++) all &= item_pass[(size_t)s * per + r];
  verdict[c] = all ? 2 : 1;
}

}  // namespace

std::vector<uint32_t> trial_tables_host() {
  // the first TRIAL_MAX_PRIMES primes by a sieve of Eratosthenes (the last one is 104729)
  std::vector<uint32_t> primes;
  std::vector<uint8_t> comp(104730, 0);
  for (uint32_t i = 2; i < comp.size() && primes.size() < TRIAL_MAX_PRIMES; i++) {
    if (comp[i]) continue;
    primes.push_back(i);
    for (uint64_t m = (uint64_t)i * i; m < comp.size(); m += i) comp[m] = 1;
  }
  std::vector<uint32_t> t(trial_table_words(), 0);
  uint32_t* P = t.data() + (size_t)TRIAL_MAX_LIMBS * TRIAL_STRIDE;
  for (uint32_t j = 0; j < primes.size(); j++) {
    const uint64_t p = primes[j];
    uint64_t c = 1 % p;
    for (uint32_t w = 0; w < TRIAL_MAX_LIMBS; w++) {
      t[(size_t)w * TRIAL_STRIDE + j] = (uint32_t)c;
      c = (c << 32) % p;
    }
    P[j] = (uint32_t)p;
    const uint64_t mu = UINT64_MAX / p;
    P[TRIAL_STRIDE + 2 * j] = (uint32_t)mu;
    P[TRIAL_STRIDE + 2 * j + 1] = (uint32_t)(mu >> 32);
  }
  return t;
}

cudaError_t launch_trial(const uint32_t* cand, uint32_t nl, uint32_t n, const uint32_t* tab, uint32_t np,
                         uint32_t* sel, uint32_t* slot, uint32_t* count, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  if (nl == 0 || nl > TRIAL_MAX_LIMBS || np == 0 || np > TRIAL_MAX_PRIMES) return cudaErrorInvalidValue;
  trial_kernel<<<(n + TRIAL_WARPS - 1) / TRIAL_WARPS, TRIAL_WARPS * 32, 0, s>>>(cand, nl, n, tab, np, sel, slot, count);
  return cudaGetLastError();
}

cudaError_t launch_prime_combine(const uint8_t* item_pass, const uint32_t* slot, uint32_t n, uint32_t per,
                                 uint8_t* verdict, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  prime_combine_kernel<<<(n + 255) / 256, 256, 0, s>>>(item_pass, slot, n, per, verdict);
  return cudaGetLastError();
}

}  // namespace mr
