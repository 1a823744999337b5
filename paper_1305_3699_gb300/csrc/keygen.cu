// RSA key assembly from candidate pools on the device (Sec. 3.3: N = pq, d = e^-1 mod (p-1)(q-1);
// Sec. 3.1: Arazi's inversion for the inverse of the public exponent; Sec. 4.3 and Sec. 3.2: the
// primes are the candidates that pass trial division and the Miller-Rabin rounds, whose verdicts
// this kernel reads).  The private parts never leave the device.
//
// One thread per key, serial multi-limb arithmetic in local memory: the work per key (a few
// multi-limb products, two short divisions, one binary inversion of about 4 * 32H steps) is a
// small fraction of the primality tests that precede it.
//   p     first candidate of the key's p pool with verdict 2 and gcd(e, p - 1) = 1
//   q     the same in the q pool, q != p
//   N     p q;   d = Arazi(e, (p-1)(q-1));   dp = Arazi(e, p - 1);   dq = Arazi(e, q - 1)
//   qinv  q^-1 mod p by the binary extended Euclidean algorithm
//   Arazi(e, f) = (1 + f t) / e with t = -f^-1 mod e (only a single-word inverse is taken)
#include <cstdint>

#include "kernels_api.h"

namespace mr {
namespace {

constexpr int KG_MAX = 2 * KEYGEN_MAX_HALF_LIMBS;  // limbs of N

__device__ bool kg_is_zero(const uint32_t* a, int n) {
  for (int i = 0; i < n; i++)
    if (a[i]) return false;
  return true;
}

__device__ bool kg_is_one(const uint32_t* a, int n) { return a[0] == 1u && kg_is_zero(a + 1, n - 1); }

__device__ int kg_cmp(const uint32_t* a, const uint32_t* b, int n) {
  for (int i = n - 1; i >= 0; i--)
    if (a[i] != b[i]) return a[i] > b[i] ? 1 : -1;
  return 0;
}

// r = a - b (n limbs); returns the borrow
__device__ uint32_t kg_sub(uint32_t* r, const uint32_t* a, const uint32_t* b, int n) {
  uint32_t br = 0;
  for (int i = 0; i < n; i++) {
    const uint64_t d = (uint64_t)a[i] - b[i] - br;
    r[i] = (uint32_t)d;
    br = (uint32_t)(d >> 32) ? 1u : 0u;
  }
  return br;
}

// r = a + b (n limbs); returns the carry
__device__ uint32_t kg_add(uint32_t* r, const uint32_t* a, const uint32_t* b, int n) {
  uint64_t c = 0;
  for (int i = 0; i < n; i++) {
    c += (uint64_t)a[i] + b[i];
    r[i] = (uint32_t)c;
    c >>= 32;
  }
  return (uint32_t)c;
}

// a = (top:a) / 2
__device__ void kg_shr1(uint32_t* a, int n, uint32_t top) {
  for (int i = 0; i < n; i++) {
    const uint32_t hi = i + 1 < n ? a[i + 1] : top;
    a[i] = (a[i] >> 1) | (hi << 31);
  }
}

// r (2n limbs) = a b
__device__ void kg_mul(uint32_t* r, const uint32_t* a, const uint32_t* b, int n) {
  for (int i = 0; i < 2 * n; i++) r[i] = 0;
  for (int i = 0; i < n; i++) {
    uint64_t c = 0;
    for (int j = 0; j < n; j++) {
      c += (uint64_t)a[i] * b[j] + r[i + j];
      r[i + j] = (uint32_t)c;
      c >>= 32;
    }
    r[i + n] = (uint32_t)c;
  }
}

__device__ uint32_t kg_mod_small(const uint32_t* a, int n, uint32_t m) {
  uint64_t r = 0;
  for (int i = n - 1; i >= 0; i--) r = ((r << 32) | a[i]) % m;
  return (uint32_t)r;
}

__device__ uint32_t kg_gcd(uint32_t a, uint32_t b) {
  while (b) {
    const uint32_t t = a % b;
    a = b;
    b = t;
  }
  return a;
}

// a^-1 mod m for gcd(a, m) = 1 (extended Euclid on words); 0 otherwise
__device__ uint32_t kg_inv_small(uint32_t a, uint32_t m) {
  int64_t r0 = m, r1 = a % m, s0 = 0, s1 = 1;
  while (r1) {
    const int64_t qt = r0 / r1;
    int64_t t = r0 - qt * r1;
    r0 = r1;
    r1 = t;
    t = s0 - qt * s1;
    s0 = s1;
    s1 = t;
  }
  if (r0 != 1) return 0;
  return (uint32_t)(((s0 % (int64_t)m) + (int64_t)m) % (int64_t)m);
}

// d (n limbs) = e^-1 mod f by Arazi's formula; false when gcd(e, f) != 1
__device__ bool kg_arazi(uint32_t* d, const uint32_t* f, int n, uint32_t e) {
  const uint32_t r = kg_mod_small(f, n, e);
  const uint32_t inv = kg_inv_small(r, e);
  if (!inv) return false;
  const uint32_t t = e - inv;  // -f^-1 mod e (inv in [1, e))
  // num = 1 + f t (n + 1 limbs), then d = num / e exactly, from the top
  uint32_t num[KG_MAX + 1];
  uint64_t c = 1;
  for (int i = 0; i < n; i++) {
    c += (uint64_t)f[i] * t;
    num[i] = (uint32_t)c;
    c >>= 32;
  }
  num[n] = (uint32_t)c;
  uint64_t rem = 0;
  for (int i = n; i >= 0; i--) {
    const uint64_t cur = (rem << 32) | num[i];
    const uint64_t qd = cur / e;
    rem = cur - qd * e;
    if (i < n) d[i] = (uint32_t)qd;  // the quotient is below f: its limb n is zero
  }
  return rem == 0;
}

// r = a mod p (n limbs each), binary long division
__device__ void kg_mod(uint32_t* r, const uint32_t* a, const uint32_t* p, int n) {
  uint32_t t[KG_MAX / 2 + 1], pe[KG_MAX / 2 + 1];
  for (int i = 0; i <= n; i++) {
    t[i] = 0;
    pe[i] = i < n ? p[i] : 0u;
  }
  for (int bit = 32 * n - 1; bit >= 0; bit--) {
    uint32_t cy = (a[bit >> 5] >> (bit & 31)) & 1u;  // t = 2 t + bit
    for (int i = 0; i <= n; i++) {
      const uint32_t nc = t[i] >> 31;
      t[i] = (t[i] << 1) | cy;
      cy = nc;
    }
    if (kg_cmp(t, pe, n + 1) >= 0) kg_sub(t, t, pe, n + 1);
  }
  for (int i = 0; i < n; i++) r[i] = t[i];
}

// r = u^-1 mod p (p odd), binary extended Euclid with a bounded step count; false when u has no
// inverse (or the bound ran out)
__device__ bool kg_inv(uint32_t* r, const uint32_t* u, const uint32_t* p, int n) {
  uint32_t a[KG_MAX / 2], b[KG_MAX / 2], x1[KG_MAX / 2], x2[KG_MAX / 2];
  kg_mod(a, u, p, n);
  for (int i = 0; i < n; i++) {
    b[i] = p[i];
    x1[i] = i == 0 ? 1u : 0u;
    x2[i] = 0;
  }
  if (kg_is_zero(a, n)) return false;
  const int limit = 8 * 32 * n + 64;
  int steps = 0;
  while (!kg_is_one(a, n) && !kg_is_one(b, n)) {
    if (kg_is_zero(a, n) || kg_is_zero(b, n) || ++steps > limit) return false;
    while ((a[0] & 1u) == 0 && steps++ <= limit) {
      kg_shr1(a, n, 0);
      const uint32_t cy = (x1[0] & 1u) ? kg_add(x1, x1, p, n) : 0u;
      kg_shr1(x1, n, cy);
    }
    while ((b[0] & 1u) == 0 && steps++ <= limit) {
      kg_shr1(b, n, 0);
      const uint32_t cy = (x2[0] & 1u) ? kg_add(x2, x2, p, n) : 0u;
      kg_shr1(x2, n, cy);
    }
    if (kg_cmp(a, b, n) >= 0) {
      kg_sub(a, a, b, n);
      if (kg_sub(x1, x1, x2, n)) kg_add(x1, x1, p, n);
    } else {
      kg_sub(b, b, a, n);
      if (kg_sub(x2, x2, x1, n)) kg_add(x2, x2, p, n);
    }
  }
  const uint32_t* x = kg_is_one(a, n) ? x1 : x2;
  for (int i = 0; i < n; i++) r[i] = x[i];
  return true;
}

// the first candidate of a pool with verdict 2, gcd(e, c - 1) = 1 and c != skip; -1 when none
__device__ int kg_pick(const uint32_t* cand, const uint8_t* verdict, uint32_t first, uint32_t pool, int H, uint32_t e,
                       const uint32_t* skip) {
  for (uint32_t j = 0; j < pool; j++) {
    const uint32_t idx = first + j;
    if (verdict[idx] != 2) continue;
    const uint32_t* c = cand + (size_t)idx * H;
    const uint32_t cm1 = (uint32_t)(((uint64_t)kg_mod_small(c, H, e) + e - 1) % e);  // (c - 1) mod e
    if (kg_gcd(e, cm1) != 1) continue;  // gcd(e, 0) = e > 1
    if (skip && kg_cmp(c, skip, H) == 0) continue;
    return (int)j;
  }
  return -1;
}

__global__ void keygen_kernel(const uint32_t* cand, const uint8_t* verdict, uint32_t n_keys, uint32_t pool, int H,
                              uint32_t e, uint32_t* out, uint8_t* status) {
  const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_keys) return;
  uint32_t* o = out + (size_t)k * 9 * H;  // N 2H | d 2H | p | q | dp | dq | qinv
  uint32_t* oN = o;
  uint32_t* od = o + 2 * H;
  uint32_t* op = o + 4 * H;
  uint32_t* oq = o + 5 * H;
  uint32_t* odp = o + 6 * H;
  uint32_t* odq = o + 7 * H;
  uint32_t* oqi = o + 8 * H;
  uint8_t st = 0;
  const uint32_t base = k * 2 * pool;
  const int jp = kg_pick(cand, verdict, base, pool, H, e, nullptr);
  const int jq = jp < 0 ? -1 : kg_pick(cand, verdict, base + pool, pool, H, e, cand + (size_t)(base + jp) * H);
  uint32_t p[KG_MAX / 2], q[KG_MAX / 2], pm1[KG_MAX / 2], qm1[KG_MAX / 2], one[KG_MAX / 2];
  uint32_t N[KG_MAX], phi[KG_MAX], t[KG_MAX];
  if (jp < 0 || jq < 0) {
    st = 5;  // MR_ERR_RANGE: a pool holds no usable prime
  } else {
    for (int i = 0; i < H; i++) {
      p[i] = cand[(size_t)(base + jp) * H + i];
      q[i] = cand[(size_t)(base + pool + jq) * H + i];
      one[i] = i == 0 ? 1u : 0u;
    }
    kg_sub(pm1, p, one, H);
    kg_sub(qm1, q, one, H);
    kg_mul(N, p, q, H);
    kg_mul(phi, pm1, qm1, H);
    bool ok = kg_arazi(t, phi, 2 * H, e);
    for (int i = 0; i < 2 * H; i++) {
      oN[i] = N[i];
      od[i] = ok ? t[i] : 0u;
    }
    ok = ok && kg_arazi(t, pm1, H, e);
    for (int i = 0; i < H; i++) odp[i] = ok ? t[i] : 0u;
    ok = ok && kg_arazi(t, qm1, H, e);
    for (int i = 0; i < H; i++) odq[i] = ok ? t[i] : 0u;
    ok = ok && kg_inv(t, q, p, H);
    for (int i = 0; i < H; i++) {
      oqi[i] = ok ? t[i] : 0u;
      op[i] = p[i];
      oq[i] = q[i];
    }
    if (!ok) st = 3;  // MR_ERR_NOT_COPRIME: an inverse does not exist (not a prime after all)
  }
  if (st == 5)
    for (int i = 0; i < 9 * H; i++) o[i] = 0u;
  if (status) status[k] = st;
}

}  // namespace

cudaError_t launch_keygen(const uint32_t* cand, const uint8_t* verdict, uint32_t n_keys, uint32_t pool,
                          uint32_t half_limbs, uint32_t e, uint32_t* out, uint8_t* status, cudaStream_t s) {
  if (n_keys == 0) return cudaSuccess;
  if (half_limbs < 2 || half_limbs > KEYGEN_MAX_HALF_LIMBS || pool == 0 || e < 3 || !(e & 1u))
    return cudaErrorInvalidValue;
  keygen_kernel<<<(n_keys + 31) / 32, 32, 0, s>>>(cand, verdict, n_keys, pool, (int)half_limbs, e, out, status);
  return cudaGetLastError();
}

}  // namespace mr
