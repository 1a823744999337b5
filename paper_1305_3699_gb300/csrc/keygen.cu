// RSA key assembly from candidate pools on the device (Sec. 3.3: N = pq, d = e^-1 mod (p-1)(q-1);
// Sec. 3.1: Arazi's inversion for the inverse of the public exponent; Sec. 4.3 and Sec. 3.2: the
// primes are the candidates that pass trial division and the Miller-Rabin rounds, whose verdicts
// this kernel reads).  The private parts never leave the device.
//
// One warp per key.  Lane 0 picks the primes and forms N, d, dp, dq with serial multi-limb code
// (a few products and three exact divisions by e); the binary inversion for qinv, about 4 * 32H
// dependent steps, runs on the whole warp with one limb per lane and register (limb i in lane
// i mod 32, register i / 32): carries of an addition are resolved for all limbs at once from
// two ballots (generate and propagate masks, added as integers), shifts move one bit between
// neighbouring lanes.
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
  bool f_is_one = f[0] == 1u;
  for (int i = n; i >= 0; i--) {
    const uint64_t cur = (rem << 32) | num[i];
    const uint64_t qd = cur / e;
    rem = cur - qd * e;
    if (i < n) d[i] = (uint32_t)qd;  // the quotient is below f for f > 1: its limb n is zero
    if (i > 0 && i < n && f[i]) f_is_one = false;
  }
  if (f_is_one)  // e^-1 mod 1 = 0 (the formula gives 1)
    for (int i = 0; i < n; i++) d[i] = 0u;
  return rem == 0;
}

// ---- warp-cooperative multi-limb arithmetic: limb i = 32 j + lane (j < R registers per lane),
// n <= 32 R limbs; limbs at or above n are zero.  Every lane of the warp calls these together.
constexpr unsigned FULL = 0xffffffffu;

// r = a + b + cin over n limbs; returns the carry out of limb n-1
template <int R>
__device__ uint32_t w_add(uint32_t (&r)[R], const uint32_t (&a)[R], const uint32_t (&b)[R], uint32_t cin, int n,
                          int lane) {
  uint32_t sm[R], C[R];
  // carry into limb i = carry into bit i of the integer sum G + (G | P) + cin, G the limbs that
  // generate a carry and P those that pass one on (32 R-bit masks from ballots, one word per register)
  uint32_t cy = cin;
#pragma unroll
  for (int j = 0; j < R; j++) {
    sm[j] = a[j] + b[j];
    const uint32_t G = __ballot_sync(FULL, sm[j] < a[j]);
    const uint32_t X = G | __ballot_sync(FULL, sm[j] == 0xffffffffu);
    const uint64_t t = (uint64_t)G + X + cy;
    cy = (uint32_t)(t >> 32);
    C[j] = (uint32_t)t ^ G ^ X;
  }
  uint32_t out = cy;  // n = 32 R: the carry out of the top word
#pragma unroll
  for (int j = 0; j < R; j++) {
    const int i = 32 * j + lane;
    r[j] = i < n ? sm[j] + ((C[j] >> lane) & 1u) : 0u;
    if (n < 32 * R && (n >> 5) == j) out = (C[j] >> (n & 31)) & 1u;
  }
  return out;
}

// r = a - b over n limbs; returns the borrow
template <int R>
__device__ uint32_t w_sub(uint32_t (&r)[R], const uint32_t (&a)[R], const uint32_t (&b)[R], int n, int lane) {
  uint32_t nb[R];
#pragma unroll
  for (int j = 0; j < R; j++) nb[j] = 32 * j + lane < n ? ~b[j] : 0u;
  return 1u - w_add<R>(r, a, nb, 1u, n, lane);
}

// v = (top : v) / 2, top in {0, 1} being limb n
template <int R>
__device__ void w_shr1(uint32_t (&v)[R], uint32_t top, int n, int lane) {
  uint32_t up[R], first[R];
#pragma unroll
  for (int j = 0; j < R; j++) {
    up[j] = __shfl_down_sync(FULL, v[j], 1);  // limb i + 1 within the register word
    first[j] = __shfl_sync(FULL, v[j], 0);    // limb 32 j, the successor of limb 32 j - 1
  }
#pragma unroll
  for (int j = 0; j < R; j++) {
    const int i = 32 * j + lane;
    const uint32_t nb = i + 1 == n ? top : (lane < 31 ? up[j] : (j + 1 < R ? first[j + 1 < R ? j + 1 : j] : 0u));
    v[j] = i < n ? (v[j] >> 1) | (nb << 31) : 0u;
  }
}

// v = 2 v + bit0 over n limbs
template <int R>
__device__ void w_shl1(uint32_t (&v)[R], uint32_t bit0, int n, int lane) {
  uint32_t dn[R], last[R];
#pragma unroll
  for (int j = 0; j < R; j++) {
    dn[j] = __shfl_up_sync(FULL, v[j], 1);  // limb i - 1 within the register word
    last[j] = __shfl_sync(FULL, v[j], 31);  // limb 32 j + 31, the predecessor of limb 32 (j + 1)
  }
#pragma unroll
  for (int j = 0; j < R; j++) {
    const int i = 32 * j + lane;
    const uint32_t lo = i == 0 ? (bit0 << 31) : (lane > 0 ? dn[j] : last[j > 0 ? j - 1 : 0]);
    v[j] = i < n ? (v[j] << 1) | (lo >> 31) : 0u;
  }
}

template <int R>
__device__ __forceinline__ bool w_is_zero(const uint32_t (&v)[R]) {
  uint32_t o = 0;
#pragma unroll
  for (int j = 0; j < R; j++) o |= v[j];
  return !__any_sync(FULL, o != 0u);
}

template <int R>
__device__ __forceinline__ bool w_is_one(const uint32_t (&v)[R], int lane) {
  uint32_t o = 0;
#pragma unroll
  for (int j = 1; j < R; j++) o |= v[j];
  return __all_sync(FULL, o == 0u && v[0] == (lane == 0 ? 1u : 0u));
}

template <int R>
__device__ __forceinline__ uint32_t w_low_bit(const uint32_t (&v)[R]) { return __shfl_sync(FULL, v[0], 0) & 1u; }

// bit `bit` of v (uniform)
template <int R>
__device__ __forceinline__ uint32_t w_bit(const uint32_t (&v)[R], int bit) {
  const int li = bit >> 5;
  uint32_t sel = v[0];
#pragma unroll
  for (int j = 1; j < R; j++)
    if ((li >> 5) == j) sel = v[j];
  const uint32_t word = __shfl_sync(FULL, sel, li & 31);
  return (word >> (bit & 31)) & 1u;
}

// r = u mod p by binary long division (32n steps)
template <int R>
__device__ void w_mod(uint32_t (&r)[R], const uint32_t (&u)[R], const uint32_t (&p)[R], int n, int lane) {
#pragma unroll
  for (int j = 0; j < R; j++) r[j] = 0u;
  for (int bit = 32 * n - 1; bit >= 0; bit--) {
    const uint32_t t = w_bit<R>(r, 32 * n - 1);  // the bit shifted out of limb n-1
    w_shl1<R>(r, w_bit<R>(u, bit), n, lane);
    uint32_t d[R];
    const uint32_t br = w_sub<R>(d, r, p, n, lane);
    if (t || !br) {  // 2r + bit >= p (the value is below 2p)
#pragma unroll
      for (int j = 0; j < R; j++) r[j] = d[j];
    }
  }
}

// r = u^-1 mod p (p odd) by the binary extended Euclidean algorithm, with a bounded step count;
// false when u has no inverse (or the bound ran out)
template <int R>
__device__ bool w_inv(uint32_t (&r)[R], const uint32_t (&u)[R], const uint32_t (&p)[R], int n, int lane) {
  uint32_t a[R], b[R], x1[R], x2[R];
#pragma unroll
  for (int j = 0; j < R; j++) {
    b[j] = p[j];
    x1[j] = (j == 0 && lane == 0) ? 1u : 0u;
    x2[j] = 0u;
  }
  w_mod<R>(a, u, p, n, lane);
  if (w_is_zero<R>(a)) return false;
  const int limit = 8 * 32 * n + 64;
  int steps = 0;
  while (!w_is_one<R>(a, lane) && !w_is_one<R>(b, lane)) {
    if (w_is_zero<R>(a) || w_is_zero<R>(b) || ++steps > limit) return false;
    while (!w_low_bit<R>(a) && steps++ <= limit) {
      w_shr1<R>(a, 0u, n, lane);
      uint32_t cy = 0u;
      if (w_low_bit<R>(x1)) cy = w_add<R>(x1, x1, p, 0u, n, lane);
      w_shr1<R>(x1, cy, n, lane);
    }
    while (!w_low_bit<R>(b) && steps++ <= limit) {
      w_shr1<R>(b, 0u, n, lane);
      uint32_t cy = 0u;
      if (w_low_bit<R>(x2)) cy = w_add<R>(x2, x2, p, 0u, n, lane);
      w_shr1<R>(x2, cy, n, lane);
    }
    uint32_t d[R];
    if (!w_sub<R>(d, a, b, n, lane)) {  // a >= b
#pragma unroll
      for (int j = 0; j < R; j++) a[j] = d[j];
      if (w_sub<R>(x1, x1, x2, n, lane)) w_add<R>(x1, x1, p, 0u, n, lane);
    } else {
      w_sub<R>(b, b, a, n, lane);
      if (w_sub<R>(x2, x2, x1, n, lane)) w_add<R>(x2, x2, p, 0u, n, lane);
    }
  }
  const bool one_a = w_is_one<R>(a, lane);
#pragma unroll
  for (int j = 0; j < R; j++) r[j] = one_a ? x1[j] : x2[j];
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

// R: registers per lane of the warp-wide inversion (32 R >= H)
template <int R>
__global__ void __launch_bounds__(32) keygen_kernel(const uint32_t* cand, const uint8_t* verdict, uint32_t pool,
                                                    int H, uint32_t e, uint32_t* out, uint8_t* status) {
  __shared__ uint32_t sp[KEYGEN_MAX_HALF_LIMBS], sq[KEYGEN_MAX_HALF_LIMBS];
  __shared__ uint32_t sst;
  const uint32_t k = blockIdx.x;  // one warp per key
  const int lane = (int)threadIdx.x;
  uint32_t* o = out + (size_t)k * 9 * H;  // N 2H | d 2H | p | q | dp | dq | qinv
  if (lane == 0) {
    uint32_t st = 0;
    const uint32_t base = k * 2 * pool;
    const int jp = kg_pick(cand, verdict, base, pool, H, e, nullptr);
    const int jq = jp < 0 ? -1 : kg_pick(cand, verdict, base + pool, pool, H, e, cand + (size_t)(base + jp) * H);
    if (jp < 0 || jq < 0) {
      st = 5;  // MR_ERR_RANGE: a pool holds no usable prime
    } else {
      uint32_t p[KG_MAX / 2], q[KG_MAX / 2], pm1[KG_MAX / 2], qm1[KG_MAX / 2], one[KG_MAX / 2];
      uint32_t N[KG_MAX], phi[KG_MAX], t[KG_MAX];
      for (int i = 0; i < H; i++) {
        p[i] = cand[(size_t)(base + jp) * H + i];
        q[i] = cand[(size_t)(base + pool + jq) * H + i];
        one[i] = i == 0 ? 1u : 0u;
        sp[i] = p[i];
        sq[i] = q[i];
        o[4 * H + i] = p[i];
        o[5 * H + i] = q[i];
      }
      kg_sub(pm1, p, one, H);
      kg_sub(qm1, q, one, H);
      kg_mul(N, p, q, H);
      kg_mul(phi, pm1, qm1, H);
      bool ok = kg_arazi(t, phi, 2 * H, e);
      for (int i = 0; i < 2 * H; i++) {
        o[i] = N[i];
        o[2 * H + i] = ok ? t[i] : 0u;
      }
      ok = ok && kg_arazi(t, pm1, H, e);
      for (int i = 0; i < H; i++) o[6 * H + i] = ok ? t[i] : 0u;
      ok = ok && kg_arazi(t, qm1, H, e);
      for (int i = 0; i < H; i++) o[7 * H + i] = ok ? t[i] : 0u;
      if (!ok) st = 3;  // MR_ERR_NOT_COPRIME: gcd(e, p-1) = gcd(e, q-1) = 1 was checked; not reached
    }
    sst = st;
  }
  __syncwarp();
  uint32_t st = sst;
  if (st == 0) {  // qinv = q^-1 mod p on the whole warp
    uint32_t pw[R], qw[R], r[R];
#pragma unroll
    for (int j = 0; j < R; j++) {
      const int i = 32 * j + lane;
      pw[j] = i < H ? sp[i] : 0u;
      qw[j] = i < H ? sq[i] : 0u;
    }
    const bool ok = w_inv<R>(r, qw, pw, H, lane);
#pragma unroll
    for (int j = 0; j < R; j++) {
      const int i = 32 * j + lane;
      if (i < H) o[8 * H + i] = ok ? r[j] : 0u;
    }
    if (!ok) st = 3;  // MR_ERR_NOT_COPRIME: q has no inverse mod p (p not prime after all)
  } else if (st == 5) {
    for (int i = lane; i < 9 * H; i += 32) o[i] = 0u;
  }
  if (lane == 0 && status) status[k] = (uint8_t)st;
}

}  // namespace

cudaError_t launch_keygen(const uint32_t* cand, const uint8_t* verdict, uint32_t n_keys, uint32_t pool,
                          uint32_t half_limbs, uint32_t e, uint32_t* out, uint8_t* status, cudaStream_t s) {
  if (n_keys == 0) return cudaSuccess;
  if (half_limbs < 2 || half_limbs > KEYGEN_MAX_HALF_LIMBS || pool == 0 || e < 3 || !(e & 1u))
    return cudaErrorInvalidValue;
  if (half_limbs <= 64)
    keygen_kernel<2><<<n_keys, 32, 0, s>>>(cand, verdict, pool, (int)half_limbs, e, out, status);
  else
    keygen_kernel<4><<<n_keys, 32, 0, s>>>(cand, verdict, pool, (int)half_limbs, e, out, status);
  return cudaGetLastError();
}

}  // namespace mr
