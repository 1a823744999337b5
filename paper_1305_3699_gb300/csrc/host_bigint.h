// Host-side multi-precision helpers used only by the one-time setup of size
// classes and moduli (never on the exponentiation path).  Little-endian
// uint32 limbs, normalised (no zero top limb; zero is the empty vector).
#pragma once
#include <algorithm>
#include <cstdint>
#include <vector>

namespace mr {

struct Big {
  std::vector<uint32_t> w;
  Big() = default;
  explicit Big(uint64_t v) {
    if (v) w.push_back((uint32_t)v);
    if (v >> 32) w.push_back((uint32_t)(v >> 32));
  }
  static Big from_limbs(const uint32_t* p, size_t n) {
    Big b;
    b.w.assign(p, p + n);
    b.norm();
    return b;
  }
  void norm() {
    while (!w.empty() && w.back() == 0) w.pop_back();
  }
  bool is_zero() const { return w.empty(); }
  size_t bits() const {
    if (w.empty()) return 0;
    uint32_t t = w.back();
    size_t b = 0;
    while (t) {
      b++;
      t >>= 1;
    }
    return 32 * (w.size() - 1) + b;
  }
  bool bit(size_t i) const {
    size_t q = i / 32;
    return q < w.size() && ((w[q] >> (i % 32)) & 1u);
  }
  uint32_t limb(size_t i) const { return i < w.size() ? w[i] : 0u; }
  std::vector<uint32_t> limbs(size_t n) const {
    std::vector<uint32_t> out(n, 0);
    for (size_t i = 0; i < n && i < w.size(); i++) out[i] = w[i];
    return out;
  }
};

inline int cmp(const Big& a, const Big& b) {
  if (a.w.size() != b.w.size()) return a.w.size() < b.w.size() ? -1 : 1;
  for (size_t i = a.w.size(); i-- > 0;)
    if (a.w[i] != b.w[i]) return a.w[i] < b.w[i] ? -1 : 1;
  return 0;
}

inline Big add(const Big& a, const Big& b) {
  Big r;
  size_t n = std::max(a.w.size(), b.w.size());
  r.w.resize(n + 1);
  uint64_t c = 0;
  for (size_t i = 0; i < n; i++) {
    c += (uint64_t)a.limb(i) + b.limb(i);
    r.w[i] = (uint32_t)c;
    c >>= 32;
  }
  r.w[n] = (uint32_t)c;
  r.norm();
  return r;
}

// a - b, requires a >= b
inline Big sub(const Big& a, const Big& b) {
  Big r;
  r.w.resize(a.w.size());
  int64_t br = 0;
  for (size_t i = 0; i < a.w.size(); i++) {
    int64_t t = (int64_t)a.w[i] - (int64_t)b.limb(i) - br;
    br = t < 0;
    r.w[i] = (uint32_t)(t + (br ? (int64_t)1 << 32 : 0));
  }
  r.norm();
  return r;
}

inline Big mul(const Big& a, const Big& b) {
  if (a.is_zero() || b.is_zero()) return Big();
  Big r;
  r.w.assign(a.w.size() + b.w.size(), 0);
  for (size_t i = 0; i < a.w.size(); i++) {
    uint64_t c = 0;
    for (size_t j = 0; j < b.w.size(); j++) {
      uint64_t t = (uint64_t)a.w[i] * b.w[j] + r.w[i + j] + c;
      r.w[i + j] = (uint32_t)t;
      c = t >> 32;
    }
    r.w[i + b.w.size()] = (uint32_t)c;
  }
  r.norm();
  return r;
}

inline Big mul_small(const Big& a, uint32_t m) { return mul(a, Big(m)); }

inline Big shl(const Big& a, size_t s) {
  if (a.is_zero()) return Big();
  Big r;
  size_t q = s / 32, b = s % 32;
  r.w.assign(a.w.size() + q + 1, 0);
  for (size_t i = 0; i < a.w.size(); i++) {
    uint64_t v = (uint64_t)a.w[i] << b;
    r.w[i + q] |= (uint32_t)v;
    r.w[i + q + 1] |= (uint32_t)(v >> 32);
  }
  r.norm();
  return r;
}

// quotient and remainder by a small divisor
inline Big divmod_small(const Big& a, uint32_t d, uint32_t* rem) {
  Big q;
  q.w.assign(a.w.size(), 0);
  uint64_t r = 0;
  for (size_t i = a.w.size(); i-- > 0;) {
    uint64_t cur = (r << 32) | a.w[i];
    q.w[i] = (uint32_t)(cur / d);
    r = cur % d;
  }
  q.norm();
  if (rem) *rem = (uint32_t)r;
  return q;
}

inline uint32_t mod_small(const Big& a, uint32_t m) {
  uint64_t r = 0;
  for (size_t i = a.w.size(); i-- > 0;) r = ((r << 32) | a.w[i]) % m;
  return (uint32_t)r;
}

// a mod n by binary long division (bit by bit); fine for one-time setup.
inline Big mod(const Big& a, const Big& n) {
  if (cmp(a, n) < 0) return a;
  Big r;
  for (size_t i = a.bits(); i-- > 0;) {
    r = shl(r, 1);
    if (a.bit(i)) {
      if (r.w.empty()) r.w.push_back(0);
      r.w[0] |= 1u;
    }
    if (cmp(r, n) >= 0) r = sub(r, n);
  }
  return r;
}

// ------------------------------------------------------------- word arithmetic

inline uint32_t mulmod32(uint64_t a, uint64_t b, uint32_t m) { return (uint32_t)((a % m) * (b % m) % m); }

inline uint32_t powmod32(uint32_t a, uint64_t e, uint32_t m) {
  uint64_t r = 1 % m, b = a % m;
  while (e) {
    if (e & 1) r = r * b % m;
    b = b * b % m;
    e >>= 1;
  }
  return (uint32_t)r;
}

// inverse modulo a prime (Fermat)
inline uint32_t invmod_prime(uint32_t a, uint32_t p) { return powmod32(a % p, p - 2, p); }

// inverse of an odd number modulo 2^32 (Newton iteration)
inline uint32_t inv32(uint32_t a) {
  uint32_t x = a;  // correct to 3 bits for odd a
  for (int i = 0; i < 5; i++) x *= 2u - a * x;
  return x;
}

inline bool is_prime_u32(uint32_t n) {
  if (n < 2) return false;
  for (uint32_t p : {2u, 3u, 5u, 7u, 11u, 13u, 17u, 19u, 23u, 29u, 31u, 37u})
    if (n % p == 0) return n == p;
  uint32_t d = n - 1;
  int s = 0;
  while ((d & 1) == 0) {
    d >>= 1;
    s++;
  }
  // bases 2, 7, 61 decide primality for every n < 4,759,123,141
  for (uint32_t a : {2u, 7u, 61u}) {
    if (a % n == 0) continue;
    uint64_t y = powmod32(a, d, n);
    if (y == 1 || y == n - 1) continue;
    bool comp = true;
    for (int r = 1; r < s; r++) {
      y = y * y % n;
      if (y == n - 1) {
        comp = false;
        break;
      }
    }
    if (comp) return false;
  }
  return true;
}

}  // namespace mr
