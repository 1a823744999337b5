// Host setup of size classes and moduli.  See setup.h.
//
// Base choice (the paper asks for a careful choice of coprime bases without
// fixing one): for k channels per base every prime lies below
// b_k = min(2^31, isqrt((2^64-1)/k)), so that the k-term dot products of the
// base extensions accumulate exactly in 64-bit words; B takes the k largest
// primes below b_k, B' the next k; k is the smallest value with
// M >= 4 (k+1)^2 2^L (products of operands below 2(k+1)N stay closed below
// (k+1)N) and M' >= 2 (k+1) 2^L (the fixed-point B'->B correction is exact).
#include "setup.h"

#include <algorithm>
#include <map>
#include <mutex>

#include "../../include/mr.h"

namespace mr {

const std::vector<uint32_t>& class_bits_list() {
  static const std::vector<uint32_t> v = {512, 1024, 1536, 2048, 3072, 4096, 8192, 16384};
  return v;
}

uint32_t class_for_bits(uint32_t bits) {
  for (uint32_t L : class_bits_list())
    if (bits <= L) return L;
  return 0;
}

static uint64_t isqrt64(uint64_t v) {
  uint64_t lo = 0, hi = 1ull << 32;
  while (hi - lo > 1) {  // invariant: lo^2 <= v < hi^2
    uint64_t mid = lo + (hi - lo) / 2;
    unsigned __int128 sq = (unsigned __int128)mid * mid;
    if (sq <= v)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

static uint64_t prime_bound(uint32_t k) {
  uint64_t b = isqrt64(~0ull / k);
  return b < (1ull << 31) ? b : (1ull << 31);
}

// the `count` largest primes strictly below `bound`, descending
static std::vector<uint32_t> primes_below(uint64_t bound, uint32_t count) {
  static std::mutex mu;
  static std::map<uint64_t, std::vector<uint32_t>> cache;
  std::lock_guard<std::mutex> g(mu);
  auto& v = cache[bound];
  uint64_t n = v.empty() ? bound - 1 : (uint64_t)v.back() - 1;
  while (v.size() < count && n >= 3) {
    if ((n & 1) && is_prime_u32((uint32_t)n)) v.push_back((uint32_t)n);
    n--;
  }
  return std::vector<uint32_t>(v.begin(), v.begin() + std::min<size_t>(count, v.size()));
}

static Big product(const std::vector<uint32_t>& xs, size_t from, size_t to) {
  Big r(1);
  for (size_t i = from; i < to; i++) r = mul_small(r, xs[i]);
  return r;
}

static uint32_t bitlen32(uint32_t v) {
  uint32_t b = 0;
  while (v) {
    b++;
    v >>= 1;
  }
  return b;
}

bool build_class(uint32_t L, ClassHost& c, std::string& err) {
  if (L == 0 || L % 32) {
    err = "class bits must be a positive multiple of 32";
    return false;
  }
  Big four_k1sq_2L, two_k1_2L;
  // every channel prime is below 2^31, so M < 2^(31k) and M >= 2^L needs k > L/31
  uint32_t k = std::max<uint32_t>(1, L / 31);
  for (;; k++) {
    if (k > 4096) {
      err = "no base found";
      return false;
    }
    uint64_t b = prime_bound(k);
    std::vector<uint32_t> pr = primes_below(b, 2 * k);
    if (pr.size() < 2 * k) {
      err = "not enough primes";
      return false;
    }
    Big M = product(pr, 0, k), Mp = product(pr, k, 2 * k);
    Big lhs1 = shl(Big((uint64_t)4 * (k + 1) * (k + 1)), L);
    Big lhs2 = shl(Big((uint64_t)2 * (k + 1)), L);
    if (cmp(M, lhs1) >= 0 && cmp(Mp, lhs2) >= 0) {
      c.L = L;
      c.k = k;
      c.bound = b;
      c.B.assign(pr.begin(), pr.begin() + k);
      c.Bp.assign(pr.begin() + k, pr.end());
      c.M = M;
      c.Mp = Mp;
      break;
    }
  }
  c.W = L / 32;
  c.WX = (uint32_t)((c.M.bits() + bitlen32(k) + 31) / 32);

  const auto& B = c.B;
  const auto& Bp = c.Bp;
  // products of all but one prime, modulo another prime, by prefix/suffix products
  auto all_but_one_mod = [&](const std::vector<uint32_t>& base, uint32_t mod, std::vector<uint32_t>& out) {
    size_t n = base.size();
    std::vector<uint64_t> pre(n + 1), suf(n + 1);
    pre[0] = 1 % mod;
    for (size_t i = 0; i < n; i++) pre[i + 1] = pre[i] * (base[i] % mod) % mod;
    suf[n] = 1 % mod;
    for (size_t i = n; i-- > 0;) suf[i] = suf[i + 1] * (base[i] % mod) % mod;
    out.resize(n);
    for (size_t i = 0; i < n; i++) out[i] = (uint32_t)(pre[i] * suf[i + 1] % mod);
    return (uint32_t)pre[n];  // product of all, mod `mod`
  };

  c.M_mi_inv.resize(k);
  c.Mp_mj_inv.resize(k);
  c.Minv_Bp.resize(k);
  c.Mp_B.resize(k);
  c.M_mi_Bp.assign((size_t)k * k, 0);
  c.Mp_mj_B.assign((size_t)k * k, 0);
  std::vector<uint32_t> tmp;
  for (uint32_t i = 0; i < k; i++) {
    all_but_one_mod(B, B[i], tmp);
    c.M_mi_inv[i] = invmod_prime(tmp[i], B[i]);
    uint32_t mp_all = all_but_one_mod(Bp, B[i], tmp);
    c.Mp_B[i] = mp_all;
    for (uint32_t j = 0; j < k; j++) c.Mp_mj_B[(size_t)j * k + i] = tmp[j];
  }
  for (uint32_t j = 0; j < k; j++) {
    all_but_one_mod(Bp, Bp[j], tmp);
    c.Mp_mj_inv[j] = invmod_prime(tmp[j], Bp[j]);
    uint32_t m_all = all_but_one_mod(B, Bp[j], tmp);
    c.Minv_Bp[j] = invmod_prime(m_all, Bp[j]);
    for (uint32_t i = 0; i < k; i++) c.M_mi_Bp[(size_t)i * k + j] = tmp[i];
  }

  // ---- device form
  ClassOff o = class_offsets(k, c.W, c.WX);
  std::vector<uint32_t>& blk = c.block;
  blk.assign(o.total, 0);
  auto chan = [&](uint32_t ch) { return ch < k ? B[ch] : Bp[ch - k]; };
  std::vector<uint32_t> r32(2 * k), r64(2 * k);
  for (uint32_t ch = 0; ch < 2 * k; ch++) {
    uint32_t m = chan(ch);
    r32[ch] = (uint32_t)((1ull << 32) % m);
    r64[ch] = mulmod32(r32[ch], r32[ch], m);
    blk[o.m + ch] = m;
    blk[o.mi + ch] = 0u - inv32(m);
    blk[o.r32 + ch] = r32[ch];
  }
  for (uint32_t j = 0; j < k; j++) {
    uint32_t m = Bp[j];
    blk[o.ahat + j] = mulmod32(c.Minv_Bp[j], r32[k + j], m);
    blk[o.ad + j] = mulmod32(c.Minv_Bp[j], c.Mp_mj_inv[j], m);
    blk[o.ubp + j] = (uint32_t)((1ull << (32 + KAW_Q)) / m);
    const uint32_t rinv = powmod32(r32[k + j], m - 2, m);  // 2^-32 mod m (m prime, Fermat)
    const uint32_t xpc = mulmod32(c.Mp_mj_inv[j], rinv, m);
    blk[o.xpc + j] = xpc;
    blk[o.xpcs + j] = (uint32_t)(((uint64_t)xpc << 32) / m);
    blk[o.ubs + j] = (uint32_t)((1ull << (KAW_Q + KAW_S)) / m);
  }
  for (uint32_t i = 0; i < k; i++) {
    uint32_t m = B[i];
    blk[o.mphh + i] = mulmod32(c.Mp_B[i], r64[i], m);
    blk[o.mmiinv + i] = c.M_mi_inv[i];
    blk[o.ub + i] = (uint32_t)((1ull << (32 + KAW_Q)) / m);
  }
  for (uint32_t i = 0; i < k; i++)
    for (uint32_t j = 0; j < k; j++)
      blk[o.T1 + (size_t)i * k + j] = mulmod32(c.M_mi_Bp[(size_t)i * k + j], r64[k + j], Bp[j]);
  for (uint32_t j = 0; j < k; j++)
    for (uint32_t i = 0; i < k; i++)
      blk[o.T2 + (size_t)j * k + i] = mulmod32(c.Mp_mj_B[(size_t)j * k + i], r64[i], B[i]);
  for (uint32_t ch = 0; ch < 2 * k; ch++) {
    uint32_t m = chan(ch);
    uint32_t v = r64[ch];  // 2^(32*0) * 2^64
    for (uint32_t w = 0; w < c.W; w++) {
      blk[o.P + (size_t)w * 2 * k + ch] = v;
      v = mulmod32(v, r32[ch], m);
    }
  }
  for (uint32_t i = 0; i < k; i++) {
    uint32_t rem = 0;
    Big q = divmod_small(c.M, B[i], &rem);
    std::vector<uint32_t> l = q.limbs(c.WX);
    for (uint32_t w = 0; w < c.WX; w++) blk[o.MD + (size_t)i * c.WX + w] = l[w];
  }
  {
    std::vector<uint32_t> l = c.M.limbs(c.WX);
    for (uint32_t w = 0; w < c.WX; w++) blk[o.ML + w] = l[w];
  }
  return true;
}

std::vector<uint32_t> residues(const ClassHost& c, const Big& X) {
  std::vector<uint32_t> r(2 * c.k);
  for (uint32_t i = 0; i < c.k; i++) r[i] = mod_small(X, c.B[i]);
  for (uint32_t j = 0; j < c.k; j++) r[c.k + j] = mod_small(X, c.Bp[j]);
  return r;
}

static void put_hat(const ClassHost& c, const Big& X, uint32_t* dst) {
  std::vector<uint32_t> r = residues(c, X);
  for (uint32_t ch = 0; ch < 2 * c.k; ch++) {
    uint32_t m = ch < c.k ? c.B[ch] : c.Bp[ch - c.k];
    uint32_t r32 = (uint32_t)((1ull << 32) % m);
    dst[ch] = mulmod32(r[ch], r32, m);
  }
}

int build_key(const ClassHost& c, const Big& N, const Big* exp, KeyHost& out, std::string& err) {
  if (N.bits() < 2 || !(N.limb(0) & 1u) || cmp(N, Big(3)) < 0) {
    err = "modulus must be odd and at least 3";
    return MR_ERR_EVEN_MODULUS;
  }
  if (N.bits() > c.L) {
    err = "modulus longer than its size class";
    return MR_ERR_SIZE;
  }
  const uint32_t k = c.k;
  std::vector<uint32_t> nres = residues(c, N);
  for (uint32_t ch = 0; ch < 2 * k; ch++)
    if (nres[ch] == 0) {
      err = "modulus is divisible by an RNS channel prime";
      return MR_ERR_NOT_COPRIME;
    }
  out.N = N;
  out.nbits = (uint32_t)N.bits();
  out.kxi.resize(k);
  out.NMinv_Bp.resize(k);
  for (uint32_t i = 0; i < k; i++) {
    uint32_t m = c.B[i];
    uint32_t ninv = invmod_prime(nres[i], m);
    out.kxi[i] = mulmod32(m - ninv, c.M_mi_inv[i], m);
  }
  for (uint32_t j = 0; j < k; j++) out.NMinv_Bp[j] = mulmod32(nres[k + j], c.Minv_Bp[j], c.Bp[j]);
  out.one = mod(c.M, N);
  out.r2 = mod(mul(out.one, out.one), N);
  out.r2h = mod(shl(out.r2, c.L), N);

  KeyOff o = key_offsets(k, c.W);
  out.block.assign(o.total, 0);
  uint32_t* b = out.block.data();
  b[o.hdr + 0] = out.nbits;
  b[o.hdr + 1] = (out.nbits + 31) / 32;
  b[o.hdr + 2] = exp ? (uint32_t)exp->bits() : 0u;
  for (uint32_t i = 0; i < k; i++) {
    const uint32_t m = c.B[i];
    b[o.kxi + i] = out.kxi[i];
    const uint32_t kxp = mulmod32(out.kxi[i], powmod32((uint32_t)((1ull << 32) % m), m - 2, m), m);
    b[o.kxp + i] = kxp;
    b[o.kxs + i] = (uint32_t)(((uint64_t)kxp << 32) / m);
  }
  for (uint32_t j = 0; j < k; j++) {
    uint32_t m = c.Bp[j];
    b[o.cmul + j] = mulmod32(out.NMinv_Bp[j], (uint32_t)((1ull << 32) % m), m);
    b[o.cd + j] = mulmod32(out.NMinv_Bp[j], c.Mp_mj_inv[j], m);
  }
  put_hat(c, out.one, b + o.one);
  put_hat(c, out.r2, b + o.r2);
  put_hat(c, out.r2h, b + o.r2h);
  std::vector<uint32_t> nl = N.limbs(c.W);
  for (uint32_t w = 0; w < c.W; w++) b[o.N + w] = nl[w];
  if (exp) {
    if (exp->bits() > 32ull * c.W) {
      err = "private exponent longer than its class";
      return MR_ERR_SIZE;
    }
    std::vector<uint32_t> el = exp->limbs(c.W);
    for (uint32_t w = 0; w < c.W; w++) b[o.exp + w] = el[w];
  }
  return MR_OK;
}

std::vector<uint32_t> build_crt(const ClassHost& c, const Big& p, const Big& q, const Big& qinv) {
  CrtOff o = crt_offsets(c.k, c.W);
  std::vector<uint32_t> blk(o.total, 0);
  Big qm = mod(mul(qinv, c.M), p);
  put_hat(c, qm, blk.data() + o.qm);
  Big twoL = shl(Big(1), c.L);
  Big t = mod(twoL, p);
  Big p2 = t.is_zero() ? twoL : add(twoL, sub(p, t));
  put_hat(c, p2, blk.data() + o.p2);
  std::vector<uint32_t> ql = q.limbs(c.W);
  for (uint32_t w = 0; w < c.W; w++) blk[o.q + w] = ql[w];
  return blk;
}

std::vector<uint32_t> build_crt_bin(uint32_t W, const Big& p, const Big& q, const Big& qinv) {
  CrtBinOff o = crt_bin_offsets(W);
  std::vector<uint32_t> blk(o.total, 0);
  Big twoW = shl(Big(1), 32 * (size_t)W);
  Big t = mod(twoW, p);
  Big p2 = t.is_zero() ? twoW : add(twoW, sub(p, t));
  std::vector<uint32_t> l = p2.limbs(W + 1);
  for (uint32_t w = 0; w <= W; w++) blk[o.p2 + w] = l[w];
  l = mod(shl(qinv, 32 * ((size_t)W + 1)), p).limbs(W);
  for (uint32_t w = 0; w < W; w++) blk[o.qr + w] = l[w];
  l = q.limbs(W);
  for (uint32_t w = 0; w < W; w++) blk[o.q + w] = l[w];
  const uint32_t p0 = p.limb(0);
  uint32_t inv = p0;  // Newton's iteration for p0^-1 mod 2^32: 3, 6, 12, 24, 48 correct bits
  for (int i = 0; i < 4; i++) inv *= 2u - p0 * inv;
  blk[o.pinv] = 0u - inv;
  return blk;
}

uint16_t half_bits(uint32_t v) {
  if (v == 0) return 0;
  uint32_t e = 0;
  while ((v >> (e + 1)) != 0) e++;  // v in [2^e, 2^(e+1))
  const uint32_t mant = (v << (10 - e)) & 0x3FFu;
  return (uint16_t)(((e + 15u) << 10) | mant);
}

bool tc_slice_table(const uint32_t* T1, const uint32_t* T2, uint32_t k, uint32_t sc, uint32_t slices,
                    std::vector<uint32_t>& out) {
  if (sc != 32) return false;
  const uint32_t KC = 64, nch = (k + KC - 1) / KC, chunk_bytes = 128u * KC * 2u;
  std::vector<uint16_t> h((size_t)slices * 2 * nch * chunk_bytes / 2, 0);
  for (uint32_t c = 0; c < slices; c++)
    for (uint32_t e = 0; e < 2; e++) {
      const uint32_t* T = e ? T2 : T1;
      for (uint32_t i = 0; i < k; i++)
        for (uint32_t j = 0; j < sc && c * sc + j < k; j++) {
          const uint32_t t = T[(size_t)i * k + c * sc + j];
          if (t >> 28) return false;
          for (uint32_t b = 0; b < 4; b++) {
            const size_t byte = (((size_t)c * 2 + e) * nch + i / KC) * chunk_bytes + tc_tile_off(128, 32 * b + j, i % KC);
            h[byte / 2] = half_bits((t >> (7 * b)) & 127u);
          }
        }
    }
  out.assign(h.size() / 2, 0);
  for (size_t w = 0; w < out.size(); w++) out[w] = (uint32_t)h[2 * w] | ((uint32_t)h[2 * w + 1] << 16);
  return true;
}

}  // namespace mr
