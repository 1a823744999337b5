// Word layout of the device-resident tables (uint32 words), shared by the
// host setup that writes them and the kernels that read them.
//
// Channel numbering: c in [0, k) are the primes of base B, c in [k, 2k) the
// primes of B'.  "hat" form of a residue v mod m is v * 2^32 mod m (the
// per-channel Montgomery form used by the kernels' word reductions); "plain"
// is v itself.
#pragma once
#include <cstdint>

#ifdef __CUDACC__
#define MR_HD __host__ __device__
#else
#define MR_HD
#endif

namespace mr {

constexpr int KAW_Q = 22;  // fixed-point bits of the B'->B correction estimate
constexpr int KAW_S = 17;  // the lane-group kernels weight xi' >> KAW_S (one 32-bit product per channel)

// ---------------------------------------------------------------- size class
// [m 2k][mi 2k][r32 2k][ahat k][ad k][ubp k][mphh k][mmiinv k][ub k][xpc k][xpcs k][ubs k]
// [T1 k*k][T2 k*k][P W*2k][MD k*WX][ML WX]
//   m      channel prime
//   mi     -m^-1 mod 2^32
//   r32    2^32 mod m  (= the hat form of 1)
//   ahat   (B') |M^-1|_{m'_j} hat
//   ad     (B') |M^-1 (M'/m'_j)^-1|_{m'_j} plain   (xi'_j = REDC(hat(s_j) ad + hat(qhat_j) cd))
//   ubp    (B') floor(2^(32+Q) / m'_j)            fixed-point factor weights
//   mphh   (B)  |M'|_{m_i} * 2^64 mod m_i          (REDC(a * mphh) = hat(a M'))
//   mmiinv (B)  |(M/m_i)^-1|_{m_i} plain           (RNS -> binary)
//   ub     (B)  floor(2^(32+Q) / m_i)
//   xpc    (B') |(M'/m'_j)^-1|_{m'_j} * 2^-32 mod m'_j  (xi'_j from the hat residue r_j by Shoup's product)
//   xpcs   (B') floor(xpc * 2^32 / m'_j)           (its quotient factor)
//   ubs    (B') floor(2^(Q+17) / m'_j)             (factor weights from the top bits: (xi' >> 17) ubs)
//   T1     row i (B), column j (B'): |M/m_i|_{m'_j} * 2^64 mod m'_j
//   T2     row j (B'), column i (B): |M'/m'_j|_{m_i} * 2^64 mod m_i
//   P      row w (limb), column c: 2^(32 w) * 2^64 mod m_c   (binary -> hat residues)
//   MD     row i: the WX limbs of M/m_i
//   ML     the WX limbs of M
struct ClassOff {
  uint32_t m, mi, r32, ahat, ad, ubp, mphh, mmiinv, ub, xpc, xpcs, ubs, T1, T2, P, MD, ML, total;
};

// Tensor-core operand layout in shared memory (K-major, no swizzling; tc_device.cuh): byte offset
// of element (r, k) of an R-row tile of fp16 values.  The unit is the core matrix of 8 rows x 16
// bytes (8 values of k), stored row after row; core matrix (r / 8, k / 8) sits at
// (k / 8) * (R / 8) * 128 + (r / 8) * 128.  The large classes' tensor-core slice table is built on the
// host in this layout.
MR_HD constexpr inline uint32_t tc_tile_off(uint32_t R, uint32_t r, uint32_t k) {
  return (k >> 3) * (R >> 3) * 128u + (r >> 3) * 128u + (r & 7u) * 16u + (k & 7u) * 2u;
}

MR_HD constexpr inline ClassOff class_offsets(uint32_t k, uint32_t W, uint32_t WX) {
  ClassOff o{};
  o.m = 0;
  o.mi = 2 * k;
  o.r32 = 4 * k;
  o.ahat = 6 * k;
  o.ad = 7 * k;
  o.ubp = 8 * k;
  o.mphh = 9 * k;
  o.mmiinv = 10 * k;
  o.ub = 11 * k;
  o.xpc = 12 * k;
  o.xpcs = 13 * k;
  o.ubs = 14 * k;
  o.T1 = 15 * k;
  o.T2 = o.T1 + k * k;
  o.P = o.T2 + k * k;
  o.MD = o.P + W * 2 * k;
  o.ML = o.MD + k * WX;
  o.total = o.ML + WX;
  return o;
}

// ------------------------------------------------------------------ modulus
// [hdr 4][kxi k][cmul k][cd k][kxp k][kxs k][one 2k][r2 2k][r2h 2k][N W][exp W]
//   hdr    nbits(N), nlimbs(N), exp_bits (private exponent bit length or 0), 0
//   kxi    (B)  |-N^-1 (M/m_i)^-1|_{m_i} plain
//   cmul   (B') |N M^-1|_{m'_j} hat
//   cd     (B') |N M^-1 (M'/m'_j)^-1|_{m'_j} plain
//   kxp    (B)  kxi * 2^-32 mod m_i          (xi_i from hat(s_i) by Shoup's product)
//   kxs    (B)  floor(kxp * 2^32 / m_i)      (its quotient factor)
//   one    hat residues of M mod N           (1 in the Montgomery domain)
//   r2     hat residues of M^2 mod N         (entry into the domain)
//   r2h    hat residues of 2^L M^2 mod N     (entry of the high chunk of a 2L-bit input)
//   N      W limbs of the modulus
//   exp    W limbs: private CRT exponent (dp or dq) of an RSA half, zero otherwise
struct KeyOff {
  uint32_t hdr, kxi, cmul, cd, kxp, kxs, one, r2, r2h, N, exp, total;
};

MR_HD constexpr inline KeyOff key_offsets(uint32_t k, uint32_t W) {
  KeyOff o{};
  o.hdr = 0;
  o.kxi = 4;
  o.cmul = o.kxi + k;
  o.cd = o.cmul + k;
  o.kxp = o.cd + k;
  o.kxs = o.kxp + k;
  o.one = o.kxs + k;
  o.r2 = o.one + 2 * k;
  o.r2h = o.r2 + 2 * k;
  o.N = o.r2h + 2 * k;
  o.exp = o.N + W;
  o.total = o.exp + W;
  return o;
}

// ----------------------------------------------------------- RSA CRT parts
// [qm 2k][p2 2k][q W]   (in the size class of p and q)
//   qm     hat residues of qinv * M mod p   (MM(d, qm) = d * qinv mod p)
//   p2     hat residues of p * ceil(2^L / p)  (a multiple of p above every m_q)
//   q      W limbs of q
struct CrtOff {
  uint32_t qm, p2, q, total;
};

MR_HD constexpr inline CrtOff crt_offsets(uint32_t k, uint32_t W) {
  CrtOff o{};
  o.qm = 0;
  o.p2 = 2 * k;
  o.q = 4 * k;
  o.total = o.q + W;
  return o;
}

// [p2 W+1][qr W][q W][pinv 1]   (binary, large size classes; W limbs of the class of p and q)
//   p2     p * ceil(2^(32W) / p): a multiple of p above every m_q, W+1 limbs
//   qr     qinv * 2^(32(W+1)) mod p   (Montgomery factor of the W+1-limb radix)
//   q      W limbs of q
//   pinv   -p^-1 mod 2^32
struct CrtBinOff {
  uint32_t p2, qr, q, pinv, total;
};

MR_HD constexpr inline CrtBinOff crt_bin_offsets(uint32_t W) {
  CrtBinOff o{};
  o.p2 = 0;
  o.qr = W + 1;
  o.q = 2 * W + 1;
  o.pinv = 3 * W + 1;
  o.total = 3 * W + 2;
  return o;
}

// ------------------------------------------------------------ work items
struct MxItem {            // one modular exponentiation
  const uint32_t* key;     // modulus block (KeyOff layout)
  const uint32_t* x;       // base, x_limbs limbs (at most 2W)
  const uint32_t* e;       // exponent, e_limbs limbs (may point into the key block)
  uint32_t* out;           // result row, out_limbs limbs
  const uint32_t* xlim;    // x must be below this number (xlim_limbs limbs)
  uint32_t x_limbs, e_limbs, out_limbs, xlim_limbs;
  uint32_t status;         // index into the status array, or 0xffffffff
  uint32_t pad_;           // host-side bookkeeping only (ignored by the kernels)
};

struct CrtItem {           // Garner recombination of one CRT decryption
  const uint32_t* keyp;    // modulus block of p
  const uint32_t* crt;     // CrtOff block (CrtBinOff for the large classes)
  const uint32_t* mp;      // W limbs, c^dp mod p
  const uint32_t* mq;      // W limbs, c^dq mod q
  uint32_t* out;           // out_limbs limbs
  uint32_t out_limbs;
  uint32_t status;
};

}  // namespace mr
