// Host setup of size classes and moduli (Sec. 3.1 of the paper: the constants
// of base extension and Montgomery multiplication are fixed once the bases are
// chosen, so they are computed once and kept resident on the GPU).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "host_bigint.h"
#include "layout.h"

namespace mr {

// Supported size classes (bits of the largest modulus each holds).
const std::vector<uint32_t>& class_bits_list();

// Smallest supported class holding a modulus of `bits` bits (0 when none).
uint32_t class_for_bits(uint32_t bits);

struct ClassHost {
  uint32_t L = 0, k = 0, W = 0, WX = 0;
  uint64_t bound = 0;                 // every channel prime is below this
  std::vector<uint32_t> B, Bp;        // bases, descending
  Big M, Mp;
  // plain tables, named as in the CPU model of the method
  std::vector<uint32_t> M_mi_inv;     // k       |(M/m_i)^-1|_{m_i}
  std::vector<uint32_t> M_mi_Bp;      // k*k     row i, col j: |M/m_i|_{m'_j}
  std::vector<uint32_t> Minv_Bp;      // k       |M^-1|_{m'_j}
  std::vector<uint32_t> Mp_mj_inv;    // k       |(M'/m'_j)^-1|_{m'_j}
  std::vector<uint32_t> Mp_mj_B;      // k*k     row j, col i: |M'/m'_j|_{m_i}
  std::vector<uint32_t> Mp_B;         // k       |M'|_{m_i}
  std::vector<uint32_t> block;        // device form (ClassOff layout)
};

// Build the bases and tables of class L.  Returns false with a message on failure.
bool build_class(uint32_t L, ClassHost& out, std::string& err);

struct KeyHost {
  Big N;
  uint32_t nbits = 0;
  std::vector<uint32_t> kxi, NMinv_Bp;  // plain
  Big one, r2, r2h;                     // M mod N, M^2 mod N, 2^L M^2 mod N
  std::vector<uint32_t> block;          // device form (KeyOff layout)
};

// Per-modulus constants of N in class c; `exp` (nullable) is stored in the
// block's exponent slot.  Returns an mr_status code (0 = ok).
int build_key(const ClassHost& c, const Big& N, const Big* exp, KeyHost& out, std::string& err);

// Garner-recombination block for RSA halves p, q of class c (CrtOff layout).
std::vector<uint32_t> build_crt(const ClassHost& c, const Big& p, const Big& q, const Big& qinv);

// Binary Garner block for halves p, q of a large size class of W limbs (CrtBinOff layout).
// p must be odd.
std::vector<uint32_t> build_crt_bin(uint32_t W, const Big& p, const Big& q, const Big& qinv);

// Operands B of the tensor-core base extensions of a large class (big_kernel.cuh, BigTcCfg): for
// each channel slice of sc = 32 columns and each extension matrix T (T1, then T2; k x k, row i =
// input channel, column j = output channel, entries below 2^28), the four 7-bit slices of the
// slice's columns as fp16 values, row 32 b + j of slice b, in chunks of 64 values of i in the
// tensor-core tile layout (tc_tile_off, 128 rows), zero past channel k.  Layout
// [slice][extension][chunk]; `out` receives the bytes as 32-bit words.  False when an entry needs
// more than 28 bits.
bool tc_slice_table(const uint32_t* T1, const uint32_t* T2, uint32_t k, uint32_t sc, uint32_t slices,
                    std::vector<uint32_t>& out);

// fp16 bit pattern of an integer 0 <= v < 2048 (exact).
uint16_t half_bits(uint32_t v);

// Residues of X in all 2k channels (plain).
std::vector<uint32_t> residues(const ClassHost& c, const Big& X);

}  // namespace mr
