/* Plain-C client of the library's C ABI (host-only calls, no device): compiles against
 * include/mr.h with a C compiler and links libmrmod.so.  Prints one line per check; exit status 0
 * when every check holds. */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "mr.h"

static int failures = 0;

static void check(int ok, const char *what) {
  printf("%s %s\n", ok ? "ok" : "FAIL", what);
  if (!ok) failures++;
}

int main(void) {
  uint32_t L = 0, k = 0;
  check(mr_class_for_bits(2048, &L, &k) == MR_OK && L == 2048 && k == 72, "class of 2048-bit moduli: k = 72");
  check(mr_class_for_bits(2049, &L, &k) == MR_OK && L == 3072, "2049 bits fall in the 3072-bit class");
  check(mr_class_for_bits(16385, &L, &k) == MR_ERR_SIZE, "16385 bits: MR_ERR_SIZE");

  /* N = 2^61 - 1 (odd, coprime to every channel prime of the 512-bit class) */
  const uint32_t N[2] = {0xffffffffu, 0x1fffffffu};
  size_t count = 0;
  check(mr_debug_key_table_host(N, 2, "kxi", NULL, 0, &count) == MR_OK && count == 18,
        "key table size query: k words for k = 18");
  uint32_t *kxi = (uint32_t *)malloc(count * sizeof(uint32_t));
  check(mr_debug_key_table_host(N, 2, "kxi", kxi, count, &count) == MR_OK, "key table copy");
  free(kxi);
  const uint32_t even[1] = {100u};
  check(mr_debug_key_table_host(even, 1, "kxi", NULL, 0, &count) == MR_ERR_EVEN_MODULUS, "even modulus refused");

  check(mr_debug_trial_table(NULL, 0, &count) == MR_OK && count == 131u * 10016u, "trial table size");
  uint32_t *tab = (uint32_t *)malloc(count * sizeof(uint32_t));
  check(mr_debug_trial_table(tab, count, &count) == MR_OK, "trial table copy");
  const uint32_t *P = tab + 128u * 10016u;
  check(P[0] == 2u && P[1] == 3u && P[9999] == 104729u, "primes 2, 3, ..., 104729");
  /* row 1, column j: 2^32 mod p_j */
  check(tab[10016u + 1] == (uint32_t)((1ull << 32) % 3u) && tab[10016u + 9999] == (uint32_t)((1ull << 32) % 104729u),
        "2^32 mod p in row 1");
  free(tab);

  /* binary Garner block for p = 2^61 - 1, q = 2^31 - 1, qinv = q^-1 mod p, W = 2 */
  const uint32_t p[2] = {0xffffffffu, 0x1fffffffu}, q[2] = {0x7fffffffu, 0u};
  /* q^-1 mod p: (2^31 - 1)^-1 mod (2^61 - 1) computed below by extended Euclid in 128-bit-free steps */
  unsigned long long pp = 0x1fffffffffffffffull, qq = 0x7fffffffull;
  long long r0 = (long long)pp, r1 = (long long)qq, s0 = 0, s1 = 1;
  while (r1) {
    long long t = r0 / r1, u = r0 - t * r1;
    r0 = r1;
    r1 = u;
    u = s0 - t * s1;
    s0 = s1;
    s1 = u;
  }
  unsigned long long qinv = (unsigned long long)((s0 % (long long)pp + (long long)pp) % (long long)pp);
  const uint32_t qi[2] = {(uint32_t)qinv, (uint32_t)(qinv >> 32)};
  uint32_t blk[8];
  check(mr_debug_crt_bin_host(p, q, qi, 2, 2, blk, 8, &count) == MR_OK && count == 8, "Garner block: 3W + 2 words");
  check((uint32_t)(blk[7] * p[0]) == 0xffffffffu, "pinv * p = -1 mod 2^32");
  check(blk[5] == q[0] && blk[6] == q[1], "q limbs");

  uint32_t nvar = 0, lanes[8];
  check(mr_class_variants(1024, &nvar, lanes, 8) == MR_OK && nvar >= 1 && lanes[0] == 4,
        "1024-bit class: variant 0 has 4 lanes per number");
  check(mr_class_variants(8192, &nvar, lanes, 8) == MR_OK && nvar == 3 && lanes[0] == 80 && lanes[1] == 84 &&
            lanes[2] == 80,
        "8192-bit class: slice widths of 10 x 8 and 7 x 12 lanes per number, tensor-core form 10 x 8");
  uint32_t v = 9, slots = 0;
  check(mr_debug_big_variant(8192, 512, 152, 1, &v, &slots) == MR_OK && v == 2 && slots == 15,
        "16 groups of the 8192-bit class take the tensor-core form in two waves of 15");
  check(mr_debug_table(NULL, 512, NULL, "B", NULL, 0, &count) == MR_OK && count == 18, "class table B: k primes");

  check(mr_init(0, NULL) == MR_ERR_ARG, "mr_init without an output pointer: MR_ERR_ARG");
  printf("%d failures\n", failures);
  return failures ? 1 : 0;
}
