"""CPU oracle for the RNS modular-exponentiation path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its CPU-baseline
leg and its reference arm) may import anything in this package.  The product
library (``paper_1305_3699_gb300``) never imports it, and this package never
imports the product: the two share no code, tables or constants.  The only
common dependency is ``synth`` (seeded random draws and limb packing).

Contents, each function citing the passage of "Secrets from the GPU"
(Chauvet & Mahe) it follows:

* ``plain``      -- the plain definitions the GPU path must reproduce exactly:
                    x^e mod N by the oracle's own left-to-right square-and-multiply
                    (Sec. 3.1), RSA encryption / decryption (Sec. 3.3), the CRT
                    (Garner) decryption, modular inverse and Arazi's inversion
                    formula (Sec. 3.1), message blocks (Sec. 3.3).
* ``primality``  -- trial division by the first 10,000 primes (Sec. 4.3), the
                    Miller-Rabin test with caller-chosen witnesses (Sec. 3.2) and the
                    two composed (prime_test_verdict).
* ``keygen``     -- seeded RSA key generation for the synthetic workloads, and keys
                    from given candidate pools (rsa_key_from_pools) (Sec. 3.3).
* ``rns``        -- a slow, step-by-step model of the RNS Montgomery
                    multiplication with base extension (Sec. 3.1), used to pin the
                    base choice, the precomputed constants and intermediate residues.

Parity status: every function here is pinned by tests in ``tests/test_oracle_*.py``
against facts independent of the function itself (library routines, closed
forms, invariants, brute force on tiny inputs, known primes and pseudoprimes).
The paper prints no worked example or test vector, so no pin is a value the paper
prints.
"""
