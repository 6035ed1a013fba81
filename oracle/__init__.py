"""Plain CPU oracle for the non-RNS CKKS/BGV hot path (test infrastructure).

This package is test infrastructure, not part of the product.  Only the
test-suite, the smoke check and the bench's CPU-baseline leg may import it.
It shares no code with the CUDA library: it receives the same seeded inputs
(from ``fhe_synth``) and computes, slowly and in the most literal form, what
the GPU path must produce bit for bit.

Modules
  bigint   limb <-> Python int conversion (the oracle's own, Sec. 4 radix form)
  ring     negacyclic products: schoolbook (Eq. schoolbook + Eq. reduction),
           Kronecker substitution, and an exact C fast path (fastmul.c)
  ntt      the negacyclic NTT/INTT as the direct sums of Eq. negacyclic_ntt
           and Eq. negacyclic_intt, NTT-friendly primes and roots
  crt      RNS decomposition, CRT composition (Eq. crt_composition), Garner's
           mixed-radix conversion (Eq. garner_mrc), centred reduction (Sec. 5)
  encode   CKKS canonical-embedding encode/decode (Eq. negacyclic_fft/ifft)
  ckks     non-RNS CKKS key generation, encryption, decryption, tensor
           product, relinearisation, rescale, rotation (Sec. 6 operations)
  bgv      non-RNS BGV with an odd modulus chain and plaintext modulus t

Every function cites the passage it follows.  Parity status of each function
is recorded in its docstring; functions with no independent pin say
"parity unpinned".
"""
