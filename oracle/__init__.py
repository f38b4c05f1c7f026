"""CPU oracle for bit-polynomial multiplication in GF(2)[x].

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call,
link or execute anything in this package.  Only the test-suite, the smoke
check (``__graft_entry__.smoke``) and the ``cpu_baseline`` / reference leg of
``bench.py`` use it.  It shares no code with the CUDA library: it has its own
field arithmetic, its own Cantor basis, its own transforms.

Modules
-------
``field``     GF(2^64) = GF(2)[x]/(x^64+x^4+x^3+x+1) (Sec. 4.3), the Cantor
              basis (Eq. 2, Sec. 2.2.1) and subspace polynomials s_i (Sec. 2.2.2).
``stages``    The steps of FP_Polymul (Alg. 5): BasisCvt / iBasisCvt (Alg. 1),
              Encode / Decode (Alg. 4), Butterfly / iButterfly (Alg. 2), the
              pointwise product, plus the definitions used to pin them
              (evaluation at the Frobenius partition, Eq. 7).
``m128``      The same method with m = 128 (Sec. 3 for general m, Sec. 4.3):
              GF(2^128) = GF(2)[x]/(x^128+x^7+x^2+x+1), its Cantor basis,
              Sigma = v_{l+64} + V_l, the 128-row Encode, Butterfly and Alg. 5.
``clmul``     The plain carry-less product (the definition the whole method
              must reproduce, Sec. 2.1) and the randomised modular checker,
              backed by the portable C code in ``oracle.c``.
"""
