"""Oracle: a plain, slow, arbitrary-precision CPU restatement of the zkVC prover path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library, its Python
binding) may import, call or link anything in this package.  Only the tests, the
``smoke()`` check of ``__graft_entry__`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` use it.

It shares no code with the CUDA path: every field, curve, NTT, R1CS and Groth16 step
here is written out with Python integers in the order the paper and the textbook
definitions give, so that a reader can check it by eye.

Modules
-------
``bn254``    BN254 parameters, Fp/Fr/Fp2/Fp12 arithmetic, G1/G2 groups, naive MSM,
             canonical serialisation.
``pairing``  optimal-ate pairing (Miller loop on the untwisted curve over Fp12) and
             plain final exponentiation.
``ntt``      textbook radix-2 NTT, O(N^2) DFT, coset variants over Fr.
``crpc``     the CRPC + PSQ rank-1 constraint system of the matmul Y = X W
             (zkVC Sec. III-A, general CRPC equation; Sec. III-B, PSQ prefix sums).
``groth16``  QAP evaluation, Groth16 setup / prove / verify, and the closed-form
             ("trapdoor") proof used to check full-size proofs.

Every function cites the passage it follows.  Parity status per function is in the
header of each module; nothing here is "parity unpinned".
"""
