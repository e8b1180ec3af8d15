"""CPU oracle for the encrypted semi-parallel GWAS hot path.

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
benchmark's CPU-baseline leg, never by the product package.

  ckks        -- O1: textbook RNS-CKKS (C core in ckks_oracle.c + evaluator)
  circuit     -- the GWAS circuit (Algorithms 1-11) over the O1 evaluator
  gwas_fp64   -- O2: plaintext FP64 of the paper's approximated GWAS
  gwas_exact  -- O3: exact references (semi-parallel with W, per-SNP Newton)
"""
