"""GB300-native CKKS-RNS engine for the encrypted semi-parallel GWAS of
"Achieving GWAS with Homomorphic Encryption" (arXiv 1902.04303).

  gwhe     -- ctypes binding of the C ABI (include/gwhe.h); the CUDA library
              libgwhe.so is built in-tree by build.build()
  datagen  -- seeded synthetic inputs of the paper's workload shape
  sharding -- SNP-batch partition across ranks and the result gather
"""
