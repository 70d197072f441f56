"""GB300-native (sm_103a) hot path of SMC with a ChEES-HMC proposal
(arXiv 2504.02627): the C-ABI library libsmcchees (include/smc.h) and its
ctypes binding.  Importing this package does not touch the GPU."""
from ._binding import (  # noqa: F401
    BANANA, GAUSS_DENSE, HIER_NORMAL, LINEAR_GAUSS, LOGISTIC, PREC_BF16, PREC_BF16C, PREC_BF16X2, PREC_BF16X3,
    PREC_FP32, JITTER_HALTON1_ITER,
    JITTER_EQUIDISTANT, JITTER_EQUIDISTANT_OFFSET, JITTER_GOLDEN, JITTER_HALTON1, JITTER_HALTON_ND,
    JITTER_HALTON_ND_INV, JITTER_NONE, JITTER_PRIMES, JITTER_PRIMES_INV, JITTER_SOBOL1, JITTER_UNIFORM,
    DevModel, ModelData, Sampler, check, lib, lib_path, make_config)
