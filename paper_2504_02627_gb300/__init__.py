"""GB300-native (sm_103a) hot path of SMC with a ChEES-HMC proposal
(arXiv 2504.02627): the C-ABI library libsmcchees (include/smc.h) and its
ctypes binding.  Importing this package does not touch the GPU."""
from ._binding import (  # noqa: F401
    BANANA, GAUSS_DENSE, HIER_NORMAL, LINEAR_GAUSS, LOGISTIC, PREC_BF16, PREC_BF16X2, PREC_BF16X3, PREC_FP32,
    DevModel, ModelData, Sampler, check, lib, lib_path, make_config)
