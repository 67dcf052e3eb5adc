"""GB300 (sm_103a) implementation of RAMBO's batched multiple-set-membership
query (arXiv 1910.02611): librambo.so (C ABI in include/rambo.h, CUDA kernels
in csrc/) and its Python binding."""
from .rambo import (  # noqa: F401
    E2BIG, EBADSEQ, ECUDA, EINVAL, EIO, ENOMEM, ENOSPC, ERANGE, ESTATE, ETIMEOUT, OK, Plan, QueryConfig, Rambo, RamboError, Server,
    RamboInfo, SIGNATURES, l2_fetch_granularity, suggest_params, suggest_params_from_sample, library_path, load_library, random_row_probe,
)
