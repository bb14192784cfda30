"""GB300 Combined Sieve (arXiv:2012.03771): CUDA kernels for sm_103a behind a
small C ABI (include/combsieve.h), with a thin ctypes binding.

Importing the package does not load the CUDA library; the first call does,
and fails loudly if libcombsieve.so has not been built.
"""
from ._binding import (  # noqa: F401
    CS_EAGAIN, CS_EDEVICE, CS_EINVAL, CS_ENOMEM, CS_EOVERFLOW, CS_ESIZE, CS_ESTATE, CS_ETIMEOUT, CS_OK,
    Batch, Cache, CSError, EXPORTS, LIB_PATH, Plan, Server, cs_atomic_rate, cs_autotune, cs_columns, cs_counts, cs_destroy, cs_device_bitset,
    cs_fetch_bitset, cs_fetch_rows, cs_info, cs_issue_rate, cs_k_mod_p, cs_kernel_times, cs_last_error, cs_modsolve, cs_plan,
    cs_plan_status, cs_primes, cs_primes_static, cs_rows, cs_sieve, cs_stats, cs_sync, load, make_tuning,
)
