"""GB300 (sm_103a) multilevel size-constrained label propagation partitioner.

The compute path is libsclap.so (hand-written CUDA behind the C ABI in
include/sclap.h); `sclap` is its ctypes binding.
"""
from .sclap import (  # noqa: F401
    CUT_STATIC_MAX_K, PENDING, ECSR, ECUDA, EINFEASIBLE, EINTERNAL, EINVAL, ENOMEM, EOVERFLOW, ETIMEOUT, OK,
    Config, Result, SclapError, Server, Served, Tuning, autotune, check_build, check_selftest, debug_inject,
    default_config, get_tuning, load,
    set_tuning, sclap_cluster,
    sclap_cluster_hierarchy, sclap_contract, sclap_cut,
    sclap_cut_static,
    sclap_initial_partition, sclap_lp_round, sclap_partition, sclap_partition_batch,
    sclap_partition_device, sclap_profile_dump, sclap_profile_enable, sclap_profile_phases, sclap_profile_read,
    sclap_profile_reset, sclap_profile_timeline,
    sclap_refine,
)
