"""All-pairs mutual information of binary variables on GB300 (sm_103a).

The computation lives in libgbmi.so (CUDA C++ with inline PTX for tcgen05,
TMA and mbarriers; C ABI in include/gbmi.h).  This package is its ctypes
binding (``gbmi``) and its build script (``build``).
"""
from .gbmi import (GbmiError, column_counts, counts_all_pairs, counts_cross, launch_count,
                   mi_all_pairs, mi_all_pairs_host, mi_cross, mi_cross_host, mi_from_counts,
                   set_option, shutdown, sync, validate_binary, version)

__all__ = ["GbmiError", "column_counts", "counts_all_pairs", "counts_cross", "launch_count",
           "mi_all_pairs", "mi_all_pairs_host", "mi_cross", "mi_cross_host", "mi_from_counts",
           "set_option", "shutdown", "sync", "validate_binary", "version"]
