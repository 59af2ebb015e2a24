"""GB300 two-site TDVP (2TDVP) for vibronic quantum dynamics.

The compute lives in libvibtdvp.so (C ABI in include/vibtdvp.h, CUDA kernels
for sm_103a in csrc/); this package is its ctypes binding. Build with
`paper_1908_10588_gb300.build.build()`.
"""
from .binding import (  # noqa: F401
    EXPORTED, VB_FP64, VB_MIXED, Mpo, Mps, VbError, lib, vb_eig_work_bytes, vb_env_left_update,
    vb_env_right_update, vb_env_work_elems, vb_heff1_apply, vb_heff2_apply, vb_heff_work_elems,
    vb_autotune, vb_herm_eig_top, vb_herm_eig_top_noalloc, vb_kernel_launches, vb_spectrum, vb_profile_enable, vb_profile_read,
    site_order_cost, site_order_rule, site_order_search, sweep_batched,
)
