"""GB300 (sm_103a) implementation of U = sign(T) for dense real upper
triangular T: recursive Parlett-Higham and Parlett-Sylvester (Stotland,
Schwartz, Toledo).  The computation lives in the CUDA library
_lib/libsigntri.so behind the C ABI of include/signtri.h; `signtri` is its
ctypes binding.
"""
from .signtri import (Info, SignTriError, Status, Variant, load, sign, sign_tri, sign_tri_host,  # noqa: F401
                      signtri_get_info, signtri_inertia, signtri_set_cutoff, signtri_set_workspace,
                      signtri_status_string, signtri_workspace_bytes, to_device, to_numpy,
                      signtri_profile_enable, signtri_profile_reset, signtri_profile_read,
                      signtri_kernel_class_name, signtri_probe_fp64_peak, sign_tri_noalloc,
                      signtri_reorder_by_sign, signtri_sylvester, signtri_set_rates,
                      signtri_gemm_emulated, signtri_set_refinement, signtri_set_verification,
                      signtri_profile_read_flops, signtri_profile_read_bytes, sign_tri_batched, signtri_set_cutoff_table,
                      signtri_get_cutoff_table, signtri_autotune, signtri_selftest_wait,
                      signtri_get_variant_table, signtri_set_variant_table, signtri_batched_cache_stats,
                      signtri_sign_schur, signtri_sign_schur_workspace_bytes, sign_schur,
                      signtri_sign_tri_complex, signtri_sign_schur_complex, signtri_complex_workspace_bytes,
                      sign_complex, sign_schur_complex, to_device_complex,
                      Phi, signtri_funm, funm, signtri_schur, signtri_schur_workspace_bytes, schur,
                      signtri_sign_general, signtri_sign_general_workspace_bytes, sign_general)
