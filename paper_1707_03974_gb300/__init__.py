"""GB300-native matrix-free Hubbard H·v and Lanczos with Paradeisos basis ranking (arXiv 1707.03974).

The compute path is libparadeisos.so (hand-written sm_103a CUDA kernels behind
the C ABI of include/paradeisos.h); this package is its thin ctypes binding.
Importing the package does not load the library; the first call does, and fails
loudly if the library has not been built.
"""
from ._binding import (HB_F32, HB_F64, HB_FX64, Batch, Handle, Inversion, Mlp, mlp_adam_step, mlp_forward, mlp_gradient,
                       mlp_last_error, mlp_start_vector, mlp_tc_gemm, mlp_activation, mlp_sample_training, hb_device_wait_selftest, hubbard_autotune, hubbard_batch_apply,
                       hubbard_batch_autotune, hubbard_batch_get_config, hubbard_batch_set_config, lanczos_batch_ground_state, lanczos_batch_wait_selftest, hubbard_convert,
                       hubbard_fixed_point_bits, hubbard_get_hv_config, hubbard_set_hv_config, HubbardError, LanczosResult, hb_tridiag_lowest,  # noqa: F401
                       hubbard_apply, hubbard_basis_create, hubbard_basis_destroy, hubbard_last_error,
                       hubbard_row_entries, hubbard_set_U, lanczos_ground_state, lanczos_ritz_vector_f32, lanczos_step,
                       lanczos_step_noalloc, lanczos_step_scratch_bytes, load, paradeisos_rank, paradeisos_unrank,
                       lanczos_ritz_vector_f64, hubbard_apply_c, hb_continued_fraction, hb_measure_ceilings,
                       hubbard_apply_timed, host_empty)

EXPORTED_SYMBOLS = ("hb_status_string", "hubbard_basis_create", "hubbard_basis_create_k", "hubbard_basis_destroy",
                    "hubbard_basis_dim",
                    "hubbard_set_U", "paradeisos_rank", "paradeisos_unrank", "hubbard_apply", "hubbard_row_entries",
                    "hubbard_last_error", "lanczos_workspace_bytes", "lanczos_ground_state", "hb_tridiag_lowest",
                    "lanczos_step_scratch_bytes", "lanczos_step", "lanczos_step_noalloc",
                    "hubbard_fixed_point_bits", "hubbard_convert", "hubbard_get_hv_config",
                    "hubbard_set_hv_config", "hubbard_autotune", "lanczos_ritz_vector_f32", "hubbard_batch_create", "hubbard_batch_destroy",
                    "hubbard_batch_layout", "hubbard_batch_apply", "hubbard_batch_autotune", "hubbard_batch_get_config",
                    "hubbard_batch_set_config",
                    "lanczos_batch_workspace_bytes", "lanczos_batch_ground_state", "lanczos_batch_wait_selftest", "paradeisos_inv_create",
                    "paradeisos_inv_destroy", "paradeisos_inv_dim", "paradeisos_inv_rank", "paradeisos_inv_unrank",
                    "paradeisos_inv_last_error", "lanczos_ritz_vector_f64", "hubbard_apply_c",
                    "hb_continued_fraction", "hb_measure_ceilings", "hubbard_apply_timed", "hb_host_alloc",
                    "hb_host_free")
MLP_SYMBOLS = ("mlp_create", "mlp_destroy", "mlp_param_count", "mlp_get_params", "mlp_set_params", "mlp_forward",
               "mlp_gradient", "mlp_adam_step", "mlp_start_vector", "mlp_last_error", "mlp_tc_gemm", "mlp_activation", "mlp_sample_workspace_bytes", "mlp_sample_training",
               "hb_device_wait_selftest")
