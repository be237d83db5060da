"""GB300 lattice Boltzmann library: the second-order force scheme of Li, Duan &
Shan (arXiv:2212.07494) as fused sm_103a CUDA kernels behind a C ABI.

This package is a thin ctypes binding of ``include/lbm.h``: the functions
``lbm_create`` ... ``lbm_destroy`` marshal arguments to the C entry points of
the same names, and ``Lattice`` wraps a handle.  Every step of the update runs
in the CUDA library; there is no CPU fallback.  If the library has not been
built, importing the binding raises ``ImportError``; build it with
``python -m paper_2212_07494_gb300.build``.

PyTorch is optional and only supplies device memory (its caching allocator)
and streams when a caller passes ``torch_stream=...``.
"""
from ._binding import (  # noqa: F401
    LBM_BGK, LBM_SMRT, LBM_SMRT_FNEQ, LBM_MRT_RAW, LBM_D2Q9, LBM_D3Q19, LBM_D3Q27, LBM_F64, LBM_F32, LBM_F16_SHIFT,
    LBM_BF16_SHIFT, LBM_G_NONE, LBM_G_UNIFORM, LBM_G_ROWS, LBM_G_FIELD, LbmError, Lattice,
    lbm_create, lbm_destroy, lbm_step, lbm_moments, lbm_moments_device, lbm_residual,
    lbm_check_device,
    lbm_set_force, lbm_set_force_schedule, lbm_set_force_scale_schedule, lbm_get_populations, lbm_set_populations, lbm_state_bytes, lbm_get_state,
    lbm_set_state, lbm_info, lbm_last_error, lbm_set_launch, lbm_set_launch_layout, lbm_get_launch,
    lbm_launch_widths, LBM_LAYOUT_STRIDED, LBM_LAYOUT_VECTOR, lbm_force_resolution, lbm_alu_peak, lbm_autotune, lbm_check_noalloc, library, library_path,
    make_desc, Batch, lbm_batch_create, lbm_batch_run_to_steady, lbm_batch_step, lbm_batch_reset,
    lbm_batch_moments, lbm_batch_get_populations, lbm_batch_set_tiles, lbm_batch_autotune,
    lbm_batch_set_spin_limit, lbm_batch_set_handoff, lbm_batch_info, lbm_batch_last_error, lbm_batch_destroy, LBM_NOT_CONVERGED,
    UNet, lbm_unet_create, lbm_unet_num_params, lbm_unet_set_params, lbm_unet_get_params, lbm_unet_forward,
    lbm_unet_grad, lbm_unet_adam, lbm_unet_train_step, lbm_unet_set_wgrad, UNET_WGRAD_AUTO, UNET_WGRAD_MMA_SYNC,
    lbm_unet_destroy, lbm_unet_last_error, Split, lbm_split_schedule, lbm_split_create, lbm_split_step,
    lbm_split_check_device, lbm_split_moments, lbm_split_state_bytes, lbm_split_get_state, lbm_split_get_populations,
    lbm_split_set_launch_layout, lbm_split_last_error, lbm_split_destroy)
