"""GB300 (sm_103a) library for the explicit electrostatic PIC-MCC model of a
dc magnetron discharge in 2D (r,z) geometry (arXiv:2507.10727).

The compute path is ``libpic_gb300.so`` (CUDA kernels behind the C ABI of
``include/pic.h``); this package holds its build script and a thin ctypes
binding with the same function names.
"""
from .pic import (  # noqa: F401
    PicError, PicConfig, PicDiag, Handle, load_library, LIB_PATH,
    pic_create, pic_destroy, pic_set_particles, pic_count, pic_get_particles,
    pic_solve_fields, pic_set_phi, pic_get_fields, pic_set_circuit, pic_set_next_id,
    pic_get_next_id, pic_step, pic_uses_graph, pic_tuned_chunk, pic_set_chunk, pic_autotune_info,
    pic_set_tile, pic_tuned_tile, pic_fp64_fma_rate, pic_sync,
    pic_diagnostics, pic_reweight, pic_get_species_charge,
    pic_region_sample, pic_region_read, pic_region_reset, PicRegions,
    pic_save, pic_load,
    pic_profile, pic_profile_read, pic_poisson_workspace_bytes, pic_poisson_solve,
    pic_unet_param_count, pic_unet_create, pic_unet_set_params, pic_unet_get_params,
    pic_unet_loss_grad, pic_unet_snapshots, pic_unet_train, pic_unet_warm_start, pic_unet_stats,
    pic_unet_set_norms, pic_unet_record,
)
