"""GB300-native relativistic PIC hot path (Runko, arXiv:1906.06306).

The API names below resolve on first use by loading libpic.so (the CUDA
kernels behind the C ABI of include/pic.h); if the library is missing that
access raises -- there is no CPU fallback.  The `build` submodule imports
without the library so that it can compile it.
"""
_API = {
    "PicError", "pic_init", "pic_set_pusher", "pic_set_field_solver", "pic_get_tuning",
    "pic_set_tuning", "pic_set_shock", "pic_particle_counts", "pic_adjoint_step", "pic_sort", "pic_gather_push",
    "pic_deposit", "pic_filter_current", "pic_field_update", "pic_step", "pic_energies",
    "pic_check", "pic_step_host", "pic_autotune", "pic_stats", "pic_timing", "pic_kernel_times",
    "pic_destroy", "pic_last_error", "pic_filter_current_static", "pic_batch_create",
    "pic_batch_step", "pic_batch_destroy", "PIC_FIELD_B_HALF", "PIC_FIELD_E",
}


def __getattr__(name):
    if name in _API:
        from . import binding

        return getattr(binding, name)
    if name in ("Simulation", "Batch"):
        from . import sim

        return getattr(sim, name)
    if name in ("Adjoint", "MagneticEnergy"):
        from . import adjoint

        return getattr(adjoint, name)
    raise AttributeError(name)
