"""GB300-native relativistic PIC hot path (Runko, arXiv:1906.06306).

The API names below resolve on first use by loading libpic.so (the CUDA
kernels behind the C ABI of include/pic.h); if the library is missing that
access raises -- there is no CPU fallback.  The `build` submodule imports
without the library so that it can compile it.

Use (device memory and the stream come from PyTorch):

    import workloads
    from paper_1906_06306_gb300 import Simulation, Batch
    sim = Simulation.from_plasma(workloads.turbulence_2d(n=256))  # periodic box
    sim.autotune()          # tile size, halo and sort cadence, by real steps
    sim.step(100)           # B half, gather+Boris+move+ZigZag, B half, filter, E
    print(sim.energies())   # 0.5 sum E^2, 0.5 sum B^2, kinetic, Gauss residual
    fields, particles = sim.download()

    sim.set_field_solver(4); sim.set_pusher("higuera_cary")   # Table 2 variants
    sim.set_shock_from_plasma(workloads.shock_tube(...))      # wall + injector
    Batch([sim_a, sim_b, ...]).step(500)                      # ensembles, one graph

    from paper_1906_06306_gb300.adjoint import MagneticEnergy, MagneticEnergyProblem
    loss = MagneticEnergy.apply(amps, u0, problem); loss.backward()  # discrete adjoint
"""
_API = {
    "PicError", "pic_init", "pic_set_pusher", "pic_set_host_chunk", "pic_set_field_solver", "pic_get_tuning",
    "pic_set_tuning", "pic_set_shock", "pic_particle_counts", "pic_adjoint_step", "pic_sort",
    "pic_sort_bins", "pic_sort_record", "pic_sort_assume", "pic_adjoint_unsort", "pic_gather_push",
    "pic_deposit", "pic_filter_current", "pic_field_update", "pic_step", "pic_energies",
    "pic_check", "pic_wait_probe", "pic_step_host", "pic_autotune", "pic_stats", "pic_timing", "pic_kernel_times",
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
