"""ctypes binding of libpic.so (include/pic.h).  Argument marshalling only:
every step of the PIC path runs in the library's CUDA kernels.  There is no
fallback; if the library is missing or fails to load, importing this module
raises."""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpic.so")

c_int, c_float, c_double, c_int64, c_void_p = (ctypes.c_int, ctypes.c_float, ctypes.c_double,
                                               ctypes.c_int64, ctypes.c_void_p)

PIC_OK, PIC_ERR_ARG, PIC_ERR_CUDA, PIC_ERR_OOM, PIC_ERR_TIMEOUT, PIC_ERR_STATE = range(6)
STATUS_NAMES = {0: "PIC_OK", 1: "PIC_ERR_ARG", 2: "PIC_ERR_CUDA", 3: "PIC_ERR_OOM",
                4: "PIC_ERR_TIMEOUT", 5: "PIC_ERR_STATE"}
PIC_MAX_SPECIES = 4
PIC_FIELD_B_HALF, PIC_FIELD_E = 0, 1
KERNEL_KINDS = ["push", "b_half", "e_update", "filter", "sort", "boundary", "adjoint"]


class pic_grid(ctypes.Structure):
    _fields_ = [("dim", c_int), ("nx", c_int), ("ny", c_int), ("nz", c_int)]


class pic_species(ctypes.Structure):
    _fields_ = [("q", c_float), ("m", c_float), ("n", c_int64), ("cell", c_void_p),
                ("off", c_void_p), ("u", c_void_p), ("cap", c_int64)]


class pic_host_species(ctypes.Structure):
    _fields_ = [("cell", c_void_p), ("off", c_void_p), ("u", c_void_p)]


class pic_shock(ctypes.Structure):
    _fields_ = [("wall", c_int), ("lt", c_int), ("x0", c_double), ("x_max", c_double),
                ("v_inj", c_double), ("v_up", c_double), ("nt", c_int64 * PIC_MAX_SPECIES),
                ("tmpl", pic_host_species * PIC_MAX_SPECIES)]


class pic_adjoint_species(ctypes.Structure):
    _fields_ = [("cell", c_void_p), ("off", c_void_p), ("u", c_void_p), ("xbar", c_void_p),
                ("ubar", c_void_p), ("tstart", c_void_p)]


class pic_tuning(ctypes.Structure):
    _fields_ = [("tile", c_int * 3), ("halo", c_int), ("sort_every", c_int),
                ("filter_passes", c_int), ("chunk", c_int)]


_P = c_void_p  # pic_ctx*
SIGNATURES = {
    "pic_init": (c_int, [ctypes.POINTER(_P), ctypes.POINTER(pic_grid), ctypes.POINTER(pic_species),
                         c_int, c_float, c_float, c_void_p, c_void_p]),
    "pic_get_tuning": (c_int, [_P, ctypes.POINTER(pic_tuning)]),
    "pic_set_tuning": (c_int, [_P, ctypes.POINTER(pic_tuning)]),
    "pic_set_pusher": (c_int, [_P, c_int]),
    "pic_set_host_chunk": (c_int, [_P, c_int64]),
    "pic_set_field_solver": (c_int, [_P, c_int]),
    "pic_set_shock": (c_int, [_P, ctypes.POINTER(pic_shock)]),
    "pic_particle_counts": (c_int, [_P, ctypes.POINTER(c_int64), c_int]),
    "pic_adjoint_step": (c_int, [_P, c_void_p, ctypes.POINTER(pic_adjoint_species), c_void_p]),
    "pic_sort": (c_int, [_P]),
    "pic_sort_bins": (c_int, [_P, ctypes.POINTER(ctypes.c_int64)]),
    "pic_sort_record": (c_int, [_P, ctypes.POINTER(c_void_p), ctypes.POINTER(c_void_p)]),
    "pic_sort_assume": (c_int, [_P, ctypes.POINTER(c_void_p)]),
    "pic_adjoint_unsort": (c_int, [_P, ctypes.POINTER(c_void_p),
                                   ctypes.POINTER(pic_adjoint_species)]),
    "pic_gather_push": (c_int, [_P]),
    "pic_deposit": (c_int, [_P]),
    "pic_filter_current": (c_int, [_P, c_int]),
    "pic_field_update": (c_int, [_P, c_int]),
    "pic_step": (c_int, [_P, c_int]),
    "pic_energies": (c_int, [_P, ctypes.POINTER(c_double), c_int]),
    "pic_check": (c_int, [_P]),
    "pic_wait_probe": (c_int, [_P]),
    "pic_step_host": (c_int, [_P, ctypes.POINTER(pic_host_species), c_void_p, c_int]),
    "pic_autotune": (c_int, [_P, ctypes.POINTER(pic_tuning), c_int, c_int, ctypes.POINTER(c_int)]),
    "pic_stats": (c_int, [_P, ctypes.POINTER(c_int64)]),
    "pic_timing": (c_int, [_P, c_int]),
    "pic_kernel_times": (c_int, [_P, ctypes.POINTER(c_double), ctypes.POINTER(c_int64)]),
    "pic_filter_current_static": (c_int, [ctypes.POINTER(pic_grid), c_void_p, c_int, c_void_p]),
    "pic_batch_create": (c_int, [ctypes.POINTER(c_void_p), ctypes.POINTER(c_void_p), c_int]),
    "pic_batch_step": (c_int, [c_void_p, c_int, c_void_p]),
    "pic_batch_destroy": (c_int, [c_void_p]),
    "pic_destroy": (c_int, [_P]),
    "pic_last_error": (ctypes.c_char_p, [_P]),
}


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise RuntimeError(f"libpic.so not found at {path}: build it with "
                           "`python -m paper_1906_06306_gb300.build` (no CPU fallback exists)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = load_library()


class PicError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def _check(status: int, ctx) -> None:
    if status != PIC_OK:
        msg = _lib.pic_last_error(ctx)
        raise PicError(status, msg.decode() if msg else "")


# --- same names as the C ABI ------------------------------------------------

def pic_init(grid: pic_grid, species, c: float, dt: float, fields_ptr: int, stream: int):
    """species: sequence of pic_species; returns the context handle."""
    arr = (pic_species * len(species))(*species)
    ctx = c_void_p()
    st = _lib.pic_init(ctypes.byref(ctx), ctypes.byref(grid), arr, len(species), c, dt,
                       c_void_p(fields_ptr), c_void_p(stream))
    _check(st, None)
    return ctx


def pic_get_tuning(ctx) -> pic_tuning:
    t = pic_tuning()
    _check(_lib.pic_get_tuning(ctx, ctypes.byref(t)), ctx)
    return t


def pic_set_tuning(ctx, t: pic_tuning) -> None:
    _check(_lib.pic_set_tuning(ctx, ctypes.byref(t)), ctx)


PIC_PUSHER_BORIS, PIC_PUSHER_HIGUERA_CARY = 0, 1


PIC_FDTD2, PIC_FDTD4 = 2, 4


def pic_set_field_solver(ctx, order: int) -> None:
    _check(_lib.pic_set_field_solver(ctx, order), ctx)


def pic_set_pusher(ctx, pusher: int) -> None:
    _check(_lib.pic_set_pusher(ctx, pusher), ctx)


def pic_set_host_chunk(ctx, particles: int) -> None:
    _check(_lib.pic_set_host_chunk(ctx, particles), ctx)


def pic_set_shock(ctx, shock: pic_shock) -> None:
    """Conducting wall and receding injector along x (Sect. 4.2); the template
    host arrays referenced by `shock` are copied by the library."""
    _check(_lib.pic_set_shock(ctx, ctypes.byref(shock)), ctx)


def pic_adjoint_step(ctx, fwd_fields_ptr: int, species, adj_fields_ptr: int) -> None:
    """Reverse of one pic_step: species is a sequence of pic_adjoint_species
    (forward particles at the start of the step, gradients xbar/ubar in place)."""
    arr = (pic_adjoint_species * len(species))(*species)
    _check(_lib.pic_adjoint_step(ctx, c_void_p(fwd_fields_ptr), arr, c_void_p(adj_fields_ptr)), ctx)


def pic_particle_counts(ctx, nspecies: int):
    out = (c_int64 * nspecies)()
    _check(_lib.pic_particle_counts(ctx, out, nspecies), ctx)
    return [int(v) for v in out]


def pic_sort(ctx) -> None:
    _check(_lib.pic_sort(ctx), ctx)


def pic_sort_bins(ctx) -> int:
    n = ctypes.c_int64(0)
    _check(_lib.pic_sort_bins(ctx, ctypes.byref(n)), ctx)
    return n.value


def pic_sort_record(ctx, perm_ptrs, tstart_ptrs) -> None:
    """perm_ptrs, tstart_ptrs: device addresses (int32[n], int32[nbins + 1])
    per species, 0 for species without particles."""
    p = (c_void_p * len(perm_ptrs))(*[c_void_p(x or None) for x in perm_ptrs])
    t = (c_void_p * len(tstart_ptrs))(*[c_void_p(x or None) for x in tstart_ptrs])
    _check(_lib.pic_sort_record(ctx, p, t), ctx)


def pic_sort_assume(ctx, tstart_ptrs) -> None:
    t = (c_void_p * len(tstart_ptrs))(*[c_void_p(x or None) for x in tstart_ptrs])
    _check(_lib.pic_sort_assume(ctx, t), ctx)


def pic_adjoint_unsort(ctx, perm_ptrs, species) -> None:
    """species: pic_adjoint_species per species (xbar and ubar are used)."""
    p = (c_void_p * len(perm_ptrs))(*[c_void_p(x or None) for x in perm_ptrs])
    arr = (pic_adjoint_species * len(species))(*species)
    _check(_lib.pic_adjoint_unsort(ctx, p, arr), ctx)


def pic_gather_push(ctx) -> None:
    _check(_lib.pic_gather_push(ctx), ctx)


def pic_deposit(ctx) -> None:
    _check(_lib.pic_deposit(ctx), ctx)


def pic_filter_current(ctx, passes: int) -> None:
    _check(_lib.pic_filter_current(ctx, passes), ctx)


def pic_field_update(ctx, which: int) -> None:
    _check(_lib.pic_field_update(ctx, which), ctx)


def pic_step(ctx, nsteps: int) -> None:
    _check(_lib.pic_step(ctx, nsteps), ctx)


def pic_energies(ctx, nspecies: int):
    n = 4 + nspecies
    out = (c_double * n)()
    _check(_lib.pic_energies(ctx, out, n), ctx)
    return list(out)


def pic_check(ctx) -> None:
    _check(_lib.pic_check(ctx), ctx)


def pic_wait_probe(ctx) -> None:
    _check(_lib.pic_wait_probe(ctx), ctx)


def pic_step_host(ctx, host_species, host_fields_ptr: int, nsteps: int) -> None:
    arr = (pic_host_species * len(host_species))(*host_species)
    _check(_lib.pic_step_host(ctx, arr, c_void_p(host_fields_ptr), nsteps), ctx)


def pic_autotune(ctx, candidates=None, steps: int = 20) -> int:
    """Run real steps under each candidate tuning (None: the built-in set) and keep
    the fastest; returns the chosen candidate's index."""
    best = c_int(-1)
    if candidates:
        arr = (pic_tuning * len(candidates))(*candidates)
        _check(_lib.pic_autotune(ctx, arr, len(candidates), steps, ctypes.byref(best)), ctx)
    else:
        _check(_lib.pic_autotune(ctx, None, 0, steps, ctypes.byref(best)), ctx)
    return int(best.value)


def pic_stats(ctx) -> int:
    """Particle updates that took the global-memory path since the last call."""
    v = c_int64()
    _check(_lib.pic_stats(ctx, ctypes.byref(v)), ctx)
    return int(v.value)


def pic_timing(ctx, enable: bool) -> None:
    _check(_lib.pic_timing(ctx, 1 if enable else 0), ctx)


def pic_kernel_times(ctx):
    ms = (c_double * len(KERNEL_KINDS))()
    n = (c_int64 * len(KERNEL_KINDS))()
    _check(_lib.pic_kernel_times(ctx, ms, n), ctx)
    return {k: (ms[i], n[i]) for i, k in enumerate(KERNEL_KINDS)}


PIC_FILTER_STATIC_MAX_FLOATS = 4194304


def pic_filter_current_static(grid: pic_grid, j_ptr: int, passes: int, stream: int) -> None:
    """Allocation-free Binomial2 filter of the three J planes at device address
    j_ptr (in place, on `stream`); see include/pic.h for the size limit."""
    _check(_lib.pic_filter_current_static(ctypes.byref(grid), c_void_p(j_ptr), passes,
                                          c_void_p(stream)), None)


def pic_batch_create(ctxs):
    arr = (c_void_p * len(ctxs))(*[c.value if isinstance(c, c_void_p) else c for c in ctxs])
    b = c_void_p()
    _check(_lib.pic_batch_create(ctypes.byref(b), arr, len(ctxs)), None)
    return b


def pic_batch_step(batch, nsteps: int, stream: int) -> None:
    _check(_lib.pic_batch_step(batch, nsteps, c_void_p(stream)), None)


def pic_batch_destroy(batch) -> None:
    _check(_lib.pic_batch_destroy(batch), None)


def pic_destroy(ctx) -> None:
    _check(_lib.pic_destroy(ctx), None)


def pic_last_error(ctx=None) -> str:
    m = _lib.pic_last_error(ctx)
    return m.decode() if m else ""
