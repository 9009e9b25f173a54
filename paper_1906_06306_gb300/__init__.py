"""GB300-native relativistic PIC hot path (Runko, arXiv:1906.06306).

Importing the package loads libpic.so (the CUDA kernels behind the C ABI of
include/pic.h); there is no CPU fallback.
"""
from . import binding  # noqa: F401  (raises if libpic.so is missing)
from .binding import (  # noqa: F401
    PicError, pic_init, pic_get_tuning, pic_set_tuning, pic_sort, pic_gather_push, pic_deposit,
    pic_filter_current, pic_field_update, pic_step, pic_energies, pic_check, pic_step_host,
    pic_timing, pic_kernel_times, pic_destroy, pic_last_error, PIC_FIELD_B_HALF, PIC_FIELD_E,
)
from .sim import Simulation  # noqa: F401
