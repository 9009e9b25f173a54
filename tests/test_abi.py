"""The C-ABI library loads and exports every entry point declared in
include/pic.h; pic_init rejects bad arguments on the host before any CUDA
work (so these run without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1906_06306_gb300 import build

    build.build()
    from paper_1906_06306_gb300 import binding

    return binding


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(pic_\w+)\s*\(", txt))
    return sorted(names)


def test_header_declares_the_boundary():
    names = _declared()
    for required in ["pic_init", "pic_gather_push", "pic_deposit", "pic_filter_current",
                     "pic_field_update", "pic_step", "pic_energies", "pic_destroy"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    so = ctypes.CDLL(lib.LIB_PATH)
    missing = [n for n in _declared() if not hasattr(so, n)]
    assert not missing, missing
    assert set(_declared()) == set(lib.SIGNATURES), "binding covers exactly the header"


def _species(lib, n=4, q=-1.0, m=1.0, ptr=0x1000, cap=0):
    return lib.pic_species(q, m, n, ptr, ptr, ptr, cap)


@pytest.mark.parametrize("case,msg", [
    (dict(dim=4), "dim"),
    (dict(dim=0), "dim"),
    (dict(nx=0), "extents"),
    (dict(dim=1, ny=2), "non-gridded"),
    (dict(dim=2, nz=3), "non-gridded"),
    (dict(c=1.0), "Courant"),
    (dict(c=0.0), "Courant"),
    (dict(dt=0.5), "dt"),
    (dict(nspecies=0), "nspecies"),
    (dict(nspecies=5), "nspecies"),
    (dict(m=0.0), "mass"),
    (dict(n=-1), "species n"),
    (dict(null_cell=True), "NULL"),
    (dict(null_fields=True), "NULL"),
    (dict(dim=3, nx=2048, ny=2048, nz=1024), "int32"),
    (dict(dim=2, nx=4, ny=70000), "65535"),
    (dict(cap=2), "cap"),
])
def test_pic_init_rejects_bad_arguments(lib, case, msg):
    dim = case.get("dim", 2)
    g = lib.pic_grid(dim, case.get("nx", 8), case.get("ny", 8 if dim >= 2 else 1),
                     case.get("nz", 1 if dim < 3 else 8))
    if "nz" in case:
        g.nz = case["nz"]
    if "ny" in case:
        g.ny = case["ny"]
    ns = case.get("nspecies", 2)
    sp = (lib.pic_species * 5)(*[_species(lib, n=case.get("n", 4), m=case.get("m", 1.0),
                                          cap=case.get("cap", 0)) for _ in range(5)])
    if case.get("null_cell"):
        sp[0].cell = None
    out = ctypes.c_void_p(123)
    fields = None if case.get("null_fields") else ctypes.c_void_p(0x2000)
    st = lib._lib.pic_init(ctypes.byref(out), ctypes.byref(g), sp, ns, case.get("c", 0.45),
                           case.get("dt", 1.0), fields, None)
    assert st == lib.PIC_ERR_ARG
    assert out.value is None
    assert msg in lib.pic_last_error(None)


def test_null_context_is_an_argument_error(lib):
    for name in ["pic_sort", "pic_gather_push", "pic_deposit", "pic_check", "pic_destroy"]:
        assert getattr(lib._lib, name)(None) == lib.PIC_ERR_ARG
    assert lib._lib.pic_step(None, 1) == lib.PIC_ERR_ARG
    assert lib._lib.pic_field_update(None, 0) == lib.PIC_ERR_ARG
    assert lib._lib.pic_set_shock(None, None) == lib.PIC_ERR_ARG
    assert lib._lib.pic_particle_counts(None, None, 0) == lib.PIC_ERR_ARG
