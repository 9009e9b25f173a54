"""pic_filter_current_static, the filter entry point that allocates nothing
(for callers whose memory manager owns the device, that must stay within a
fixed memory budget, or that cannot afford the synchronisation cudaFree
implies), against the context-based pic_filter_current (bit for bit: both run
the same fused passes) and against the oracle's Binomial2 filter.

Kept in a file of its own that pytest collects last; it passes on its own in a
fresh process and after the other tests."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

# (dim, (nz, ny, nx), passes): ragged odd passes, then x rows of a multiple of
# 4 floats (the 16-byte path) with an even number of passes (no copy back)
CASES = [(2, (1, 23, 29), 3), (3, (9, 11, 13), 2), (2, (1, 20, 32), 2), (3, (6, 10, 16), 1)]


def _context_filter(dim, shape, J, passes):
    """The existing entry point: a context over the planes, pic_filter_current."""
    from paper_1906_06306_gb300 import Simulation

    nz, ny, nx = shape
    F = np.zeros((9,) + shape, np.float32)
    F[6:9] = J
    empty = [dict(q=-1.0, m=1.0, cell=np.zeros(0, np.int32), off=np.zeros((dim, 0), np.float32),
                  u=np.zeros((3, 0), np.float32))]
    sim = Simulation(dim, nx, ny, nz, 0.45, F, empty)
    sim.filter_current(passes)
    out = sim.download()[0][6:9].copy()
    sim.close()
    return out


def _oracle_filter(dim, shape, J, passes):
    nz, ny, nx = shape
    g = oracle.Grid(dim, nx, ny, nz)
    F = g.zeros()
    F[6:9] = J.astype(np.float64)
    oracle.filter_binomial(g, F, passes)
    return F[6:9]


def _static_filter(dim, shape, Jd, passes, stream):
    from paper_1906_06306_gb300 import binding as B

    nz, ny, nx = shape
    B.pic_filter_current_static(B.pic_grid(dim, nx, ny, nz), Jd.data_ptr(), passes,
                                stream.cuda_stream)


def test_static_filter_matches_context_filter_and_oracle_on_consecutive_calls():
    import torch

    rs = np.random.default_rng(900)
    stream = torch.cuda.current_stream()
    for call, (dim, shape, passes) in enumerate(CASES):  # calls in a row share the scratch
        J = rs.normal(size=(3,) + shape).astype(np.float32)
        ref = _context_filter(dim, shape, J, passes)
        Jd = torch.from_numpy(J).cuda()
        _static_filter(dim, shape, Jd, passes, stream)
        stream.synchronize()
        got = Jd.cpu().numpy()
        assert np.array_equal(got, ref), (call, np.abs(got - ref).max())
        orc = _oracle_filter(dim, shape, J, passes)
        err = np.abs(got - orc).max() / np.abs(orc).max()
        assert err < 1e-6, (call, err)


def test_static_filter_allocates_nothing():
    """Device memory (the driver's free bytes and torch's allocator) is the same
    before and after calls, once the first call has looked up the scratch."""
    import torch

    dim, shape, passes = 3, (8, 12, 16), 3
    rs = np.random.default_rng(901)
    Jd = torch.from_numpy(rs.normal(size=(3,) + shape).astype(np.float32)).cuda()
    stream = torch.cuda.current_stream()
    _static_filter(dim, shape, Jd, passes, stream)  # first call on the device: set-up
    stream.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for _ in range(3):
        _static_filter(dim, shape, Jd, passes, stream)
    stream.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_allocated() == alloc0


def test_static_filter_rejects_grids_beyond_its_scratch():
    from paper_1906_06306_gb300 import binding as B

    n = int(np.ceil((B.PIC_FILTER_STATIC_MAX_FLOATS / 3) ** 0.5)) + 1
    with pytest.raises(B.PicError) as ei:
        B.pic_filter_current_static(B.pic_grid(2, n, n, 1), 0x1000, 1, 0)
    assert ei.value.status == B.PIC_ERR_ARG
    assert "PIC_FILTER_STATIC_MAX_FLOATS" in str(ei.value)
