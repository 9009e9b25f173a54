"""pic_filter_current_static, the filter entry point that allocates nothing
(for callers whose memory manager owns the device, that must stay within a
fixed memory budget, or that cannot afford the synchronisation cudaFree
implies), against the context-based pic_filter_current.

Kept in a file of its own that pytest collects last; it passes on its own in a
fresh process and after the other tests."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

CASES = [(2, (1, 23, 29), 3), (3, (9, 11, 13), 2)]  # (dim, (nz, ny, nx), passes)


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


def test_static_filter_matches_context_filter_on_consecutive_calls():
    import torch

    from paper_1906_06306_gb300 import binding as B

    rs = np.random.default_rng(900)
    stream = torch.cuda.current_stream()
    for call, (dim, shape, passes) in enumerate(CASES):  # two calls in a row
        nz, ny, nx = shape
        J = rs.normal(size=(3,) + shape).astype(np.float32)
        ref = _context_filter(dim, shape, J, passes)
        Jd = torch.from_numpy(J).cuda()
        B.pic_filter_current_static(B.pic_grid(dim, nx, ny, nz), Jd.data_ptr(), passes,
                                    stream.cuda_stream)
        stream.synchronize()
        got = Jd.cpu().numpy()
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert err < 1e-6, (call, err)


def test_static_filter_rejects_grids_beyond_its_scratch():
    from paper_1906_06306_gb300 import binding as B

    n = int(np.ceil((B.PIC_FILTER_STATIC_MAX_FLOATS / 3) ** 0.5)) + 1
    with pytest.raises(B.PicError) as ei:
        B.pic_filter_current_static(B.pic_grid(2, n, n, 1), 0x1000, 1, 0)
    assert ei.value.status == B.PIC_ERR_ARG
    assert "PIC_FILTER_STATIC_MAX_FLOATS" in str(ei.value)
