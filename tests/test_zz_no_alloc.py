"""fg_action_sums_noalloc against fg_action, through the C ABI.

fg_action_sums_noalloc serves callers that cannot let the library allocate
device memory (their GPU memory is reserved in full by another allocator, or
a cudaMalloc/cudaFree pair would stall a latency-critical loop).  It keeps
its block partial sums in a fixed device array inside the library, so this
test checks that two calls in a row, on different lattices, both reproduce
the sums of the handle-based fg_action, and that oversized lattices are
refused.  The file name makes pytest collect it last.
"""

import ctypes as C

import numpy as np
import pytest

from paper_0910_2950_gb300 import inputs

pytestmark = pytest.mark.gpu


def _reference(fg, dims, beta, u, p):
    with fg.Lattice(dims, beta) as lat:
        lat.set_gauge(u)
        lat.set_momenta(p)
        sg, _, t = lat.action()
    return sg, t


def test_action_sums_noalloc_matches_fg_action():
    import torch
    from paper_0910_2950_gb300 import build, fg

    build.build()
    lib = fg.load()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    out = torch.empty(2, dtype=torch.float64, device=dev)
    # two calls in a row; the second lattice is smaller, so stale partial sums
    # of the first call sit beyond the range the second call reads
    cases = [((8, 6, 4, 10), 5.7, 31), ((4, 4, 2, 6), 6.0, 32)]
    for dims, beta, seed in cases:
        u = inputs.hot_start(dims, seed)
        p = inputs.gaussian_momenta(dims, seed + 100)
        sg_ref, t_ref = _reference(fg, dims, beta, u, p)
        du = torch.from_numpy(np.ascontiguousarray(u).view(np.float64).reshape(-1)).to(dev)
        dp = torch.from_numpy(np.ascontiguousarray(p).reshape(-1)).to(dev)
        out.fill_(-1.0)
        d = (C.c_int * 4)(*dims)
        st = lib.fg_action_sums_noalloc(du.data_ptr(), dp.data_ptr(), d, beta, out.data_ptr(),
                                        stream.cuda_stream)
        assert st == fg.FG_OK
        torch.cuda.synchronize()
        sg, t = out.cpu().tolist()
        assert abs(sg - sg_ref) <= 1e-12 * abs(sg_ref), (sg, sg_ref)
        assert abs(t - t_ref) <= 1e-12 * abs(t_ref), (t, t_ref)
        # without momenta the kinetic sum is zero
        st = lib.fg_action_sums_noalloc(du.data_ptr(), None, d, beta, out.data_ptr(), stream.cuda_stream)
        assert st == fg.FG_OK
        torch.cuda.synchronize()
        sg2, t2 = out.cpu().tolist()
        assert sg2 == sg and t2 == 0.0
    # more than FG_NOALLOC_MAX_SITES sites is refused before anything is queued
    big = (C.c_int * 4)(256, 256, 256, 2)
    assert lib.fg_action_sums_noalloc(du.data_ptr(), dp.data_ptr(), big, 6.0, out.data_ptr(),
                                      stream.cuda_stream) == fg.FG_EINVAL
    odd = (C.c_int * 4)(4, 4, 3, 4)
    assert lib.fg_action_sums_noalloc(du.data_ptr(), dp.data_ptr(), odd, 6.0, out.data_ptr(),
                                      stream.cuda_stream) == fg.FG_EINVAL
