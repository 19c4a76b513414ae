"""The allocation-free cube entry point against the library's own cube.

``ucp_root_cube_static`` serves callers that cannot allocate GPU memory when
they call in (for instance while a CUDA graph is being captured, or under a
device-memory budget owned by another allocator): it keeps its partial results
in a fixed device array.  Its cube must equal the one ``ucp_tree_build`` makes
(min/max reductions are exact, so the comparison is bit for bit), call after
call, and it must refuse sizes beyond its fixed scratch.
"""
import ctypes as C

import numpy as np
import pytest

from paper_0709_3331_gb300.inputs import gaussian_cloud

pytestmark = pytest.mark.gpu

UCP_STATIC_MAX_N = 1024 * 2048


def _entry():
    from paper_0709_3331_gb300 import build as B
    B.build()
    from paper_0709_3331_gb300 import lib
    L = lib()
    f = L.ucp_root_cube_static
    f.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]
    f.restype = C.c_int
    return f


def test_root_cube_static_matches_tree_build():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0709_3331_gb300 import Context
    f = _entry()
    stream = torch.cuda.current_stream().cuda_stream
    # two calls in a row, the second with fewer tiles than the first
    for n, sigma, seed in ((524288, 8.0, 3), (6002, 2.0, 7)):
        c = gaussian_cloud(n, sigma, seed)
        pos = torch.from_numpy(c.pos).cuda()
        out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
        assert f(pos.data_ptr(), n, out.data_ptr(), stream) == 0
        torch.cuda.synchronize()
        with Context(n, c.q, c.m, leaf_cap=16) as ctx:
            ctx.set_state(c.pos, c.vel, c.species)
            ctx.tree_build()
            ref = ctx.get_cube()
        np.testing.assert_array_equal(out.cpu().numpy(), ref)
    # sizes outside [1, UCP_STATIC_MAX_N] are refused before anything is launched
    assert f(pos.data_ptr(), UCP_STATIC_MAX_N + 1, out.data_ptr(), stream) == -1
    assert f(pos.data_ptr(), 0, out.data_ptr(), stream) == -1
    assert f(None, 16, out.data_ptr(), stream) == -1
