"""The allocation-free cube entry point against the library's own cube and the
oracle's.

``ucp_root_cube_static`` serves callers that cannot allocate GPU memory when
they call in (for instance while a CUDA graph is being captured, or under a
device-memory budget owned by another allocator): it keeps its partial results
in a fixed device array.  Its cube must equal the one ``ucp_tree_build`` makes
and the oracle's (min/max reductions are exact, so the comparison is bit for
bit), call after call, and it must refuse sizes beyond its fixed scratch.
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


def _static_cube(torch, f, pos_np, stream):
    pos = torch.from_numpy(np.ascontiguousarray(pos_np)).cuda()
    out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
    assert f(pos.data_ptr(), pos_np.shape[0], out.data_ptr(), stream) == 0
    torch.cuda.synchronize()
    return out.cpu().numpy(), pos, out


def test_root_cube_static_matches_tree_build(orc):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0709_3331_gb300 import Context
    f = _entry()
    stream = torch.cuda.current_stream().cuda_stream
    # two calls in a row, the second with fewer tiles than the first; then a
    # cloud whose z axis holds only +0 and -0 (the centre's zero sign must agree)
    zeros = gaussian_cloud(4096, 1.0, 8)
    zpos = zeros.pos.copy()
    zpos[:, 2] = np.where(np.arange(zeros.n) % 3 == 0, -0.0, 0.0)
    for c, pos_np in ((gaussian_cloud(524288, 8.0, 3), None), (gaussian_cloud(6002, 2.0, 7), None),
                      (zeros, zpos)):
        pos_np = c.pos if pos_np is None else pos_np
        got, pos, out = _static_cube(torch, f, pos_np, stream)
        with Context(c.n, c.q, c.m, leaf_cap=16) as ctx:
            ctx.set_state(pos_np, c.vel, c.species)
            ctx.tree_build()
            ref = ctx.get_cube()
        assert got.tobytes() == ref.tobytes()          # bit for bit, zero signs included
        np.testing.assert_array_equal(got, orc.root_cube(pos_np))
    # exactly the largest size the fixed scratch holds (every one of its 1024 tile slots)
    big = gaussian_cloud(UCP_STATIC_MAX_N, 8.0, 11)
    got, _, _ = _static_cube(torch, f, big.pos, stream)
    with Context(big.n, big.q, big.m, leaf_cap=16) as ctx:
        ctx.set_state(big.pos, big.vel, big.species)
        ctx.tree_build()
        ref = ctx.get_cube()
    assert got.tobytes() == ref.tobytes()
    np.testing.assert_array_equal(got, orc.root_cube(big.pos))
    # a NaN coordinate: the library refuses such a state; here the axis's centre is NaN
    bad = gaussian_cloud(1000, 1.0, 9).pos.copy()
    bad[17, 1] = np.nan
    got, _, _ = _static_cube(torch, f, bad, stream)
    assert np.isnan(got[1]) and np.isfinite(got[0]) and np.isfinite(got[2])
    # sizes outside [1, UCP_STATIC_MAX_N] are refused before anything is launched
    assert f(pos.data_ptr(), UCP_STATIC_MAX_N + 1, out.data_ptr(), stream) == -1
    assert f(pos.data_ptr(), 0, out.data_ptr(), stream) == -1
    assert f(None, 16, out.data_ptr(), stream) == -1
