"""The library used from plain C through include/ucp.h with host pointers: a C
client compiled here with gcc gives the same bits as the Python binding on the
same cloud (force, 10-substep state, energy), in both precisions."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_0709_3331_gb300.inputs import gaussian_cloud

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def client(tmp_path_factory):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    from paper_0709_3331_gb300 import build as b
    lib = b.build()
    d = tmp_path_factory.mktemp("c_abi")
    exe = str(d / "ucp_c_client")
    subprocess.run(["gcc", "-O2", "-std=c99", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c_abi", "ucp_c_client.c"), "-o", exe,
                    "-L", os.path.dirname(lib), "-lucp", "-Wl,-rpath," + os.path.dirname(lib)],
                   check=True)
    return exe, d


@pytest.mark.parametrize("prec", [0, 1])
def test_c_client_matches_binding(client, prec):
    exe, d = client
    import paper_0709_3331_gb300 as P
    c = gaussian_cloud(3000, 1.4, 71)
    inp, out = str(d / f"in{prec}.txt"), str(d / f"out{prec}.txt")
    with open(inp, "w") as f:
        f.write(f"{c.n}\n")
        for i in range(c.n):
            f.write(" ".join(repr(float(v)) for v in (*c.pos[i], *c.vel[i])) +
                    f" {int(c.species[i])}\n")
    subprocess.run([exe, inp, out, str(prec)], check=True)
    rows = [np.array(ln.split(), dtype=np.float64) for ln in open(out)]
    acc_c = np.array([r[:3] for r in rows[:c.n]])
    phi_c = np.array([r[3] for r in rows[:c.n]])
    st_c = np.array(rows[c.n:2 * c.n])
    en_c = rows[2 * c.n]
    with P.Context(c.n, c.q, c.m, leaf_cap=16, precision=prec) as ctx:
        ctx.set_state(c.pos, c.vel, c.species)
        acc, phi = ctx.tree_force(0.5, 0.01)
        ctx.step(1e-3, 5, 10, 0.5, 0.01)
        p, v = ctx.get_state()
        en = ctx.energy(0.5, 0.01)
    assert np.array_equal(acc_c, acc) and np.array_equal(phi_c, phi)
    assert np.array_equal(st_c[:, :3], p) and np.array_equal(st_c[:, 3:], v)
    assert np.array_equal(en_c, en)
