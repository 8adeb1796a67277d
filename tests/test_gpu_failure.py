"""Failure detection without a GPU fault: errors are made on the host (a
refused allocation, a NaN planted in a field, a malformed request) and
must come back as status codes with the context still usable; checkpoint
and resume through the public API reproduce an uninterrupted run bit for bit."""
import os
import subprocess
import sys

import numpy as np
import pytest

import meshgen as mg

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1207_1571_gb300 import build as B
    B.build()
    import paper_1207_1571_gb300 as P
    P.load()
    return P


def test_nan_in_field_reports_diverged(P):
    m = mg.cavity3d(8)
    mesh = P.Mesh(m)
    case = P.Case(mesh, 0.01)
    u = np.zeros((3, m.n_cells))
    u[0, 17] = np.nan
    case.set_fields_host(u, np.zeros(m.n_cells), np.zeros(m.n_faces))
    s = case.piso_step(0.01, 2, p_ref_cell=0)
    assert s["status"] == 5          # FV_E_DIVERGED, reported not raised
    # the context is still usable
    case2 = P.Case(mesh, 0.01)
    assert case2.piso_step(0.01, 2, p_ref_cell=0)["status"] == 0


def test_refused_allocation_returns_nomem():
    code = (
        "import sys; sys.path.insert(0, %r)\n"
        "import meshgen as mg, paper_1207_1571_gb300 as P\n"
        "try:\n"
        "    P.Mesh(mg.cavity3d(6))\n"
        "    print('NO ERROR')\n"
        "except P.FvError as e:\n"
        "    print('STATUS', e.status)\n" % ROOT)
    env = dict(os.environ, FVGB_FAIL_ALLOC_AFTER="5")
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                         timeout=300)
    assert "STATUS 3" in out.stdout, out.stdout + out.stderr


def test_bad_requests_are_rejected(P):
    m = mg.cavity2d(6)
    mesh = P.Mesh(m)
    case = P.Case(mesh, 0.1)
    with pytest.raises(P.FvError) as e:
        case.piso_step(-1.0, 2, p_ref_cell=0)
    assert e.value.status == 1
    with pytest.raises(P.FvError) as e:
        case.piso_step(0.01, 99, p_ref_cell=0)
    assert e.value.status == 1
    with pytest.raises(P.FvError) as e:
        case.piso_step(0.01, 2, p_ref_cell=10 ** 6)
    assert e.value.status == 1
    assert case.piso_step(0.01, 2, p_ref_cell=0)["status"] == 0


def test_checkpoint_resume_is_bit_exact(P, tmp_path):
    m = mg.permute_cells(mg.cavity3d(10), mg.random_permutation(1000, 4))
    mesh = P.Mesh(m)
    a = P.Case(mesh, 0.01)
    for _ in range(10):
        a.piso_step(0.01, 2, p_ref_cell=m.corner_cell)
    b = P.Case(mesh, 0.01)
    for _ in range(5):
        b.piso_step(0.01, 2, p_ref_cell=m.corner_cell)
    path = str(tmp_path / "ck.npz")
    b.save(path, step=5)
    c = P.Case(mesh, 0.01)
    extra = c.load(path)
    assert int(extra["step"]) == 5
    for _ in range(5):
        c.piso_step(0.01, 2, p_ref_cell=m.corner_cell)
    for x, y in zip(a.get_fields_host(), c.get_fields_host()):
        assert np.array_equal(x, y)
