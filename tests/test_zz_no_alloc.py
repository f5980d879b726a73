"""nufft_gridding_static: gridding for callers that cannot allocate device
memory when they call in (a process under a fixed memory budget, or code that
must not enter an allocator from where it runs).  Its partial tiles live in the
library's fixed 16 MiB device array instead of plan-owned memory, so the call
allocates nothing.  These tests call it through the C ABI and compare it with
nufft_gridding (the plan-scratch path) on two calls in a row, so leftovers
from the first call cannot hide in the second.  The file is collected last.
"""
import ctypes

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_OP = 2e-5


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


@pytest.fixture(scope="module")
def nf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1710_03197_gb300 as nf
    return nf


def _call_static(nf, plan, y, grid):
    rc = nf.lib.nufft_gridding_static(plan.handle, ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(grid.data_ptr()))
    nf.check(rc, plan.handle)


@pytest.mark.parametrize("name,Nd,Kd,Jd,gen", [
    ("radial2d_256", (256, 256), (512, 512), (6, 6), lambda: W.radial2d_golden(403, 512)),
    ("koosh3d_small", (24, 24, 24), (64, 64, 32), (6, 6, 6), lambda: W.kooshball3d(200, 64)),
])
def test_static_gridding_matches_plan_gridding_on_consecutive_calls(nf, name, Nd, Kd, Jd, gen):
    dev = torch.device("cuda:0")
    om = gen()
    with nf.NufftPlan(torch.from_numpy(om).to(dev), Nd, Kd, Jd) as plan:
        for call in range(2):
            rng = np.random.default_rng(100 + call)
            y = torch.from_numpy((rng.standard_normal(om.shape[0]) + 1j * rng.standard_normal(om.shape[0]))
                                 .astype(np.complex64)).to(dev)
            ref = plan.gridding(y)
            out = torch.full(Kd, float("nan"), dtype=torch.complex64, device=dev)
            _call_static(nf, plan, y, out)
            torch.cuda.synchronize()
            a, b = out.cpu().numpy(), ref.cpu().numpy()
            assert np.all(np.isfinite(a))
            assert _rel(a, b) < TOL_OP, (name, call)


def test_static_gridding_rejects_plans_beyond_its_scratch(nf):
    dev = torch.device("cuda:0")
    om = W.uniform_random_om(40000, 3, seed=7)        # 512 tiles of 21^3 cells: 38 MB of partial tiles
    with nf.NufftPlan(torch.from_numpy(om).to(dev), (64, 64, 64), (128, 128, 128), (6, 6, 6)) as plan:
        y = torch.zeros(om.shape[0], dtype=torch.complex64, device=dev)
        grid = torch.zeros((128, 128, 128), dtype=torch.complex64, device=dev)
        with pytest.raises(nf.NufftError) as ei:
            _call_static(nf, plan, y, grid)
        assert ei.value.code == 1 and "static scratch" in str(ei.value)
