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
    ("uniform1d_J6", (200,), (512,), (6,), lambda: W.uniform_random_om(5000, 1, seed=5)),
    ("uniform1d_J5", (96,), (256,), (5,), lambda: W.uniform_random_om(3000, 1, seed=6)),
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


# A 2D plan on a 1024^2 grid has 64 x 64 tiles of 16^2 cells; each partial tile
# is 21^2 cells of 8 bytes (J = 6), 3528 bytes, so 16 MiB holds 4755 of them.
# One point per tile gives 4096 chunks; a tile with 257 points gives two.
_PAD_BYTES = 21 * 21 * 8
_LIMIT = 16 << 20


def _om_with_chunks(nchunks):
    K, T, J = 1024, 16, 6
    gamma = 2 * np.pi / K
    extra = nchunks - 64 * 64                 # tiles with a second chunk
    rng = np.random.default_rng(8)
    pts = []
    for t in range(64 * 64):
        c = np.array([t // 64, t % 64]) * T + T // 2       # first neighbour at the tile centre
        n = 257 if t < extra else 1
        u = c + J / 2 - 1 + 0.5 + rng.uniform(-0.4, 0.4, size=(n, 2))
        pts.append(u * gamma)
    return np.concatenate(pts).astype(np.float32)


def test_static_gridding_accepts_a_plan_just_under_the_limit_and_rejects_one_over(nf):
    dev = torch.device("cuda:0")
    assert 4755 * _PAD_BYTES <= _LIMIT < 4756 * _PAD_BYTES
    for nchunks, fits in ((4755, True), (4756, False)):
        om = _om_with_chunks(nchunks)
        with nf.NufftPlan(torch.from_numpy(om).to(dev), (512, 512), (1024, 1024), (6, 6)) as plan:
            assert plan.info()["nchunks"] == nchunks
            rng = np.random.default_rng(9)
            y = torch.from_numpy((rng.standard_normal(om.shape[0]) + 1j * rng.standard_normal(om.shape[0]))
                                 .astype(np.complex64)).to(dev)
            out = torch.full((1024, 1024), float("nan"), dtype=torch.complex64, device=dev)
            if fits:
                for _ in range(2):
                    _call_static(nf, plan, y, out)
                    ref = plan.gridding(y)
                    torch.cuda.synchronize()
                    assert _rel(out.cpu().numpy(), ref.cpu().numpy()) < TOL_OP
            else:
                with pytest.raises(nf.NufftError) as ei:
                    _call_static(nf, plan, y, out)
                assert ei.value.code == 1 and "static scratch" in str(ei.value)


def test_static_gridding_runs_on_the_plans_device(nf):
    """A plan made on device 1 and called while device 0 is current uses
    device 1's array and stream, and leaves device 0 current."""
    if torch.cuda.device_count() < 2:
        pytest.skip("needs two CUDA devices")
    dev = torch.device("cuda:1")
    om = W.uniform_random_om(3000, 2, seed=10)
    with torch.cuda.device(1):
        plan = nf.NufftPlan(torch.from_numpy(om).to(dev), (32, 32), (64, 64), (6, 6))
        y = torch.from_numpy(np.random.default_rng(11).standard_normal(3000).astype(np.complex64)).to(dev)
        ref = plan.gridding(y)
        torch.cuda.synchronize(dev)
    out = torch.full((64, 64), float("nan"), dtype=torch.complex64, device=dev)
    with torch.cuda.device(0):
        _call_static(nf, plan, y, out)
        assert torch.cuda.current_device() == 0
    torch.cuda.synchronize(dev)
    assert _rel(out.cpu().numpy(), ref.cpu().numpy()) < TOL_OP
    with torch.cuda.device(1):
        plan.close()
