"""Out-of-memory paths, injected on the host.

Every device buffer the library owns is allocated through one wrapper;
nufft_debug_fail_allocation(n) makes the n-th allocation from then on fail as
if the device were full, without calling CUDA.  So these tests reach every
NUFFT_ENOMEM path of plan creation, the solver work space, batch growth and
the Toeplitz set-up on a healthy GPU, and check that each failure returns
NUFFT_ENOMEM, releases what the failed call had allocated
(nufft_debug_device_bytes), leaves no CUDA error behind, and leaves the plan
usable.  Nothing here faults or hangs the GPU.
"""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ENOMEM = 2
DEV = "cuda:0"
Nd, Kd, Jd = (32, 32), (64, 64), (6, 6)


@pytest.fixture(scope="module")
def nf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1710_03197_gb300 as nf
    yield nf
    nf.lib.nufft_debug_fail_allocation(-1)


def _om():
    return torch.from_numpy(W.uniform_random_om(3000, 2, seed=81)).to(DEV)


def _cn(shape, seed):
    rng = np.random.default_rng(seed)
    return torch.from_numpy((rng.standard_normal(shape) + 1j * rng.standard_normal(shape))
                            .astype(np.complex64)).to(DEV)


def _held(nf):
    torch.cuda.synchronize()
    return nf.lib.nufft_debug_device_bytes()


def _device_is_clean():
    torch.cuda.synchronize()
    t = torch.arange(1000, device=DEV, dtype=torch.float32)
    assert float(t.sum().item()) == 499500.0


def test_plan_creation_fails_cleanly_at_every_allocation(nf):
    om = _om()
    failures = 0
    for n in range(0, 64):
        before = _held(nf)
        nf.lib.nufft_debug_fail_allocation(n)
        try:
            plan = nf.NufftPlan(om, Nd, Kd, Jd)
        except nf.NufftError as e:
            assert e.code == ENOMEM, (n, str(e))
            failures += 1
            assert _held(nf) == before, n          # nothing of the failed plan is left
            _device_is_clean()
            continue
        nf.lib.nufft_debug_fail_allocation(-1)
        plan.close()
        assert _held(nf) == before
        break
    else:
        pytest.fail("plan creation made more than 64 allocations")
    assert failures >= 10                            # every plan-owned buffer was reached


def test_solver_work_space_failure_leaves_the_plan_usable(nf):
    om = _om()
    y = _cn(3000, 82)
    with nf.NufftPlan(om, Nd, Kd, Jd) as plan:
        before = _held(nf)
        nf.lib.nufft_debug_fail_allocation(0)
        with pytest.raises(nf.NufftError) as ei:
            plan.solve_cg(y, maxiter=3)
        assert ei.value.code == ENOMEM
        assert _held(nf) == before
        _device_is_clean()
        x1 = plan.solve_cg(y, maxiter=3)             # eager: allocates the work space now
        x2 = plan.solve_cg(y, maxiter=3)             # recorded
        x3 = plan.solve_cg(y, maxiter=3)             # replayed
        ref = oracle.cg(oracle.make_plan(om.cpu().numpy(), Nd, Kd, Jd), y.cpu().numpy(), np.zeros(Nd), 3)
        for x in (x1, x2, x3):
            xx = x.cpu().numpy()
            assert np.linalg.norm(xx - ref) / np.linalg.norm(ref) < 1e-4


def test_batch_growth_failure_leaves_the_plan_usable(nf):
    om = _om()
    xs = _cn((3,) + Nd, 83)
    with nf.NufftPlan(om, Nd, Kd, Jd) as plan:
        y1 = plan.forward(xs[0])
        before = _held(nf)
        for n in range(4):                           # the batched grids, tiles, samples, images
            nf.lib.nufft_debug_fail_allocation(n)
            with pytest.raises(nf.NufftError) as ei:
                plan.forward_batch(xs)
            assert ei.value.code == ENOMEM
            assert _held(nf) == before, n
            _device_is_clean()
            torch.testing.assert_close(plan.forward(xs[0]), y1, rtol=0, atol=0)
        nf.lib.nufft_debug_fail_allocation(-1)
        yb = plan.forward_batch(xs)
        # the batched interpolation is a different kernel from the single one
        # (same arithmetic order, different fusing of multiply-adds)
        assert float(torch.linalg.norm(yb[0] - y1) / torch.linalg.norm(y1)) < 1e-6


def test_toeplitz_set_up_failure_leaves_the_plan_usable(nf):
    om = _om()
    x = _cn(Nd, 84)
    with nf.NufftPlan(om, Nd, Kd, Jd) as plan:
        ref = plan.selfadjoint(x)
        before = _held(nf)
        failures = 0
        for n in range(0, 200):                     # three nested plans: dozens of allocations
            nf.lib.nufft_debug_fail_allocation(n)
            try:
                plan.toeplitz_init()
            except nf.NufftError as e:
                assert e.code == ENOMEM, (n, str(e))
                failures += 1
                assert _held(nf) == before, n
                _device_is_clean()
                torch.testing.assert_close(plan.selfadjoint(x), ref, rtol=0, atol=0)
                continue
            nf.lib.nufft_debug_fail_allocation(-1)
            break
        else:
            pytest.fail("the Toeplitz set-up made more than 200 allocations")
        assert failures >= 10
        t = plan.selfadjoint_toeplitz(x)
        assert float(torch.linalg.norm(t - ref) / torch.linalg.norm(ref)) < 1e-4
