"""nufft_plan_set_trajectory: a plan moved to a new trajectory must behave as a
plan built on it (the same interpolator and sort, hence a bit-identical
forward), through recorded graphs, batch buffers, the trajectory derivative,
frame sets and a discarded Toeplitz kernel; a rejected trajectory leaves the
plan as it was."""
import numpy as np
import pytest

import oracle
import workloads as W
from oracle import extensions as X

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_OP = 2e-5
DEV = "cuda:0"


@pytest.fixture(scope="module")
def nf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1710_03197_gb300 as nf
    return nf


def rel(a, b):
    a, b = np.asarray(a).ravel(), np.asarray(b).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def cn(shape, seed):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def clustered(M, d, seed, width=0.05):
    """All points inside one small region: few tiles, several chunks each."""
    rng = np.random.default_rng(seed)
    return (0.3 + width * rng.standard_normal((M, d))).astype(np.float32)


def _same_plan(a, b):
    ia, ib = a.interpolator(), b.interpolator()
    for u, v in zip(ia, ib):
        if isinstance(u, list):
            for s, t in zip(u, v):
                assert torch.equal(s, t)
        else:
            assert torch.equal(u, v)
    assert a.info()["nchunks"] == b.info()["nchunks"]


@pytest.mark.parametrize("Nd,Kd,Jd,M", [((32, 32), (64, 64), (6, 6), 3000), ((16, 16, 16), (32, 32, 32), (6, 6, 6), 4000),
                                        ((40,), (128,), (6,), 900)])
def test_set_trajectory_equals_a_fresh_plan(nf, Nd, Kd, Jd, M):
    d = len(Nd)
    trajs = [clustered(M, d, 1), W.uniform_random_om(M, d, seed=2), clustered(M, d, 3, 0.5)]
    x = cn(Nd, 4)
    xd = dev(x)
    y = torch.empty(M, dtype=torch.complex64, device=DEV)
    with nf.NufftPlan(dev(trajs[0]), Nd, Kd, Jd) as plan:
        for _ in range(3):                         # eager, record, replay on the first trajectory
            plan.forward(xd, y)
        xb = dev(np.stack([cn(Nd, 5), cn(Nd, 6)]))
        plan.selfadjoint_batch(xb)                 # batch buffers sized for the first chunk list
        for om in trajs[1:] + trajs[:1]:
            plan.set_trajectory(dev(om))
            with nf.NufftPlan(dev(om), Nd, Kd, Jd) as fresh:
                _same_plan(plan, fresh)
                for _ in range(3):                 # the dropped graphs are recorded again
                    plan.forward(xd, y)
                    assert torch.equal(y, fresh.forward(xd))
                ref = oracle.make_plan(om, Nd, Kd, Jd)
                assert rel(host(y), oracle.forward(ref, x)) < TOL_OP
                yh = cn(M, 7)
                assert rel(host(plan.adjoint(dev(yh))), oracle.adjoint(ref, yh)) < TOL_OP
                got = host(plan.selfadjoint_batch(xb))
                for b in range(2):
                    assert rel(got[b], host(fresh.selfadjoint(xb[b].contiguous()))) < 1e-6


def test_set_trajectory_recomputes_the_derivative(nf):
    Nd, Kd, Jd = (32, 32), (64, 64), (6, 6)
    om1, om2 = W.spiral2d(4, 300), W.uniform_random_om(1200, 2, seed=8)
    x, g = cn(Nd, 9), cn(1200, 10)
    with nf.NufftPlan(dev(om1[:1200]), Nd, Kd, Jd) as plan:
        plan.trajectory_gradient(dev(x), dev(g))   # derivative coefficients now kept by the plan
        plan.set_trajectory(dev(om2))
        gom = host(plan.trajectory_gradient(dev(x), dev(g)))
        assert rel(gom, X.trajectory_gradient(oracle.make_plan(om2, Nd, Kd, Jd), x, g)) < 1e-4


def test_set_trajectory_discards_the_toeplitz_kernel(nf):
    Nd, Kd, Jd = (32, 32), (64, 64), (6, 6)
    om1, om2 = W.uniform_random_om(1000, 2, seed=11), W.uniform_random_om(1000, 2, seed=12)
    with nf.NufftPlan(dev(om1), Nd, Kd, Jd) as plan:
        plan.toeplitz_init()
        plan.set_normal_operator(True)
        plan.set_trajectory(dev(om2))
        with pytest.raises(nf.NufftError):
            plan.selfadjoint_toeplitz(dev(cn(Nd, 13)))
        y = cn(1000, 14)
        ref = oracle.make_plan(om2, Nd, Kd, Jd)
        x = plan.solve_cg(dev(y), torch.zeros(Nd, dtype=torch.complex64, device=DEV), maxiter=5)
        assert rel(host(x), oracle.cg(ref, y, np.zeros(Nd), 5)) < 1e-4   # V^H V again, new points


def test_rejected_trajectory_leaves_the_plan_unchanged(nf):
    Nd, Kd, Jd = (32, 32), (64, 64), (6, 6)
    om = W.uniform_random_om(800, 2, seed=15)
    bad = om.copy()
    bad[17, 1] = np.nan
    x = dev(cn(Nd, 16))
    with nf.NufftPlan(dev(om), Nd, Kd, Jd) as plan:
        before = host(plan.forward(x))
        with pytest.raises(nf.NufftError):
            plan.set_trajectory(dev(bad))
        with pytest.raises(ValueError):
            plan.set_trajectory(dev(om[:700]))
        assert np.array_equal(host(plan.forward(x)), before)


def test_frame_set_follows_a_moved_plan(nf):
    """A frame set's recorded graph is re-recorded after one of its plans moves."""
    Nd, Kd, Jd = (32, 32), (64, 64), (6, 6)
    frames = W.dynamic_radial_frames(3, 64)
    nc = 2
    coils = dev(W.coil_maps(nc, Nd))
    xs = dev(cn((len(frames),) + Nd, 17))
    plans = [nf.NufftPlan(dev(om), Nd, Kd, Jd) for om in frames]
    try:
        with nf.NufftFrames(plans) as fs:
            out = torch.empty_like(xs)
            for _ in range(3):                     # eager, record, replay
                fs.selfadjoint_multicoil(coils, xs, out)
            moved = clustered(frames[1].shape[0], 2, 18, 0.4)
            plans[1].set_trajectory(dev(moved))
            for _ in range(3):
                out.zero_()
                fs.selfadjoint_multicoil(coils, xs, out)
                got = host(out)
                for f, p in enumerate(plans):
                    assert rel(got[f], host(p.selfadjoint_multicoil(coils, xs[f]))) < 1e-5
    finally:
        for p in plans:
            p.close()
