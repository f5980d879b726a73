"""GPU vs oracle for density compensation (Eqs. 5-6), the paper's k-space CG
(Eqs. 7-9) and the multi-coil operators and CG (Eqs. 32-33), through the C ABI.

Tolerances: 2e-5 relative L2 for operators, 1e-4 after solver iterations
where the iteration is stable to FP32 rounding (checked on the oracle:
density compensation and multi-coil CG move by ~2e-6 under 1e-6 operator
noise, the k-space CG by ~1e-6 at 10 iterations on the overdetermined case).
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from oracle import extensions as X

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_OP = 2e-5
TOL_SOLVER = 1e-4
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
    return t.cpu().numpy()


def _cartesian_om(N):
    k = 2 * math.pi * (np.arange(N) - N // 2) / N
    g0, g1 = np.meshgrid(k, k, indexing="ij")
    return np.stack([g0.ravel(), g1.ravel()], 1).astype(np.float32)


@pytest.mark.parametrize("traj,iters", [("cartesian", 1), ("cartesian", 3), ("radial", 1), ("radial", 3),
                                        ("radial", 5)])
def test_density_compensation_matches_oracle(nf, traj, iters):
    if traj == "cartesian":
        om, Nd, Kd = _cartesian_om(16), (16, 16), (32, 32)
    else:
        om, Nd, Kd = W.radial2d_uniform(32, 64), (32, 32), (64, 64)
    ref = oracle.make_plan(om, Nd, Kd, (6, 6))
    with nf.NufftPlan(dev(om), Nd, Kd, (6, 6)) as plan:
        w = host(plan.density_compensation(iters))
    assert rel(w, X.density_compensation(ref, iters)) < TOL_SOLVER


def test_gridding_recon_matches_oracle(nf):
    om = W.radial2d_golden(60, 128)
    Nd, Kd = (64, 64), (128, 128)
    ref = oracle.make_plan(om, Nd, Kd, (6, 6))
    y = cn(om.shape[0], 3)
    w = np.abs(cn(om.shape[0], 4)).astype(np.float32)
    with nf.NufftPlan(dev(om), Nd, Kd, (6, 6)) as plan:
        x = host(plan.gridding_recon(dev(y), dev(w)))
    assert rel(x, X.gridding_recon(ref, y, w)) < TOL_OP


def _overdetermined():
    Nd, Kd = (8, 8), (16, 16)
    om = W.uniform_random_om(600, 2, seed=9)
    ref = oracle.make_plan(om, Nd, Kd, (6, 6))
    xt = cn(Nd, 5)
    return Nd, Kd, om, ref, xt, oracle.forward(ref, xt).astype(np.complex64)


def test_kspace_cg_matches_oracle(nf):
    Nd, Kd, om, ref, xt, y = _overdetermined()
    with nf.NufftPlan(dev(om), Nd, Kd, (6, 6)) as plan:
        x = host(plan.solve_cg_kspace(dev(y), maxiter=10))
    assert rel(x, X.cg_kspace(ref, y, 10)) < TOL_SOLVER


def test_kspace_cg_recovers_the_image(nf):
    """Consistent, overdetermined data: many iterations return x itself."""
    Nd, Kd, om, ref, xt, y = _overdetermined()
    with nf.NufftPlan(dev(om), Nd, Kd, (6, 6)) as plan:
        x = host(plan.solve_cg_kspace(dev(y), maxiter=400))
    assert rel(x, xt) < 5e-3


def _multicoil_case(nc=4):
    Nd, Kd = (32, 32), (64, 64)
    om = W.uniform_random_om(1500, 2, seed=6)
    ref = oracle.make_plan(om, Nd, Kd, (6, 6))
    coils = W.coil_maps(nc, Nd)
    return Nd, Kd, om, ref, coils


def test_multicoil_operators_match_oracle(nf):
    Nd, Kd, om, ref, coils = _multicoil_case()
    x = cn(Nd, 6)
    y = cn(4 * om.shape[0], 7)
    with nf.NufftPlan(dev(om), Nd, Kd, (6, 6)) as plan:
        cd = dev(coils)
        yf = host(plan.forward_multicoil(cd, dev(x)))
        xa = host(plan.adjoint_multicoil(cd, dev(y)))
        xs = host(plan.selfadjoint_multicoil(cd, dev(x)))
    c128 = coils.astype(np.complex128)
    assert rel(yf, X.forward_multicoil(ref, c128, x)) < TOL_OP
    assert rel(xa, X.adjoint_multicoil(ref, c128, y)) < TOL_OP
    assert rel(xs, X.selfadjoint_multicoil(ref, c128, x)) < TOL_OP


def test_multicoil_cg_matches_oracle(nf):
    Nd, Kd, om, ref, coils = _multicoil_case()
    c128 = coils.astype(np.complex128)
    y = X.forward_multicoil(ref, c128, W.complex_normal_image(Nd)).astype(np.complex64)
    with nf.NufftPlan(dev(om), Nd, Kd, (6, 6)) as plan:
        x = host(plan.solve_cg_multicoil(dev(coils), dev(y), maxiter=20))
    assert rel(x, X.cg_multicoil(ref, c128, y, np.zeros(Nd), 20)) < TOL_SOLVER


def test_multicoil_full_size_frame_matches_oracle(nf):
    """The batched multi-coil dynamic workload at its real size, one frame: the
    first golden-angle frame of the series (256^2 image, 512^2 grid, J = 6x6)
    with 4 of its coil maps; the normal operator (Eq. 33) and the adjoint of
    the stacked coil data against the oracle."""
    frames = W.dynamic_radial_frames(8, 512)
    om = frames[0]
    Nd, Kd = (256, 256), (512, 512)
    nc = 4
    coils = W.coil_maps(32, Nd)[:nc]
    ref = oracle.make_plan(om, Nd, Kd, (6, 6))
    x = W.ellipse_phantom(256)
    y = cn(nc * om.shape[0], 31)
    c128 = coils.astype(np.complex128)
    with nf.NufftPlan(dev(om), Nd, Kd, (6, 6)) as plan:
        cd = dev(coils)
        got = host(plan.selfadjoint_multicoil(cd, dev(x)))
        assert rel(got, X.selfadjoint_multicoil(ref, c128, x.astype(np.complex128))) < TOL_OP
        assert rel(host(plan.adjoint_multicoil(cd, dev(y))), X.adjoint_multicoil(ref, c128, y)) < TOL_OP


def test_multicoil_rejects_bad_coil_shape(nf):
    Nd, Kd, om, ref, coils = _multicoil_case()
    with nf.NufftPlan(dev(om), Nd, Kd, (6, 6)) as plan:
        with pytest.raises(ValueError):
            plan.forward_multicoil(dev(coils[:, :16]), dev(cn(Nd, 1)))
        assert nf.lib.nufft_forward_multicoil(plan.handle, None, 4, None, None) == 1     # EINVAL


@pytest.mark.parametrize("nb", [5, 19])   # 19: batch groups of 8, 8 and 3 in the grouped kernels
@pytest.mark.parametrize("name,Nd,Kd,Jd,gen", [
    ("2d", (32, 32), (64, 64), (6, 6), lambda: W.radial2d_golden(30, 64)),
    ("2d_oddJ", (32, 32), (64, 64), (5, 7), lambda: W.uniform_random_om(1800, 2, seed=26)),
    ("3d", (16, 16, 16), (32, 32, 32), (6, 6, 6), lambda: W.kooshball3d(80, 32)),
])
def test_batched_operators_equal_single_calls(nf, name, Nd, Kd, Jd, gen, nb):
    om = gen()
    xs = cn((nb,) + Nd, 21)
    ys = cn((nb, om.shape[0]), 22)
    ref = oracle.make_plan(om, Nd, Kd, Jd)
    with nf.NufftPlan(dev(om), Nd, Kd, Jd) as plan:
        yb = host(plan.forward_batch(dev(xs)))
        xb = host(plan.adjoint_batch(dev(ys)))
        sb = host(plan.selfadjoint_batch(dev(xs)))
        for b in range(nb):
            assert rel(yb[b], host(plan.forward(dev(xs[b])))) < 1e-6
            assert rel(xb[b], host(plan.adjoint(dev(ys[b])))) < 1e-6
            assert rel(sb[b], host(plan.selfadjoint(dev(xs[b])))) < 1e-6
            assert rel(yb[b], oracle.forward(ref, xs[b])) < TOL_OP
            assert rel(xb[b], oracle.adjoint(ref, ys[b])) < TOL_OP


def test_single_coil_multicoil_equals_plain_operators(nf):
    Nd, Kd, om, ref, coils = _multicoil_case(nc=1)
    x = cn(Nd, 8)
    y = cn(om.shape[0], 9)
    with nf.NufftPlan(dev(om), Nd, Kd, (6, 6)) as plan:
        cd = dev(coils)
        c128 = coils.astype(np.complex128)
        assert rel(host(plan.forward_multicoil(cd, dev(x))), X.forward_multicoil(ref, c128, x)) < TOL_OP
        assert rel(host(plan.adjoint_multicoil(cd, dev(y))), X.adjoint_multicoil(ref, c128, y)) < TOL_OP
        assert rel(host(plan.selfadjoint_multicoil(cd, dev(x))), X.selfadjoint_multicoil(ref, c128, x)) < TOL_OP


@pytest.mark.parametrize("Nd,gen", [
    ((32, 32), lambda: W.radial2d_golden(40, 64)),
    ((64, 48), lambda: W.uniform_random_om(4000, 2, seed=41)),
    ((12, 16, 8), lambda: W.kooshball3d(60, 32)),
    ((40,), lambda: W.uniform_random_om(300, 1, seed=42)),
])
def test_toeplitz_selfadjoint_matches_oracle(nf, Nd, gen):
    om = gen()
    d = len(Nd)
    Kd = tuple(2 * n if 2 * n >= 16 else 16 for n in Nd)
    Kd = tuple(1 << (k - 1).bit_length() for k in Kd)
    Jd = (6,) * d
    ref = oracle.make_plan(om, Nd, Kd, Jd)
    T = X.toeplitz_kernel(ref)
    x = cn(Nd, 43)
    with nf.NufftPlan(dev(om), Nd, Kd, Jd) as plan:
        plan.toeplitz_init()
        out = host(plan.selfadjoint_toeplitz(dev(x)))
    assert rel(out, X.selfadjoint_toeplitz(ref, T, x)) < TOL_OP
    assert rel(out, oracle.selfadjoint(ref, x)) < 1e-4


def test_solvers_in_toeplitz_mode_match_oracle(nf):
    Nd, Kd, Jd = (64, 64), (128, 128), (6, 6)
    om = W.uniform_random_om(3 * 64 * 64, 2, seed=3)
    ref = oracle.make_plan(om, Nd, Kd, Jd)
    T = X.toeplitz_kernel(ref)
    y = oracle.forward(ref, W.complex_normal_image(Nd)).astype(np.complex64)
    from oracle.solvers import cg_solve
    x_ref = cg_solve(lambda v: X.selfadjoint_toeplitz(ref, T, v), oracle.adjoint(ref, y), np.zeros(Nd), 30)
    coils = W.coil_maps(4, Nd)
    c128 = coils.astype(np.complex128)
    ymc = X.forward_multicoil(ref, c128, W.complex_normal_image(Nd)).astype(np.complex64)
    mc_ref = cg_solve(lambda v: sum(np.conj(c) * X.selfadjoint_toeplitz(ref, T, c * v) for c in c128),
                      X.adjoint_multicoil(ref, c128, ymc), np.zeros(Nd), 15)
    with nf.NufftPlan(dev(om), Nd, Kd, Jd) as plan:
        plan.toeplitz_init()
        plan.set_normal_operator(True)
        x = host(plan.solve_cg(dev(y), maxiter=30))
        xm = host(plan.solve_cg_multicoil(dev(coils), dev(ymc), maxiter=15))
        plan.set_normal_operator(False)
        x_grid = host(plan.solve_cg(dev(y), maxiter=30))
    assert rel(x, x_ref) < TOL_SOLVER
    assert rel(xm, mc_ref) < TOL_SOLVER
    assert rel(x_grid, oracle.cg(ref, y, np.zeros(Nd), 30)) < TOL_SOLVER


def test_toeplitz_errors(nf):
    om = W.uniform_random_om(100, 2, seed=44)
    with nf.NufftPlan(dev(om), (16, 16), (32, 32), (6, 6)) as plan:
        with pytest.raises(nf.NufftError):
            plan.selfadjoint_toeplitz(dev(cn((16, 16), 1)))
        with pytest.raises(nf.NufftError):
            plan.set_normal_operator(True)
    with nf.NufftPlan(dev(om), (512, 16), (1024, 32), (6, 6)) as plan:
        with pytest.raises(nf.NufftError):
            plan.toeplitz_init()                 # period P = 1024, grid 2P = 2048 exceeds the FFT sizes


def test_frame_set_multicoil_normal_operator(nf):
    """A frame set records every frame's multi-coil normal operator (Eq. 33 per
    frame, uneven point counts) as one graph with concurrent branches: eager,
    recording and replayed calls match the per-frame calls and the oracle."""
    Nd, Kd, Jd = (32, 32), (64, 64), (6, 6)
    frames = W.dynamic_radial_frames(4, 64)
    nc = 3
    coils = W.coil_maps(nc, Nd)
    xs = cn((len(frames),) + Nd, 81)
    plans = [nf.NufftPlan(dev(om), Nd, Kd, Jd) for om in frames]
    try:
        ref = [X.selfadjoint_multicoil(oracle.make_plan(om, Nd, Kd, Jd), coils.astype(np.complex128), xs[f])
               for f, om in enumerate(frames)]
        cd, xd = dev(coils), dev(xs)
        single = [host(p.selfadjoint_multicoil(cd, xd[f])) for f, p in enumerate(plans)]
        with nf.NufftFrames(plans) as fs:
            out = torch.empty_like(xd)
            for _ in range(4):                   # eager, record, replay, replay
                out.zero_()
                fs.selfadjoint_multicoil(cd, xd, out)
                got = host(out)
                for f in range(len(frames)):
                    assert rel(got[f], single[f]) < 1e-5
                    assert rel(got[f], ref[f]) < TOL_OP
            with pytest.raises(nf.NufftError):
                fs.selfadjoint_multicoil(cd, xd, xd)     # aliasing rejected
    finally:
        for p in plans:
            p.close()


def test_frame_set_rejects_mismatched_plans(nf):
    a = nf.NufftPlan(dev(W.uniform_random_om(200, 2, seed=82)), (16, 16), (32, 32), (6, 6))
    b = nf.NufftPlan(dev(W.uniform_random_om(200, 2, seed=83)), (32, 32), (64, 64), (6, 6))
    try:
        with pytest.raises(nf.NufftError):
            nf.NufftFrames([a, b])
        with pytest.raises(nf.NufftError):
            nf.NufftFrames([a, a])
    finally:
        a.close()
        b.close()
