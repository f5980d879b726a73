"""Pins of the oracle's density compensation, k-space CG and multi-coil operators."""
import math

import numpy as np

import oracle
import workloads as W
from oracle import extensions as X

RNG = np.random.default_rng(77)


def _cn(shape):
    return RNG.standard_normal(shape) + 1j * RNG.standard_normal(shape)


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


def _cartesian(N, K):
    k = 2 * math.pi * (np.arange(N) - N // 2) / N
    g0, g1 = np.meshgrid(k, k, indexing="ij")
    om = np.stack([g0.ravel(), g1.ravel()], 1)
    return oracle.make_plan(om, (N, N), (K, K), (6, 6))


def test_density_compensation_is_uniform_on_a_cartesian_grid():
    """Full Cartesian sampling: A A^H = N^d I, so one step gives w = 1/N^d."""
    p = _cartesian(16, 32)
    w = X.density_compensation(p, 1)
    assert np.abs(w * 256 - 1).max() < 1e-4
    w3 = X.density_compensation(p, 3)
    assert np.abs(w3 * 256 - 1).max() < 1e-4


def test_gridding_recon_inverts_cartesian_sampling():
    p = _cartesian(16, 32)
    x = _cn((16, 16))
    w = X.density_compensation(p, 1)
    assert _rel(X.gridding_recon(p, oracle.forward(p, x), w), x) < 1e-4


def test_density_compensation_first_steps_reduce_the_residual():
    """The iteration drives |A A^H w| towards 1 (its fixed point) over its first
    steps: the typical (median) deviation falls from step 1 to step 5."""
    om = W.radial2d_uniform(32, 64)
    p = oracle.make_plan(om, (32, 32), (64, 64), (6, 6))
    def resid(w):
        return np.median(np.abs(np.abs(oracle.forward(p, oracle.adjoint(p, w.astype(complex)))) - 1))
    r0 = resid(np.ones(om.shape[0]))
    r1 = resid(X.density_compensation(p, 1))
    r5 = resid(X.density_compensation(p, 5))
    assert r1 < 1e-3 * r0 and r5 < r1


def test_VHV_is_hermitian():
    om = W.uniform_random_om(300, 2, seed=3)
    p = oracle.make_plan(om, (8, 8), (16, 16), (6, 6))
    a, b = _cn((16, 16)), _cn((16, 16))
    lhs, rhs = np.vdot(X.VHV(p, a), b), np.vdot(a, X.VHV(p, b))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_kspace_cg_recovers_the_image_from_consistent_overdetermined_data():
    """M = 600 > K^d = 256: V has full column rank, y = A x gives k = F S x,
    and S^{-1} F^{-1} k returns x."""
    Nd, Kd = (8, 8), (16, 16)
    om = W.uniform_random_om(600, 2, seed=9)
    p = oracle.make_plan(om, Nd, Kd, (6, 6))
    xt = _cn(Nd)
    x = X.cg_kspace(p, oracle.forward(p, xt), 400)
    assert _rel(x, xt) < 1e-4


def test_multicoil_with_a_unit_coil_equals_single_coil():
    om = W.uniform_random_om(200, 2, seed=4)
    p = oracle.make_plan(om, (16, 16), (32, 32), (6, 6))
    c = np.ones((1, 16, 16), dtype=complex)
    x, y = _cn((16, 16)), _cn(200)
    np.testing.assert_allclose(X.forward_multicoil(p, c, x), oracle.forward(p, x), atol=1e-12)
    np.testing.assert_allclose(X.adjoint_multicoil(p, c, y), oracle.adjoint(p, y), atol=1e-10)
    np.testing.assert_allclose(X.selfadjoint_multicoil(p, c, x), oracle.selfadjoint(p, x), atol=1e-9)


def test_multicoil_adjoint_identity_and_normal_operator():
    om = W.uniform_random_om(150, 2, seed=5)
    p = oracle.make_plan(om, (12, 12), (24, 24), (6, 6))
    coils = W.coil_maps(4, (12, 12)).astype(complex)
    x, y = _cn((12, 12)), _cn(4 * 150)
    lhs = np.vdot(X.forward_multicoil(p, coils, x), y)
    rhs = np.vdot(x, X.adjoint_multicoil(p, coils, y))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    np.testing.assert_allclose(X.selfadjoint_multicoil(p, coils, x),
                               X.adjoint_multicoil(p, coils, X.forward_multicoil(p, coils, x)), atol=1e-9)


def test_multicoil_cg_reaches_dense_solution():
    Nd = (8, 8)
    om = W.uniform_random_om(80, 2, seed=6)            # one coil alone is underdetermined
    p = oracle.make_plan(om, Nd, (16, 16), (6, 6))
    coils = W.coil_maps(4, Nd).astype(complex)
    A = np.stack([X.forward_multicoil(p, coils, e.reshape(Nd)) for e in np.eye(64)], axis=1)
    y = A @ _cn(64)
    x_ls = np.linalg.solve(A.conj().T @ A, A.conj().T @ y).reshape(Nd)
    x = X.cg_multicoil(p, coils, y, np.zeros(Nd), 200)
    assert _rel(x, x_ls) < 1e-6


def test_coil_maps_are_smooth_and_distinct():
    c = W.coil_maps(8, (32, 32))
    assert c.shape == (8, 32, 32)
    mags = np.abs(c).reshape(8, -1)
    assert np.all(mags.max(1) <= 1.0 + 1e-6) and np.all(mags.max(1) > 0.5)
    # neighbouring pixels differ little (smooth), different coils peak in different places
    assert np.abs(np.diff(np.abs(c), axis=-1)).max() < 0.1
    assert len(set(int(np.argmax(m)) for m in mags)) == 8


def _fd_case():
    Nd, Kd, Jd = (16, 16), (32, 32), (6, 6)
    om = W.uniform_random_om(200, 2, seed=12).astype(np.float64)
    x = W.complex_normal_image(Nd).astype(complex)
    return Nd, Kd, Jd, om, x


def test_trajectory_derivative_matches_central_differences():
    """FP64 central differences, step 1e-6, on points away from cell boundaries
    (the neighbourhood jumps there and the interpolator is discontinuous)."""
    Nd, Kd, Jd, om, x = _fd_case()
    p = oracle.make_plan(om, Nd, Kd, Jd)
    dy = X.forward_domega(p, x)
    h = 1e-6
    u = om / (2 * math.pi / Kd[0])
    away = (np.abs(u - np.round(u)) > 1e-3).all(1)
    for a in range(2):
        op, omn = om.copy(), om.copy()
        op[:, a] += h
        omn[:, a] -= h
        fd = (oracle.forward(oracle.make_plan(op, Nd, Kd, Jd), x) -
              oracle.forward(oracle.make_plan(omn, Nd, Kd, Jd), x)) / (2 * h)
        assert _rel(dy[away, a], fd[away]) < 1e-7


def test_trajectory_derivative_approximates_the_exact_nudft_derivative():
    Nd, Kd, Jd, om, x = _fd_case()
    p = oracle.make_plan(om, Nd, Kd, Jd)
    dy = X.forward_domega(p, x)
    t = np.arange(16) - 8
    T0, T1 = np.meshgrid(t, t, indexing="ij")
    E = np.exp(-1j * (om[:, :1] * T0.ravel()[None] + om[:, 1:] * T1.ravel()[None]))
    for a, Ta in enumerate((T0, T1)):
        exact = (E * (-1j * Ta.ravel()[None])) @ x.ravel()
        assert _rel(dy[:, a], exact) < 1e-4


def test_trajectory_gradient_of_a_quadratic_loss():
    """L = ||A(w) x - y0||^2 has dL/dw = Re(conj(2 (A x - y0)) dy/dw); checked by FD on L."""
    Nd, Kd, Jd, om, x = _fd_case()
    y0 = _cn(om.shape[0])
    p = oracle.make_plan(om, Nd, Kd, Jd)
    r = oracle.forward(p, x) - y0
    g = X.trajectory_gradient(p, x, 2 * r)
    h = 1e-6
    m, a = 17, 1
    op, omn = om.copy(), om.copy()
    op[m, a] += h
    omn[m, a] -= h
    L = lambda o: np.sum(np.abs(oracle.forward(oracle.make_plan(o, Nd, Kd, Jd), x) - y0) ** 2)
    assert abs((L(op) - L(omn)) / (2 * h) - g[m, a]) < 1e-6 * abs(g[m, a]) + 1e-8


def test_toeplitz_normal_operator_matches_exact_nudft_normal_operator():
    for Nd in [(16, 16), (8, 8, 8), (24,)]:
        d = len(Nd)
        om = W.uniform_random_om(300, d, seed=3)
        p = oracle.make_plan(om, Nd, tuple(2 * n for n in Nd), (6,) * d)
        T = X.toeplitz_kernel(p)
        x = _cn(Nd)
        exact = oracle.nudft_adjoint(om, oracle.nudft_forward(om, x), Nd)
        assert _rel(X.selfadjoint_toeplitz(p, T, x), exact) < 1e-4
        assert _rel(X.selfadjoint_toeplitz(p, T, x), oracle.selfadjoint(p, x)) < 1e-4


def test_toeplitz_normal_operator_is_hermitian_to_the_nufft_error():
    """t[-D] = conj(t[D]) holds for the exact sum; the kernel computed by the
    NUFFT keeps it to the NUFFT's accuracy (~1e-6 relative here)."""
    om = W.radial2d_uniform(16, 32)
    p = oracle.make_plan(om, (16, 16), (32, 32), (6, 6))
    T = X.toeplitz_kernel(p)
    a, b = _cn((16, 16)), _cn((16, 16))
    lhs = np.vdot(X.selfadjoint_toeplitz(p, T, a), b)
    rhs = np.vdot(a, X.selfadjoint_toeplitz(p, T, b))
    assert abs(lhs - rhs) < 1e-5 * abs(lhs)
