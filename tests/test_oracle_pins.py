"""Pins of the FP64 oracle against facts fixed outside the oracle itself.

Each test ties one oracle function to something independent: the exact NUDFT
(brute force), the adjoint identity, closed forms, a least-squares definition
solved by LAPACK on the explicit matrix, numerical quadrature, and dense
solves.  A dropped term, wrong sign, wrong centring, transposed operand or
wrong offset in the oracle fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

import oracle
import workloads as W
from oracle.minmax import centred_coords

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
RNG = np.random.default_rng(1234)


def _cn(shape):
    return RNG.standard_normal(shape) + 1j * RNG.standard_normal(shape)


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


# ---------------------------------------------------------------- interpolator

@pytest.mark.parametrize("N,K,J", [(16, 32, 6), (32, 64, 6), (20, 40, 5), (16, 24, 4)])
def test_scaling_matches_kb_fourier_transform_by_quadrature(N, K, J):
    """s_n is 1 / (Fourier transform of the KB kernel of width J, alpha = 2.34 J)."""
    from scipy.integrate import quad
    from scipy.special import i0
    a = 2.34 * J

    def ft(t):
        f = lambda u: i0(a * math.sqrt(max(0.0, 1.0 - (2.0 * u / J) ** 2))) * math.cos(2 * math.pi * u * t / K)
        return quad(f, -J / 2, J / 2, limit=200, epsabs=1e-13, epsrel=1e-13)[0]

    ref = np.array([1.0 / ft(t) for t in centred_coords(N)])
    ref /= ref.max()
    np.testing.assert_allclose(oracle.kb_scaling_1d(N, K, J), ref, rtol=0, atol=1e-12)


@pytest.mark.parametrize("J", [4, 5, 6, 7])
def test_offsets_bracket_the_frequency(J):
    K = 32
    gamma = 2 * math.pi / K
    om = np.concatenate([np.linspace(-math.pi, math.pi, 997), [0.0, -math.pi, gamma * 3, -gamma * 5]])
    k0 = oracle.offsets_1d(om, K, J)
    u = om / gamma
    for m in range(om.size):
        nb = k0[m] + np.arange(1, J + 1)                     # neighbours (unwrapped)
        # every neighbour within J/2 cells of the frequency, and they are the J nearest
        dist = np.abs(nb - u[m])
        assert dist.max() <= J / 2 + 1e-12
        others = np.concatenate([np.arange(nb[0] - 3, nb[0]), np.arange(nb[-1] + 1, nb[-1] + 4)])
        assert np.abs(others - u[m]).min() >= dist.max() - 1e-12


@pytest.mark.parametrize("N,K,J", [(16, 32, 6), (12, 24, 5), (16, 32, 4)])
def test_minmax_coefficients_are_least_squares_solution(N, K, J):
    """c = argmin ||b - A c||_2 on the explicit N x J matrix (LAPACK lstsq)."""
    s = oracle.kb_scaling_1d(N, K, J)
    t = centred_coords(N)
    gamma = 2 * math.pi / K
    om = np.array([-3.0, -1.234, 0.0, 0.05, 1.7, 3.1])
    k0, c, _ = oracle.minmax_coefficients_1d(om, N, K, J)
    for m in range(om.size):
        A = s[:, None] * np.exp(-1j * gamma * (k0[m] + np.arange(1, J + 1))[None, :] * t[:, None])
        b = np.exp(-1j * om[m] * t)
        c_ls = np.linalg.lstsq(A, b, rcond=None)[0]
        np.testing.assert_allclose(c[m], c_ls, rtol=0, atol=1e-9 * np.abs(c_ls).max())
        # optimality: no perturbation lowers the worst-case error
        e0 = np.linalg.norm(b - A @ c[m])
        for _ in range(5):
            dc = 1e-3 * _cn(J)
            assert np.linalg.norm(b - A @ (c[m] + dc)) >= e0


@pytest.mark.parametrize("N,K,J", [(16, 32, 6), (12, 24, 5), (32, 32, 4)])
def test_minmax_coefficients_depend_only_on_the_offset(N, K, J):
    """Shifting w by whole grid steps (gamma) shifts the neighbourhood by the
    same number of cells and leaves the coefficients unchanged: they depend on
    w only through delta = w / gamma - k0 - J/2 in [0, 1), so one smooth
    function of delta per dimension describes every point."""
    gamma = 2 * math.pi / K
    base = np.array([-2.9, -1.234, 0.0, 0.05, 1.0 / 3.0, 1.7])
    k0, c, _ = oracle.minmax_coefficients_1d(base, N, K, J)
    delta = base / gamma - k0 - J / 2
    assert np.all((delta >= 0) & (delta < 1))
    for shift in (1, 3, -5):
        k1, c1, _ = oracle.minmax_coefficients_1d(base + shift * gamma, N, K, J)
        np.testing.assert_array_equal(k1, k0 + shift)
        np.testing.assert_allclose(c1, c, rtol=0, atol=1e-10 * np.abs(c).max())


def test_separable_coefficients_solve_the_2d_minmax_problem():
    """The Kronecker product of 1D solutions is the 2D least-squares solution."""
    Nd, Kd, Jd = (8, 10), (16, 20), (4, 5)
    om = np.array([[0.3, -2.2], [-1.1, 0.9], [3.0, 0.0]])
    p = oracle.make_plan(om, Nd, Kd, Jd)
    t0, t1 = centred_coords(Nd[0]), centred_coords(Nd[1])
    s2 = np.multiply.outer(p.s[0], p.s[1]).ravel()
    T0, T1 = np.meshgrid(t0, t1, indexing="ij")
    for m in range(om.shape[0]):
        cols = []
        for j0 in range(1, Jd[0] + 1):
            for j1 in range(1, Jd[1] + 1):
                k = (p.k0[m, 0] + j0, p.k0[m, 1] + j1)
                ph = 2 * math.pi * (k[0] * T0 / Kd[0] + k[1] * T1 / Kd[1])
                cols.append(s2 * np.exp(-1j * ph.ravel()))
        A = np.stack(cols, axis=1)
        b = np.exp(-1j * (om[m, 0] * T0 + om[m, 1] * T1)).ravel()
        c_ls = np.linalg.lstsq(A, b, rcond=None)[0]
        c_kron = np.kron(p.coef[0][m], p.coef[1][m])
        np.testing.assert_allclose(c_kron, c_ls, rtol=0, atol=1e-8 * np.abs(c_ls).max())


# ---------------------------------------------------------------- NUFFT vs NUDFT

@pytest.mark.parametrize("Nd,Kd,Jd,M", [
    ((32,), (64,), (6,), 400),
    ((32, 32), (64, 64), (6, 6), 500),
    ((16, 24), (32, 48), (6, 6), 300),
    ((12, 12, 12), (24, 24, 24), (6, 6, 6), 200),
    ((8, 10, 12), (16, 20, 24), (6, 6, 6), 150),
])
def test_forward_matches_brute_force_nudft(Nd, Kd, Jd, M):
    om = W.uniform_random_om(M, len(Nd), seed=5)
    x = _cn(Nd)
    p = oracle.make_plan(om, Nd, Kd, Jd)
    err = _rel(oracle.forward(p, x), oracle.nudft_forward(om, x))
    assert err < 2e-5, err          # J=6, K=2N: ~7e-6 expected; 1e-3 is the bound asked for


@pytest.mark.parametrize("Jd", [(4, 4), (5, 5)])
def test_forward_error_decreases_with_J(Jd):
    Nd, Kd = (16, 16), (32, 32)
    om = W.uniform_random_om(300, 2, seed=6)
    x = _cn(Nd)
    ref = oracle.nudft_forward(om, x)
    e = _rel(oracle.forward(oracle.make_plan(om, Nd, Kd, Jd), x), ref)
    e6 = _rel(oracle.forward(oracle.make_plan(om, Nd, Kd, (6, 6)), x), ref)
    assert e6 < e < 1e-3


def test_adjoint_matches_brute_force_nudft_adjoint():
    Nd, Kd, Jd = (16, 16), (32, 32), (6, 6)
    om = W.uniform_random_om(300, 2, seed=7)
    y = _cn(300)
    p = oracle.make_plan(om, Nd, Kd, Jd)
    assert _rel(oracle.adjoint(p, y), oracle.nudft_adjoint(om, y, Nd)) < 2e-5


def test_golden_nudft_fixture():
    """Stored exact NUDFT values (tests/golden/nudft_2d_tiny.txt)."""
    data = np.loadtxt(os.path.join(GOLDEN, "nudft_2d_tiny.txt"))
    y_gold = data[:, 1] + 1j * data[:, 2]
    om = W.uniform_random_om(40, 2, seed=11)
    x = W.complex_normal_image((16, 8), seed=12)
    p = oracle.make_plan(om, (16, 8), (32, 16), (6, 6))
    assert _rel(oracle.forward(p, x), y_gold) < 2e-5
    assert _rel(oracle.nudft_forward(om, x), y_gold) < 1e-13


def test_shifted_delta_closed_form():
    """x = delta[n - n0] has spectrum exp(-i w . (n0 - N/2))."""
    Nd, Kd, Jd = (32, 32), (64, 64), (6, 6)
    n0 = (5, 27)
    om = W.uniform_random_om(400, 2, seed=8)
    x = np.zeros(Nd, dtype=complex)
    x[n0] = 1.0
    p = oracle.make_plan(om, Nd, Kd, Jd)
    y = oracle.forward(p, x)
    exact = np.exp(-1j * (om.astype(np.float64) @ (np.array(n0) - np.array(Nd) / 2)))
    assert np.abs(y - exact).max() < 1e-4


def test_parseval_on_uniform_frequencies():
    """With w on the uniform N-grid the NUDFT is a unitary DFT times sqrt(N^d)."""
    Nd, Kd, Jd = (16, 16), (32, 32), (6, 6)
    k = 2 * math.pi * (np.arange(16) - 8) / 16
    g0, g1 = np.meshgrid(k, k, indexing="ij")
    om = np.stack([g0.ravel(), g1.ravel()], axis=1)
    x = _cn(Nd)
    p = oracle.make_plan(om, Nd, Kd, Jd)
    y = oracle.forward(p, x)
    ratio = np.vdot(y, y).real / (256 * np.vdot(x, x).real)
    assert abs(ratio - 1.0) < 1e-4


# ---------------------------------------------------------------- stages

def test_fft_stages_match_direct_dft():
    K = (8, 16)
    z = _cn(K)
    g = [np.arange(k) for k in K]
    D0 = np.exp(-2j * math.pi * np.outer(g[0], g[0]) / K[0])
    D1 = np.exp(-2j * math.pi * np.outer(g[1], g[1]) / K[1])
    np.testing.assert_allclose(oracle.fft_forward(z), D0 @ z @ D1.T, atol=1e-12)
    np.testing.assert_allclose(oracle.fft_adjoint(z), D0.conj() @ z @ D1.conj().T, atol=1e-12)


def test_stage_adjoint_identities():
    Nd, Kd, Jd = (16, 12), (32, 24), (6, 6)
    om = W.uniform_random_om(200, 2, seed=9)
    p = oracle.make_plan(om, Nd, Kd, Jd)
    x, z, Y, y = _cn(Nd), _cn(Kd), _cn(Kd), _cn(200)
    # S + pad vs crop + S^H
    assert abs(np.vdot(oracle.scale_pad(p, x), z) - np.vdot(x, oracle.crop_rescale(p, z))) < 1e-12 * 1e3
    # F vs F^H
    lhs, rhs = np.vdot(oracle.fft_forward(z), Y), np.vdot(z, oracle.fft_adjoint(Y))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    # V vs V^H
    lhs, rhs = np.vdot(oracle.interp_V(p, Y), y), np.vdot(Y, oracle.gridding_VH(p, y))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    # A vs A^H
    lhs, rhs = np.vdot(oracle.forward(p, x), y), np.vdot(x, oracle.adjoint(p, y))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_pad_crop_placement():
    """The image centre n = N/2 lands on grid index 0; crop undoes pad."""
    Nd, Kd = (8, 6), (16, 12)
    p = oracle.make_plan(np.zeros((1, 2)), Nd, Kd, (4, 4))
    x = np.zeros(Nd, dtype=complex)
    x[4, 3] = 1.0
    z = oracle.scale_pad(p, x)
    assert np.count_nonzero(z) == 1 and z[0, 0] != 0
    s2 = np.multiply.outer(p.s[0], p.s[1])
    xx = _cn(Nd)
    np.testing.assert_allclose(oracle.crop_rescale(p, oracle.scale_pad(p, xx)), s2 * s2 * xx, atol=1e-14)


# ---------------------------------------------------------------- solver pieces

def test_gradient_adjoint_and_constant():
    x, g = _cn((6, 7, 5)), _cn((6, 7, 5))
    for ax in range(3):
        assert abs(np.vdot(oracle.grad(x, ax), g) - np.vdot(x, oracle.grad_T(g, ax))) < 1e-12
        assert np.abs(oracle.grad(np.full((6, 7, 5), 2 + 1j), ax)).max() == 0
    ramp = np.arange(5.0)[None, :] * np.ones((3, 1))
    np.testing.assert_array_equal(oracle.grad(ramp, 1), np.array([[1, 1, 1, 1, -4]] * 3))


def test_shrink_closed_form():
    z = np.array([5.0, 1.0, -3.0, 0.0, 3 + 4j, 0.3j])
    out = oracle.shrink(z, 2.0)
    np.testing.assert_allclose(out, [3.0, 0.0, -1.0, 0.0, (3 + 4j) * 3 / 5, 0.0], atol=1e-15)


def _tiny_problem(M=300, seed=10):
    Nd, Kd, Jd = (8, 8), (16, 16), (6, 6)
    om = W.uniform_random_om(M, 2, seed=seed)
    p = oracle.make_plan(om, Nd, Kd, Jd)
    A = np.stack([oracle.forward(p, e.reshape(Nd)) for e in np.eye(64)], axis=1)
    xt = _cn(Nd)
    return p, A, xt, Nd


def test_cg_reaches_dense_normal_equation_solution():
    p, A, xt, Nd = _tiny_problem()
    y = A @ xt.ravel() + 0.01 * _cn(A.shape[0])
    x_ls = np.linalg.solve(A.conj().T @ A, A.conj().T @ y).reshape(Nd)
    x = oracle.cg(p, y, np.zeros(Nd), 64)
    assert _rel(x, x_ls) < 1e-10


def test_cg_residuals_orthogonal():
    from oracle.solvers import cg_solve
    p, A, xt, Nd = _tiny_problem()
    H = A.conj().T @ A
    b = _cn(64)
    rs = []
    for it in range(1, 6):
        x = cg_solve(lambda v: H @ v, b, np.zeros(64), it)
        rs.append(b - H @ x)
    for i in range(len(rs)):
        for j in range(i):
            assert abs(np.vdot(rs[i], rs[j])) < 1e-9 * np.linalg.norm(rs[i]) * np.linalg.norm(rs[j]) + 1e-12


def test_l1tv_ols_reduces_to_least_squares_as_lambda_vanishes():
    """lambda -> 0: the split Bregman loop becomes iterated CG on A^H A."""
    p, A, xt, Nd = _tiny_problem()
    y = A @ xt.ravel()
    x_ls = np.linalg.solve(A.conj().T @ A, A.conj().T @ y).reshape(Nd)
    x = oracle.l1tv_ols(p, y, np.zeros(Nd), 20, 1, 10, 1.0, 1e-12)
    assert _rel(x, x_ls) < 1e-9


def test_l1tv_lad_recovers_consistent_data_as_lambda_vanishes():
    p, A, xt, Nd = _tiny_problem()
    y = A @ xt.ravel()
    x = oracle.l1tv_lad(p, y, np.zeros(Nd), 20, 2, 10, 1.0, 1e-12)
    assert _rel(x, xt) < 1e-9


def test_l1tv_ols_tv_term_smooths_a_noisy_piecewise_constant_image():
    """With the shrink active the TV solution is closer to the piecewise-constant
    truth than the plain least-squares solve on noisy, undersampled data."""
    Nd, Kd, Jd = (16, 16), (32, 32), (6, 6)
    om = W.radial2d_uniform(12, 32)
    xt = np.zeros(Nd, dtype=complex)
    xt[4:12, 5:11] = 1.0
    p = oracle.make_plan(om, Nd, Kd, Jd)
    rng = np.random.default_rng(3)
    y = oracle.forward(p, xt) + 0.3 * (rng.standard_normal(om.shape[0]) + 1j * rng.standard_normal(om.shape[0]))
    x_cg = oracle.cg(p, y, np.zeros(Nd), 30)
    x_tv = oracle.l1tv_ols(p, y, np.zeros(Nd), 10, 2, 5, 1.0, 2.0)
    assert _rel(x_tv, xt) < _rel(x_cg, xt)
