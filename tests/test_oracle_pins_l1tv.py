"""Pins of the oracle's L1TV-OLS and L1TV-LAD outer (Bregman) loops.

Section 2.2.3 (Eqs. 11-20 for OLS, Eqs. 21-31 for LAD) solves the
TV-regularised problems by variable splitting inside a Bregman iteration
that adds the data residual A^H y - A^H A x back to the right-hand side after
every outer step.  Bregman iteration of this kind converges to a solution of
the constrained problem

    minimise TV(x) = sum_i |grad_i x|_1   subject to   A x = y

for any positive mu and lambda (the threshold 1/lambda sets only the speed),
so its limit is fixed by the mathematics, not by the oracle:

* with A of full column rank and consistent data y = A x_true, the only
  feasible point is x_true, so both loops must reach it;
* with fewer measurements than unknowns, the limit must be feasible
  (A x = y), have TV no larger than any other feasible point (x_true, the
  least-norm solution), and here, where x_true is piecewise constant with
  few edges and the samples are random, it is the unique TV minimiser x_true.

The shrink is active in these cases: 1/lambda = 1 lies inside the range of
the true image's non-zero gradient magnitudes, so the thresholding both zeroes
and passes real gradients (checked below).

The planted-mistake test rewrites one line of a copy of each loop (the sign
of the b update, d + b for d - b in the right-hand side, the sign of the
Bregman add-back, the shrink argument, LAD's b_f update and the sign of its
d_f - b_f term) and checks that every rewritten copy fails a pin.
"""
import inspect

import numpy as np
import pytest

import oracle
import oracle.solvers as S
import workloads as W

Nd, Kd, Jd = (8, 8), (16, 16), (6, 6)
LAM, MU = 1.0, 1.0          # threshold 1/lambda = 1
INNER, CG_ITERS = 2, 10


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


def _x_true():
    """Piecewise-constant complex image: a block of 1 + 0.5i and an overlapping bar of -0.7."""
    x = np.zeros(Nd, dtype=complex)
    x[2:6, 3:7] = 1.0 + 0.5j
    x[5:7, 1:3] += -0.7
    return x


def _tv(x):
    return float(sum(np.abs(oracle.grad(x, a)).sum() for a in range(x.ndim)))


def _problem(M, seed):
    om = W.uniform_random_om(M, 2, seed=seed)
    p = oracle.make_plan(om, Nd, Kd, Jd)
    A = np.stack([oracle.forward(p, e.reshape(Nd)) for e in np.eye(int(np.prod(Nd)))], axis=1)
    xt = _x_true()
    return p, A, xt, A @ xt.ravel()


@pytest.fixture(scope="module")
def full_rank():
    p, A, xt, y = _problem(300, 10)
    assert np.linalg.matrix_rank(A) == A.shape[1]
    return p, A, xt, y


@pytest.fixture(scope="module")
def underdetermined():
    p, A, xt, y = _problem(32, 11)
    assert A.shape[0] < A.shape[1]          # 32 complex equations, 64 complex unknowns
    return p, A, xt, y


def test_shrink_is_active_at_this_lambda():
    xt = _x_true()
    g = np.concatenate([oracle.grad(xt, a).ravel() for a in range(2)])
    nz = g[np.abs(g) > 0]
    kept = np.abs(oracle.shrink(nz, 1.0 / LAM)) > 0
    assert 0.2 < kept.mean() < 0.9           # some non-zero gradients zeroed, some passed
    assert np.median(np.abs(nz)) > 1.0 / LAM  # 1/lambda lies below the median


def _solve(fn, prob, outer):
    p, _, _, y = prob
    return fn(p, y, np.zeros(Nd), outer, INNER, CG_ITERS, MU, LAM)


def _full_rank_ok(fn, prob):
    _, _, xt, _ = prob
    with np.errstate(all="ignore"):
        x = _solve(fn, prob, 30)
    return bool(np.all(np.isfinite(x))) and _rel(x, xt) < 1e-8


def _underdetermined_ok(fn, prob):
    _, A, xt, y = prob
    with np.errstate(all="ignore"):
        x = _solve(fn, prob, 80)
        if not np.all(np.isfinite(x)):
            return False
        feasible = np.linalg.norm(A @ x.ravel() - y) <= 1e-8 * np.linalg.norm(y)
        x_ln = (np.linalg.pinv(A) @ y).reshape(Nd)
        tv_ok = _tv(x) <= _tv(xt) * (1 + 1e-8) and _tv(x) < _tv(x_ln)
    return bool(feasible and tv_ok and _rel(x, xt) < 1e-8)


@pytest.mark.parametrize("name", ["l1tv_ols", "l1tv_lad"])
def test_full_column_rank_consistent_data_reaches_x_true(full_rank, name):
    assert _full_rank_ok(getattr(oracle, name), full_rank)


@pytest.mark.parametrize("name", ["l1tv_ols", "l1tv_lad"])
def test_underdetermined_limit_is_the_tv_minimiser(underdetermined, name):
    _, A, xt, y = underdetermined
    x_ln = (np.linalg.pinv(A) @ y).reshape(Nd)
    assert _tv(x_ln) > 1.2 * _tv(xt)         # the least-norm solution is not TV-minimal
    assert _underdetermined_ok(getattr(oracle, name), underdetermined)


_MUTATIONS = {
    "b update sign": ("b[ax] = b[ax] + (g - d[ax])", "b[ax] = b[ax] - (g - d[ax])"),
    "d + b in the right-hand side": ("grad_T(d[ax] - b[ax], ax)", "grad_T(d[ax] + b[ax], ax)"),
    "add-back sign": ("AHy_k = AHy_k + AHy - selfadjoint(plan, x)", "AHy_k = AHy_k - AHy + selfadjoint(plan, x)"),
    "shrink argument": ("shrink(g + b[ax], 1.0 / lam)", "shrink(g - b[ax], 1.0 / lam)"),
    "b_f update sign": ("b_f = b_f + (resid - d_f)", "b_f = b_f - (resid - d_f)"),
    "d_f - b_f sign": ("mu * (AHy_k + d_f - b_f)", "mu * (AHy_k - d_f + b_f)"),
}


def _mutant(name, old, new):
    src = inspect.getsource(getattr(S, name))
    if old not in src:
        return None
    ns = dict(S.__dict__)
    exec(compile(src.replace(old, new), "<mutant>", "exec"), ns)
    return ns[name]


@pytest.mark.parametrize("mutation", sorted(_MUTATIONS))
@pytest.mark.parametrize("name", ["l1tv_ols", "l1tv_lad"])
def test_planted_mistakes_fail_a_pin(full_rank, underdetermined, name, mutation):
    fn = _mutant(name, *_MUTATIONS[mutation])
    if fn is None:
        pytest.skip(f"{name} has no such line")
    assert not (_full_rank_ok(fn, full_rank) and _underdetermined_ok(fn, underdetermined))
