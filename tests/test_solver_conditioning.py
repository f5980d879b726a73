"""Why the solver parity cases are chosen as they are (CPU, oracle only).

The GPU path computes in FP32 (as the paper's own benchmarks do, Section 2.4),
so a solver can match the FP64 oracle only as closely as the iteration lets
rounding through.  These tests record, on the oracle alone, that radial
problems amplify a 1e-7 relative perturbation of the normal operator far past
the 1e-4 solver tolerance within 20 CG iterations, while the uniform random
problems used for the 1e-4 parity tests do not; and that the L1TV parity
cases do exercise the shrink step.
"""
import numpy as np

import oracle
import oracle.solvers as S
import workloads as W


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _perturbed_cg(plan, y, Nd, iters, eps, seed, monkeypatch):
    exact = S.selfadjoint
    rng = np.random.default_rng(seed)
    monkeypatch.setattr(S, "selfadjoint", lambda p, v: (lambda o: o * (1 + eps * rng.standard_normal(o.shape)))(exact(p, v)))
    try:
        return oracle.cg(plan, y, np.zeros(Nd), iters)
    finally:
        monkeypatch.setattr(S, "selfadjoint", exact)


def test_radial_cg_amplifies_rounding_beyond_solver_tolerance(monkeypatch):
    spec, om, x, _ = W.make_workload("radial2d_64")
    p = oracle.make_plan(om, spec["Nd"], spec["Kd"], spec["Jd"])
    y = oracle.forward(p, x)
    ref = oracle.cg(p, y, np.zeros(spec["Nd"]), 20)
    alt = _perturbed_cg(p, y, spec["Nd"], 20, 1e-7, 1, monkeypatch)
    assert _rel(alt, ref) > 1e-3


def test_uniform_random_cg_is_stable_to_rounding(monkeypatch):
    Nd, Kd, Jd = (64, 64), (128, 128), (6, 6)
    om = W.uniform_random_om(3 * 64 * 64, 2, seed=3)
    p = oracle.make_plan(om, Nd, Kd, Jd)
    y = oracle.forward(p, W.complex_normal_image(Nd))
    ref = oracle.cg(p, y, np.zeros(Nd), 50)
    alt = _perturbed_cg(p, y, Nd, 50, 1e-6, 1, monkeypatch)
    assert _rel(alt, ref) < 2e-5


def test_l1tv_parity_cases_exercise_the_shrink():
    """lambda = 50 (threshold 1/lambda = 0.02, near the median gradient): a real
    share of the gradients is zeroed by the shrink and a real share passes."""
    Nd, Kd, Jd = (64, 64), (128, 128), (6, 6)
    om = W.uniform_random_om(3 * 64 * 64, 2, seed=3)
    p = oracle.make_plan(om, Nd, Kd, Jd)
    y = (oracle.forward(p, W.ellipse_phantom(64)) + W.complex_noise(om.shape[0], 0.5)).astype(np.complex64)
    x = oracle.l1tv_ols(p, y, np.zeros(Nd), 2, 1, 5, 1.0, 50.0)
    d = oracle.shrink(oracle.grad(x, 0), 1.0 / 50.0)
    assert 0.1 < np.mean(d == 0) < 0.9
