"""Write tests/golden/solver_baselines.json from the FP64 oracle alone.

The solver runs of the benchmark configurations (Section 2.2.2 CG and
Section 2.2.3 L1TV-OLS / L1TV-LAD on the 64^2 and 256^2 radial workloads and
the 256^2 spiral) take the oracle minutes each, too long for every test run,
so their results are stored here.  Per configuration:

* the final iterate's norm, anisotropic TV and data residual ||A x - y|| / ||y||
  (A the oracle's forward operator);
* a 64-dimensional complex Gaussian sketch s = G^H x / sqrt(64) of the final
  iterate (rows of G drawn from numpy.random.default_rng(SKETCH_SEED), one row
  of n complex values at a time); for any v, |s(v)|^2 estimates ||v||^2 within
  about 1/sqrt(128), so ||s(x) - s(x_ref)|| / ||s(x_ref)|| estimates the
  relative L2 distance of an iterate x to the oracle's;
* the spread of the final iterate when the oracle's normal operator output is
  multiplied by (1 + eps * N(0, 1)) elementwise (eps = 1e-7 and 1e-6, two
  seeds each): the largest relative L2 distance to the unperturbed run, and
  the largest relative change of its norm.  A spread above the solver
  tolerance says that no FP32 implementation can meet it on this
  configuration, and bounds how far a correct one can land.

The inputs are the seeded workloads of workloads.py; y is the oracle's forward
of the workload image plus its noise, rounded to complex64 (the GPU tests use
the same bytes).  Runs in a process pool; about 20 minutes on 8 cores.

    python tests/golden/make_solver_golden.py
"""
from __future__ import annotations

import json
import multiprocessing as mp
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "solver_baselines.json")
SKETCH_SEED = 20260101
SKETCH_DIM = 64
EPS = (1e-7, 1e-6)
SEEDS = (1, 2)

L1TV = dict(maxiter=50, inner=2, cg_iters=5, mu=1.0, lam=0.01)
CONFIGS = {
    "c1_radial2d_64_cg20": ("radial2d_64", "cg", dict(maxiter=20)),
    "c2_radial2d_256_cg100": ("radial2d_256", "cg", dict(maxiter=100)),
    "c2_radial2d_256_l1tv_ols50": ("radial2d_256", "l1tv_ols", L1TV),
    "c2_radial2d_256_l1tv_lad50": ("radial2d_256", "l1tv_lad", L1TV),
    "c5_spiral2d_256_l1tv_lad50": ("spiral2d_256", "l1tv_lad", L1TV),
}


def sketch(x: np.ndarray, k: int = SKETCH_DIM, seed: int = SKETCH_SEED) -> np.ndarray:
    """s_j = <g_j, x> / sqrt(k), g_j complex with N(0, 1/2) real and imaginary parts."""
    v = np.asarray(x, dtype=np.complex128).ravel()
    rng = np.random.default_rng(seed)
    s = np.empty(k, dtype=np.complex128)
    for j in range(k):
        g = (rng.standard_normal(v.size) + 1j * rng.standard_normal(v.size)) / np.sqrt(2.0)
        s[j] = np.vdot(g, v)
    return s / np.sqrt(k)


def workload_data(name):
    import oracle
    import workloads as W
    spec, om, x, noise = W.make_workload(name)
    plan = oracle.make_plan(om, spec["Nd"], spec["Kd"], spec["Jd"])
    y = oracle.forward(plan, x)
    if noise is not None:
        y = y + noise
    return spec, plan, y.astype(np.complex64)


def run_solver(plan, y, Nd, solver, kw):
    import oracle
    x0 = np.zeros(Nd)
    if solver == "cg":
        return oracle.cg(plan, y, x0, kw["maxiter"])
    fn = getattr(oracle, solver)
    return fn(plan, y, x0, kw["maxiter"], kw["inner"], kw["cg_iters"], kw["mu"], kw["lam"])


def _job(args):
    key, eps, seed = args
    import oracle
    import oracle.solvers as S
    name, solver, kw = CONFIGS[key]
    spec, plan, y = workload_data(name)
    if eps > 0:
        exact = S.selfadjoint
        rng = np.random.default_rng(seed)
        S.selfadjoint = lambda p, v: (lambda o: o * (1 + eps * rng.standard_normal(o.shape)))(exact(p, v))
    x = run_solver(plan, y, spec["Nd"], solver, kw)
    return key, eps, seed, x


def tv(x):
    import oracle
    return float(sum(np.abs(oracle.grad(x, a)).sum() for a in range(x.ndim)))


def main():
    import oracle
    jobs = [(k, 0.0, 0) for k in CONFIGS] + [(k, e, s) for k in CONFIGS for e in EPS for s in SEEDS]
    jobs.sort(key=lambda j: 0 if "256_l1tv" in j[0] else 1)     # longest first
    results = {}
    with mp.get_context("spawn").Pool(min(len(jobs), max(1, (os.cpu_count() or 2) - 1))) as pool:
        for key, eps, seed, x in pool.imap_unordered(_job, jobs):
            results[(key, eps, seed)] = x
            print(key, eps, seed, flush=True)
    out = {"sketch_seed": SKETCH_SEED, "sketch_dim": SKETCH_DIM, "configs": {}}
    for key, (name, solver, kw) in CONFIGS.items():
        spec, plan, y = workload_data(name)
        x = results[(key, 0.0, 0)]
        res = float(np.linalg.norm(oracle.forward(plan, x) - y) / np.linalg.norm(y))
        spread, norm_spread = {}, {}
        for eps in EPS:
            spread[f"{eps:g}"] = max(float(np.linalg.norm(results[(key, eps, s)] - x) / np.linalg.norm(x))
                                     for s in SEEDS)
            norm_spread[f"{eps:g}"] = max(abs(float(np.linalg.norm(results[(key, eps, s)]) / np.linalg.norm(x)) - 1)
                                          for s in SEEDS)
        out["configs"][key] = {
            "workload": name, "solver": solver, "params": kw,
            "norm": float(np.linalg.norm(x)), "tv": tv(x), "residual": res,
            "sketch": [[float(v.real), float(v.imag)] for v in sketch(x)],
            "spread": spread, "norm_spread": norm_spread,
        }
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
