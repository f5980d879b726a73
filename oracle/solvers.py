"""FP64 solvers on the NUFFT normal operator: CG, L1TV-OLS, L1TV-LAD.

TEST INFRASTRUCTURE ONLY (see the package docstring).

* ``cg``: conjugate gradient (Hestenes-Stiefel) on the normal equation
  A^H A x = A^H y (Section 2.1.5, Eq. 4; Section 2.2.2), a fixed number of
  iterations with no early exit.  The paper's own CG is written on the k-space
  system V^H V k = V^H y (Eqs. 7-9); the image-domain form is the reading used
  here, because the normal operator is what the solvers below iterate on.
* ``grad`` / ``grad_T``: periodic forward difference along axis i and its
  transpose, the "image rolling" of Section 2.2.3 (Eq. 10).
* ``shrink``: complex soft threshold z/|z| max(|z| - t, 0), 0 at z = 0
  (Eqs. 14-15, 24-26).
* ``l1tv_ols``: variable splitting of Eqs. 11-20 (Section 2.2.3).
* ``l1tv_lad``: variable splitting of Eqs. 21-31 (Section 2.2.3).

Readings (the paper leaves these open):
* the split system x = K^{-1} rhs (Eq. 13, Eq. 23) is solved by ``cg_iters``
  CG steps on K = mu A^H A + lambda sum_i grad_i^T grad_i, warm-started from
  the current x;
* ``maxiter`` counts outer (Bregman) iterations, ``inner`` the split
  iterations inside each one; d = b = 0 and A^H y^0 = A^H y at the start;
* the threshold is literally 1/lambda (1/mu for the LAD data term);
* in the LAD d_f update (Eq. 26) the Bregman variable added is b_f (the
  printed "b_y" reads as a typo); d_f, b_f live in the image domain;
* TV is anisotropic (sum over axes of |grad_i x|), with every axis of the
  image used (x, y and, in 3D, z).
* CG guards: alpha = 0 when <p, A p> = 0, beta = 0 when <r, r> = 0.

Pins: the Bregman loops of ``l1tv_ols`` and ``l1tv_lad`` converge to a
solution of min TV(x) subject to A x = y; ``tests/test_oracle_pins_l1tv.py``
checks that limit on full-rank and underdetermined problems with the shrink
active.
"""
from __future__ import annotations

import numpy as np

from .nufft import Plan, adjoint, selfadjoint


def grad(x: np.ndarray, axis: int) -> np.ndarray:
    """grad_i x [.., a_i, ..] = x[.., a_i + 1, ..] - x[.., a_i, ..] (periodic)."""
    return np.roll(x, -1, axis=axis) - x


def grad_T(g: np.ndarray, axis: int) -> np.ndarray:
    """Transpose of ``grad``: (grad_i^T g)[a_i] = g[a_i - 1] - g[a_i] (periodic)."""
    return np.roll(g, 1, axis=axis) - g


def shrink(z: np.ndarray, t: float) -> np.ndarray:
    z = np.asarray(z, dtype=np.complex128)
    mag = np.abs(z)
    out = np.zeros_like(z)
    nz = mag > 0
    out[nz] = z[nz] / mag[nz] * np.maximum(mag[nz] - t, 0.0)
    return out


def _dot(a: np.ndarray, b: np.ndarray) -> complex:
    """<a, b> = sum conj(a) b."""
    return complex(np.vdot(a.ravel(), b.ravel()))


def cg_solve(apply, b: np.ndarray, x0: np.ndarray, iters: int) -> np.ndarray:
    """Textbook CG for a Hermitian positive semi-definite operator."""
    x = np.array(x0, dtype=np.complex128, copy=True)
    r = b - apply(x)
    p = r.copy()
    rr = _dot(r, r).real
    for _ in range(iters):
        q = apply(p)
        pq = _dot(p, q).real
        alpha = rr / pq if pq != 0.0 else 0.0
        x = x + alpha * p
        r = r - alpha * q
        rr_new = _dot(r, r).real
        beta = rr_new / rr if rr != 0.0 else 0.0
        p = r + beta * p
        rr = rr_new
    return x


def cg(plan: Plan, y: np.ndarray, x0: np.ndarray, maxiter: int) -> np.ndarray:
    """CG on A^H A x = A^H y from x0, ``maxiter`` iterations."""
    b = adjoint(plan, y)
    return cg_solve(lambda v: selfadjoint(plan, v), b, x0, maxiter)


def _K_apply(plan: Plan, mu: float, lam: float):
    def apply(v):
        out = mu * selfadjoint(plan, v)
        for ax in range(v.ndim):
            out = out + lam * grad_T(grad(v, ax), ax)
        return out
    return apply


def l1tv_ols(plan: Plan, y, x0, maxiter: int, inner: int, cg_iters: int,
             mu: float, lam: float) -> np.ndarray:
    """L1TV-OLS by variable splitting (Eqs. 11-20)."""
    Kop = _K_apply(plan, mu, lam)
    AHy = adjoint(plan, y)
    AHy_k = AHy.copy()
    x = np.array(x0, dtype=np.complex128, copy=True)
    nax = x.ndim
    d = [np.zeros_like(x) for _ in range(nax)]
    b = [np.zeros_like(x) for _ in range(nax)]
    for _ in range(maxiter):
        for _ in range(inner):
            rhs = mu * AHy_k
            for ax in range(nax):
                rhs = rhs + lam * grad_T(d[ax] - b[ax], ax)
            x = cg_solve(Kop, rhs, x, cg_iters)
            for ax in range(nax):
                g = grad(x, ax)
                d[ax] = shrink(g + b[ax], 1.0 / lam)
                b[ax] = b[ax] + (g - d[ax])
        AHy_k = AHy_k + AHy - selfadjoint(plan, x)
    return x


def l1tv_lad(plan: Plan, y, x0, maxiter: int, inner: int, cg_iters: int,
             mu: float, lam: float) -> np.ndarray:
    """L1TV-LAD by variable splitting (Eqs. 21-31)."""
    Kop = _K_apply(plan, mu, lam)
    AHy = adjoint(plan, y)
    AHy_k = AHy.copy()
    x = np.array(x0, dtype=np.complex128, copy=True)
    nax = x.ndim
    d = [np.zeros_like(x) for _ in range(nax)]
    b = [np.zeros_like(x) for _ in range(nax)]
    d_f = np.zeros_like(x)
    b_f = np.zeros_like(x)
    for _ in range(maxiter):
        for _ in range(inner):
            rhs = mu * (AHy_k + d_f - b_f)
            for ax in range(nax):
                rhs = rhs + lam * grad_T(d[ax] - b[ax], ax)
            x = cg_solve(Kop, rhs, x, cg_iters)
            for ax in range(nax):
                g = grad(x, ax)
                d[ax] = shrink(g + b[ax], 1.0 / lam)
                b[ax] = b[ax] + (g - d[ax])
            resid = selfadjoint(plan, x) - AHy
            d_f = shrink(resid + b_f, 1.0 / mu)
            b_f = b_f + (resid - d_f)
        AHy_k = AHy_k + AHy - selfadjoint(plan, x)
    return x
