"""FP64 NUFFT operators A = V F S, A^H = S^H F^H V^H and A^H A.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Each function is one stage of the operator chain of Section 2.1 (Eq. 1) and
Section 2.1.4 (Eq. 2), in the paper's order, with C-order (row-major) arrays
as the paper uses (Section 2.1.3):

* S     scaling, elementwise multiply by s = prod_d s_d (Section 2.1.1);
* pad   copy the N^d image into the K^d grid at g = (n - N/2) mod K
        (Section 2.1.2; the centred placement is the reading that matches
        t_n = n - N/2 in the interpolator);
* F     unnormalised forward FFT, exp(-2 pi i k g / K) (Section 2.1.2);
* V     y_m = sum_{j in [1,J]^d} prod_d c[m,d,j_d] Y[(k0_m + j) mod K]
        (Section 2.1.3, min-max interpolator of the oracle's minmax module);
* V^H   conjugate-transpose scatter of V (Section 2.1.3, "gridding");
* F^H   unnormalised inverse FFT, exp(+2 pi i k g / K) (Section 2.1.2);
* crop + S^H: read the N^d region back and multiply by s (s is real).

The exact target the method approximates (the NUDFT) is also here:
y_m = sum_n x[n] exp(-i sum_d w_{m,d} (n_d - N_d/2)).
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass

import numpy as np

from .minmax import minmax_coefficients_1d, centred_coords


@dataclass
class Plan:
    Nd: tuple
    Kd: tuple
    Jd: tuple
    om: np.ndarray          # (M, d) float64 (the float32 input, widened exactly)
    s: list                 # per-dim scaling (N_d,) float64
    k0: np.ndarray          # (M, d) int64
    coef: list              # per-dim (M, J_d) complex128

    @property
    def d(self) -> int:
        return len(self.Nd)

    @property
    def M(self) -> int:
        return self.om.shape[0]


def make_plan(om, Nd, Kd, Jd) -> Plan:
    """Per-dimension min-max precompute (the paper's interpolator set-up)."""
    om = np.asarray(om)
    if om.ndim == 1:
        om = om[:, None]
    om64 = om.astype(np.float64)
    d = om64.shape[1]
    Nd, Kd, Jd = tuple(int(v) for v in Nd), tuple(int(v) for v in Kd), tuple(int(v) for v in Jd)
    assert len(Nd) == len(Kd) == len(Jd) == d
    s_list, k0_cols, c_list = [], [], []
    for dim in range(d):
        k0, c, s = minmax_coefficients_1d(om64[:, dim], Nd[dim], Kd[dim], Jd[dim])
        s_list.append(s)
        k0_cols.append(k0)
        c_list.append(c)
    return Plan(Nd, Kd, Jd, om64, s_list, np.stack(k0_cols, axis=1), c_list)


def _pad_indices(plan: Plan):
    return [(np.arange(N) - N // 2) % K for N, K in zip(plan.Nd, plan.Kd)]


def _scaling_nd(plan: Plan) -> np.ndarray:
    s = np.ones((), dtype=np.float64)
    for sd in plan.s:
        s = np.multiply.outer(s, sd)
    return s


def scale_pad(plan: Plan, x: np.ndarray) -> np.ndarray:
    """S then zero-padding: z[(n - N/2) mod K] = s[n] x[n]."""
    z = np.zeros(plan.Kd, dtype=np.complex128)
    z[np.ix_(*_pad_indices(plan))] = _scaling_nd(plan) * np.asarray(x, dtype=np.complex128)
    return z


def fft_forward(z: np.ndarray) -> np.ndarray:
    """F: unnormalised forward DFT over all axes."""
    return np.fft.fftn(z)


def interp_V(plan: Plan, Y: np.ndarray) -> np.ndarray:
    """V: J^d-neighbour tensor-product interpolation of the grid."""
    y = np.zeros(plan.M, dtype=np.complex128)
    for taps in itertools.product(*[range(1, J + 1) for J in plan.Jd]):
        idx = tuple((plan.k0[:, dim] + taps[dim]) % plan.Kd[dim] for dim in range(plan.d))
        w = np.ones(plan.M, dtype=np.complex128)
        for dim in range(plan.d):
            w = w * plan.coef[dim][:, taps[dim] - 1]
        y += w * Y[idx]
    return y


def gridding_VH(plan: Plan, y: np.ndarray) -> np.ndarray:
    """V^H: scatter conj(prod_d c) y_m onto the K^d grid (the transpose of V)."""
    y = np.asarray(y, dtype=np.complex128)
    Z = np.zeros(plan.Kd, dtype=np.complex128)
    for taps in itertools.product(*[range(1, J + 1) for J in plan.Jd]):
        idx = tuple((plan.k0[:, dim] + taps[dim]) % plan.Kd[dim] for dim in range(plan.d))
        w = np.ones(plan.M, dtype=np.complex128)
        for dim in range(plan.d):
            w = w * plan.coef[dim][:, taps[dim] - 1]
        np.add.at(Z, idx, np.conj(w) * y)
    return Z


def fft_adjoint(Z: np.ndarray) -> np.ndarray:
    """F^H: unnormalised inverse DFT over all axes (no 1/K^d)."""
    return np.fft.ifftn(Z) * float(np.prod(Z.shape))


def crop_rescale(plan: Plan, z: np.ndarray) -> np.ndarray:
    """Copy the N^d region back and apply S^H (= S, s is real)."""
    return _scaling_nd(plan) * z[np.ix_(*_pad_indices(plan))]


def forward(plan: Plan, x: np.ndarray) -> np.ndarray:
    """A x = V F S x (Eq. 1)."""
    return interp_V(plan, fft_forward(scale_pad(plan, x)))


def adjoint(plan: Plan, y: np.ndarray) -> np.ndarray:
    """A^H y = S^H F^H V^H y (Eq. 2)."""
    return crop_rescale(plan, fft_adjoint(gridding_VH(plan, y)))


def selfadjoint(plan: Plan, x: np.ndarray) -> np.ndarray:
    """A^H A x (the normal operator of Section 2.1.5)."""
    return adjoint(plan, forward(plan, x))


def _phase_matrix(om: np.ndarray, Nd) -> np.ndarray:
    om = np.asarray(om, dtype=np.float64)
    if om.ndim == 1:
        om = om[:, None]
    grids = np.meshgrid(*[centred_coords(N) for N in Nd], indexing="ij")
    tn = np.stack([g.ravel() for g in grids], axis=1)          # (prod N, d)
    return np.exp(-1j * (om @ tn.T))                           # (M, prod N)


def nudft_forward(om: np.ndarray, x: np.ndarray) -> np.ndarray:
    """Brute-force non-uniform DFT, the exact value A approximates."""
    x = np.asarray(x, dtype=np.complex128)
    return _phase_matrix(om, x.shape) @ x.ravel()


def nudft_adjoint(om: np.ndarray, y: np.ndarray, Nd) -> np.ndarray:
    """Conjugate transpose of the brute-force NUDFT."""
    E = _phase_matrix(om, Nd)
    return (E.conj().T @ np.asarray(y, dtype=np.complex128)).reshape(Nd)
