"""FP64 oracle for the paper's remaining reconstruction methods.

TEST INFRASTRUCTURE ONLY (see the package docstring).

* density compensation (Section 2.2.1, Eqs. 5-6): the Pipe-Menon iteration
  w <- w / (A A^H w) and the gridding reconstruction x = A^H (y . w);
* the paper's own two-step CG (Section 2.2.2, Eqs. 7-9): solve
  V^H V k = V^H y for the oversampled k-space k by CG, then
  x = S^{-1} F^{-1} k (normalised inverse FFT, crop, divide by s);
* multi-coil operators (Section 2.2.3, Eqs. 32-33): A_i x = A (c_i . x),
  A_multi^H A_multi x = sum_i conj(c_i) . A^H A (c_i . x), and CG on the
  multi-coil normal equation.

Readings (the paper leaves these open):
* A A^H w is complex for real w (the Dirichlet kernel of a centred grid
  carries a half-sample phase); the update divides by its magnitude,
  w <- w / |A A^H w|, which keeps w real and positive.  w starts at 1.
* F^{-1} is the normalised inverse DFT (1/K^d), S^{-1} divides by s after the
  crop back to N^d; CG starts from k = 0.
* coil maps c_i are complex images of the image's shape; multi-coil k-space
  data are the coils' M-vectors stacked in coil order.
"""
from __future__ import annotations

import numpy as np

from .nufft import (Plan, forward, adjoint, selfadjoint, interp_V, gridding_VH, _pad_indices, _scaling_nd)
from .solvers import cg_solve


# ---------------------------------------------------------------- density compensation
def density_compensation(plan: Plan, iters: int, w0=None) -> np.ndarray:
    """Pipe-Menon iteration (Eq. 5): w_{i+1} = w_i / |A A^H w_i|."""
    w = np.ones(plan.M) if w0 is None else np.array(w0, dtype=np.float64)
    for _ in range(iters):
        d = forward(plan, adjoint(plan, w.astype(np.complex128)))
        w = w / np.abs(d)
    return w


def gridding_recon(plan: Plan, y: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Density-compensated gridding reconstruction (Eq. 6): x = A^H (y . w)."""
    return adjoint(plan, np.asarray(y, dtype=np.complex128) * np.asarray(w, dtype=np.float64))


# ---------------------------------------------------------------- two-step k-space CG
def VHV(plan: Plan, k: np.ndarray) -> np.ndarray:
    """The interpolation-gridding operator V^H V on the oversampled grid."""
    return gridding_VH(plan, interp_V(plan, k))


def cg_kspace(plan: Plan, y: np.ndarray, iters: int) -> np.ndarray:
    """Eqs. 7-9: k from CG on V^H V k = V^H y, then x = S^{-1} F^{-1} k."""
    b = gridding_VH(plan, np.asarray(y, dtype=np.complex128))
    k = cg_solve(lambda v: VHV(plan, v), b, np.zeros(plan.Kd, dtype=np.complex128), iters)
    z = np.fft.ifftn(k)                                   # normalised inverse DFT
    return z[np.ix_(*_pad_indices(plan))] / _scaling_nd(plan)


# ---------------------------------------------------------------- multi-coil
def forward_multicoil(plan: Plan, coils: np.ndarray, x: np.ndarray) -> np.ndarray:
    """Stacked coil data: [A (c_0 . x); A (c_1 . x); ...] (Eq. 32's A_i)."""
    return np.concatenate([forward(plan, c * x) for c in coils])


def adjoint_multicoil(plan: Plan, coils: np.ndarray, y: np.ndarray) -> np.ndarray:
    """sum_i conj(c_i) . A^H y_i, the adjoint of forward_multicoil."""
    M = plan.M
    return sum(np.conj(c) * adjoint(plan, y[i * M:(i + 1) * M]) for i, c in enumerate(coils))


def selfadjoint_multicoil(plan: Plan, coils: np.ndarray, x: np.ndarray) -> np.ndarray:
    """Eq. 33: sum_i conj(c_i) . A^H A (c_i . x)."""
    return sum(np.conj(c) * selfadjoint(plan, c * x) for c in coils)


def cg_multicoil(plan: Plan, coils: np.ndarray, y: np.ndarray, x0: np.ndarray, iters: int) -> np.ndarray:
    """CG on the multi-coil normal equation A_multi^H A_multi x = A_multi^H y."""
    b = adjoint_multicoil(plan, coils, y)
    return cg_solve(lambda v: selfadjoint_multicoil(plan, coils, v), b, x0, iters)


# ---------------------------------------------------------------- trajectory derivative
def _dr_domega(om_1d: np.ndarray, k0: np.ndarray, s: np.ndarray, K: int, J: int) -> np.ndarray:
    """d r_j / d w = sum_n s_n (-i t_n) exp(-i (w - gamma (k0 + j)) t_n), shape (M, J)."""
    from .minmax import centred_coords
    t = centred_coords(s.shape[0])
    gamma = (2.0 * np.pi) / K
    M = om_1d.shape[0]
    dr = np.empty((M, J), dtype=np.complex128)
    for j in range(1, J + 1):
        u = om_1d - gamma * (k0 + j)
        E = np.exp(-1j * u[:, None] * t[None, :])
        dr[:, j - 1] = E @ (s * (-1j) * t)
    return dr


def coefficient_derivatives(plan: Plan) -> list:
    """Per dimension, d c / d w (M, J): the min-max coefficients c = G^{-1} r
    with G independent of w and the neighbourhood k0 held fixed, so
    dc/dw = G^{-1} dr/dw.  (k0 jumps at cell boundaries, where the interpolator
    is discontinuous; the derivative is the one-sided one inside a cell.)"""
    from .minmax import minmax_G
    out = []
    for dim in range(plan.d):
        K, J = plan.Kd[dim], plan.Jd[dim]
        G = minmax_G(plan.s[dim], K, J)
        dr = _dr_domega(plan.om[:, dim], plan.k0[:, dim], plan.s[dim], K, J)
        out.append(np.linalg.solve(G, dr.T).T)
    return out


def forward_domega(plan: Plan, x: np.ndarray) -> np.ndarray:
    """d y_m / d w_{m,a} for every point and dimension, shape (M, d)."""
    import itertools
    from .nufft import scale_pad, fft_forward
    Y = fft_forward(scale_pad(plan, x))
    dc = coefficient_derivatives(plan)
    out = np.zeros((plan.M, plan.d), dtype=np.complex128)
    for taps in itertools.product(*[range(1, J + 1) for J in plan.Jd]):
        idx = tuple((plan.k0[:, dim] + taps[dim]) % plan.Kd[dim] for dim in range(plan.d))
        v = Y[idx]
        for a in range(plan.d):
            w = np.ones(plan.M, dtype=np.complex128)
            for dim in range(plan.d):
                w = w * (dc[dim][:, taps[dim] - 1] if dim == a else plan.coef[dim][:, taps[dim] - 1])
            out[:, a] += w * v
    return out


def trajectory_gradient(plan: Plan, x: np.ndarray, g: np.ndarray) -> np.ndarray:
    """Gradient of a real loss L(y), y = A(w) x, with respect to w (M, d), given
    g = dL/dRe(y) + i dL/dIm(y): dL/dw_{m,a} = Re(conj(g_m) dy_m/dw_{m,a})."""
    dy = forward_domega(plan, x)
    return np.real(np.conj(np.asarray(g, dtype=np.complex128))[:, None] * dy)


# ---------------------------------------------------------------- Toeplitz-embedded normal operator
def toeplitz_period(N: int) -> int:
    """Embedding period: 2N rounded up to a power of two (at least 16)."""
    P = 16
    while P < 2 * N:
        P *= 2
    return P


def toeplitz_kernel(plan: Plan) -> np.ndarray:
    """Spectrum of the Toeplitz embedding of A^H A (the precomputed normal
    operator of Section 2.1.5, in the Toeplitz form the paper cites).

    (A^H A x)[n] = sum_n' x[n'] t[n - n'],  t[D] = sum_m exp(i w_m . D).
    With P = toeplitz_period(N) >= 2N per dimension, t on D in [-P/2, P/2)^d is
    the adjoint NUFFT of all-ones on an image of size P (oversampled grid 2P,
    same J), whose centred coordinates q - P/2 give t[q - P/2].  Placed
    circularly on the P grid (t_circ[D mod P] = t[D]) its unnormalised DFT is
    the returned kernel; the circular convolution equals the linear one on the
    N^d image because P >= 2N."""
    from .nufft import make_plan as _mk, adjoint as _adj
    Pd = tuple(toeplitz_period(N) for N in plan.Nd)
    big = _mk(plan.om, Pd, tuple(2 * P for P in Pd), plan.Jd)
    x2 = _adj(big, np.ones(plan.M, dtype=np.complex128))
    t_circ = np.fft.ifftshift(x2)               # move D = 0 (q = P/2) to index 0
    return np.fft.fftn(t_circ)


def selfadjoint_toeplitz(plan: Plan, T: np.ndarray, x: np.ndarray) -> np.ndarray:
    """A^H A x by the circular embedding: centred zero-pad of x to the P grid,
    DFT, multiply by the kernel spectrum, inverse DFT, crop."""
    x = np.asarray(x, dtype=np.complex128)
    idx = [(np.arange(N) - N // 2) % P for N, P in zip(plan.Nd, T.shape)]
    z = np.zeros(T.shape, dtype=np.complex128)
    z[np.ix_(*idx)] = x
    w = np.fft.ifftn(np.fft.fftn(z) * T)
    return w[np.ix_(*idx)]
