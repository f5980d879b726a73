"""Min-max interpolator of the NUFFT, one dimension at a time (FP64).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper names the min-max interpolator of Fessler and Sutton as its default
kernel (Section 2.1; Section 2.1.3) but prints none of its formulas.  The
construction below is the published least-squares form, restated:

For an image x[n], n = 0..N-1 with centred coordinate t_n = n - N/2, the
exact spectrum at frequency w is X(w) = sum_n x[n] exp(-i w t_n).  The NUFFT
approximates it from the oversampled DFT of the scaled image,
Y[k] = sum_n s_n x[n] exp(-i gamma k t_n), gamma = 2 pi / K, by
X^(w) = sum_{j=1..J} c_j(w) Y[k0(w) + j].  The error is x^T (b - A c) with
b_n = exp(-i w t_n) and A[n, j] = s_n exp(-i gamma (k0 + j) t_n).  Its worst
case over unit-norm images is ||b - A c||_2, minimised by the least-squares
solution c = (A^H A)^{-1} A^H b = G^{-1} r with

  G[j, j'] = sum_n s_n^2 exp(+i gamma (j - j') t_n)          (J x J, no w)
  r_j(w)   = sum_n s_n exp(-i (w - gamma (k0 + j)) t_n).

With separable scaling s and a tensor-product neighbourhood, the d-dimensional
min-max coefficients are the Kronecker product of these 1D solutions (G and r
factor as Kronecker products), so only the 1D pieces are stored.

Readings where the paper is silent:
* scaling s: reciprocal of the Fourier transform of a Kaiser-Bessel kernel of
  width J grid cells with alpha = 2.34 J, i.e. s(t) = z / sinh(z),
  z = sqrt(alpha^2 - (pi J t / K)^2) (sin for a negative radicand), then
  normalised so that max_n s_n = 1;
* neighbourhood: k0 = floor(w / gamma) - J/2 for even J,
  k0 = floor(w / gamma + 1/2) - (J + 1)/2 for odd J, neighbours k0 + j,
  j = 1..J, wrapped modulo K; the floor is taken in FP64 on w / gamma with
  gamma = (2 pi) / K.
"""
from __future__ import annotations

import math

import numpy as np


def centred_coords(N: int) -> np.ndarray:
    """t_n = n - N/2 for n = 0..N-1 (image centre at n = N/2)."""
    return np.arange(N, dtype=np.float64) - N / 2.0


def kb_scaling_1d(N: int, K: int, J: int) -> np.ndarray:
    """Scaling factors s_n (FP64, length N), max-normalised to 1."""
    alpha = 2.34 * J
    t = centred_coords(N)
    s = np.empty(N, dtype=np.float64)
    for i in range(N):
        q = alpha * alpha - (math.pi * J * t[i] / K) ** 2
        if q > 0.0:
            z = math.sqrt(q)
            ft = math.sinh(z) / z
        elif q < 0.0:
            z = math.sqrt(-q)
            ft = math.sin(z) / z
        else:
            ft = 1.0
        s[i] = 1.0 / ft
    return s / s.max()


def offsets_1d(om: np.ndarray, K: int, J: int) -> np.ndarray:
    """First-neighbour offset k0 per point (int64; may be negative or >= K)."""
    gamma = (2.0 * math.pi) / K
    u = np.asarray(om, dtype=np.float64) / gamma
    if J % 2 == 0:
        k0 = np.floor(u) - J // 2
    else:
        k0 = np.floor(u + 0.5) - (J + 1) // 2
    return k0.astype(np.int64)


def minmax_G(s: np.ndarray, K: int, J: int) -> np.ndarray:
    """G[j, j'] = sum_n s_n^2 exp(i gamma (j - j') t_n), j, j' = 1..J."""
    N = s.shape[0]
    t = centred_coords(N)
    gamma = (2.0 * math.pi) / K
    G = np.empty((J, J), dtype=np.complex128)
    for a in range(J):
        for b in range(J):
            G[a, b] = np.sum(s * s * np.exp(1j * gamma * (a - b) * t))
    return G


def minmax_r(om: np.ndarray, k0: np.ndarray, s: np.ndarray, K: int, J: int) -> np.ndarray:
    """r[m, j-1] = sum_n s_n exp(-i (w_m - gamma (k0_m + j)) t_n), shape (M, J)."""
    om = np.asarray(om, dtype=np.float64)
    N = s.shape[0]
    t = centred_coords(N)
    gamma = (2.0 * math.pi) / K
    M = om.shape[0]
    r = np.empty((M, J), dtype=np.complex128)
    chunk = 4096
    for lo in range(0, M, chunk):
        hi = min(M, lo + chunk)
        for j in range(1, J + 1):
            u = om[lo:hi] - gamma * (k0[lo:hi] + j)              # (P,)
            E = np.exp(-1j * u[:, None] * t[None, :])             # (P, N)
            r[lo:hi, j - 1] = E @ s
    return r


def minmax_coefficients_1d(om: np.ndarray, N: int, K: int, J: int):
    """Return (k0 (M,), c (M, J) complex128, s (N,)) for one dimension."""
    s = kb_scaling_1d(N, K, J)
    k0 = offsets_1d(om, K, J)
    G = minmax_G(s, K, J)
    r = minmax_r(om, k0, s, K, J)
    c = np.linalg.solve(G, r.T).T
    return k0, c, s
