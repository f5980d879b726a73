"""GB300 (sm_103a) min-max NUFFT: Python binding of the C-ABI library.

The functions below carry the names of the C entry points in
``include/nufft_gb300.h`` and only marshal arguments (device pointers, sizes,
the current CUDA stream); every step of the computation runs in the library's
CUDA kernels.  PyTorch supplies device memory and streams.  There is no CPU
fallback: if the compiled library is missing, importing the binding raises.

Operators (PyNUFFT, arXiv:1710.03197): forward A = V F S (Section 2.1, Eq. 1),
adjoint A^H = S^H F^H V^H (Section 2.1.4, Eq. 2), self-adjoint A^H A
(Section 2.1.5), solvers CG (Section 2.2.2), L1TV-OLS (Eqs. 11-20) and
L1TV-LAD (Eqs. 21-31).
"""
from __future__ import annotations

from ._lib import lib, LIB_PATH, NufftError, check, symbols_declared
from .plan import (
    NufftPlan,
    NufftFrames,
    nufft_plan,
    nufft_plan_tuned,
    nufft_plan_set_trajectory,
    nufft_forward,
    nufft_adjoint,
    nufft_selfadjoint,
    nufft_forward_host,
    nufft_adjoint_host,
    nufft_scale_pad_fft,
    nufft_interp,
    nufft_gridding,
    nufft_gridding_static,
    nufft_ifft_crop_rescale,
    solve_cg,
    solve_l1tv_ols,
    solve_l1tv_lad,
    nufft_density_compensation,
    nufft_gridding_recon,
    solve_cg_kspace,
    nufft_forward_multicoil,
    nufft_adjoint_multicoil,
    nufft_selfadjoint_multicoil,
    solve_cg_multicoil,
    nufft_trajectory_gradient,
    nufft_trajectory_gradient_grid,
    nufft_forward_batch,
    nufft_adjoint_batch,
    nufft_selfadjoint_batch,
    nufft_toeplitz_init,
    nufft_selfadjoint_toeplitz,
    nufft_set_normal_operator,
)
from .autograd import NufftFunction, nufft_apply

__all__ = [
    "lib", "LIB_PATH", "NufftError", "check", "symbols_declared", "NufftPlan", "NufftFrames",
    "nufft_plan", "nufft_plan_tuned", "nufft_plan_set_trajectory", "nufft_forward", "nufft_adjoint", "nufft_selfadjoint",
    "nufft_forward_host", "nufft_adjoint_host", "nufft_scale_pad_fft", "nufft_interp",
    "nufft_gridding", "nufft_gridding_static", "nufft_ifft_crop_rescale", "solve_cg", "solve_l1tv_ols", "solve_l1tv_lad",
    "nufft_density_compensation", "nufft_gridding_recon", "solve_cg_kspace", "nufft_forward_multicoil",
    "nufft_adjoint_multicoil", "nufft_selfadjoint_multicoil", "solve_cg_multicoil",
    "nufft_trajectory_gradient", "nufft_trajectory_gradient_grid", "NufftFunction", "nufft_apply",
    "nufft_forward_batch", "nufft_adjoint_batch", "nufft_selfadjoint_batch",
    "nufft_toeplitz_init", "nufft_selfadjoint_toeplitz", "nufft_set_normal_operator",
]
