"""FP64 CPU oracle for the min-max NUFFT and its solvers.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or run
anything in this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference arm of ``bench.py`` use it.  It shares no code with
the CUDA library (no kernels, headers, tables or constant generators); the only
common module is ``workloads.py``, which draws seeded inputs and holds none of
the method's arithmetic.

The oracle is written for a reader checking it against the paper, not for
speed: every step follows the operator chain A = V F S (Section 2.1, Eq. 1),
its adjoint A^H = S^H F^H V^H (Section 2.1.4, Eq. 2), the self-adjoint normal
operator A^H A (Section 2.1.5), and the solvers of Section 2.2.  Library
primitives used as single steps: ``numpy.fft.fftn``/``ifftn`` (the FFT),
``numpy.linalg.solve`` (the J x J min-max system), ``numpy.add.at`` (scatter).

Pins: every function is checked in ``tests/test_oracle_pins.py`` against
brute-force NUDFT, the adjoint identity, closed forms, least-squares
definitions solved by LAPACK, and dense solves; the L1TV-OLS and L1TV-LAD
outer (Bregman) loops are pinned in ``tests/test_oracle_pins_l1tv.py`` to the
limit the constrained problem fixes (x_true for full-rank consistent data, a
feasible TV minimiser for underdetermined data), with planted mistakes in
their update lines failing those pins.
"""
from .minmax import kb_scaling_1d, offsets_1d, minmax_G, minmax_r, minmax_coefficients_1d
from .nufft import Plan, make_plan, forward, adjoint, selfadjoint, nudft_forward, nudft_adjoint
from .nufft import scale_pad, fft_forward, interp_V, gridding_VH, fft_adjoint, crop_rescale
from .solvers import grad, grad_T, shrink, cg, l1tv_ols, l1tv_lad

__all__ = [
    "kb_scaling_1d", "offsets_1d", "minmax_G", "minmax_r", "minmax_coefficients_1d",
    "Plan", "make_plan", "forward", "adjoint", "selfadjoint", "nudft_forward", "nudft_adjoint",
    "scale_pad", "fft_forward", "interp_V", "gridding_VH", "fft_adjoint", "crop_rescale",
    "grad", "grad_T", "shrink", "cg", "l1tv_ols", "l1tv_lad",
]
