"""C-ABI checks that need no GPU: the library loads, exports every function the
public header declares, and rejects invalid arguments before touching CUDA."""
import ctypes

import pytest

from paper_1710_03197_gb300 import _lib

L = _lib.lib
EINVAL = 1


def test_library_exports_every_declared_function():
    declared = _lib.symbols_declared()
    assert len(declared) >= 18
    for name in declared:
        assert hasattr(L, name), name
    # and the binding wraps exactly what the header declares
    assert set(_lib._SIGS) == set(declared)


def _plan(d, N, K, J, M=10, om=1):
    h = ctypes.c_void_p(0)
    arr = lambda v: (ctypes.c_int * len(v))(*v)
    rc = L.nufft_plan(d, arr(N), arr(K), arr(J), M, ctypes.c_void_p(om), None, ctypes.byref(h))
    return rc, h


@pytest.mark.parametrize("d,N,K,J,M,om,frag", [
    (4, [8] * 4, [16] * 4, [4] * 4, 10, 1, "d = 4"),
    (0, [8], [16], [4], 10, 1, "d = 0"),
    (2, [8, 8], [16, 98], [4, 4], 10, 1, "prime factor"),      # 98 = 2 * 7^2
    (2, [8, 8], [16, 2048], [4, 4], 10, 1, "in [16, 1024]"),
    (2, [8, 8], [16, 45], [4, 4], 10, 1, "must be even"),       # odd K
    (1, [8], [14], [4], 10, 1, "in [16, 1024]"),
    (2, [7, 8], [16, 16], [4, 4], 10, 1, "even"),
    (2, [32, 8], [16, 16], [4, 4], 10, 1, "even"),
    (2, [8, 8], [16, 16], [0, 4], 10, 1, "J[0]"),
    (2, [8, 8], [16, 16], [4, 17], 10, 1, "J[1]"),
    (1, [8], [16], [4], -1, 1, "M ="),
    (1, [8], [16], [4], 10, 0, "om_dev is NULL"),
    (3, [8, 8, 8], [16, 16, 16], [16, 16, 16], 10, 1, "shared memory"),
])
def test_plan_rejects_bad_arguments(d, N, K, J, M, om, frag):
    """Argument checks that run before any CUDA call.  Kd must be even, in
    16..1024, with prime factors 2, 3 and 5 only (the FFT passes' radices)."""
    rc, h = _plan(d, N, K, J, M, om)
    assert rc == EINVAL
    assert not h.value
    assert frag in _lib.last_error(None)


def test_calls_reject_null_plan():
    null = ctypes.c_void_p(0)
    x = ctypes.c_void_p(1)
    for name in ["nufft_forward", "nufft_adjoint", "nufft_selfadjoint", "nufft_forward_host", "nufft_adjoint_host",
                 "nufft_scale_pad_fft", "nufft_interp", "nufft_gridding", "nufft_ifft_crop_rescale"]:
        assert getattr(L, name)(null, x, x) == EINVAL, name
    assert L.solve_cg(null, x, x, 3) == EINVAL
    assert L.solve_l1tv_ols(null, x, x, 1, 1, 1, 1.0, 1.0) == EINVAL
    assert L.solve_l1tv_lad(null, x, x, 1, 1, 1, 1.0, 1.0) == EINVAL
    for name in ["nufft_trajectory_gradient", "nufft_trajectory_gradient_grid"]:
        assert getattr(L, name)(null, x, x, x) == EINVAL, name
    assert L.nufft_plan_set_trajectory(null, x) == EINVAL
    assert L.nufft_set_stream(null, None) == EINVAL
    assert L.nufft_plan_info(null, None) == EINVAL
    assert L.nufft_plan_destroy(null) == 0
    assert "is NULL" in _lib.last_error(None)


def test_plan_out_pointer_required():
    arr = lambda v: (ctypes.c_int * len(v))(*v)
    assert L.nufft_plan(1, arr([8]), arr([16]), arr([4]), 0, None, None, None) == EINVAL
