"""ctypes loader for libnufft_gb300.so (built in-tree by ``build.py``)."""
from __future__ import annotations

import ctypes
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnufft_gb300.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "nufft_gb300.h")

NUFFT_OK, NUFFT_EINVAL, NUFFT_ENOMEM, NUFFT_ECUDA, NUFFT_ETIMEOUT = 0, 1, 2, 3, 4
_NAMES = {1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ETIMEOUT"}


class NufftError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"NUFFT_{_NAMES.get(code, code)}: {msg}")
        self.code = code


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build the CUDA library first "
            "(python -c 'import __graft_entry__ as g; g.build()')")
    return ctypes.CDLL(LIB_PATH)


lib = _load()

_vp, _i, _i64, _d = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
_PLAN = ctypes.c_void_p

_SIGS = {
    "nufft_plan": (_i, [_i, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_i), _i64, _vp, _vp,
                        ctypes.POINTER(_PLAN)]),
    "nufft_plan_tuned": (_i, [_i, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_i), _i64, _vp, _vp,
                              ctypes.POINTER(_PLAN)]),
    "nufft_plan_destroy": (_i, [_PLAN]),
    "nufft_last_error": (ctypes.c_char_p, [_PLAN]),
    "nufft_set_stream": (_i, [_PLAN, _vp]),
    "nufft_plan_set_trajectory": (_i, [_PLAN, _vp]),
    "nufft_set_graphs": (_i, [_PLAN, _i]),
    "nufft_plan_info": (_i, [_PLAN, ctypes.POINTER(_i64)]),
    "nufft_plan_get_interpolator": (_i, [_PLAN, _vp, _vp, _vp, _vp]),
    "nufft_forward": (_i, [_PLAN, _vp, _vp]),
    "nufft_adjoint": (_i, [_PLAN, _vp, _vp]),
    "nufft_selfadjoint": (_i, [_PLAN, _vp, _vp]),
    "nufft_forward_host": (_i, [_PLAN, _vp, _vp]),
    "nufft_adjoint_host": (_i, [_PLAN, _vp, _vp]),
    "nufft_scale_pad_fft": (_i, [_PLAN, _vp, _vp]),
    "nufft_interp": (_i, [_PLAN, _vp, _vp]),
    "nufft_gridding": (_i, [_PLAN, _vp, _vp]),
    "nufft_gridding_static": (_i, [_PLAN, _vp, _vp]),
    "nufft_ifft_crop_rescale": (_i, [_PLAN, _vp, _vp]),
    "solve_cg": (_i, [_PLAN, _vp, _vp, _i]),
    "solve_l1tv_ols": (_i, [_PLAN, _vp, _vp, _i, _i, _i, _d, _d]),
    "solve_l1tv_lad": (_i, [_PLAN, _vp, _vp, _i, _i, _i, _d, _d]),
    "nufft_density_compensation": (_i, [_PLAN, _vp, _i]),
    "nufft_gridding_recon": (_i, [_PLAN, _vp, _vp, _vp]),
    "solve_cg_kspace": (_i, [_PLAN, _vp, _vp, _i]),
    "nufft_forward_multicoil": (_i, [_PLAN, _vp, _i, _vp, _vp]),
    "nufft_adjoint_multicoil": (_i, [_PLAN, _vp, _i, _vp, _vp]),
    "nufft_selfadjoint_multicoil": (_i, [_PLAN, _vp, _i, _vp, _vp]),
    "solve_cg_multicoil": (_i, [_PLAN, _vp, _i, _vp, _vp, _i]),
    "nufft_frames_create": (_i, [ctypes.POINTER(_PLAN), _i, _vp, ctypes.POINTER(_vp)]),
    "nufft_frames_destroy": (_i, [_vp]),
    "nufft_frames_set_stream": (_i, [_vp, _vp]),
    "nufft_frames_selfadjoint_multicoil": (_i, [_vp, _vp, _i, _vp, _vp]),
    "nufft_trajectory_gradient": (_i, [_PLAN, _vp, _vp, _vp]),
    "nufft_trajectory_gradient_grid": (_i, [_PLAN, _vp, _vp, _vp]),
    "nufft_forward_batch": (_i, [_PLAN, _i, _vp, _vp]),
    "nufft_adjoint_batch": (_i, [_PLAN, _i, _vp, _vp]),
    "nufft_selfadjoint_batch": (_i, [_PLAN, _i, _vp, _vp]),
    "nufft_toeplitz_init": (_i, [_PLAN]),
    "nufft_selfadjoint_toeplitz": (_i, [_PLAN, _vp, _vp]),
    "nufft_set_normal_operator": (_i, [_PLAN, _i]),
    "nufft_debug_fail_allocation": (_i, [_i64]),
    "nufft_debug_device_bytes": (_i64, []),
}

for _name, (_res, _args) in _SIGS.items():
    _fn = getattr(lib, _name)
    _fn.restype = _res
    _fn.argtypes = _args


def last_error(plan=None) -> str:
    msg = lib.nufft_last_error(plan)
    return msg.decode() if msg else ""


def check(rc: int, plan=None) -> None:
    if rc != NUFFT_OK:
        raise NufftError(rc, last_error(plan))


def symbols_declared(header: str = HEADER):
    """Names of every function the public header declares."""
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([a-z_][a-z0-9_]*)\s*\(",
                                 text, flags=re.M)))
