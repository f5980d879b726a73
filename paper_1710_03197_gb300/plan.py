"""Plan object and same-named wrappers of the C entry points.

Argument marshalling only: tensors are checked for device, dtype, contiguity
and size, then their data pointers and the current CUDA stream are handed to
the library.  Complex tensors are complex64 (interleaved float pairs).
"""
from __future__ import annotations

import ctypes

import torch

from ._lib import lib, check

_c_int_arr = lambda v: (ctypes.c_int * len(v))(*[int(t) for t in v])


def _stream_ptr(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


# torch's current stream as a raw handle without building a Stream object
# (about 3 us per call less); torch.cuda.current_stream where it is missing
_raw_current_stream = getattr(torch._C, "_cuda_getCurrentRawStream", None)


def _current_stream_handle(device_index: int) -> int:
    if _raw_current_stream is not None:
        return int(_raw_current_stream(device_index))
    return torch.cuda.current_stream(device_index).cuda_stream


def _dev_ptr(t: torch.Tensor, numel: int, name: str, dtype=torch.complex64):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.numel() != numel:
        raise ValueError(f"{name} has {t.numel()} elements, expected {numel}")
    return ctypes.c_void_p(t.data_ptr())


def _host_ptr(t: torch.Tensor, numel: int, name: str):
    if t.is_cuda or t.dtype != torch.complex64 or not t.is_contiguous() or t.numel() != numel:
        raise ValueError(f"{name} must be a contiguous complex64 host tensor with {numel} elements")
    return ctypes.c_void_p(t.data_ptr())


class NufftPlan:
    """Min-max NUFFT plan for one trajectory (C: ``nufft_plan``).

    om: (M, d) float32 CUDA tensor of frequencies in radians; Nd, Kd, Jd: image
    size, oversampled grid (even, prime factors 2, 3, 5) and neighbours per dimension.
    """

    def __init__(self, om: torch.Tensor, Nd, Kd, Jd, stream=None, autotune: bool = False):
        if om.dim() == 1:
            om = om[:, None]
        d = len(Nd)
        if om.dim() != 2 or om.shape[1] != d:
            raise ValueError("om must have shape (M, d)")
        M = om.shape[0]
        om_ptr = _dev_ptr(om.contiguous(), M * d, "om", dtype=torch.float32) if M > 0 else ctypes.c_void_p(0)
        self._om = om
        h = ctypes.c_void_p(0)
        make = lib.nufft_plan_tuned if autotune else lib.nufft_plan   # autotune: tile edge by measurement
        sp = _stream_ptr(stream)
        rc = make(d, _c_int_arr(Nd), _c_int_arr(Kd), _c_int_arr(Jd), M, om_ptr, sp, ctypes.byref(h))
        check(rc, None)
        self._h = h
        self._stream_key = sp.value or 0
        self.d, self.M = d, M
        self.Nd, self.Kd, self.Jd = tuple(int(v) for v in Nd), tuple(int(v) for v in Kd), tuple(int(v) for v in Jd)
        self.device = om.device
        self._dev_index = om.device.index if om.device.index is not None else torch.cuda.current_device()

    # ---------------------------------------------------------------- lifetime
    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib.nufft_plan_destroy(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_stream(self, stream=None):
        sp = _stream_ptr(stream)
        check(lib.nufft_set_stream(self._h, sp), self._h)
        self._stream_key = sp.value or 0

    def set_trajectory(self, om: torch.Tensor):
        """New trajectory of the same M points (C: nufft_plan_set_trajectory):
        only the per-point interpolator and the tile sort are redone."""
        if om.dim() == 1:
            om = om[:, None]
        if om.dim() != 2 or tuple(om.shape) != (self.M, self.d):
            raise ValueError(f"om must have shape ({self.M}, {self.d})")
        om = om.detach().to(torch.float32).contiguous()
        self._sync_stream()
        ptr = _dev_ptr(om, self.M * self.d, "om", dtype=torch.float32) if self.M > 0 else ctypes.c_void_p(0)
        check(lib.nufft_plan_set_trajectory(self._h, ptr), self._h)
        self._om = om

    def set_graphs(self, enable: bool):
        check(lib.nufft_set_graphs(self._h, 1 if enable else 0), self._h)

    def _sync_stream(self):
        # order the plan's work on torch's current stream; the library keeps the
        # stream it was last given, so the call is skipped when it is unchanged
        s = _current_stream_handle(self._dev_index)
        if s != self._stream_key:
            check(lib.nufft_set_stream(self._h, ctypes.c_void_p(s)), self._h)
            self._stream_key = s

    # ---------------------------------------------------------------- sizes
    @property
    def Nprod(self):
        n = 1
        for v in self.Nd:
            n *= v
        return n

    @property
    def Kprod(self):
        n = 1
        for v in self.Kd:
            n *= v
        return n

    def info(self):
        buf = (ctypes.c_int64 * 16)()
        check(lib.nufft_plan_info(self._h, buf), self._h)
        v = list(buf)
        return {"d": v[0], "M": v[1], "N": v[2:5][: self.d], "K": v[5:8][: self.d], "J": v[8:11][: self.d],
                "nbins": v[11], "nchunks": v[12], "device_bytes": v[13], "tile_first": v[14], "tile_last": v[15]}

    def interpolator(self):
        """(kfirst (M,d) int32, [coef_i (M,J_i) complex64], [s_i (N_i,) float32], perm (M,) int32) on host."""
        M, d = self.M, self.d
        kf = torch.empty((M, d), dtype=torch.int32)
        ncoef = sum(M * J for J in self.Jd)
        coef = torch.empty(ncoef, dtype=torch.complex64)
        s = torch.empty(sum(self.Nd), dtype=torch.float32)
        perm = torch.empty(M, dtype=torch.int32)
        check(lib.nufft_plan_get_interpolator(self._h, ctypes.c_void_p(kf.data_ptr()), ctypes.c_void_p(coef.data_ptr()),
                                              ctypes.c_void_p(s.data_ptr()), ctypes.c_void_p(perm.data_ptr())), self._h)
        coefs, off = [], 0
        for J in self.Jd:
            coefs.append(coef[off: off + M * J].reshape(M, J))
            off += M * J
        ss, off = [], 0
        for N in self.Nd:
            ss.append(s[off: off + N])
            off += N
        return kf, coefs, ss, perm

    # ---------------------------------------------------------------- operators
    def forward(self, x: torch.Tensor, y: torch.Tensor | None = None) -> torch.Tensor:
        if y is None:
            y = torch.empty(self.M, dtype=torch.complex64, device=self.device)
        self._sync_stream()
        check(lib.nufft_forward(self._h, _dev_ptr(x, self.Nprod, "x"), _dev_ptr(y, self.M, "y")), self._h)
        return y

    def adjoint(self, y: torch.Tensor, x: torch.Tensor | None = None) -> torch.Tensor:
        if x is None:
            x = torch.empty(self.Nd, dtype=torch.complex64, device=self.device)
        self._sync_stream()
        check(lib.nufft_adjoint(self._h, _dev_ptr(y, self.M, "y"), _dev_ptr(x, self.Nprod, "x")), self._h)
        return x

    def selfadjoint(self, x: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        if out is None:
            out = torch.empty(self.Nd, dtype=torch.complex64, device=self.device)
        self._sync_stream()
        check(lib.nufft_selfadjoint(self._h, _dev_ptr(x, self.Nprod, "x"), _dev_ptr(out, self.Nprod, "out")), self._h)
        return out

    def forward_host(self, x_host: torch.Tensor, y_host: torch.Tensor | None = None) -> torch.Tensor:
        if y_host is None:
            y_host = torch.empty(self.M, dtype=torch.complex64, pin_memory=True)
        self._sync_stream()
        check(lib.nufft_forward_host(self._h, _host_ptr(x_host, self.Nprod, "x_host"),
                                     _host_ptr(y_host, self.M, "y_host")), self._h)
        return y_host

    def adjoint_host(self, y_host: torch.Tensor, x_host: torch.Tensor | None = None) -> torch.Tensor:
        if x_host is None:
            x_host = torch.empty(self.Nd, dtype=torch.complex64, pin_memory=True)
        self._sync_stream()
        check(lib.nufft_adjoint_host(self._h, _host_ptr(y_host, self.M, "y_host"),
                                     _host_ptr(x_host, self.Nprod, "x_host")), self._h)
        return x_host

    # ---------------------------------------------------------------- stages
    def scale_pad_fft(self, x, grid=None):
        grid = torch.empty(self.Kd, dtype=torch.complex64, device=self.device) if grid is None else grid
        self._sync_stream()
        check(lib.nufft_scale_pad_fft(self._h, _dev_ptr(x, self.Nprod, "x"), _dev_ptr(grid, self.Kprod, "grid")), self._h)
        return grid

    def interp(self, grid, y=None):
        y = torch.empty(self.M, dtype=torch.complex64, device=self.device) if y is None else y
        self._sync_stream()
        check(lib.nufft_interp(self._h, _dev_ptr(grid, self.Kprod, "grid"), _dev_ptr(y, self.M, "y")), self._h)
        return y

    def gridding(self, y, grid=None):
        grid = torch.empty(self.Kd, dtype=torch.complex64, device=self.device) if grid is None else grid
        self._sync_stream()
        check(lib.nufft_gridding(self._h, _dev_ptr(y, self.M, "y"), _dev_ptr(grid, self.Kprod, "grid")), self._h)
        return grid

    def gridding_static(self, y, grid):
        """V^H y with the partial tiles in the library's fixed device array
        (no allocation by the call; see nufft_gridding_static in the header)."""
        self._sync_stream()
        check(lib.nufft_gridding_static(self._h, _dev_ptr(y, self.M, "y"), _dev_ptr(grid, self.Kprod, "grid")),
              self._h)
        return grid

    def ifft_crop_rescale(self, grid, x=None):
        x = torch.empty(self.Nd, dtype=torch.complex64, device=self.device) if x is None else x
        self._sync_stream()
        check(lib.nufft_ifft_crop_rescale(self._h, _dev_ptr(grid, self.Kprod, "grid"), _dev_ptr(x, self.Nprod, "x")),
              self._h)
        return x

    # ---------------------------------------------------------------- solvers
    def solve_cg(self, y, x=None, maxiter=20):
        x = torch.zeros(self.Nd, dtype=torch.complex64, device=self.device) if x is None else x
        self._sync_stream()
        check(lib.solve_cg(self._h, _dev_ptr(y, self.M, "y"), _dev_ptr(x, self.Nprod, "x"), int(maxiter)), self._h)
        return x

    def solve_l1tv_ols(self, y, x=None, maxiter=50, inner=2, cg_iters=5, mu=1.0, lam=0.01):
        x = torch.zeros(self.Nd, dtype=torch.complex64, device=self.device) if x is None else x
        self._sync_stream()
        check(lib.solve_l1tv_ols(self._h, _dev_ptr(y, self.M, "y"), _dev_ptr(x, self.Nprod, "x"), int(maxiter),
                                 int(inner), int(cg_iters), float(mu), float(lam)), self._h)
        return x

    def solve_l1tv_lad(self, y, x=None, maxiter=50, inner=2, cg_iters=5, mu=1.0, lam=0.01):
        x = torch.zeros(self.Nd, dtype=torch.complex64, device=self.device) if x is None else x
        self._sync_stream()
        check(lib.solve_l1tv_lad(self._h, _dev_ptr(y, self.M, "y"), _dev_ptr(x, self.Nprod, "x"), int(maxiter),
                                 int(inner), int(cg_iters), float(mu), float(lam)), self._h)
        return x


    # ---------------------------------------------------------------- batches (one plan, nb transforms)
    def _batch(self, t, per, name):
        nb = t.numel() // per
        if nb < 1 or nb * per != t.numel():
            raise ValueError(f"{name} must hold a whole number of elements of size {per}")
        return nb

    def forward_batch(self, x, y=None):
        nb = self._batch(x, self.Nprod, "x")
        y = torch.empty((nb, self.M), dtype=torch.complex64, device=self.device) if y is None else y
        self._sync_stream()
        check(lib.nufft_forward_batch(self._h, nb, _dev_ptr(x, nb * self.Nprod, "x"), _dev_ptr(y, nb * self.M, "y")),
              self._h)
        return y

    def adjoint_batch(self, y, x=None):
        nb = self._batch(y, self.M, "y")
        x = torch.empty((nb,) + self.Nd, dtype=torch.complex64, device=self.device) if x is None else x
        self._sync_stream()
        check(lib.nufft_adjoint_batch(self._h, nb, _dev_ptr(y, nb * self.M, "y"), _dev_ptr(x, nb * self.Nprod, "x")),
              self._h)
        return x

    def selfadjoint_batch(self, x, out=None):
        nb = self._batch(x, self.Nprod, "x")
        out = torch.empty((nb,) + self.Nd, dtype=torch.complex64, device=self.device) if out is None else out
        self._sync_stream()
        check(lib.nufft_selfadjoint_batch(self._h, nb, _dev_ptr(x, nb * self.Nprod, "x"),
                                          _dev_ptr(out, nb * self.Nprod, "out")), self._h)
        return out

    # ---------------------------------------------------------------- Toeplitz normal operator
    def toeplitz_init(self):
        self._sync_stream()
        check(lib.nufft_toeplitz_init(self._h), self._h)

    def selfadjoint_toeplitz(self, x, out=None):
        out = torch.empty(self.Nd, dtype=torch.complex64, device=self.device) if out is None else out
        self._sync_stream()
        check(lib.nufft_selfadjoint_toeplitz(self._h, _dev_ptr(x, self.Nprod, "x"), _dev_ptr(out, self.Nprod, "out")),
              self._h)
        return out

    def set_normal_operator(self, toeplitz: bool):
        check(lib.nufft_set_normal_operator(self._h, 1 if toeplitz else 0), self._h)

    # ---------------------------------------------------------------- trajectory gradient
    def trajectory_gradient(self, x, g, gom=None):
        """Re(conj(g) dy/dom) as an (M, d) float32 tensor (C: nufft_trajectory_gradient)."""
        gom = torch.empty((self.M, self.d), dtype=torch.float32, device=self.device) if gom is None else gom
        self._sync_stream()
        check(lib.nufft_trajectory_gradient(self._h, _dev_ptr(x, self.Nprod, "x"), _dev_ptr(g, self.M, "g"),
                                            _dev_ptr(gom, self.M * self.d, "gom", dtype=torch.float32)), self._h)
        return gom

    def trajectory_gradient_grid(self, grid, g, gom=None):
        """The same gradient from the oversampled spectrum F S x (C: nufft_trajectory_gradient_grid)."""
        gom = torch.empty((self.M, self.d), dtype=torch.float32, device=self.device) if gom is None else gom
        self._sync_stream()
        check(lib.nufft_trajectory_gradient_grid(self._h, _dev_ptr(grid, self.Kprod, "grid"), _dev_ptr(g, self.M, "g"),
                                                 _dev_ptr(gom, self.M * self.d, "gom", dtype=torch.float32)), self._h)
        return gom

    # ---------------------------------------------------------------- density compensation, k-space CG
    def density_compensation(self, iters: int, w=None):
        """Pipe-Menon weights (Eq. 5); w: float32 CUDA tensor of M starting weights (default ones)."""
        w = torch.ones(self.M, dtype=torch.float32, device=self.device) if w is None else w
        self._sync_stream()
        check(lib.nufft_density_compensation(self._h, _dev_ptr(w, self.M, "w", dtype=torch.float32), int(iters)),
              self._h)
        return w

    def gridding_recon(self, y, w, x=None):
        x = torch.empty(self.Nd, dtype=torch.complex64, device=self.device) if x is None else x
        self._sync_stream()
        check(lib.nufft_gridding_recon(self._h, _dev_ptr(y, self.M, "y"), _dev_ptr(w, self.M, "w", dtype=torch.float32),
                                       _dev_ptr(x, self.Nprod, "x")), self._h)
        return x

    def solve_cg_kspace(self, y, x=None, maxiter=20):
        x = torch.empty(self.Nd, dtype=torch.complex64, device=self.device) if x is None else x
        self._sync_stream()
        check(lib.solve_cg_kspace(self._h, _dev_ptr(y, self.M, "y"), _dev_ptr(x, self.Nprod, "x"), int(maxiter)),
              self._h)
        return x

    # ---------------------------------------------------------------- multi-coil
    def _coils(self, coils):
        if coils.dim() != self.d + 1 or tuple(coils.shape[1:]) != self.Nd:
            raise ValueError("coils must have shape (nc, *Nd)")
        return _dev_ptr(coils, coils.shape[0] * self.Nprod, "coils"), int(coils.shape[0])

    def forward_multicoil(self, coils, x, y=None):
        cp, nc = self._coils(coils)
        y = torch.empty(nc * self.M, dtype=torch.complex64, device=self.device) if y is None else y
        self._sync_stream()
        check(lib.nufft_forward_multicoil(self._h, cp, nc, _dev_ptr(x, self.Nprod, "x"), _dev_ptr(y, nc * self.M, "y")),
              self._h)
        return y

    def adjoint_multicoil(self, coils, y, x=None):
        cp, nc = self._coils(coils)
        x = torch.empty(self.Nd, dtype=torch.complex64, device=self.device) if x is None else x
        self._sync_stream()
        check(lib.nufft_adjoint_multicoil(self._h, cp, nc, _dev_ptr(y, nc * self.M, "y"), _dev_ptr(x, self.Nprod, "x")),
              self._h)
        return x

    def selfadjoint_multicoil(self, coils, x, out=None):
        cp, nc = self._coils(coils)
        out = torch.empty(self.Nd, dtype=torch.complex64, device=self.device) if out is None else out
        self._sync_stream()
        check(lib.nufft_selfadjoint_multicoil(self._h, cp, nc, _dev_ptr(x, self.Nprod, "x"),
                                              _dev_ptr(out, self.Nprod, "out")), self._h)
        return out

    def solve_cg_multicoil(self, coils, y, x=None, maxiter=20):
        cp, nc = self._coils(coils)
        x = torch.zeros(self.Nd, dtype=torch.complex64, device=self.device) if x is None else x
        self._sync_stream()
        check(lib.solve_cg_multicoil(self._h, cp, nc, _dev_ptr(y, nc * self.M, "y"), _dev_ptr(x, self.Nprod, "x"),
                                     int(maxiter)), self._h)
        return x


class NufftFrames:
    """A dynamic series (C: ``nufft_frames_create``): plans of equal image size
    over per-frame trajectories; the multi-coil normal operator of all frames
    is recorded as one CUDA graph with the frames as concurrent branches.  The
    plans must outlive the set."""

    def __init__(self, plans, stream=None):
        if not plans:
            raise ValueError("at least one plan")
        self.plans = list(plans)
        self.Nd = self.plans[0].Nd
        self.device = self.plans[0].device
        arr = (ctypes.c_void_p * len(self.plans))(*[p.handle.value for p in self.plans])
        h = ctypes.c_void_p(0)
        check(lib.nufft_frames_create(arr, len(self.plans), _stream_ptr(stream), ctypes.byref(h)), None)
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib.nufft_frames_destroy(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def selfadjoint_multicoil(self, coils, x, out=None):
        """out[f] = sum_i conj(c_i) A_f^H A_f (c_i x[f]); x, out: (nframes, *Nd)."""
        nf = len(self.plans)
        n = 1
        for v in self.Nd:
            n *= v
        if coils.dim() != len(self.Nd) + 1 or tuple(coils.shape[1:]) != self.Nd:
            raise ValueError("coils must have shape (nc, *Nd)")
        nc = int(coils.shape[0])
        out = torch.empty((nf,) + self.Nd, dtype=torch.complex64, device=self.device) if out is None else out
        check(lib.nufft_frames_set_stream(self._h, _stream_ptr()), None)
        check(lib.nufft_frames_selfadjoint_multicoil(self._h, _dev_ptr(coils, nc * n, "coils"), nc,
                                                     _dev_ptr(x, nf * n, "x"), _dev_ptr(out, nf * n, "out")), None)
        return out


# ---------------------------------------------------------------- same names as the C ABI
def nufft_plan(om, Nd, Kd, Jd, stream=None) -> NufftPlan:
    return NufftPlan(om, Nd, Kd, Jd, stream)


def nufft_plan_tuned(om, Nd, Kd, Jd, stream=None) -> NufftPlan:
    return NufftPlan(om, Nd, Kd, Jd, stream, autotune=True)


def nufft_plan_set_trajectory(plan: NufftPlan, om) -> None:
    plan.set_trajectory(om)


def nufft_forward(plan: NufftPlan, x, y=None):
    return plan.forward(x, y)


def nufft_adjoint(plan: NufftPlan, y, x=None):
    return plan.adjoint(y, x)


def nufft_selfadjoint(plan: NufftPlan, x, out=None):
    return plan.selfadjoint(x, out)


def nufft_forward_host(plan: NufftPlan, x_host, y_host=None):
    return plan.forward_host(x_host, y_host)


def nufft_adjoint_host(plan: NufftPlan, y_host, x_host=None):
    return plan.adjoint_host(y_host, x_host)


def nufft_scale_pad_fft(plan: NufftPlan, x, grid=None):
    return plan.scale_pad_fft(x, grid)


def nufft_interp(plan: NufftPlan, grid, y=None):
    return plan.interp(grid, y)


def nufft_gridding(plan: NufftPlan, y, grid=None):
    return plan.gridding(y, grid)


def nufft_gridding_static(plan: NufftPlan, y, grid):
    return plan.gridding_static(y, grid)


def nufft_ifft_crop_rescale(plan: NufftPlan, grid, x=None):
    return plan.ifft_crop_rescale(grid, x)


def solve_cg(plan: NufftPlan, y, x=None, maxiter=20):
    return plan.solve_cg(y, x, maxiter)


def solve_l1tv_ols(plan: NufftPlan, y, x=None, maxiter=50, inner=2, cg_iters=5, mu=1.0, lam=0.01):
    return plan.solve_l1tv_ols(y, x, maxiter, inner, cg_iters, mu, lam)


def solve_l1tv_lad(plan: NufftPlan, y, x=None, maxiter=50, inner=2, cg_iters=5, mu=1.0, lam=0.01):
    return plan.solve_l1tv_lad(y, x, maxiter, inner, cg_iters, mu, lam)


def nufft_density_compensation(plan: NufftPlan, iters: int, w=None):
    return plan.density_compensation(iters, w)


def nufft_gridding_recon(plan: NufftPlan, y, w, x=None):
    return plan.gridding_recon(y, w, x)


def solve_cg_kspace(plan: NufftPlan, y, x=None, maxiter=20):
    return plan.solve_cg_kspace(y, x, maxiter)


def nufft_forward_multicoil(plan: NufftPlan, coils, x, y=None):
    return plan.forward_multicoil(coils, x, y)


def nufft_adjoint_multicoil(plan: NufftPlan, coils, y, x=None):
    return plan.adjoint_multicoil(coils, y, x)


def nufft_selfadjoint_multicoil(plan: NufftPlan, coils, x, out=None):
    return plan.selfadjoint_multicoil(coils, x, out)


def solve_cg_multicoil(plan: NufftPlan, coils, y, x=None, maxiter=20):
    return plan.solve_cg_multicoil(coils, y, x, maxiter)


def nufft_trajectory_gradient(plan: NufftPlan, x, g, gom=None):
    return plan.trajectory_gradient(x, g, gom)


def nufft_trajectory_gradient_grid(plan: NufftPlan, grid, g, gom=None):
    return plan.trajectory_gradient_grid(grid, g, gom)


def nufft_forward_batch(plan: NufftPlan, x, y=None):
    return plan.forward_batch(x, y)


def nufft_adjoint_batch(plan: NufftPlan, y, x=None):
    return plan.adjoint_batch(y, x)


def nufft_selfadjoint_batch(plan: NufftPlan, x, out=None):
    return plan.selfadjoint_batch(x, out)


def nufft_toeplitz_init(plan: NufftPlan):
    return plan.toeplitz_init()


def nufft_selfadjoint_toeplitz(plan: NufftPlan, x, out=None):
    return plan.selfadjoint_toeplitz(x, out)


def nufft_set_normal_operator(plan: NufftPlan, mode: int):
    return plan.set_normal_operator(bool(mode))
