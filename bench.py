"""Benchmark: min-max NUFFT forward + adjoint throughput on GB300.

One step = y = A x (scale+pad+FFT, interpolation) then x' = A^H y (gridding,
inverse FFT + crop + rescale) on one batch of synthetic input: the operator
pair of Section 2.1 (Eq. 1) and Section 2.1.4 (Eq. 2).  Metric: non-uniform
points per second (M points per forward+adjoint pair), inputs resident in
HBM, device-timed with CUDA events per step, L2 flushed between steps.

Workload (default): 2D, 256x256 image, 512x512 grid, J = 6x6, golden-angle
radial 403 spokes x 512 samples (206,336 points).  The 3D kooshball (128^3
image, 256^3 grid, J = 6^3, 2,097,152 points) is measured in the same run and
reported under "also".

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun) every rank runs an independent replica of the workload
(the operator has no data-parallel exchange); time is the max over ranks and
the value counts the points of all ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "NUFFT fwd+adj nonuniform pts/s (2D 256^2, 3D 128^3); % HBM roofline vs plain"
UNIT = "points/s"
FALLBACK_HBM_GBS = 6800.0


# ------------------------------------------------------------------ helpers (host logic, tested on CPU)

def algorithmic_bytes(spec: dict) -> dict:
    """Minimum bytes each stage must move (complex64 data, int32 offsets)."""
    d, M = spec["d"], spec["M"]
    Nprod = int(np.prod(spec["Nd"]))
    Kprod = int(np.prod(spec["Kd"]))
    point = 4 * d + 8 * int(sum(spec["Jd"])) + 8          # first neighbours + coefficients + sample
    return {
        "scale_pad_fft": 8 * Nprod + 8 * Kprod,             # image read once, grid written once
        "interp": 8 * Kprod + M * point,
        "gridding": 8 * Kprod + M * point,
        "ifft_crop_rescale": 8 * Kprod + 8 * Nprod,
    }


def launches_per_step(spec: dict, nchunks: int) -> int:
    d = spec["d"]
    fwd = d + 1                                   # d FFT passes + interpolation
    adj = (1 if nchunks > 0 else 0) + 1 + d       # gridding chunks + tile reduction + d inverse passes
    return fwd + adj


def reduce_over_ranks(elapsed_s: float, units: float, world: int):
    """Max elapsed time and summed units over ranks (identity for one rank)."""
    if world <= 1:
        return elapsed_s, units
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([elapsed_s], dtype=torch.float64, device=dev)
    u = torch.tensor([units], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, out_path: str | None = None):
        self.gpu_index = gpu_index
        self.proc = None
        self.out_path = out_path

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu_index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]
        if self.out_path:
            with open(self.out_path, "w") as f:
                f.write("\n".join(self.lines) + "\n")

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() in ("active", "1"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ our arm

STAGES = ("scale_pad_fft", "interp", "gridding", "ifft_crop_rescale")

WORKLOAD_TEXT = {
    "radial2d_256": "radial2d_256: 2D 256x256 image, 512x512 grid, J=6x6, golden-angle radial 403 spokes x 512 "
                    "samples (206,336 points), ellipse phantom",
    "kooshball3d_128": "kooshball3d_128: 3D 128^3 image, 256^3 grid, J=6^3, kooshball 8192 Fibonacci spokes x 256 "
                       "samples (2,097,152 points), complex normal image",
    "radial2d_64": "radial2d_64: 2D 64x64 image, 128x128 grid, J=6x6, 64 uniform spokes x 128 samples (8192 points)",
    "radial2d_256_K384": "radial2d_256_K384: the radial2d_256 image and trajectory on a 1.5x oversampled 384x384 "
                         "grid (mixed-radix FFT passes, radix 3), J=6x6, 206,336 points",
}


def run_workload(nf, torch, name: str, steps: int, warmup: int, dev, flush_bytes: int, solvers: bool = False,
                 extra_rows: bool = True, autotune: bool = True):
    spec, om, x, noise = W.make_workload(name)
    M = spec["M"]
    om_d = torch.from_numpy(om).to(dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plan = nf.NufftPlan(om_d, spec["Nd"], spec["Kd"], spec["Jd"])
    torch.cuda.synchronize()
    plan_ms = (time.perf_counter() - t0) * 1e3
    default_tile = plan.info()["tile_last"]
    plan.close()
    # the timed steps use the autotuned plan (tile edge chosen by measurement);
    # --no-autotune keeps the default plan (profiling runs: no candidate plans)
    t0 = time.perf_counter()
    plan = nf.NufftPlan(om_d, spec["Nd"], spec["Kd"], spec["Jd"], autotune=autotune)
    torch.cuda.synchronize()
    tuned_ms = (time.perf_counter() - t0) * 1e3 if autotune else None
    info = plan.info()
    xd = torch.from_numpy(x).to(dev)
    grid = torch.empty(spec["Kd"], dtype=torch.complex64, device=dev)
    y = torch.empty(M, dtype=torch.complex64, device=dev)
    xo = torch.empty(spec["Nd"], dtype=torch.complex64, device=dev)
    flush = torch.empty(flush_bytes // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        # the same kernel sequence as nufft_forward + nufft_adjoint, called stage by stage
        plan.scale_pad_fft(xd, grid)
        plan.interp(grid, y)
        plan.gridding(y, grid)
        plan.ifft_crop_rescale(grid, xo)

    for _ in range(warmup):
        step()
        flush.fill_(1.0)
    torch.cuda.synchronize()
    # Per-stage GPU times: the staged step is captured into a CUDA graph with
    # timing events between the stage calls (the library's calls launch into
    # the caller's capture), so host call overhead does not enter the stage
    # times; the graph is replayed once per step with L2 flushed in between.
    try:
        evs = [torch.cuda.Event(enable_timing=True, external=True) for _ in range(len(STAGES) + 1)]
        cap = torch.cuda.Stream()
        cap.wait_stream(stream)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(cap):
            with torch.cuda.graph(g, stream=cap):
                evs[0].record()
                plan.scale_pad_fft(xd, grid)
                evs[1].record()
                plan.interp(grid, y)
                evs[2].record()
                plan.gridding(y, grid)
                evs[3].record()
                plan.ifft_crop_rescale(grid, xo)
                evs[4].record()
        torch.cuda.synchronize()
        stage_ms = {s: [] for s in STAGES}
        staged_ms = []
        for k in range(steps):
            flush.fill_(float(k))                      # evict the previous step's data from L2
            g.replay()
            torch.cuda.synchronize()
            for i, s_ in enumerate(STAGES):
                stage_ms[s_].append(evs[i].elapsed_time(evs[i + 1]))
            staged_ms.append(evs[0].elapsed_time(evs[-1]))
        del g
        stage_timing = "graph replay"
    except (RuntimeError, TypeError):
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(len(STAGES) + 1)] for _ in range(steps)]
        for k in range(steps):
            flush.fill_(float(k))
            e = ev[k]
            e[0].record(stream)
            plan.scale_pad_fft(xd, grid)
            e[1].record(stream)
            plan.interp(grid, y)
            e[2].record(stream)
            plan.gridding(y, grid)
            e[3].record(stream)
            plan.ifft_crop_rescale(grid, xo)
            e[4].record(stream)
        torch.cuda.synchronize()
        staged_ms = [ev[k][0].elapsed_time(ev[k][-1]) for k in range(steps)]
        stage_ms = {s: [ev[k][i].elapsed_time(ev[k][i + 1]) for k in range(steps)] for i, s in enumerate(STAGES)}
        stage_timing = "eager calls"

    # The timed step: the operator entry points a user calls (nufft_forward,
    # nufft_adjoint), which replay their recorded CUDA graphs after the first
    # two calls.  The staged loop above gives the per-stage breakdown.
    for _ in range(max(3, warmup)):
        plan.forward(xd, y)
        plan.adjoint(y, xo)
        flush.fill_(1.0)
    torch.cuda.synchronize()
    evm = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        flush.fill_(float(k))
        evm[k][0].record(stream)
        plan.forward(xd, y)
        plan.adjoint(y, xo)
        evm[k][1].record(stream)
    torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in evm]

    rows = {"a1_plan_ms": round(plan_ms, 3), "a1_plan_tuned_ms": None if tuned_ms is None else round(tuned_ms, 3),
            "tile_edge": {"default": default_tile, "tuned": info["tile_last"]}}
    if extra_rows:
        rows.update(_extra_rows(plan, torch, spec, x, xd, xo, noise, steps, flush, stream, dev, solvers))

    # end to end through the host-buffer entry points (pinned host memory)
    x_h = torch.from_numpy(x).pin_memory()
    y_h = torch.empty(M, dtype=torch.complex64).pin_memory()
    xo_h = torch.empty(spec["Nd"], dtype=torch.complex64).pin_memory()
    for _ in range(2):
        plan.forward_host(x_h, y_h)
        plan.adjoint_host(y_h, xo_h)
    t0 = time.perf_counter()
    for _ in range(steps):
        plan.forward_host(x_h, y_h)
        plan.adjoint_host(y_h, xo_h)
    e2e_s = (time.perf_counter() - t0) / steps
    nprod = int(np.prod(spec["Nd"]))
    plan.close()
    return dict(spec=spec, info=info, step_ms=step_ms, stage_ms=stage_ms, staged_ms=staged_ms, e2e_s=e2e_s,
                stage_timing=stage_timing,
                h2d=8 * (nprod + M), d2h=8 * (M + nprod), rows=rows)


def _extra_rows(plan, torch, spec, x, xd, xo, noise, steps, flush, stream, dev, solvers):
    """Rows beyond the timed step: A^H A, the Toeplitz operator, the solvers."""
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # the self-adjoint operator A^H A (one call per step, L2 flushed between)
    sa = []
    for k in range(steps):
        flush.fill_(float(k))
        e0.record(stream)
        plan.selfadjoint(xd, xo)
        e1.record(stream)
        e1.synchronize()
        sa.append(e0.elapsed_time(e1))
    rows = {"a8_selfadjoint_ms": round(statistics.mean(sa), 5)}
    # the Toeplitz-embedded normal operator (init once, then per call)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plan.toeplitz_init()
    torch.cuda.synchronize()
    rows["f4_toeplitz_init_ms"] = round((time.perf_counter() - t0) * 1e3, 3)
    st_ = []
    for k in range(steps):
        flush.fill_(float(k))
        e0.record(stream)
        plan.selfadjoint_toeplitz(xd, xo)
        e1.record(stream)
        e1.synchronize()
        st_.append(e0.elapsed_time(e1))
    rows["f4_selfadjoint_toeplitz_ms"] = round(statistics.mean(st_), 5)
    # cuFFT (through torch.fft) on the same oversampled grid, for comparison
    # only: the full unpruned transform, no scaling or padding, L2 flushed
    gfull = torch.randn(*spec["Kd"], dtype=torch.complex64, device=dev)
    for key, fn in (("cufft_fft_ms", lambda: torch.fft.fftn(gfull)), ("cufft_ifft_ms", lambda: torch.fft.ifftn(gfull))):
        fn()
        t_ = []
        for k in range(steps):
            flush.fill_(float(k))
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            t_.append(e0.elapsed_time(e1))
        rows[key] = round(statistics.mean(t_), 5)
    del gfull
    if solvers:
        # the reconstruction runs of the paper's solvers on this workload's
        # data.  Each solve runs three times on the same buffers (reset to the
        # start value): the first call launches eagerly, the second records
        # the library's graph, the third replays it and is the reported time;
        # the first is reported beside it as *_eager_ms.
        yd = plan.forward(xd)
        if noise is not None:
            yd = yd + torch.from_numpy(noise).to(dev)
        yd = yd.contiguous()
        xb = torch.zeros(spec["Nd"], dtype=torch.complex64, device=dev)
        wb = torch.ones(plan.M, dtype=torch.float32, device=dev)

        def timed(key, fn, reset):
            t_ = []
            for _ in range(3):
                reset()
                torch.cuda.synchronize()
                e0.record(stream)
                fn()
                e1.record(stream)
                e1.synchronize()
                t_.append(e0.elapsed_time(e1))
            rows[key] = round(t_[-1], 3)
            rows[key.replace("_ms", "_eager_ms")] = round(t_[0], 3)

        zero_x = xb.zero_
        timed("a9_cg_100_iterations_ms", lambda: plan.solve_cg(yd, xb, maxiter=100), zero_x)
        timed("a9_l1tv_ols_50_iterations_ms",
              lambda: plan.solve_l1tv_ols(yd, xb, maxiter=50, inner=2, cg_iters=5, mu=1.0, lam=0.01), zero_x)
        timed("a9_l1tv_lad_50_iterations_ms",
              lambda: plan.solve_l1tv_lad(yd, xb, maxiter=50, inner=2, cg_iters=5, mu=1.0, lam=0.01), zero_x)
        rows["a9_solver_settings"] = "CG x0=0; L1TV: inner=2, cg_iters=5, mu=1, lambda=0.01"
        # density compensation (Pipe-Menon, 5 iterations from w = 1) and the
        # gridding reconstruction A^H (y w); the paper's k-space CG (20 steps)
        timed("f3_density_compensation_5_iterations_ms", lambda: plan.density_compensation(5, wb),
              lambda: wb.fill_(1.0))
        timed("f3_gridding_recon_ms", lambda: plan.gridding_recon(yd, wb, xb), lambda: None)
        timed("f4_cg_kspace_20_iterations_ms", lambda: plan.solve_cg_kspace(yd, xb, maxiter=20), lambda: None)
        # the same solves with the Toeplitz normal operator
        plan.set_normal_operator(True)
        timed("f4_cg_100_iterations_toeplitz_ms", lambda: plan.solve_cg(yd, xb, maxiter=100), zero_x)
        timed("f4_l1tv_ols_50_iterations_toeplitz_ms",
              lambda: plan.solve_l1tv_ols(yd, xb, maxiter=50, inner=2, cg_iters=5, mu=1.0, lam=0.01), zero_x)
        plan.set_normal_operator(False)
    return rows


def roofline_for(res, peak_gbs: float, peak_kind: str, traffic: dict):
    alg = algorithmic_bytes(res["spec"])
    per_stage = {}
    for s in STAGES:
        ms = statistics.mean(res["stage_ms"][s])
        gbs = alg[s] / (ms * 1e-3) / 1e9
        per_stage[s] = {"ms": round(ms, 5), "alg_bytes": alg[s], "achieved_gbs": round(gbs, 1),
                        "frac": round(gbs / peak_gbs, 4)}
    dom = max(STAGES, key=lambda s: per_stage[s]["ms"])
    r = per_stage[dom]
    return dom, per_stage, {
        "bound": "hbm", "kernel": dom, "achieved": r["achieved_gbs"], "peak": peak_gbs, "unit": "GB/s",
        "frac": r["frac"], "peak_kind": f"{peak_kind} hbm_gbs", "traffic": traffic.get(dom),
    }


def ours(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    import paper_1710_03197_gb300 as nf

    flush_bytes = 512 * 1024 * 1024
    clocks_path = args.clocks_csv   # optional copy of the raw nvidia-smi samples
    if world > 1:
        torch.distributed.barrier()
    names = [w.strip() for w in args.workloads.split(",") if w.strip()]
    with ClockSampler(torch.cuda.current_device() if world == 1 else local, clocks_path) as clk:
        results = {n: run_workload(nf, torch, n, args.steps, args.warmup, dev, flush_bytes,
                                   solvers=(i == 0 and not args.no_solvers), extra_rows=not args.no_rows,
                                   autotune=not args.no_autotune)
                   for i, n in enumerate(names)}
        next_rows = None
        if not args.no_solvers and not args.no_rows:
            next_rows = {"f1_multicoil_dynamic": run_multicoil_dynamic(nf, torch, dev),
                         "f2_differentiable_spiral": run_differentiable(nf, torch, dev)}
    torch.cuda.synchronize()
    res2 = results[names[0]]

    M2 = res2["spec"]["M"]
    tot_ms = sum(res2["step_ms"])
    elapsed, units = reduce_over_ranks(tot_ms * 1e-3, M2 * args.steps, world)
    value = units / elapsed
    e2e_el, e2e_units = reduce_over_ranks(res2["e2e_s"] * args.steps, M2 * args.steps, world)
    others = {}
    for n in names[1:]:
        r = results[n]
        others[n] = (r, reduce_over_ranks(sum(r["step_ms"]) * 1e-3, r["spec"]["M"] * args.steps, world))
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return

    peak, peak_kind = load_peaks()
    traffic_all = {}
    tpath = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tpath):
        with open(tpath) as f:
            traffic_all = json.load(f)
    dom2, stages2, roof2 = roofline_for(res2, peak, peak_kind, traffic_all.get(names[0], {}))

    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline(seconds=args.cpu_seconds)

    line = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(elapsed * 1e3 / args.steps, 5), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c64", "data": "synthetic",
        "config": {"workload": WORKLOAD_TEXT[names[0]],
                   "step": "A x then A^H y (nufft_forward + nufft_adjoint, recorded CUDA graphs replayed)",
                   "l2": "flushed between timed steps (512 MB write)",
                   "parallelism": f"replicas x{world}"},
        "e2e": {"value": round(e2e_units / e2e_el, 1), "unit": UNIT, "h2d_bytes_per_step": res2["h2d"],
                "d2h_bytes_per_step": res2["d2h"]},
        "gpu_launches": launches_per_step(res2["spec"], res2["info"]["nchunks"]) * args.steps,
        "roofline": roof2,
        "stages": stages2,
        "staged_ms_per_step": round(statistics.mean(res2["staged_ms"]), 5),
        "stage_timing": res2["stage_timing"],
        "rows": res2["rows"],
        "next_rows": next_rows,
        "clocks": clk.summary(),
        "cpu_baseline": cpu,
    }
    if others:
        line["also"] = {}
        for n, (r, (el_n, un_n)) in others.items():
            _, stages_n, roof_n = roofline_for(r, peak, peak_kind, traffic_all.get(n, {}))
            line["also"][n] = {
                "workload": WORKLOAD_TEXT[n],
                "value": round(un_n / el_n, 1), "unit": UNIT, "ms_per_step": round(el_n * 1e3 / args.steps, 5),
                "e2e": {"value": round(r["spec"]["M"] / r["e2e_s"], 1), "unit": UNIT,
                        "h2d_bytes_per_step": r["h2d"], "d2h_bytes_per_step": r["d2h"]},
                "gpu_launches": launches_per_step(r["spec"], r["info"]["nchunks"]) * args.steps,
                "roofline": roof_n, "stages": stages_n, "rows": r["rows"],
                "staged_ms_per_step": round(statistics.mean(r["staged_ms"]), 5)}
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


# ------------------------------------------------------------------ next rows: batched multi-coil, differentiable

def run_multicoil_dynamic(nf, torch, dev, reps: int = 5):
    """32 coils x 8 frames, 256^2, uneven golden-angle frames: the multi-coil
    normal operator sum_i conj(c_i) A_f^H A_f (c_i x_f) for every frame, batched
    (one launch per stage for all coils of a frame) against the plain form
    (one single-coil A^H A call per coil, coil products as tensor ops)."""
    frames = W.dynamic_radial_frames(8, 512)
    Nd, Kd, Jd = (256, 256), (512, 512), (6, 6)
    nc = 32
    coils = torch.from_numpy(W.coil_maps(nc, Nd)).to(dev)
    x = torch.from_numpy(W.ellipse_phantom(256)).to(dev)
    plans = [nf.NufftPlan(torch.from_numpy(om).to(dev), Nd, Kd, Jd) for om in frames]
    out = torch.empty(Nd, dtype=torch.complex64, device=dev)
    tmp = torch.empty(Nd, dtype=torch.complex64, device=dev)

    def batched():
        for p in plans:
            p.selfadjoint_multicoil(coils, x, out)

    def plain():
        for p in plans:
            out.zero_()
            for c in range(nc):
                p.selfadjoint(coils[c] * x, tmp)
                out.add_(coils[c].conj() * tmp)

    # all frames in one recorded graph (frames as concurrent branches)
    fs = nf.NufftFrames(plans)
    xs = x.unsqueeze(0).repeat(len(plans), 1, 1).contiguous()
    outs = torch.empty_like(xs)

    def frames_graph():
        fs.selfadjoint_multicoil(coils, xs, outs)

    res = {}
    for key, fn in (("batched", batched), ("frames_graph", frames_graph), ("plain", plain)):
        fn()
        fn()                                   # second call records the graphs
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        e1.synchronize()
        res[key] = e0.elapsed_time(e1) / reps
    samples = nc * sum(om.shape[0] for om in frames)
    fs.close()
    for p in plans:
        p.close()
    return {"workload": "32 coils x 8 frames, 256^2, golden-angle frames of U{13..89} spokes x 512 samples "
                        f"({samples} coil samples), grid 512^2, J=6x6",
            "batched_ms": round(res["batched"], 4), "frames_graph_ms": round(res["frames_graph"], 4),
            "plain_ms": round(res["plain"], 4),
            "batched_coil_samples_per_s": round(samples / (res["batched"] * 1e-3), 1),
            "plain_coil_samples_per_s": round(samples / (res["plain"] * 1e-3), 1)}


def run_differentiable(nf, torch, dev, reps: int = 5):
    """256^2 spiral (16 x 2048, om + N(0, 1e-3)): forward + backward through the
    autograd function with a plan rebuilt each step, with one plan moved to
    each step's trajectory (nufft_plan_set_trajectory) and with a fixed plan,
    against the plain forward + adjoint; then 50 L1TV-LAD iterations."""
    spec, om, x, noise = W.make_workload("spiral2d_256")
    Nd, Kd, Jd = spec["Nd"], spec["Kd"], spec["Jd"]
    om_d = torch.from_numpy(om).to(dev)
    x_d = torch.from_numpy(x).to(dev)
    plan = nf.NufftPlan(om_d, Nd, Kd, Jd)
    y0 = (plan.forward(x_d) + torch.from_numpy(noise).to(dev)).contiguous()

    def diff_step():
        om_t = om_d.clone().requires_grad_(True)
        x_t = x_d.clone().requires_grad_(True)
        y = nf.nufft_apply(om_t, x_t, Nd, Kd, Jd)
        torch.sum(torch.abs(y - y0) ** 2).backward()

    def diff_step_fixed_plan():
        om_t = om_d.clone().requires_grad_(True)
        x_t = x_d.clone().requires_grad_(True)
        y = nf.nufft_apply(om_t, x_t, Nd, Kd, Jd, plan)
        torch.sum(torch.abs(y - y0) ** 2).backward()

    def plain_step():
        y = plan.forward(x_d)
        plan.adjoint((y - y0).contiguous())

    # a trajectory that moves every step (an optimisation loop over om): one
    # plan moved by nufft_plan_set_trajectory instead of a new plan per step
    g = torch.Generator(device=dev).manual_seed(5)
    moved = [(om_d + 1e-4 * torch.randn(om_d.shape, device=dev, generator=g)).contiguous() for _ in range(4)]
    plan_r = nf.NufftPlan(om_d, Nd, Kd, Jd)
    it = [0]

    def diff_step_moving_plan():
        om_t = moved[it[0] % len(moved)].clone().requires_grad_(True)
        it[0] += 1
        x_t = x_d.clone().requires_grad_(True)
        y = nf.nufft_apply(om_t, x_t, Nd, Kd, Jd, plan_r, refresh=True)
        torch.sum(torch.abs(y - y0) ** 2).backward()

    def set_trajectory_only():
        plan_r.set_trajectory(moved[it[0] % len(moved)])
        it[0] += 1

    res = {}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for key, fn in (("autograd_with_plan_ms", diff_step), ("autograd_fixed_plan_ms", diff_step_fixed_plan),
                    ("autograd_moving_plan_ms", diff_step_moving_plan), ("set_trajectory_ms", set_trajectory_only),
                    ("plain_fwd_adj_ms", plain_step)):
        fn()
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        res[key] = round((time.perf_counter() - t0) / reps * 1e3, 4)          # wall time, Python included
        res[key.replace("_ms", "_gpu_ms")] = round(e0.elapsed_time(e1) / reps, 4)   # stream time
    res.update(_differentiable_graph(nf, torch, plan, om_d, x_d, y0, Nd, Kd, Jd, reps))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    plan.solve_l1tv_lad(y0, maxiter=50, inner=2, cg_iters=5, mu=1.0, lam=0.01)
    e1.record()
    e1.synchronize()
    res["l1tv_lad_50_iterations_ms"] = round(e0.elapsed_time(e1), 3)
    plan_r.close()
    res["workload"] = "256^2 ellipse phantom, 16 spiral interleaves x 2048 samples (32,768 points), grid 512^2, J=6x6"
    res["points"] = int(om.shape[0])
    plan.close()
    return res


def _differentiable_graph(nf, torch, plan, om_d, x_d, y0, Nd, Kd, Jd, reps):
    """The fixed-plan autograd step (forward, loss, backward to x and om)
    captured once in a torch CUDA graph and replayed: the step's stream time
    without the Python and ATen launch overhead of its ~20 small loss ops.
    Beside it, the library calls of the step on their own: the forward as
    its two stages, the adjoint and the trajectory gradient from the kept
    spectrum."""
    om_s = om_d.clone().requires_grad_(True)
    x_s = x_d.clone().requires_grad_(True)

    def step():
        om_s.grad = None
        x_s.grad = None
        y = nf.nufft_apply(om_s, x_s, Nd, Kd, Jd, plan)
        torch.sum(torch.abs(y - y0) ** 2).backward()

    out = {}
    try:
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            for _ in range(3):
                step()
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            step()
        for _ in range(2):
            graph.replay()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            graph.replay()
        e1.record()
        e1.synchronize()
        out["autograd_fixed_plan_graph_gpu_ms"] = round(e0.elapsed_time(e1) / reps, 4)
        del graph
    except RuntimeError as exc:   # capture refused by the runtime: report, do not fail the bench
        out["autograd_fixed_plan_graph_gpu_ms"] = None
        out["autograd_graph_error"] = str(exc).splitlines()[0][:200]
    grid = plan.scale_pad_fft(x_d)
    y = plan.interp(grid)
    g = (y - y0).contiguous()
    gx = plan.adjoint(g)
    gom = plan.trajectory_gradient_grid(grid, g)
    calls = (("scale_pad_fft_gpu_ms", lambda: plan.scale_pad_fft(x_d, grid)),
             ("interp_gpu_ms", lambda: plan.interp(grid, y)),
             ("adjoint_gpu_ms", lambda: plan.adjoint(g, gx)),
             ("trajectory_gradient_grid_gpu_ms", lambda: plan.trajectory_gradient_grid(grid, g, gom)))
    for key, fn in calls:
        for _ in range(3):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps * 4):
            fn()
        e1.record()
        e1.synchronize()
        out[key] = round(e0.elapsed_time(e1) / (reps * 4), 4)
    return out


# ------------------------------------------------------------------ oracle timing (CPU baseline / reference arm)

def _oracle_setup(name="radial2d_256"):
    import oracle
    spec, om, x, noise = W.make_workload(name)
    plan = oracle.make_plan(om, spec["Nd"], spec["Kd"], spec["Jd"])
    return oracle, spec, plan, x


def _oracle_pair(oracle, plan, x):
    y = oracle.forward(plan, x)
    oracle.adjoint(plan, y)


def _cpu_worker(name, lo, hi, slot, shm_names, conn):
    """One process of the all-cores baseline: the oracle's V and V^H for the
    points [lo, hi) of the workload, on data in shared memory."""
    from multiprocessing import shared_memory
    import oracle
    spec, om, _, _ = W.make_workload(name)
    plan = oracle.make_plan(om[lo:hi], spec["Nd"], spec["Kd"], spec["Jd"])
    M, Kd = spec["M"], tuple(spec["Kd"])
    shms = [shared_memory.SharedMemory(name=n) for n in shm_names]
    Y = np.ndarray(Kd, dtype=np.complex128, buffer=shms[0].buf)
    y = np.ndarray((M,), dtype=np.complex128, buffer=shms[1].buf)
    Z = np.ndarray(Kd, dtype=np.complex128, buffer=shms[2].buf, offset=slot * int(np.prod(Kd)) * 16)
    conn.send("ready")
    while True:
        cmd = conn.recv()
        if cmd == "V":
            y[lo:hi] = oracle.interp_V(plan, Y)
        elif cmd == "VH":
            Z[...] = oracle.gridding_VH(plan, y[lo:hi])
        else:
            break
        conn.send("done")
    for sh in shms:
        sh.close()


def _cpu_all_cores(name, cores, pairs):
    """The oracle's forward + adjoint with V and V^H split over `cores`
    processes by point range (S, F, F^H and the crop in this process):
    median seconds per pair over `pairs` pairs."""
    import multiprocessing as mp
    from multiprocessing import shared_memory
    import oracle
    spec, om, x, _ = W.make_workload(name)
    M, Kd = spec["M"], tuple(spec["Kd"])
    kprod = int(np.prod(Kd))
    plan0 = oracle.make_plan(om[:1], spec["Nd"], spec["Kd"], spec["Jd"])   # S only depends on N, K, J
    shms = [shared_memory.SharedMemory(create=True, size=kprod * 16),
            shared_memory.SharedMemory(create=True, size=M * 16),
            shared_memory.SharedMemory(create=True, size=cores * kprod * 16)]
    ctx = mp.get_context("spawn")
    bounds = np.linspace(0, M, cores + 1).astype(int)
    procs, conns = [], []
    try:
        for c in range(cores):
            a, b = ctx.Pipe()
            pr = ctx.Process(target=_cpu_worker, args=(name, int(bounds[c]), int(bounds[c + 1]), c,
                                                        [sh.name for sh in shms], b))
            pr.start()
            procs.append(pr)
            conns.append(a)
        for cn in conns:
            assert cn.recv() == "ready"
        Y = np.ndarray(Kd, dtype=np.complex128, buffer=shms[0].buf)
        Zs = np.ndarray((cores,) + Kd, dtype=np.complex128, buffer=shms[2].buf)

        def pair():
            Y[...] = oracle.fft_forward(oracle.scale_pad(plan0, x))
            for cmd in ("V", "VH"):
                for cn in conns:
                    cn.send(cmd)
                for cn in conns:
                    assert cn.recv() == "done"
            Z = Zs[0].copy()
            for c in range(1, cores):
                Z += Zs[c]
            oracle.crop_rescale(plan0, oracle.fft_adjoint(Z))

        pair()
        ts = []
        for _ in range(pairs):
            t0 = time.perf_counter()
            pair()
            ts.append(time.perf_counter() - t0)
        for cn in conns:
            cn.send("quit")
        for pr in procs:
            pr.join(timeout=30)
        return statistics.median(ts)
    finally:
        for pr in procs:
            if pr.is_alive():
                pr.terminate()
        for sh in shms:
            sh.close()
            sh.unlink()


def cpu_baseline(seconds: float = 10.0, pairs: int = 20):
    """The FP64 oracle's forward + adjoint on the full 2D workload, timed on the
    host (plan precompute excluded): the median of `pairs` timed pairs on one
    core (the oracle as it stands), and the same with V and V^H split by point
    range over all host cores.  `seconds` caps the one-core sample."""
    oracle, spec, plan, x = _oracle_setup()
    _oracle_pair(oracle, plan, x)
    ts, t_start = [], time.perf_counter()
    for _ in range(pairs):
        t0 = time.perf_counter()
        _oracle_pair(oracle, plan, x)
        ts.append(time.perf_counter() - t0)
        if time.perf_counter() - t_start > seconds:
            break
    one = statistics.median(ts)
    cores = os.cpu_count() or 1
    try:
        allc = _cpu_all_cores("radial2d_256", cores, pairs)
    except Exception as exc:   # report, do not fail the bench
        allc, err = None, str(exc).splitlines()[0][:200] if str(exc) else type(exc).__name__
    else:
        err = None
    M = spec["M"]
    line = {"value": round(M / allc, 1) if allc else round(M / one, 1), "unit": UNIT,
            "cores": cores if allc else 1, "kind": "oracle",
            "sample": f"median of {len(ts)} (one core) and {pairs} (all cores) forward+adjoint pairs on the full "
                      "radial2d_256 workload (206,336 points), FP64 numpy, plan excluded; all cores: V and V^H "
                      f"split by point range over {cores} processes, S, F, F^H and the crop in one",
            "single_core": {"value": round(M / one, 1), "unit": UNIT, "cores": 1, "median_pair_s": round(one, 4)}}
    if allc:
        line["all_cores_median_pair_s"] = round(allc, 4)
    if err:
        line["all_cores_error"] = err
    return line


def reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1 and rank != 0:
        return
    oracle, spec, plan, x = _oracle_setup()
    for _ in range(args.warmup):
        oracle.adjoint(plan, oracle.forward(plan, x))
    t0, c0 = time.perf_counter(), time.process_time()
    for _ in range(args.steps):
        oracle.adjoint(plan, oracle.forward(plan, x))
    el = time.perf_counter() - t0
    cores = max(1, round((time.process_time() - c0) / el))   # threads the timed loop kept busy
    value = spec["M"] * args.steps / el
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(el * 1e3 / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
        "config": {"workload": "radial2d_256: 2D 256x256 image, 512x512 grid, J=6x6, golden-angle radial "
                               "403 spokes x 512 samples (206,336 points), ellipse phantom",
                   "step": "A x then A^H y (forward + adjoint)", "parallelism": "host CPU"},
        "cpu_baseline": {"value": round(value, 1), "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} timed forward+adjoint pairs on the full workload, FP64 numpy, "
                                   f"plan excluded"},
        "e2e": {"value": round(value, 1), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-solvers", action="store_true", help="skip the solver timings (rows a9)")
    ap.add_argument("--clocks-csv", default=None,
                    help="also write the raw nvidia-smi clock samples of the timed region to this file")
    ap.add_argument("--no-autotune", action="store_true",
                    help="time the default plan instead of the tile-autotuned one (no candidate plans are built)")
    ap.add_argument("--no-rows", action="store_true",
                    help="time only the forward+adjoint step (no A^H A, Toeplitz, solver or extension rows)")
    ap.add_argument("--workloads", default="radial2d_256,kooshball3d_128,radial2d_256_K384",
                    help="comma list; the first sets value/roofline, the others are reported under 'also'")
    args = ap.parse_args(argv)
    args.warmup = max(3, args.warmup)           # at least 3 untimed warm-up steps
    if args.impl == "reference":
        reference(args)
    else:
        ours(args)


if __name__ == "__main__":
    main()
