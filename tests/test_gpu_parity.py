"""GPU (CUDA, through the C ABI) against the FP64 oracle.

Tolerances (relative L2 over the compared outputs): 2e-5 per operator and per
stage, 1e-4 after solver iterations, integers bit-exact.  Small cases run
element by element and span several tiles with ragged tails; the full-size
2D workload runs element by element too; the full-size 3D workload is checked
on sampled points and through identities that hold at any size.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_OP = 2e-5
TOL_SOLVER = 1e-4


@pytest.fixture(scope="module")
def nf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1710_03197_gb300 as nf
    return nf


DEV = "cuda:0"


def rel(a, b):
    a, b = np.asarray(a).ravel(), np.asarray(b).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def cn(shape, seed):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64)


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


CASES = [
    # (name, Nd, Kd, Jd, om generator)
    ("1d", (40,), (128,), (6,), lambda: W.uniform_random_om(777, 1, seed=21)),
    ("2d_radial_c1", (64, 64), (128, 128), (6, 6), lambda: W.radial2d_uniform(64, 128)),
    ("2d_rect_ragged", (24, 40), (64, 128), (6, 6), lambda: W.uniform_random_om(3001, 2, seed=22)),
    ("2d_oddJ", (32, 32), (64, 64), (5, 7), lambda: W.uniform_random_om(2049, 2, seed=23)),
    ("2d_J1_NeqK", (16, 32), (16, 32), (1, 3), lambda: W.uniform_random_om(513, 2, seed=24)),
    ("2d_spiral", (48, 48), (128, 128), (6, 6), lambda: W.spiral2d(8, 500)),
    ("3d_koosh", (24, 32, 16), (64, 64, 32), (6, 6, 6), lambda: W.kooshball3d(300, 64)),
    ("3d_mixedJ", (16, 16, 16), (32, 32, 32), (4, 5, 6), lambda: W.uniform_random_om(1500, 3, seed=25)),
    # grids that are not powers of two (mixed-radix FFT passes, tiles of the
    # largest power of two dividing K): 1.5x and 1.25x oversampling, a 1D grid
    # of 2-cell tiles, factors 3 and 5 on different axes
    ("2d_radial_K1.5", (256, 256), (384, 384), (6, 6), lambda: W.radial2d_golden(60, 384)),
    ("3d_koosh_K1.25", (64, 64, 64), (80, 80, 80), (6, 6, 6), lambda: W.kooshball3d(300, 80)),
    ("1d_K90", (40,), (90,), (6,), lambda: W.uniform_random_om(900, 1, seed=26)),
    ("2d_K72x80_oddJ", (48, 60), (72, 80), (5, 6), lambda: W.uniform_random_om(4000, 2, seed=27)),
    # a 1024-point strided pass: two columns per CTA, exactly 48 KB of line buffers
    ("2d_K1024", (512, 48), (1024, 128), (6, 6), lambda: W.uniform_random_om(3000, 2, seed=28)),
]


@pytest.fixture(scope="module", params=CASES, ids=[c[0] for c in CASES])
def case(request, nf):
    name, Nd, Kd, Jd, gen = request.param
    om = gen()
    plan = nf.NufftPlan(to_dev(om), Nd, Kd, Jd)
    ref = oracle.make_plan(om, Nd, Kd, Jd)
    yield dict(name=name, Nd=Nd, Kd=Kd, Jd=Jd, om=om, plan=plan, ref=ref)
    plan.close()


# ------------------------------------------------------------------ a1: plan precompute

def test_interpolator_matches_oracle(case):
    plan, ref = case["plan"], case["ref"]
    kf, coefs, ss, perm = plan.interpolator()
    kf = kf.numpy()
    for a in range(len(case["Nd"])):
        want = (ref.k0[:, a] + 1) % case["Kd"][a]
        np.testing.assert_array_equal(kf[:, a], want)                      # bit-exact
        c_ref = ref.coef[a]
        err = np.abs(coefs[a].numpy() - c_ref).max() / np.abs(c_ref).max()
        assert err < 1e-6, (a, err)
        np.testing.assert_allclose(ss[a].numpy(), ref.s[a], rtol=2e-7, atol=0)


def test_tile_sort_and_bank_order(case):
    plan = case["plan"]
    kf, _, _, perm = plan.interpolator()
    perm, kf = perm.numpy().astype(np.int64), kf.numpy().astype(np.int64)
    M = case["om"].shape[0]
    np.testing.assert_array_equal(np.sort(perm), np.arange(M))
    info = plan.info()
    d = len(case["Nd"])
    base = {1: 1024, 2: 16, 3: 16}[d]

    def edge(K, J):   # the largest divisor of K up to the base edge, else the smallest from J - 1 up
        t = max(v for v in range(1, min(base, K) + 1) if K % v == 0)
        return t if t >= J - 1 else min(v for v in range(J - 1, K + 1) if K % v == 0)
    T = [edge(K, J) for K, J in zip(case["Kd"], case["Jd"])]
    nb = [K // t for K, t in zip(case["Kd"], T)]
    bins = np.zeros(M, dtype=np.int64)
    for a in range(d):
        bins = bins * nb[a] + kf[:, a] // T[a]
    sb = bins[perm]
    assert np.all(np.diff(sb) >= 0)                                          # sorted by tile
    assert info["nbins"] == int(np.prod(nb))
    # chunks: each tile's points cut into runs of at most C points; inside a run,
    # every aligned group of G = 32 // J_last points covers disjoint bank windows
    # whenever the run's points allow it (greedy): check the groups are no worse
    # than the plain trajectory order, and that each chunk holds the same points
    # as the stable (trajectory-order) sort would.
    C = {1: 1024, 2: 256, 3: 2048}[d]
    JL = case["Jd"][-1]
    G = 32 // JL
    P = [t + j - 1 for t, j in zip(T, case["Jd"])]
    stable = np.lexsort((np.arange(M), bins))
    tot_got = tot_plain = 0
    b0 = 0
    while b0 < M:
        b1 = b0
        while b1 < M and sb[b1] == sb[b0]:
            b1 += 1
        for c0 in range(b0, b1, C):
            c1 = min(b1, c0 + C)
            assert set(perm[c0:c1]) == set(stable[c0:c1])
            tile = np.array(np.unravel_index(sb[c0], nb)) * np.array(T)
            loc = kf[perm[c0:c1]] - tile
            cell = np.ravel_multi_index(tuple(loc.T), P) & 31
            def mult(cells):
                cnt = np.zeros(32, int)
                for cb in cells:
                    cnt[(cb + np.arange(JL)) % 32] += 1
                return cnt.max()
            got = sum(mult(cell[g:g + G]) for g in range(0, len(cell), G))
            loc_s = kf[stable[c0:c1]] - tile
            cell_s = np.ravel_multi_index(tuple(loc_s.T), P) & 31
            plain = sum(mult(cell_s[g:g + G]) for g in range(0, len(cell_s), G))
            # exactly the greedy: per group of G, take from the fullest bucket
            # (bank b) whose window [b, b + J_last) is free, lowest b on ties,
            # else the fullest bucket; each bucket in chunk (stable) order
            buckets = [[q for q in range(c1 - c0) if cell_s[q] == b] for b in range(32)]
            want = []
            while len(want) < c1 - c0:
                used = 0
                for _ in range(G):
                    if len(want) == c1 - c0:
                        break
                    def win(b):
                        return sum(1 << ((b + j) % 32) for j in range(JL))
                    free = [b for b in range(32) if buckets[b] and not (win(b) & used)]
                    pool = free or [b for b in range(32) if buckets[b]]
                    best = max(pool, key=lambda b: (len(buckets[b]), -b))
                    want.append(stable[c0 + buckets[best].pop(0)])
                    used |= win(best)
            np.testing.assert_array_equal(perm[c0:c1], want)
            if c1 - c0 >= 4 * G:   # the greedy is a heuristic: compare where the order has room to matter
                tot_got += got
                tot_plain += plain
        b0 = b1
    assert tot_got <= tot_plain


# ------------------------------------------------------------------ a2..a7: stages

def test_scale_pad_fft_matches_oracle(case):
    plan, ref = case["plan"], case["ref"]
    x = cn(case["Nd"], 1)
    g = host(plan.scale_pad_fft(to_dev(x)))
    assert rel(g, oracle.fft_forward(oracle.scale_pad(ref, x))) < TOL_OP


def test_interp_matches_oracle(case):
    plan, ref = case["plan"], case["ref"]
    Y = cn(case["Kd"], 2)
    y = host(plan.interp(to_dev(Y)))
    assert rel(y, oracle.interp_V(ref, Y)) < TOL_OP


def test_gridding_matches_oracle(case):
    plan, ref = case["plan"], case["ref"]
    y = cn(case["om"].shape[0], 3)
    Z = host(plan.gridding(to_dev(y)))
    assert rel(Z, oracle.gridding_VH(ref, y)) < TOL_OP


def test_ifft_crop_rescale_matches_oracle(case):
    plan, ref = case["plan"], case["ref"]
    Z = cn(case["Kd"], 4)
    x = host(plan.ifft_crop_rescale(to_dev(Z)))
    assert rel(x, oracle.crop_rescale(ref, oracle.fft_adjoint(Z))) < TOL_OP


# ------------------------------------------------------------------ operators

def test_forward_matches_oracle(case):
    plan, ref = case["plan"], case["ref"]
    x = cn(case["Nd"], 5)
    assert rel(host(plan.forward(to_dev(x))), oracle.forward(ref, x)) < TOL_OP


def test_adjoint_matches_oracle(case):
    plan, ref = case["plan"], case["ref"]
    y = cn(case["om"].shape[0], 6)
    assert rel(host(plan.adjoint(to_dev(y))), oracle.adjoint(ref, y)) < TOL_OP


def test_selfadjoint_matches_oracle(case):
    plan, ref = case["plan"], case["ref"]
    x = cn(case["Nd"], 7)
    assert rel(host(plan.selfadjoint(to_dev(x))), oracle.selfadjoint(ref, x)) < TOL_OP


def test_gridding_operators_are_bit_identical_run_to_run(case):
    """V^H accumulates in fixed point (integer atomics, a per-chunk power-of-two
    scale from a fixed-order bound), so the order in which warps add has no
    effect: repeated calls give bit-identical grids, adjoints and normal
    operators."""
    plan = case["plan"]
    y = to_dev(cn(case["om"].shape[0], 10))
    x = to_dev(cn(case["Nd"], 11))
    for op, arg in ((plan.gridding, y), (plan.adjoint, y), (plan.selfadjoint, x)):
        first = host(op(arg))
        for _ in range(3):
            np.testing.assert_array_equal(host(op(arg)), first)


def test_dense_cluster_gridding_is_bit_identical_and_accurate(nf):
    """The worst case for the fixed-point scale: thousands of random-phase samples
    piled into one cell of a tile, so one chunk's bound is far above any single
    contribution.  The grid still matches the oracle to the operator tolerance,
    run after run identically, in 1D, 2D and 3D."""
    rng = np.random.default_rng(90)
    for Nd, Kd, Jd, n in (((64,), (128,), (6,), 4000), ((32, 32), (64, 64), (6, 6), 3000),
                          ((16, 16, 16), (32, 32, 32), (6, 6, 6), 6000)):
        d = len(Nd)
        om = np.concatenate([(0.3 + 0.02 * rng.standard_normal((n, d))).astype(np.float32),
                             W.uniform_random_om(300, d, seed=91)])
        ref = oracle.make_plan(om, Nd, Kd, Jd)
        y = cn(om.shape[0], 92)
        y[:5] *= 1e3                               # a few large samples set the chunk's scale
        with nf.NufftPlan(to_dev(om), Nd, Kd, Jd) as plan:
            Z = host(plan.gridding(to_dev(y)))
            np.testing.assert_array_equal(host(plan.gridding(to_dev(y))), Z)
        assert rel(Z, oracle.gridding_VH(ref, y)) < TOL_OP, (d, rel(Z, oracle.gridding_VH(ref, y)))


def test_gridding_propagates_non_finite_samples(nf):
    om = W.uniform_random_om(500, 2, seed=93)
    y = cn(500, 94)
    y[7] = np.inf
    with nf.NufftPlan(to_dev(om), (16, 16), (32, 32), (6, 6)) as plan:
        Z = host(plan.gridding(to_dev(y)))
    assert np.isnan(Z).any()


@pytest.mark.parametrize("Nd,Kd,Jd,gen", [
    ((64, 64), (128, 128), (6, 6), lambda: W.radial2d_uniform(64, 128)),
    ((24, 40), (64, 128), (6, 6), lambda: W.uniform_random_om(3001, 2, seed=22)),
    ((32, 32), (64, 64), (5, 7), lambda: W.uniform_random_om(2049, 2, seed=23)),
    ((16, 32), (16, 32), (1, 3), lambda: W.uniform_random_om(513, 2, seed=24)),
    ((24, 32, 16), (64, 64, 32), (6, 6, 6), lambda: W.kooshball3d(300, 64)),
    ((16, 16, 16), (32, 32, 32), (4, 5, 6), lambda: W.uniform_random_om(1500, 3, seed=25)),
])
def test_fused_normal_operator_equals_forward_then_adjoint(nf, Nd, Kd, Jd, gen):
    """2D A^H A runs V^H V as one gather-then-scatter pass per tile chunk (1D
    and 3D run V then V^H); it
    must agree with the separate forward and adjoint calls (the same
    arithmetic up to the float rounding of the gathered samples), singly and
    batched; the batched form is bit-identical run to run."""
    om = gen()
    with nf.NufftPlan(to_dev(om), Nd, Kd, Jd) as plan:
        xs = [cn(Nd, 80 + b) for b in range(3)]
        for x in xs[:1]:
            xd = to_dev(x)
            two = host(plan.adjoint(plan.forward(xd)))
            assert rel(host(plan.selfadjoint(xd)), two) < 1e-6
        xb = to_dev(np.stack(xs))
        outb = host(plan.selfadjoint_batch(xb))
        np.testing.assert_array_equal(host(plan.selfadjoint_batch(xb)), outb)
        for b, x in enumerate(xs):
            two = host(plan.adjoint(plan.forward(to_dev(x))))
            assert rel(outb[b], two) < 1e-6


def test_host_buffer_calls_match_device_calls(case):
    plan = case["plan"]
    x = cn(case["Nd"], 8)
    y_dev = host(plan.forward(to_dev(x)))
    y_host = plan.forward_host(torch.from_numpy(x).pin_memory()).numpy()
    assert rel(y_host, y_dev) < 1e-6
    y = cn(case["om"].shape[0], 9)
    x_dev = host(plan.adjoint(to_dev(y)))
    x_host = plan.adjoint_host(torch.from_numpy(y).pin_memory()).numpy()
    assert rel(x_host, x_dev) < 1e-6


def test_golden_nudft_fixture(nf):
    import os
    data = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", "nudft_2d_tiny.txt"))
    y_gold = data[:, 1] + 1j * data[:, 2]
    om = W.uniform_random_om(40, 2, seed=11)
    x = W.complex_normal_image((16, 8), seed=12)
    with nf.NufftPlan(to_dev(om), (16, 8), (32, 16), (6, 6)) as plan:
        y = host(plan.forward(to_dev(x)))
    assert rel(y, y_gold) < 2e-5


# ------------------------------------------------------------------ full-size workloads

def test_full_2d_256_forward_adjoint_elementwise(nf, oracle_workload):
    spec, om, x, noise, ref = oracle_workload("radial2d_256")
    with nf.NufftPlan(to_dev(om), spec["Nd"], spec["Kd"], spec["Jd"]) as plan:
        y = host(plan.forward(to_dev(x)))
        y_in = (oracle.forward(ref, x) + noise).astype(np.complex64)
        xa = host(plan.adjoint(to_dev(y_in)))
    assert rel(y, oracle.forward(ref, x)) < TOL_OP
    assert rel(xa, oracle.adjoint(ref, y_in)) < TOL_OP


def test_full_3d_128_forward_sampled_and_identities(nf):
    spec, om, x, _ = W.make_workload("kooshball3d_128")
    rng = np.random.default_rng(31)
    idx = np.sort(rng.choice(om.shape[0], 3000, replace=False))
    # include the densest region (the kooshball centre) and the first/last points
    centre = np.argsort(np.abs(om.astype(np.float64)).sum(1))[:500]
    idx = np.unique(np.concatenate([idx, centre, [0, om.shape[0] - 1]]))
    with nf.NufftPlan(to_dev(om), spec["Nd"], spec["Kd"], spec["Jd"]) as plan:
        xd = to_dev(x)
        y = plan.forward(xd)
        y_h = host(y)
        # sampled forward vs oracle (the oracle grid is exact; coefficients only for the sample)
        ref_s = oracle.make_plan(om[idx], spec["Nd"], spec["Kd"], spec["Jd"])
        Y = oracle.fft_forward(oracle.scale_pad(ref_s, x))
        assert rel(y_h[idx], oracle.interp_V(ref_s, Y)) < TOL_OP
        # adjoint identity <A x, v> = <x, A^H v> in FP64 over the GPU outputs
        v = cn(om.shape[0], 32)
        ahv = host(plan.adjoint(to_dev(v)))
        lhs = np.vdot(y_h.astype(np.complex128), v.astype(np.complex128))
        rhs = np.vdot(x.astype(np.complex128), ahv.astype(np.complex128))
        assert abs(lhs - rhs) / abs(lhs) < 1e-5
        # A^H A x = A^H (A x)
        aha = host(plan.selfadjoint(xd))
        ah_ax = host(plan.adjoint(y))
        assert rel(aha, ah_ax) < 1e-6


def test_full_3d_128_adjoint_on_a_point_subset_elementwise(nf):
    """The full kooshball plan (2.1M points, every chunk and tile of the
    workload) applied to samples that are zero except on ~3,500 points,
    including the 500 nearest the centre, where the tiles are densest and are
    cut into several chunks.  Zero samples add nothing, so the exact result is
    the oracle's adjoint on those points alone, checked element by element
    over the whole 128^3 image."""
    spec, om, x, _ = W.make_workload("kooshball3d_128")
    rng = np.random.default_rng(33)
    centre = np.argsort(np.abs(om.astype(np.float64)).sum(1))[:500]
    idx = np.unique(np.concatenate([rng.choice(om.shape[0], 3000, replace=False), centre, [0, om.shape[0] - 1]]))
    v = np.zeros(om.shape[0], dtype=np.complex64)
    v[idx] = cn(idx.size, 34)
    with nf.NufftPlan(to_dev(om), spec["Nd"], spec["Kd"], spec["Jd"]) as plan:
        assert plan.info()["nchunks"] > plan.info()["nbins"] // 2
        xa = host(plan.adjoint(to_dev(v)))
    ref_s = oracle.make_plan(om[idx], spec["Nd"], spec["Kd"], spec["Jd"])
    assert rel(xa, oracle.adjoint(ref_s, v[idx])) < TOL_OP


# ------------------------------------------------------------------ solvers

def _solver_problem(name):
    spec, om, x, noise = W.make_workload(name)
    ref = oracle.make_plan(om, spec["Nd"], spec["Kd"], spec["Jd"])
    y = oracle.forward(ref, x)
    if noise is not None:
        y = y + noise
    return spec, om, ref, y.astype(np.complex64)


def _well_conditioned():
    """Uniform random trajectory with M = 3 N^2: CG is stable to FP32 rounding here."""
    Nd, Kd, Jd = (64, 64), (128, 128), (6, 6)
    om = W.uniform_random_om(3 * 64 * 64, 2, seed=3)
    ref = oracle.make_plan(om, Nd, Kd, Jd)
    y = oracle.forward(ref, W.complex_normal_image(Nd)).astype(np.complex64)
    return Nd, Kd, Jd, om, ref, y


def test_cg_50_iterations_well_conditioned(nf):
    Nd, Kd, Jd, om, ref, y = _well_conditioned()
    with nf.NufftPlan(to_dev(om), Nd, Kd, Jd) as plan:
        xg = host(plan.solve_cg(to_dev(y), maxiter=50))
    assert rel(xg, oracle.cg(ref, y, np.zeros(Nd), 50)) < TOL_SOLVER


def test_cg_warm_start_and_zero_iterations(nf):
    Nd, Kd, Jd, om, ref, y = _well_conditioned()
    x0 = cn(Nd, 40)
    with nf.NufftPlan(to_dev(om), Nd, Kd, Jd) as plan:
        x_same = host(plan.solve_cg(to_dev(y), to_dev(x0), maxiter=0))
        xg = host(plan.solve_cg(to_dev(y), to_dev(x0), maxiter=12))
    np.testing.assert_array_equal(x_same, x0)
    assert rel(xg, oracle.cg(ref, y, x0, 12)) < TOL_SOLVER


def test_cg_5_iterations_radial2d_64(nf):
    spec, om, ref, y = _solver_problem("radial2d_64")
    with nf.NufftPlan(to_dev(om), spec["Nd"], spec["Kd"], spec["Jd"]) as plan:
        xg = host(plan.solve_cg(to_dev(y), maxiter=5))
    assert rel(xg, oracle.cg(ref, y, np.zeros(spec["Nd"]), 5)) < TOL_SOLVER


def _l1tv_well_conditioned(d):
    if d == 2:
        Nd, Kd, Jd = (64, 64), (128, 128), (6, 6)
        om = W.uniform_random_om(3 * 64 * 64, 2, seed=3)
        xt = W.ellipse_phantom(64)
    else:
        Nd, Kd, Jd = (16, 16, 16), (32, 32, 32), (6, 6, 6)
        om = W.uniform_random_om(3 * 4096, 3, seed=4)
        xt = W.complex_normal_image(Nd)
    ref = oracle.make_plan(om, Nd, Kd, Jd)
    y = (oracle.forward(ref, xt) + W.complex_noise(om.shape[0], 0.5)).astype(np.complex64)
    return Nd, Kd, Jd, om, ref, y


@pytest.mark.parametrize("d,lam", [(2, 0.01), (2, 2.0), (2, 50.0), (3, 0.5)])
def test_l1tv_ols_matches_oracle(nf, d, lam):
    Nd, Kd, Jd, om, ref, y = _l1tv_well_conditioned(d)
    outer, inner, cgi = (6, 2, 5) if d == 2 else (3, 1, 4)
    with nf.NufftPlan(to_dev(om), Nd, Kd, Jd) as plan:
        xg = host(plan.solve_l1tv_ols(to_dev(y), maxiter=outer, inner=inner, cg_iters=cgi, mu=1.0, lam=lam))
    xr = oracle.l1tv_ols(ref, y, np.zeros(Nd), outer, inner, cgi, 1.0, lam)
    assert rel(xg, xr) < TOL_SOLVER


@pytest.mark.parametrize("d,mu,lam", [(2, 1.0, 0.01), (2, 0.05, 2.0), (2, 0.05, 50.0), (3, 1.0, 0.5)])
def test_l1tv_lad_matches_oracle(nf, d, mu, lam):
    Nd, Kd, Jd, om, ref, y = _l1tv_well_conditioned(d)
    outer, inner, cgi = (6, 2, 5) if d == 2 else (3, 1, 4)
    with nf.NufftPlan(to_dev(om), Nd, Kd, Jd) as plan:
        xg = host(plan.solve_l1tv_lad(to_dev(y), maxiter=outer, inner=inner, cg_iters=cgi, mu=mu, lam=lam))
    xr = oracle.l1tv_lad(ref, y, np.zeros(Nd), outer, inner, cgi, mu, lam)
    assert rel(xg, xr) < TOL_SOLVER


# ------------------------------------------------------------------ edge cases

@pytest.mark.parametrize("Nd,Kd,Jd", [((64,), (128,), (16,)), ((32, 32), (64, 64), (12, 12)), ((40,), (64,), (9,))])
def test_wide_neighbourhoods(nf, Nd, Kd, Jd):
    """Large J makes G ill-conditioned (the plan's check of its Chebyshev
    expansion may then fall back to the direct sums); the operator must still
    match the oracle to the operator tolerance."""
    d = len(Nd)
    om = W.uniform_random_om(700 * d, d, seed=71)
    ref = oracle.make_plan(om, Nd, Kd, Jd)
    x = cn(Nd, 72)
    with nf.NufftPlan(to_dev(om), Nd, Kd, Jd) as plan:
        y = host(plan.forward(to_dev(x)))
        xa = host(plan.adjoint(to_dev(y)))
    assert rel(y, oracle.forward(ref, x)) < TOL_OP
    assert rel(xa, oracle.adjoint(ref, y.astype(np.complex128))) < TOL_OP


def test_empty_trajectory(nf):
    with nf.NufftPlan(torch.empty((0, 2), dtype=torch.float32, device=DEV), (16, 16), (32, 32), (6, 6)) as plan:
        y = plan.forward(to_dev(cn((16, 16), 1)))
        assert y.numel() == 0
        x = host(plan.adjoint(torch.empty(0, dtype=torch.complex64, device=DEV)))
        assert np.all(x == 0)
        assert plan.info()["nchunks"] == 0


def test_dense_tile_splits_into_chunks(nf):
    """5000 points in one tile (more than one gridding chunk) plus a sparse rest."""
    rng = np.random.default_rng(50)
    dense = (0.01 * rng.standard_normal((5000, 2))).astype(np.float32)
    om = np.concatenate([dense, W.uniform_random_om(700, 2, seed=51)])
    Nd, Kd, Jd = (32, 32), (64, 64), (6, 6)
    ref = oracle.make_plan(om, Nd, Kd, Jd)
    y = cn(om.shape[0], 52)
    x = cn(Nd, 53)
    with nf.NufftPlan(to_dev(om), Nd, Kd, Jd) as plan:
        info = plan.info()
        assert info["nchunks"] >= info["nbins"] + 2        # the dense tile holds 3 chunks
        assert rel(host(plan.adjoint(to_dev(y))), oracle.adjoint(ref, y)) < TOL_OP
        assert rel(host(plan.forward(to_dev(x))), oracle.forward(ref, x)) < TOL_OP


def test_boundary_and_wrapped_frequencies(nf):
    K = 64
    gam = 2 * math.pi / K
    vals = np.array([-math.pi, -math.pi + 1e-7, 0.0, gam * 5, -gam * 7, math.pi - 1e-6, math.pi, 3.5, -4.0, 7.0,
                     2 * math.pi, -2 * math.pi + 0.1, 1000.0], dtype=np.float32)
    g0, g1 = np.meshgrid(vals, vals[::-1], indexing="ij")
    om = np.stack([g0.ravel(), g1.ravel()], 1).astype(np.float32)
    Nd, Kd, Jd = (32, 32), (K, K), (6, 6)
    ref = oracle.make_plan(om, Nd, Kd, Jd)
    x = cn(Nd, 54)
    y = cn(om.shape[0], 55)
    with nf.NufftPlan(to_dev(om), Nd, Kd, Jd) as plan:
        kf, _, _, _ = plan.interpolator()
        np.testing.assert_array_equal(kf.numpy(), (ref.k0 + 1) % K)
        assert rel(host(plan.forward(to_dev(x))), oracle.forward(ref, x)) < TOL_OP
        assert rel(host(plan.adjoint(to_dev(y))), oracle.adjoint(ref, y)) < TOL_OP


def test_invalid_trajectory_is_rejected(nf):
    om = W.uniform_random_om(100, 2, seed=56)
    om[17, 1] = np.nan
    with pytest.raises(nf.NufftError) as ei:
        nf.NufftPlan(to_dev(om), (16, 16), (32, 32), (6, 6))
    assert ei.value.code == 1
    om[17, 1] = 3e7
    with pytest.raises(nf.NufftError):
        nf.NufftPlan(to_dev(om), (16, 16), (32, 32), (6, 6))


def test_selfadjoint_rejects_aliasing(nf):
    om = W.uniform_random_om(100, 2, seed=57)
    with nf.NufftPlan(to_dev(om), (16, 16), (32, 32), (6, 6)) as plan:
        x = to_dev(cn((16, 16), 1))
        with pytest.raises(nf.NufftError):
            plan.selfadjoint(x, x)


def test_runs_on_a_side_stream(nf):
    om = W.uniform_random_om(2000, 2, seed=58)
    Nd, Kd, Jd = (32, 32), (64, 64), (6, 6)
    ref = oracle.make_plan(om, Nd, Kd, Jd)
    x = cn(Nd, 59)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        plan = nf.NufftPlan(to_dev(om), Nd, Kd, Jd)
        y = plan.forward(to_dev(x))
    s.synchronize()
    assert rel(y.cpu().numpy(), oracle.forward(ref, x)) < TOL_OP
    plan.close()


@pytest.mark.parametrize("name,Nd,Kd,Jd,gen", [
    ("2d", (64, 64), (128, 128), (6, 6), lambda: W.radial2d_golden(60, 128)),
    ("3d", (16, 16, 16), (32, 32, 32), (6, 6, 6), lambda: W.kooshball3d(80, 32)),
    ("1d", (200,), (512,), (6,), lambda: W.uniform_random_om(3000, 1, seed=73)),
])
def test_autotuned_plan_matches_oracle(nf, name, Nd, Kd, Jd, gen):
    """nufft_plan_tuned picks one of its candidate tile edges and gives the
    same operators as the default plan."""
    om = gen()
    ref = oracle.make_plan(om, Nd, Kd, Jd)
    x = cn(Nd, 74)
    yin = cn(om.shape[0], 75)
    with nf.NufftPlan(to_dev(om), Nd, Kd, Jd, autotune=True) as plan:
        info = plan.info()
        edge = {1: (256, 512, 1024), 2: (8, 16, 32), 3: (8, 16)}[len(Nd)]
        for a, t in zip((0, len(Nd) - 1), ("tile_first", "tile_last")):
            assert info[t] in [min(e, Kd[a]) for e in edge]
        assert rel(host(plan.forward(to_dev(x))), oracle.forward(ref, x)) < TOL_OP
        assert rel(host(plan.adjoint(to_dev(yin))), oracle.adjoint(ref, yin)) < TOL_OP
