"""Differentiable NUFFT on the GPU: trajectory and image gradients against the
FP64 oracle's analytic gradient (itself pinned to FP64 central differences in
test_oracle_pins_ext.py).  Tolerance: 1e-4 relative L2 over all gradient
entries (a derivative sum in FP32, like a forward operator)."""
import numpy as np
import pytest

import oracle
import workloads as W
from oracle import extensions as X

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_GRAD = 1e-4
TOL_OP = 2e-5
DEV = "cuda:0"


@pytest.fixture(scope="module")
def nf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1710_03197_gb300 as nf
    return nf


def rel(a, b):
    a, b = np.asarray(a).ravel(), np.asarray(b).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def cn(shape, seed):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.mark.parametrize("Nd,Kd,Jd,gen", [
    ((40,), (128,), (6,), lambda: W.uniform_random_om(500, 1, seed=31)),
    ((32, 48), (64, 128), (6, 6), lambda: W.uniform_random_om(1500, 2, seed=32)),
    ((32, 32), (64, 64), (5, 7), lambda: W.spiral2d(4, 300)),
    ((16, 16, 16), (32, 32, 32), (6, 6, 6), lambda: W.kooshball3d(100, 32)),
])
def test_trajectory_gradient_matches_oracle(nf, Nd, Kd, Jd, gen):
    om = gen()
    x = cn(Nd, 1)
    g = cn(om.shape[0], 2)
    ref = oracle.make_plan(om, Nd, Kd, Jd)
    with nf.NufftPlan(dev(om), Nd, Kd, Jd) as plan:
        gom = plan.trajectory_gradient(dev(x), dev(g))
        torch.cuda.synchronize()
        gom = gom.cpu().numpy()
        assert rel(gom, X.trajectory_gradient(ref, x, g)) < TOL_GRAD
        # eager, recording and replayed calls on the same buffers, new contents each time
        xd, gd = dev(x), dev(g)
        out = torch.empty((om.shape[0], len(Nd)), dtype=torch.float32, device=DEV)
        for it in range(3):
            x2, g2 = cn(Nd, 10 + it), cn(om.shape[0], 20 + it)
            xd.copy_(torch.from_numpy(x2))
            gd.copy_(torch.from_numpy(g2))
            plan.trajectory_gradient(xd, gd, out)
            assert rel(host(out), X.trajectory_gradient(ref, x2, g2)) < TOL_GRAD
        # from the oversampled spectrum: the same kernel on the same grid, so bit-identical
        grid = plan.scale_pad_fft(xd)
        out_g = torch.empty_like(out)
        for it in range(3):
            g3 = cn(om.shape[0], 30 + it)
            gd.copy_(torch.from_numpy(g3))
            plan.trajectory_gradient_grid(grid, gd, out_g)
            plan.trajectory_gradient(xd, gd, out)
            assert np.array_equal(host(out_g), host(out))


def test_autograd_quadratic_loss_matches_oracle(nf):
    Nd, Kd, Jd = (32, 32), (64, 64), (6, 6)
    om = W.spiral2d(6, 400)
    x = cn(Nd, 3)
    y0 = cn(om.shape[0], 4)
    om_t = dev(om).requires_grad_(True)
    x_t = dev(x).requires_grad_(True)
    y = nf.nufft_apply(om_t, x_t, Nd, Kd, Jd)
    y.retain_grad()
    loss = torch.sum(torch.abs(y - dev(y0)) ** 2)
    loss.backward()
    ref = oracle.make_plan(om, Nd, Kd, Jd)
    r = oracle.forward(ref, x) - y0
    assert abs(loss.item() - np.sum(np.abs(r) ** 2)) < 1e-4 * np.sum(np.abs(r) ** 2)
    g = y.grad.cpu().numpy().astype(np.complex128)      # = 2 (y - y0), from the GPU forward
    assert rel(g, 2 * r) < 1e-4
    assert rel(x_t.grad.cpu().numpy(), oracle.adjoint(ref, g)) < TOL_OP
    assert rel(om_t.grad.cpu().numpy(), X.trajectory_gradient(ref, x, g)) < TOL_GRAD


@pytest.mark.parametrize("which", ["x", "om"])
def test_autograd_one_input_needs_grad(nf, which):
    """Only one of x, om requires a gradient: the forward then runs as one call
    (x) or as its two stages with the spectrum kept (om)."""
    Nd, Kd, Jd = (24, 40), (64, 128), (6, 6)
    om = W.uniform_random_om(900, 2, seed=41)
    x = cn(Nd, 5)
    y0 = cn(om.shape[0], 6)
    om_t = dev(om).requires_grad_(which == "om")
    x_t = dev(x).requires_grad_(which == "x")
    y = nf.nufft_apply(om_t, x_t, Nd, Kd, Jd)
    y.retain_grad()
    torch.sum(torch.abs(y - dev(y0)) ** 2).backward()
    ref = oracle.make_plan(om, Nd, Kd, Jd)
    assert rel(host(y.detach()), oracle.forward(ref, x)) < TOL_OP
    g = y.grad.cpu().numpy().astype(np.complex128)
    if which == "x":
        assert om_t.grad is None
        assert rel(x_t.grad.cpu().numpy(), oracle.adjoint(ref, g)) < TOL_OP
    else:
        assert x_t.grad is None
        assert rel(om_t.grad.cpu().numpy(), X.trajectory_gradient(ref, x, g)) < TOL_GRAD


def test_spiral2d_256_gradients_full_size(nf):
    """The 256^2 spiral workload (16 x 2048 points, om perturbed by N(0, 1e-3))."""
    spec, om, x, noise = W.make_workload("spiral2d_256")
    ref = oracle.make_plan(om, spec["Nd"], spec["Kd"], spec["Jd"])
    y0 = (oracle.forward(ref, x) + noise).astype(np.complex64)
    om_t = dev(om).requires_grad_(True)
    x_t = dev(x).requires_grad_(True)
    y = nf.nufft_apply(om_t, x_t, spec["Nd"], spec["Kd"], spec["Jd"])
    y.retain_grad()
    loss = torch.sum(torch.abs(y - dev(y0)) ** 2)
    loss.backward()
    # near the optimum the residual y - y0 cancels (|noise| << |A x|), so the
    # backward kernels are checked on the gradient the GPU forward produced
    g = y.grad.cpu().numpy().astype(np.complex128)
    assert rel(x_t.grad.cpu().numpy(), oracle.adjoint(ref, g)) < TOL_OP
    assert rel(om_t.grad.cpu().numpy(), X.trajectory_gradient(ref, x, g)) < TOL_GRAD


def test_autograd_step_in_a_torch_cuda_graph(nf):
    """Forward, loss and backward captured in one torch CUDA graph (the library
    calls launch into the caller's capture) and replayed with new image
    contents: gradients match the oracle's on every replay."""
    Nd, Kd, Jd = (32, 32), (64, 64), (6, 6)
    om = W.spiral2d(6, 400)
    y0 = cn(om.shape[0], 7)
    ref = oracle.make_plan(om, Nd, Kd, Jd)
    plan = nf.NufftPlan(dev(om), Nd, Kd, Jd)
    om_s = dev(om).requires_grad_(True)
    x_s = dev(cn(Nd, 8)).requires_grad_(True)
    y0d = dev(y0)
    holder = {}

    def step():
        om_s.grad = None
        x_s.grad = None
        y = nf.nufft_apply(om_s, x_s, Nd, Kd, Jd, plan)
        y.retain_grad()
        torch.sum(torch.abs(y - y0d) ** 2).backward()
        holder["y"] = y

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
    for it in range(3):
        x = cn(Nd, 50 + it)
        with torch.no_grad():
            x_s.copy_(torch.from_numpy(x))
        graph.replay()
        torch.cuda.synchronize()
        r = oracle.forward(ref, x) - y0
        g = holder["y"].grad.cpu().numpy().astype(np.complex128)
        assert rel(g, 2 * r) < 1e-4
        assert rel(x_s.grad.cpu().numpy(), oracle.adjoint(ref, g)) < TOL_OP
        assert rel(om_s.grad.cpu().numpy(), X.trajectory_gradient(ref, x, g)) < TOL_GRAD
    del graph
    plan.close()
