"""Differentiation of the MAR-DEAM objective on the GPU: deam_gradient against
the FP64 oracle's gradient and against central finite differences of the
oracle's objective, and the torch.autograd.Function built on it."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2202_00116_gb300 import build
    build.build()
    import oracle
    oracle.build()
    import paper_2202_00116_gb300 as p
    return p


def _case(name):
    case = synth.make_case(name)
    d, metal = synth.measure(case, seed=1)
    truth, _ = synth.voxelize(case)
    mask = (metal >= case.metal_threshold).to(torch.uint8)
    c0 = synth.initial_image(case, truth)
    return case, d, mask, c0


def _rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("name", ["t3d", "c0"])
def test_gradient_matches_oracle(pkg, name):
    import oracle
    case, d, mask, c0 = _case(name)
    gpu = pkg.from_case(case)
    gpu.set_data(d.cuda())
    gpu.set_metal_mask(mask.cuda(), "ray")
    g, F = gpu.gradient(c0.cuda())
    O = oracle.from_case(case)
    go = O.gradient(c0.double().numpy(), d.double().numpy(), mask.numpy())
    assert _rel(g.cpu().numpy(), go) < 1e-4
    assert F == pytest.approx(O.objective(c0.double().numpy(), d.double().numpy(), mask.numpy()), rel=1e-5)


def test_gradient_central_differences(pkg):
    # relative step 1e-3 on 64 random (voxel, component) pairs, differences of
    # the FP64 oracle objective
    import oracle
    case, d, mask, c0 = _case("t3d")
    gpu = pkg.from_case(case)
    gpu.set_data(d.cuda())
    gpu.set_metal_mask(mask.cuda(), "ray")
    g, _ = gpu.gradient(c0.cuda())
    g = g.cpu().double().numpy().reshape(-1)
    O = oracle.from_case(case)
    dn, mn = d.double().numpy(), mask.numpy()
    flat = c0.double().numpy().reshape(-1)
    rng = np.random.default_rng(4)
    big = np.flatnonzero(np.abs(g) > 1e-3 * np.abs(g).max())
    for p in rng.choice(big, size=64, replace=False):
        h = 1e-3 * max(abs(flat[p]), 0.1)
        cp, cm = flat.copy(), flat.copy()
        cp[p] += h
        cm[p] -= h
        fd = (O.objective(cp.reshape(c0.shape), dn, mn) - O.objective(cm.reshape(c0.shape), dn, mn)) / (2 * h)
        assert g[p] == pytest.approx(fd, rel=2e-3, abs=2e-5 * np.abs(g).max())


def test_autograd_function_and_descent(pkg):
    case, d, mask, c0 = _case("t3d")
    gpu = pkg.from_case(case)
    gpu.set_data(d.cuda())
    gpu.set_metal_mask(mask.cuda(), "ray")
    c = c0.clone().cuda().requires_grad_(True)
    F = pkg.i_divergence(c, gpu)
    F.backward()
    g_direct, F_direct = gpu.gradient(c0.cuda())
    assert F.item() == F_direct
    assert torch.equal(c.grad, g_direct)
    # gradient descent with backtracking decreases F monotonically; the DEAM
    # update (a preconditioned step) decreases it too
    x = c0.clone().cuda()
    Fs = [gpu.objective(x)]
    step = 1e-7
    for _ in range(5):
        g, Fx = gpu.gradient(x)
        for _ in range(60):
            y = x - step * g
            Fy = gpu.objective(y)
            if Fy < Fx:
                break
            step *= 0.5
        else:
            pytest.fail("no descent along -grad")
        x = y
        Fs.append(Fy)
        step *= 1.5
    assert all(b < a for a, b in zip(Fs, Fs[1:]))
    xd = c0.clone().cuda()
    hist = gpu.iterate(xd, 5)
    assert np.all(np.diff(hist) < 0)


def test_gradient_solver_is_monotone_and_trails_deam(pkg):
    # Barzilai-Borwein descent on the adjoint kernel's gradient never raises F
    # (the monotone safeguard), and each accepted step lowers it; DEAM's
    # majorise-minimise steps also decrease F (Sec. 2.3).  Both start from c0.
    from paper_2202_00116_gb300 import solvers
    case, d, mask, c0 = _case("t3d")
    gpu = pkg.from_case(case)
    gpu.set_data(d.cuda())
    gpu.set_metal_mask(mask.cuda(), "ray")
    c = c0.clone().cuda()
    res = solvers.gradient_descent(gpu, c, 30)
    F = res["objective"]
    assert len(F) >= 2 and np.all(np.diff(F) <= 0) and F[-1] < F[0]
    assert F[-1] == pytest.approx(gpu.objective(c), rel=1e-12)
    assert np.all(np.diff(res["evaluations"]) >= 1)
    h = gpu.iterate(c0.clone().cuda(), 10)
    assert np.all(np.diff(h) < 0) and h[0] == pytest.approx(F[0], rel=1e-12)


@pytest.mark.parametrize("name", ["t3d", "c0"])
def test_backprojected_sums_match_oracle(pkg, name):
    # (b~, delta = b^ - b~) of the c-step at c0 against the oracle's FP64 sums;
    # delta equals deam_gradient bitwise (same payload, same accumulation
    # order), and applying the c-step to them gives one deam_iterate step.
    import oracle
    case, d, mask, c0 = _case(name)
    gpu = pkg.from_case(case)
    gpu.set_data(d.cuda())
    gpu.set_metal_mask(mask.cuda(), "ray")
    sums, F, Z = gpu.backprojected_sums(c0.cuda())
    O = oracle.from_case(case)
    bt, bh, Fo = O.backprojected_sums(c0.double().numpy(), d.double().numpy(), mask.numpy())
    s = sums.cpu().double().numpy()
    assert _rel(s[..., :2], bt) < 1e-5
    assert np.linalg.norm(s[..., 2:] - (bh - bt)) / np.linalg.norm(bh) < 1e-5
    assert F == pytest.approx(Fo, rel=1e-5)
    assert Z == pytest.approx(O.normaliser(), rel=1e-5)
    g, Fg = gpu.gradient(c0.cuda())
    assert torch.equal(g, sums[..., 2:].contiguous()) and Fg == F
    c = c0.clone().cuda()
    gpu.iterate(c, 1)
    b, dl = sums[..., :2].double(), sums[..., 2:].double()
    ok = (b > 0) & (dl / b.clamp_min(1e-300) > -1)
    step = torch.where(ok, -torch.log1p(dl / torch.where(ok, b, torch.ones_like(b))) / Z, torch.zeros_like(b))
    ref = c0.cuda().double() + step
    assert float((c.double() - ref).abs().max()) <= 1e-6 * float(ref.abs().max()) + 1e-7


def test_preconditioned_gradient_solver(pkg):
    # the 1/(Z b~) preconditioned descent (DEAM's c-step is its exact-surrogate
    # form) keeps F monotone under the BB steps and the halving safeguard
    from paper_2202_00116_gb300 import solvers
    case, d, mask, c0 = _case("t3d")
    gpu = pkg.from_case(case)
    gpu.set_data(d.cuda())
    gpu.set_metal_mask(mask.cuda(), "ray")
    c = c0.clone().cuda()
    res = solvers.gradient_descent(gpu, c, 20, precondition=True)
    F = res["objective"]
    assert len(F) >= 2 and np.all(np.diff(F) <= 0) and F[-1] < F[0]
    assert F[0] == pytest.approx(gpu.objective(c0.cuda()), rel=1e-12)
    assert F[-1] == pytest.approx(gpu.objective(c), rel=1e-12)


def test_c1_full_size_gradient(pkg):
    # At the differentiation workload's size (256x256x32 helical, 3480 views x
    # 16 x 672): the adjoint kernel's gradient against the oracle's FP64
    # gradient over every voxel, and the directional derivative of the GPU
    # objective (central difference along a random sign pattern on the body)
    # against <gradient, direction>.
    import oracle
    dev = torch.device("cuda")
    case = synth.make_case("c1")
    d, metal = synth.measure(case, device=dev, seed=1)
    truth, _ = synth.voxelize(case, device=dev)
    mask = (metal >= case.metal_threshold).to(torch.uint8)
    c0 = synth.initial_image(case, truth).to(dev)
    gpu = pkg.from_case(case)
    gpu.set_data(d)
    gpu.set_metal_mask(mask, "ray")
    g, F = gpu.gradient(c0)
    O = oracle.from_case(case)
    go = O.gradient(c0.cpu().double().numpy(), d.cpu().double().numpy(), mask.cpu().numpy())
    assert _rel(g.cpu().numpy(), go) < 1e-4
    gen = torch.Generator(device="cpu").manual_seed(3)
    v = (torch.randint(0, 2, c0.shape, generator=gen).float() * 2 - 1).to(dev) * (truth[..., :1] > 0.3)
    eps = 1e-3
    fd = (gpu.objective(c0 + eps * v) - gpu.objective(c0 - eps * v)) / (2 * eps)
    dd = float((g.double() * v.double()).sum())
    assert fd == pytest.approx(dd, rel=1e-3)
