"""Regularised MAR-DEAM on the GPU (Eqs. 6-7 with the convex phi reading):
parity with the FP64 oracle's regularised c-step, the penalty value, and the
monotone decrease of F + R."""
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


def _rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("name,lam,delta", [("t2d", 2e3, 0.05), ("t3d", 5e3, 0.02)])
def test_regularised_iterations_match_oracle(pkg, name, lam, delta):
    import oracle
    case = synth.make_case(name)
    d, metal = synth.measure(case, seed=1)
    truth, _ = synth.voxelize(case)
    mask = (metal >= case.metal_threshold).to(torch.uint8)
    c0 = synth.initial_image(case, truth)
    gpu = pkg.from_case(case, penalty_lambda=lam, penalty_delta=delta)
    gpu.set_data(d.cuda())
    gpu.set_metal_mask(mask.cuda(), "ray")
    O = oracle.from_case(case)
    assert gpu.penalty(c0.cuda()) == pytest.approx(O.penalty(c0.double().numpy(), lam, delta), rel=1e-5)
    c = c0.clone().cuda()
    Fs, Rs = [], []
    for _ in range(5):
        Rs.append(gpu.penalty(c))
        Fs.append(gpu.iterate(c, 1)[0])
    c_ref, hF, hR, _ = O.iterate_reg(c0.double().numpy(), d.double().numpy(), mask.numpy(), n_iter=5, lam=lam,
                                     delta=delta)
    assert _rel(c.cpu().numpy(), c_ref) < 1e-4
    np.testing.assert_allclose(Fs, hF, rtol=1e-5)
    np.testing.assert_allclose(Rs, hR, rtol=1e-4)
    assert np.all(np.diff(np.array(Fs) + np.array(Rs)) < 0)
    # the plain and the regularised iterations differ
    plain = pkg.from_case(case)
    plain.set_data(d.cuda())
    plain.set_metal_mask(mask.cuda(), "ray")
    cp = c0.clone().cuda()
    plain.iterate(cp, 5)
    assert _rel(c.cpu().numpy(), cp.cpu().numpy()) > 1e-5


def test_regularised_scan_in_a_batch(pkg):
    cases = synth.make_batch_cases(2, small=True)
    scans, imgs, refs = [], [], []
    for j, case in enumerate(cases):
        d, metal = synth.measure(case, seed=2)
        truth, _ = synth.voxelize(case)
        mask = (metal >= case.metal_threshold).to(torch.uint8)
        c0 = synth.initial_image(case, truth)
        g = pkg.from_case(case, penalty_lambda=1e3 if j == 0 else 0.0, penalty_delta=0.05)
        g.set_data(d.cuda())
        g.set_metal_mask(mask.cuda(), "ray")
        c = c0.clone().cuda()
        g.iterate(c, 2)
        scans.append(g)
        refs.append(c)
        imgs.append(c0.clone().cuda())
    b = pkg.DeamBatch(scans, autotune=False)
    b.iterate(imgs, 2)
    for x, r in zip(imgs, refs):
        assert _rel(x.cpu().numpy(), r.cpu().numpy()) < 1e-6
    b.close()
