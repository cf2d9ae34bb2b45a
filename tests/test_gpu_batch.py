"""Batched MAR-DEAM (deam_batch_*): scans of uneven size and view count iterated
together must give what deam_iterate gives for each scan alone (same per-ray
code; the backprojection tile shape the autotuner picks may differ from the
single-scan one, which changes only the FP32 summation grouping)."""
import dataclasses

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
    import paper_2202_00116_gb300 as p
    return p


def _rel(a, b):
    a, b = a.double(), b.double()
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


def _scans(pkg, n=4):
    out = []
    for case in synth.make_batch_cases(n, small=True):
        d, metal = synth.measure(case, seed=2)
        truth, _ = synth.voxelize(case)
        mask = (metal >= case.metal_threshold).to(torch.uint8)
        c0 = synth.initial_image(case, truth)
        g = pkg.from_case(case)
        g.set_data(d.cuda())
        g.set_metal_mask(mask.cuda(), "ray")
        out.append((g, c0))
    return out


@pytest.mark.parametrize("autotune", [True, False])   # tuned plan / the persistent plan
def test_batch_matches_single_scans(pkg, autotune):
    scans = _scans(pkg)
    ref_imgs, ref_hist = [], []
    for g, c0 in scans:
        c = c0.clone().cuda()
        ref_hist.append(g.iterate(c, 3))
        ref_imgs.append(c)
    batch = pkg.DeamBatch([g for g, _ in scans], autotune=autotune)
    imgs = [c0.clone().cuda() for _, c0 in scans]
    H = batch.iterate(imgs, 3)
    assert H.shape == (len(scans), 3)
    for i in range(len(scans)):
        assert _rel(imgs[i], ref_imgs[i]) < 1e-6
        np.testing.assert_allclose(H[i, 0], ref_hist[i][0], rtol=1e-12)
        np.testing.assert_allclose(H[i], ref_hist[i], rtol=1e-7)
        assert np.all(np.diff(H[i]) < 0)
    info = batch.info()
    if autotune:
        assert min(info["tuning_ms"]["forward"]) > 0 and len(info["tuning_ms"]["backprojection"]) >= 2
        assert {b["slab"] for b in info["backprojection"]} <= {2, 8, 16}
        assert min(info["tuning_ms"]["plans"]) > 0 and info["plan"] in ("persistent", "per-scan graph branches")
    # new image buffers: the graph is captured again and the iterations continue
    imgs2 = [c.clone() for c in imgs]
    H2 = batch.iterate(imgs2, 2)
    for i, (g, _) in enumerate(scans):
        c = ref_imgs[i].clone()
        h = g.iterate(c, 2)
        assert _rel(imgs2[i], c) < 2e-6
        np.testing.assert_allclose(H2[i], h, rtol=1e-6)
    batch.close()


@pytest.mark.parametrize("plan", ["persistent", "per_scan"])
def test_batch_spectral_models(pkg, plan):
    # every scan with its own source spectra (I0 scaled per scan): each work
    # item of the persistent forward must use its own scan's spectral tables
    scans = []
    for i, case in enumerate(synth.make_batch_cases(6, small=True)):
        case = dataclasses.replace(case, I0=case.I0 * (1.0 + 0.25 * i))
        d, metal = synth.measure(case, seed=2)
        truth, _ = synth.voxelize(case)
        g = pkg.from_case(case)
        g.set_data(d.cuda())
        g.set_metal_mask((metal >= case.metal_threshold).to(torch.uint8).cuda(), "ray")
        scans.append((g, synth.initial_image(case, truth)))
    ref = []
    for g, c0 in scans:
        c = c0.clone().cuda()
        ref.append((c, g.iterate(c, 2)))
    batch = pkg.DeamBatch([g for g, _ in scans], autotune=False, plan=plan if plan == "per_scan" else None)
    imgs = [c0.clone().cuda() for _, c0 in scans]
    H = batch.iterate(imgs, 2)
    assert batch.info()["plan"] == {"persistent": "persistent", "per_scan": "per-scan graph branches"}[plan]
    for i, (c, h) in enumerate(ref):
        assert _rel(imgs[i], c) < 1e-6, i
        np.testing.assert_allclose(H[i], h, rtol=1e-7)
    batch.close()
    for g, _ in scans:
        g.close()


def test_batch_rejects_bad_input(pkg):
    scans = _scans(pkg, 2)
    g0 = scans[0][0]
    with pytest.raises(pkg.DeamError):
        pkg.DeamBatch([g0, g0])                 # a context twice
    batch = pkg.DeamBatch([g for g, _ in scans], autotune=False)
    with pytest.raises(ValueError):
        batch.iterate([scans[0][1].cuda()], 1)  # one image for two scans
    with pytest.raises(ValueError):
        batch.iterate([c0 for _, c0 in scans], 1)  # host images are refused by the binding
    batch.close()


def test_full_batch_workload_persistent_plan(pkg):
    # The batching workload at full size: 24 seeded scans (2D slices 128^2 to
    # 512^2, 3D helical slabs 256^2x16 to 512^2x48, 180-1160 views, 1-3 metal
    # inserts) in the persistent plan (one forward launch over all scans, one
    # backprojection launch per slab class, captured in a CUDA graph) against
    # each scan's own deam_iterate.
    dev = torch.device("cuda")
    scans, imgs = [], []
    for case in synth.make_batch_cases(24):
        d, metal = synth.measure(case, device=dev, seed=1)
        truth, _ = synth.voxelize(case, device=dev)
        g = pkg.from_case(case)
        g.set_data(d)
        g.set_metal_mask((metal >= case.metal_threshold).to(torch.uint8), "ray")
        scans.append(g)
        imgs.append(synth.initial_image(case, truth).to(dev))
        del d, metal, truth
    ref = []
    for g, c0 in zip(scans, imgs):
        c = c0.clone()
        ref.append((c, g.iterate(c, 2)))
    batch = pkg.DeamBatch(scans, autotune=False)
    cb = [c.clone() for c in imgs]
    H = batch.iterate(cb, 2)
    assert batch.info()["plan"] == "persistent"
    for i, (c, h) in enumerate(ref):
        assert _rel(cb[i], c) < 1e-6, i
        np.testing.assert_allclose(H[i], h, rtol=1e-7)
    batch.close()


def test_context_in_a_live_batch_is_not_destroyed(pkg):
    scans = _scans(pkg, 2)
    batch = pkg.DeamBatch([g for g, _ in scans], autotune=False)
    with pytest.raises(pkg.DeamError) as e:
        scans[0][0].close()
    assert e.value.code == pkg.DEAM_ERR_STATE
    imgs = [c0.clone().cuda() for _, c0 in scans]
    assert batch.iterate(imgs, 1).shape == (2, 1)      # the batch still works
    batch.close()
    scans[0][0].close()                                # now allowed


@pytest.mark.parametrize("plan", ["persistent", "per_scan"])
def test_batch_matches_oracle(pkg, plan):
    # the batched forms against the FP64 oracle directly (not only against the
    # single-scan path): four small scans of uneven size, three iterations,
    # images to the parity tolerance 1e-4 and objective histories to 1e-5
    import oracle
    oracle.build()
    cases = synth.make_batch_cases(4, small=True)
    scans, c0s, refs = [], [], []
    for case in cases:
        d, metal = synth.measure(case, seed=2)
        truth, _ = synth.voxelize(case)
        mask = (metal >= case.metal_threshold).to(torch.uint8)
        c0 = synth.initial_image(case, truth)
        g = pkg.from_case(case)
        g.set_data(d.cuda())
        g.set_metal_mask(mask.cuda(), "ray")
        scans.append(g)
        c0s.append(c0)
        O = oracle.from_case(case)
        refs.append(O.iterate(c0.double().numpy(), d.double().numpy(), mask.numpy(), n_iter=3)[:2])
    batch = pkg.DeamBatch(scans, autotune=False, plan=plan if plan == "per_scan" else None)
    imgs = [c.clone().cuda() for c in c0s]
    H = batch.iterate(imgs, 3)
    assert batch.info()["plan"] == {"persistent": "persistent", "per_scan": "per-scan graph branches"}[plan]
    for i, (c_ref, h_ref) in enumerate(refs):
        rel = float(np.linalg.norm(imgs[i].cpu().double().numpy() - c_ref) / np.linalg.norm(c_ref))
        assert rel < 1e-4, (i, rel)
        np.testing.assert_allclose(H[i], h_ref, rtol=1e-5)
    batch.close()
