"""MAR initialisation on the GPU (Sec. 2.2, Eq. 4) against the FP64 oracle on
the same seeded inputs.

Tolerances from the arithmetic: log sinograms and trace completion are a few
FP32 roundings per element (relative L2 <= 1e-6).  FBP: the ramp sums and the
backprojection sums are compensated, so the error is set by the FP32 geometry
(fan angle from atan2f, ~1e-7 rad, i.e. ~1e-4 of a channel, times the
filtered sinogram's channel-to-channel variation): relative L2 <= 1e-4 over
the image.  The prior (one pass of the in-plane smoothing, then the thresholds) is
decided in FP32 on the GPU:
the full pipeline is compared with the oracle run on the GPU's prior, and the
GPU's prior is checked against the oracle's classification, which may differ
only where the oracle's FBP value lies within 1e-4 (relative) of a threshold."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

MAR = dict(t_air=0.005, t_bone=0.026, soft_value=0.0195, prior_spectrum=1)


@pytest.fixture(scope="module")
def pkg():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2202_00116_gb300 import build
    build.build()
    import oracle
    oracle.build()
    import paper_2202_00116_gb300 as p
    return p


_CACHE = {}


def _case(name):
    if name not in _CACHE:
        case = synth.make_case(name)
        d, metal = synth.measure(case, seed=1)
        truth, M = synth.voxelize(case)
        mask = (metal >= case.metal_threshold).to(torch.uint8)
        _CACHE[name] = (case, d, mask, truth, M)
    return _CACHE[name]


def _rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _gpu(pkg, case, d, mask=None):
    g = pkg.from_case(case)
    g.set_data(d.cuda())
    if mask is not None:
        g.set_metal_mask(mask.cuda(), "ray")
    return g


def _calib(pkg, case):
    """Eq. (4) weights from two noiseless calibration scans (a body-sized disk of
    basis 1, then the same disk with 0.3 of basis 2) through the GPU FBP."""
    geo = case.geo
    rad = 0.35 * min(geo.nx * geo.dx, geo.ny * geo.dy)
    scans = []
    for c2 in (0.0, 0.3):
        cal = synth.Case("cal", geo, case.energies, case.I0, case.mu, case.mu_metal,
                         [synth.Obj("cylinder", (0.0, 0.0, 0.0), (rad, rad, 1e4), 0.0, c1=1.0, c2=c2)],
                         case.i0_total)
        dc, _ = synth.measure(cal, seed=0, noiseless=True)
        scans.append((_gpu(pkg, case, dc), (1.0, c2)))
    x, y, _ = synth.voxel_centres(geo)
    roi = (torch.hypot(x[None, :], y[:, None]) < 0.5 * rad)[None].expand(geo.nz, -1, -1)
    return pkg.calibrate_decomposition(scans, roi)


def _calib_oracle(case):
    """The same Eq. (4) calibration through the oracle's own FBP (ROI means,
    least squares): the weights both sides use in the oracle comparisons, so
    that no oracle input comes from the CUDA path."""
    import oracle
    geo = case.geo
    O = oracle.from_case(case)
    rad = 0.35 * min(geo.nx * geo.dx, geo.ny * geo.dy)
    x, y, _ = synth.voxel_centres(geo)
    roi = np.broadcast_to((np.hypot(x.numpy()[None, :], y.numpy()[:, None]) < 0.5 * rad)[None],
                          (geo.nz, geo.ny, geo.nx))
    A, b = [], []
    for c2 in (0.0, 0.3):
        cal = synth.Case("cal", geo, case.energies, case.I0, case.mu, case.mu_metal,
                         [synth.Obj("cylinder", (0.0, 0.0, 0.0), (rad, rad, 1e4), 0.0, c1=1.0, c2=c2)],
                         case.i0_total)
        dc, _ = synth.measure(cal, seed=0, noiseless=True)
        p = O.log_sinogram(dc.double().numpy())
        b.append([float(O.fbp(p[j])[roi].mean()) for j in range(2)])
        A.append([1.0, c2])
    sol = np.linalg.lstsq(np.asarray(A), np.asarray(b), rcond=None)[0]
    return np.array([sol[0, 0], sol[1, 0], sol[0, 1], sol[1, 1]])


@pytest.mark.parametrize("name", ["t2d", "t3d"])
def test_log_sinogram_and_trace_completion(pkg, name):
    import oracle
    case, d, mask, _, _ = _case(name)
    g = _gpu(pkg, case, d, mask)
    O = oracle.from_case(case)
    p = g.log_sinogram(count_floor=1.0)
    po = O.log_sinogram(d.double().numpy(), 1.0)
    assert _rel(p.cpu().numpy(), po) < 1e-6
    bits = O.mask_bits(mask.numpy())
    prior = torch.rand(O.ray_shape, generator=torch.Generator().manual_seed(5)) * 3.0
    prior[0, 0, :3] = 0.0                                   # exercises the eps floor
    for j in range(2):
        # the same sinogram on both sides, the oracle's own (rounded to FP32 for
        # the GPU): the completion step alone is compared
        pj = torch.from_numpy(po[j]).float().contiguous().cuda()
        li = g.complete_trace(pj, j).cpu().numpy()
        nm = g.complete_trace(pj, j, prior_proj=prior.cuda(), eps=1e-3).cpu().numpy()
        pin = pj.cpu().double().numpy()
        li_o = O.complete_trace(pin, bits, j)
        nm_o = O.complete_trace(pin, bits, j, prior_proj=prior.double().numpy(), eps=1e-3)
        off = (bits & (1 << j)) == 0
        assert np.array_equal(li[off], pj.cpu().numpy()[off]) and np.array_equal(nm[off], pj.cpu().numpy()[off])
        assert _rel(li, li_o) < 1e-6 and _rel(nm, nm_o) < 1e-6
    # in place
    pj = p[1].contiguous()
    ref = g.complete_trace(pj, 1).clone()
    g.complete_trace(pj, 1, out=pj)
    assert torch.equal(pj, ref)


@pytest.mark.parametrize("name", ["t2d", "t3d", "c0"])
def test_fbp_matches_oracle(pkg, name):
    import oracle
    case, d, mask, _, _ = _case(name)
    g = _gpu(pkg, case, d, mask)
    O = oracle.from_case(case)
    # the oracle's log sinograms, rounded to FP32, are the input of both FBPs
    p = torch.from_numpy(O.log_sinogram(d.double().numpy(), 1.0)).float().contiguous()
    img = g.fbp(p.cuda())                                   # both spectra in one launch
    for j in range(2):
        ref = O.fbp(p[j].double().numpy())
        assert _rel(img[j].cpu().numpy(), ref) < 1e-4, j
        one = g.fbp(p[j].contiguous().cuda())
        assert _rel(one.cpu().numpy(), img[j].cpu().numpy()) < 1e-6


@pytest.mark.parametrize("name", ["t2d", "t3d"])
def test_mar_init_matches_oracle(pkg, name):
    import oracle
    case, d, mask, truth, M = _case(name)
    g = _gpu(pkg, case, d, mask)
    O = oracle.from_case(case)
    calib = _calib_oracle(case)
    # the binding's calibration through the GPU FBP gives the same weights
    np.testing.assert_allclose(_calib(pkg, case), calib, rtol=1e-3)
    dn = d.double().numpy()
    # the whole initialisation, each side on its own data: the oracle runs its
    # own pipeline end to end (its own FBP, thresholds and prior), and the GPU
    # runs the same pipeline with the oracle's prior handed in (the one input
    # where FP32 and FP64 may classify a voxel differently at a threshold), so
    # nothing the oracle uses comes from the CUDA path
    co, po_own, mLo, mHo = O.mar_init(dn, mask.numpy(), calib, **MAR)
    c_o, prior_o, mu_o = g.mar_init(calib, prior=torch.from_numpy(po_own).float().cuda(), **MAR)
    assert np.array_equal(prior_o.cpu().double().numpy(), po_own.astype(np.float32).astype(np.float64))
    assert _rel(mu_o[0].cpu().numpy(), mLo) < 1e-4 and _rel(mu_o[1].cpu().numpy(), mHo) < 1e-4
    assert _rel(c_o.cpu().numpy(), co) < 1e-4
    # the GPU's own prior: its threshold decisions against the oracle's
    c, prior, mu = g.mar_init(calib, **MAR)
    bits = O.mask_bits(mask.numpy())
    f = oracle.smooth_inplane(O.fbp(O.complete_trace(O.log_sinogram(dn)[1], bits, 1)), 1)
    pg = prior.cpu().double().numpy()

    def classes(x):   # 0 air, 1 soft tissue, 2 kept (bone) value
        return np.where(x == 0, 0, np.where(np.abs(x - MAR["soft_value"]) < 1e-6, 1, 2))

    diff = classes(po_own) != classes(pg)
    near = np.minimum(np.abs(f - MAR["t_air"]), np.abs(f - MAR["t_bone"])) <= 1e-4 * np.abs(f).max()
    assert np.all(near[diff]), int(diff.sum())
    kept = (classes(pg) == 2) & ~diff
    assert np.all(np.abs(pg[kept] - f[kept]) <= 1e-4 * np.abs(f).max())
    # a prior handed in is used as it is
    c2, prior2, _ = g.mar_init(calib, prior=prior, **MAR)
    assert torch.equal(prior2, prior) and torch.equal(c2, c)


def test_mar_init_improves_on_uncorrected_fbp(pkg):
    # the point of the initialisation: away from the metal, the NMAR image is
    # closer to the same pipeline's image of the phantom without its metal than
    # the decomposition without trace completion is (noiseless counts, so that
    # metal streaks rather than noise or beam hardening are measured)
    import dataclasses
    case, _, mask, truth, M = _case("c0")
    d, _ = synth.measure(case, seed=1, noiseless=True)
    d_ref, _ = synth.measure(dataclasses.replace(case, objects=[o for o in case.objects if not o.metal]),
                             seed=1, noiseless=True)
    calib = _calib(pkg, case)
    c, _, _ = _gpu(pkg, case, d, mask).mar_init(calib, **MAR)
    c_raw, _, _ = _gpu(pkg, case, d).mar_init(calib, **MAR)      # no metal mask: nothing completed
    c_ref, _, _ = _gpu(pkg, case, d_ref).mar_init(calib, **MAR)
    from scipy.ndimage import binary_dilation
    t = truth.numpy()
    away = ~binary_dilation(M.numpy()[0] > 0, iterations=4)[None] & (t[..., 0] > 0.5)
    ref = c_ref.cpu().numpy()[away]
    err = np.linalg.norm(c.cpu().numpy()[away] - ref) / np.linalg.norm(ref)
    err_raw = np.linalg.norm(c_raw.cpu().numpy()[away] - ref) / np.linalg.norm(ref)
    assert err < 0.6 * err_raw, (err, err_raw)


def test_mar_init_argument_errors(pkg):
    case, d, mask, _, _ = _case("t2d")
    g = _gpu(pkg, case, d, mask)
    with pytest.raises(pkg.DeamError):
        g.mar_init([1.0, 2.0, 2.0, 4.0], **MAR)             # singular calibration
    with pytest.raises(pkg.DeamError):
        g.mar_init([0.02, 0.04, 0.018, 0.03], count_floor=0.0, **MAR)
    with pytest.raises(pkg.DeamError):
        g.mar_init([0.02, 0.04, 0.018, 0.03], prior_smooth=17, **MAR)
    fresh = pkg.from_case(case)
    with pytest.raises(pkg.DeamError):
        fresh.log_sinogram()                                # no data yet


def test_c2_full_size_sampled(pkg):
    # The MAR initialisation's steps at the benchmark's full size (512x512x64,
    # 5800 views x 16 x 816), as bench.py times them: log sinograms and the
    # trace completion of every ray against the oracle, and the FBP of the
    # completed high-kVp sinogram at 2000 seeded voxels against the oracle's
    # FBP of the same sinogram at those voxels.
    import oracle
    dev = torch.device("cuda")
    case = synth.make_case("c2")
    d, metal = synth.measure(case, device=dev, seed=1)
    mask = (metal >= case.metal_threshold).to(torch.uint8)
    del metal
    g = pkg.from_case(case)
    g.set_data(d)
    g.set_metal_mask(mask, "ray")
    O = oracle.from_case(case)
    p = g.log_sinogram()
    po = O.log_sinogram(d.cpu().double().numpy(), 1.0)
    for j in range(2):
        assert _rel(p[j].cpu().numpy(), po[j]) < 1e-6
    # each later step on both sides from the oracle's own high-kVp sinogram
    # (rounded to FP32 for the GPU), so no oracle input comes from the GPU
    ph = torch.from_numpy(po[1]).float().contiguous()
    del po, p
    bits = O.mask_bits(mask.cpu().numpy())
    li = g.complete_trace(ph.to(dev), 1)
    li_o = O.complete_trace(ph.double().numpy(), bits, 1)
    assert _rel(li.cpu().numpy(), li_o) < 1e-6
    img = g.fbp(li)
    q = O.ramp_filter(li_o)
    del li_o
    vox = np.sort(np.random.default_rng(5).choice(case.geo.n_voxels, size=2000, replace=False))
    ref = O.fbp_backproject_at(q, vox)
    assert _rel(img.reshape(-1)[torch.from_numpy(vox).to(dev)].cpu().numpy(), ref) < 1e-4
