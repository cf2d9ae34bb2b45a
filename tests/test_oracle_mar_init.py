"""Pins of the oracle's MAR initialisation (Sec. 2.2, Eq. 4): log sinograms,
NMAR / linear trace completion, fan- and helical-beam FBP, the thresholded
prior and the image-domain decomposition, each against something fixed by the
mathematics rather than by the oracle's own formulas: Beer-Lambert inversion,
exactness of linear interpolation on linear data, NMAR's exactness when the
data are proportional to the prior's projection, analytic line integrals of
uniform disks and z-invariant cylinders reconstructed to their attenuation,
the object's position, and the inverse of a known 2x2 mixing."""
import math

import numpy as np
import pytest
import torch

import oracle
import synth


def _geo2d(n=96, dx=1.0, V=540, K=400, offset=0.25, start=0.37):
    fov = n * dx
    return synth.Geometry(synth.FAN2D, n, n, 1, dx, dx, 1.0, 0.0, 0.0, 0.0, 570.0, 1040.0, V, V, start, 0.0, 0.0,
                          1, 1.0, K, synth.fan_pitch(fov / 2.0 * 1.05, 570.0, K), offset, 0.0)


def _line_integrals(geo, objs):
    """Analytic sum over objects of c1 x chord length (mm) for every ray."""
    case = synth.Case("pin", geo, np.array([60.0]), np.ones((2, 1)), np.ones((2, 1)), np.zeros(1), objs, (1.0, 1.0))
    l1, _, _ = synth._chords(case, torch.arange(geo.n_views), "cpu")
    return l1.numpy()


def _oracle(geo, nE=3, bowtie=None):
    I0 = np.array([[1e4, 2e4, 3e4][:nE], [5e3, 1e4, 4e4][:nE]])
    mu = np.array([[0.02, 0.018, 0.017][:nE], [0.05, 0.03, 0.025][:nE]])
    return oracle.Oracle(geo, I0, mu, bowtie)


def test_log_sinogram_inverts_beer_lambert():
    geo = _geo2d(n=8, V=5, K=12)
    bow = np.linspace(0.5, 1.5, geo.n_channels)
    O = _oracle(geo, bowtie=bow)
    rng = np.random.default_rng(0)
    ell = rng.uniform(0.0, 6.0, (2,) + O.ray_shape)
    tot = O.I0.sum(axis=1)
    d = tot[:, None, None, None] * bow[None, None, None, :] * np.exp(-ell)
    p = O.log_sinogram(d, floor_counts=1e-30)
    np.testing.assert_allclose(p, ell, rtol=0, atol=1e-12)
    d[0, 1, 0, 3] = -4.0  # nonpositive counts are floored
    p = O.log_sinogram(d, floor_counts=0.5)
    assert p[0, 1, 0, 3] == pytest.approx(math.log(tot[0] * bow[3] / 0.5), rel=1e-14)


def _trace_case():
    geo = _geo2d(n=8, V=4, K=40)
    O = _oracle(geo)
    mask = np.zeros(O.ray_shape, dtype=np.uint8)
    mask[0, 0, 10:17] = 3      # interior segment, both spectra
    mask[1, 0, 0:5] = 1        # touching the row start, spectrum L only
    mask[2, 0, 33:40] = 2      # touching the row end, spectrum H only
    mask[3, 0, 5:8] = 3
    mask[3, 0, 20:26] = 3      # two segments in one row
    return geo, O, mask


def test_linear_interpolation_is_exact_on_linear_rows():
    geo, O, mask = _trace_case()
    k = np.arange(geo.n_channels)
    p = np.stack([0.3 + 0.07 * (v + 1) * k for v in range(geo.n_views)])[:, None, :]
    corrupt = p.copy()
    corrupt[mask != 0] = 50.0
    for bit in (0, 1):
        out = O.complete_trace(corrupt, mask, bit)
        on = (mask & (1 << bit)) != 0
        np.testing.assert_array_equal(out[~on], corrupt[~on])        # off the trace: untouched
        interior = on.copy()
        interior[1, 0, :5] = False                                    # row-start / row-end runs are
        interior[2, 0, 33:] = False                                   # extended constantly instead
        np.testing.assert_allclose(out[interior], p[interior], rtol=0, atol=1e-12)
    out = O.complete_trace(corrupt, mask, 0)
    assert np.all(out[1, 0, :5] == p[1, 0, 5])
    out = O.complete_trace(corrupt, mask, 1)
    assert np.all(out[2, 0, 33:] == p[2, 0, 32])


def test_nmar_is_exact_when_data_follow_the_prior():
    # NMAR divides by the prior's projection before interpolating: data that
    # are a (per-row) multiple of a nonlinear prior projection come back exactly,
    # where plain linear interpolation does not.
    geo, O, mask = _trace_case()
    k = np.arange(geo.n_channels)
    prior = (1.0 + 0.5 * np.sin(k / 3.0) + 0.02 * k)[None, None, :].repeat(geo.n_views, 0)
    scale = np.array([1.3, 0.7, 2.0, 1.1])[:, None, None]
    p = scale * prior
    corrupt = p.copy()
    corrupt[mask != 0] = -9.0
    out = O.complete_trace(corrupt, mask, 0, prior_proj=prior, eps=1e-6)
    on = (mask & 1) != 0
    np.testing.assert_allclose(out[on], p[on], rtol=1e-13)
    np.testing.assert_array_equal(out[~on], corrupt[~on])
    li = O.complete_trace(corrupt, mask, 0)
    assert np.max(np.abs(li[on] - p[on])) > 1e-2


def test_no_trace_is_identity():
    geo, O, mask = _trace_case()
    p = np.random.default_rng(1).normal(size=O.ray_shape)
    out = O.complete_trace(p, np.zeros_like(mask), 0, prior_proj=np.abs(p) + 1)
    np.testing.assert_array_equal(out, p)


def _disk(x0, y0, r, mu):
    return synth.Obj("cylinder", (x0, y0, 0.0), (r, r, 1e4), 0.0, c1=mu)


def _centroid(img, geo, thr):
    x, y, _ = synth.voxel_centres(geo)
    w = (img > thr).astype(np.float64)
    return float((w * x.numpy()[None, :]).sum() / w.sum()), float((w * y.numpy()[:, None]).sum() / w.sum())


def test_fan_beam_fbp_reconstructs_a_uniform_disk():
    geo = _geo2d()
    O = _oracle(geo)
    mu, x0, y0, R = 0.02, 9.0, -6.0, 25.0
    p = _line_integrals(geo, [_disk(x0, y0, R, mu)])
    img = O.fbp(p)[0]
    x, y, _ = synth.voxel_centres(geo)
    rr = np.hypot(x.numpy()[None, :] - x0, y.numpy()[:, None] - y0)
    inner = img[rr < R - 3]
    outer = img[(rr > R + 3) & (np.hypot(x.numpy()[None, :], y.numpy()[:, None]) < 40)]
    # the fan pre-weight cos(gamma) alone is a 0.2-0.4 % effect at this fan angle
    assert abs(inner.mean() / mu - 1) < 1e-3 and inner.std() / mu < 2e-3
    assert abs(outer.mean()) / mu < 1e-3
    cx, cy = _centroid(img, geo, mu / 2)
    assert abs(cx - x0) < 0.2 and abs(cy - y0) < 0.2


def test_fbp_backprojection_follows_the_rays():
    # A filtered sinogram that is one at a single (view, channel) backprojects
    # onto that ray's line: seen from the source, the image's weight is centred
    # on the ray direction given by the scanner's ray vectors (synth), to a small
    # fraction of a channel.  Coarse channels make a quarter-channel offset error
    # (0.5 mm at the centre here) plain to see.
    geo = _geo2d(n=64, dx=1.0, V=12, K=32, offset=0.25)
    O = _oracle(geo)
    s, u = synth.ray_endpoints(geo, torch.arange(geo.n_views))
    x, y, _ = synth.voxel_centres(geo)
    X, Y = np.meshgrid(x.numpy(), y.numpy())
    for v, k in ((0, 9), (5, 16), (11, 23)):
        q = np.zeros(O.ray_shape)
        q[v, 0, k] = 1.0
        img = O.fbp_backproject(q)[0]
        sx, sy = s[v, 0].item(), s[v, 1].item()
        ux, uy = u[v, 0, k, 0].item(), u[v, 0, k, 1].item()
        ang = np.arctan2(ux * (Y - sy) - uy * (X - sx), ux * (X - sx) + uy * (Y - sy))
        w = img * ((X - sx) ** 2 + (Y - sy) ** 2)
        assert w.sum() > 0
        assert abs((w * ang).sum() / w.sum()) < 0.05 * geo.channel_pitch, (v, k)


def test_fbp_is_linear_and_shift_consistent():
    # two disks reconstruct to the sum of their single-disk reconstructions
    geo = _geo2d(n=48, dx=2.0, V=360, K=200)
    O = _oracle(geo)
    a, b = _disk(-15.0, 5.0, 10.0, 0.02), _disk(12.0, 14.0, 6.0, 0.05)
    pa, pb = _line_integrals(geo, [a]), _line_integrals(geo, [b])
    fa, fb, fab = O.fbp(pa), O.fbp(pb), O.fbp(pa + pb)
    np.testing.assert_allclose(fab, fa + fb, rtol=0, atol=1e-12)


def test_helical_fbp_reconstructs_a_z_invariant_cylinder():
    # For an object that does not vary along z every tilted ray integral is the
    # in-plane one over the cosine of the cone angle, so the cone pre-weight
    # makes the helical FBP a fan-beam FBP of the cross-section.
    nx, nz, dx, dz, R, K, vpr = 48, 6, 2.0, 2.0, 8, 160, 240
    row_iso = 1.5
    feed = 0.8 * R * row_iso
    V = int(vpr * 2.2)
    fov = nx * dx
    geo = synth.Geometry(synth.HELICAL, nx, nx, nz, dx, dx, dz, 0.0, 0.0, 0.0, 570.0, 1040.0, V, vpr, 0.2, feed,
                         -feed * V / vpr / 2.0, R, row_iso * 1040.0 / 570.0, K,
                         synth.fan_pitch(fov / 2.0 * 1.05, 570.0, K), 0.25, 0.0)
    O = _oracle(geo)
    mu, x0, y0, r = 0.03, -8.0, 6.0, 20.0
    p = _line_integrals(geo, [_disk(x0, y0, r, mu)])
    img = O.fbp(p)
    x, y, _ = synth.voxel_centres(geo)
    rr = np.hypot(x.numpy()[None, :] - x0, y.numpy()[:, None] - y0)
    for iz in range(nz):
        inner = img[iz][rr < r - 5]
        assert abs(inner.mean() / mu - 1) < 0.02, iz
    cx, cy = _centroid(img[nz // 2], geo, mu / 2)
    assert abs(cx - x0) < 0.5 and abs(cy - y0) < 0.5


def test_helical_backprojection_follows_the_rays():
    # the 3D counterpart: a one-ray filtered sinogram lands on voxels whose
    # height matches the ray's height at their position (row interpolation at
    # w = (z - z_s) SDD / L), centred to a small fraction of a row
    nx, nz, dx, dz, R, K, vpr = 32, 24, 2.0, 1.0, 8, 48, 60
    row_iso = 1.5
    feed = 0.8 * R * row_iso
    geo = synth.Geometry(synth.HELICAL, nx, nx, nz, dx, dx, dz, 0.0, 0.0, 0.0, 570.0, 1040.0, 2 * vpr, vpr, 0.2,
                         feed, -feed, R, row_iso * 1040.0 / 570.0, K,
                         synth.fan_pitch(nx * dx / 2.0 * 1.05, 570.0, K), 0.25, 0.3)
    O = _oracle(geo)
    s, u = synth.ray_endpoints(geo, torch.arange(geo.n_views))
    x, y, z = synth.voxel_centres(geo)
    Z, Y, X = np.meshgrid(z.numpy(), y.numpy(), x.numpy(), indexing="ij")
    for v, r, k in ((55, 3, 20), (61, 5, 30), (70, 2, 24)):
        q = np.zeros(O.ray_shape)
        q[v, r, k] = 1.0
        img = O.fbp_backproject(q)
        assert img.sum() > 0
        sx, sy, sz = (s[v, i].item() for i in range(3))
        ux, uy, uz = (u[v, r, k, i].item() for i in range(3))
        t = ((X - sx) * ux + (Y - sy) * uy) / (ux * ux + uy * uy)
        zr = sz + t * uz
        w = img * ((X - sx) ** 2 + (Y - sy) ** 2)
        row_at_voxel = geo.row_pitch * np.sqrt((X - sx) ** 2 + (Y - sy) ** 2) / geo.sdd
        dev = (w * (Z - zr) / row_at_voxel).sum() / w.sum()
        assert abs(dev) < 0.05, (v, r, k, dev)


def test_prior_and_decomposition():
    f = np.array([-0.001, 0.0004, 0.002, 0.019, 0.025, 0.06])
    pr = oracle.prior_image(f, t_air=0.005, t_bone=0.024, soft_value=0.019)
    np.testing.assert_array_equal(pr, [0.0, 0.0, 0.0, 0.019, 0.025, 0.06])
    rng = np.random.default_rng(3)
    calib = np.array([0.021, 0.066, 0.018, 0.041])   # [[m1L, m2L], [m1H, m2H]]
    c = rng.uniform(-0.5, 1.5, (5, 7, 2))
    muL = calib[0] * c[..., 0] + calib[1] * c[..., 1]
    muH = calib[2] * c[..., 0] + calib[3] * c[..., 1]
    np.testing.assert_allclose(oracle.decompose(muL, muH, calib), c, rtol=1e-12, atol=1e-14)


def test_mar_init_reduces_metal_artifacts():
    # end to end on a small fan-beam case with a titanium insert, noiseless
    # data: away from the metal, the NMAR-initialised image is much closer to
    # the same pipeline's image of the phantom without its metal than the
    # pipeline without trace completion is; the prior override reproduces the
    # thresholded run
    import dataclasses
    from scipy.ndimage import binary_dilation
    case = synth.make_case("t2d")
    d, metal = synth.measure(case, seed=1, noiseless=True)
    d_ref, _ = synth.measure(dataclasses.replace(case, objects=[o for o in case.objects if not o.metal]),
                             seed=1, noiseless=True)
    truth, M = synth.voxelize(case)
    mask = (metal >= case.metal_threshold).to(torch.uint8).numpy()
    none = np.zeros_like(mask)
    O = oracle.from_case(case)
    calib = mar_calibration(case, O)
    kw = dict(calib=calib, t_air=0.005, t_bone=0.026, soft_value=0.0195, prior_spectrum=1)
    c, prior, mL, mH = O.mar_init(d.double().numpy(), mask, **kw)
    c_raw, *_ = O.mar_init(d.double().numpy(), none, **kw)
    c_ref, *_ = O.mar_init(d_ref.double().numpy(), none, **kw)
    t = truth.double().numpy()
    away = ~binary_dilation(M.numpy()[0] > 0, iterations=4)[None] & (t[..., 0] > 0.5)
    ref = c_ref[away]
    err = np.linalg.norm(c[away] - ref) / np.linalg.norm(ref)
    err_raw = np.linalg.norm(c_raw[away] - ref) / np.linalg.norm(ref)
    assert err < 0.4 * err_raw, (err, err_raw)
    assert abs(np.median(c[..., 0][t[..., 0] > 0.5]) - 1.0) < 0.1
    c2, *_ = O.mar_init(d.double().numpy(), mask, prior=prior, **kw)
    np.testing.assert_array_equal(c2, c)


def mar_calibration(case, O):
    """mu~_ij of Eq. (4) from two noiseless calibration scans through the same
    pipeline (no metal): a body-sized disk of basis 1 at unit density, and the
    same disk with 0.3 of basis 2 added; FBP means over a central ROI."""
    geo = case.geo
    rad = 0.35 * geo.nx * geo.dx
    mus = []
    for c2 in (0.0, 0.3):
        cal = synth.Case("cal", geo, case.energies, case.I0, case.mu, case.mu_metal,
                         [synth.Obj("cylinder", (0.0, 0.0, 0.0), (rad, rad, 1e4), 0.0, c1=1.0, c2=c2)],
                         case.i0_total)
        dc, _ = synth.measure(cal, seed=0, noiseless=True)
        p = O.log_sinogram(dc.double().numpy())
        x, y, _ = synth.voxel_centres(geo)
        roi = np.hypot(x.numpy()[None, :], y.numpy()[:, None]) < 0.5 * rad
        mus.append([O.fbp(p[j])[:, roi].mean() for j in range(2)])
    (aL, aH), (bL, bH) = mus
    return np.array([aL, (bL - aL) / 0.3, aH, (bH - aH) / 0.3])


def test_fbp_at_listed_voxels_equals_the_full_image():
    # the voxel-list form (used for sampled parity at full size) is the same
    # per-voxel sum as the full backprojection
    geo = _geo2d(n=48, dx=2.0, V=360, K=200)
    O = _oracle(geo)
    q = O.ramp_filter(_line_integrals(geo, [_disk(-15.0, 5.0, 10.0, 0.02)]))
    full = O.fbp_backproject(q).reshape(-1)
    vox = np.array([0, 5, 100, 1151, 2303])
    np.testing.assert_array_equal(O.fbp_backproject_at(q, vox), full[vox])


def test_prior_smoothing_closed_forms():
    # the in-plane [1,2,1]/4 filter: a delta spreads into the binomial kernel
    # ([1,2,1] x [1,2,1] / 16 after one pass, [1,4,6,4,1] x [1,4,6,4,1] / 256
    # after two), constants and linear ramps are kept, slices do not mix
    f = np.zeros((3, 9, 11))
    f[1, 4, 5] = 1.0
    one = oracle.smooth_inplane(f, 1)
    k1 = np.outer([1, 2, 1], [1, 2, 1]) / 16.0
    np.testing.assert_allclose(one[1, 3:6, 4:7], k1, rtol=0, atol=1e-15)
    assert abs(one[1].sum() - 1.0) < 1e-15 and not one[0].any() and not one[2].any()
    two = oracle.smooth_inplane(f, 2)
    b = np.array([1, 4, 6, 4, 1])
    np.testing.assert_allclose(two[1, 2:7, 3:8], np.outer(b, b) / 256.0, rtol=0, atol=1e-15)
    const = np.full((2, 5, 6), 0.7)
    np.testing.assert_allclose(oracle.smooth_inplane(const, 3), const, rtol=1e-15)
    ramp = np.broadcast_to(0.1 * np.arange(11.0)[None, None, :] + 0.3 * np.arange(9.0)[None, :, None], (2, 9, 11))
    out = oracle.smooth_inplane(ramp, 1)
    np.testing.assert_allclose(out[:, 1:-1, 1:-1], ramp[:, 1:-1, 1:-1], rtol=1e-14)
