"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the
same seeded inputs, element by element, plus invariants that hold at any size.

Tolerances (written from the arithmetic): projections (l, g, payload sums) are
FP32 sums of FP32 samples with compensated spectral sums, relative L2 <= 1e-5;
images after 10 iterations relative L2 <= 1e-4; objective values relative
1e-5.  Rays whose dominant axis is a near tie (|u_x| and |u_y| within 1e-6) are
left out of element-wise comparisons: the two choices are both valid Joseph
samplings and FP32/FP64 may pick differently there."""
import math

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


_CACHE = {}


def case_data(name):
    if name not in _CACHE:
        case = synth.make_case(name)
        d, metal = synth.measure(case, seed=1)
        truth, M = synth.voxelize(case)
        mask = (metal >= case.metal_threshold).to(torch.uint8)
        c0 = synth.initial_image(case, truth)
        _CACHE[name] = (case, d, mask, M, c0)
    return _CACHE[name]


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def near_tie(geo, views=None):
    """Rays whose |cos(beta+gamma)| and |sin(beta+gamma)| agree to 1e-6."""
    v = np.arange(geo.n_views) if views is None else np.asarray(views)
    beta = geo.start_angle + 2 * math.pi * v / geo.views_per_rotation
    k = np.arange(geo.n_channels)
    gam = (k - (geo.n_channels - 1) / 2 + geo.channel_offset) * geo.channel_pitch
    a = beta[:, None] + gam[None, :]
    t = np.abs(np.abs(np.cos(a)) - np.abs(np.sin(a))) < 1e-6
    return np.broadcast_to(t[:, None, :], (len(v), geo.n_rows, geo.n_channels))


def oracle_of(case):
    import oracle
    return oracle.from_case(case)


@pytest.mark.parametrize("name", ["t2d", "t3d", "c0"])
def test_forward_line_integrals(pkg, name):
    case, d, mask, M, c0 = case_data(name)
    gpu = pkg.from_case(case)
    l, g = gpu.forward(c0.cuda(), want_l=True, want_g=True)
    O = oracle_of(case)
    lo = O.forward(c0.double().numpy())
    lg = l.cpu().double().numpy()
    keep = ~near_tie(case.geo)
    for i in range(2):
        assert rel_l2(lg[..., i][keep], lo[..., i][keep]) < 1e-5
    err = np.abs(lg - lo)[keep]
    assert err.max() <= 1e-4 * np.abs(lo).max()
    go = O.expected(lo)
    assert rel_l2(g.cpu().double().numpy()[:, keep], go[:, keep]) < 1e-5


@pytest.mark.parametrize("name", ["t2d", "t3d", "c0"])
def test_backprojection_is_the_oracle_adjoint(pkg, name):
    case, *_ = case_data(name)
    gpu = pkg.from_case(case)
    y = synth.random_rays(case.geo, 21).float()
    img = gpu.backproject(y.cuda())
    ref = oracle_of(case).adjoint(y.double().numpy())
    ig = img.cpu().double().numpy()
    assert rel_l2(ig, ref) < 1e-5
    assert np.abs(ig - ref).max() <= 1e-4 * np.abs(ref).max()


@pytest.mark.parametrize("name", ["t3d", "c1"])
def test_adjoint_identity_on_gpu(pkg, name):
    case = synth.make_case(name)
    gpu = pkg.from_case(case)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(5)
    x = torch.rand(gpu.img_shape, generator=gen, device="cuda")
    y = torch.rand(gpu.ray_shape + (2,), generator=gen, device="cuda")
    Ax, _ = gpu.forward(x)
    Aty = gpu.backproject(y)
    lhs = torch.sum(Ax.double() * y.double()).item()
    rhs = torch.sum(x.double() * Aty.double()).item()
    assert abs(lhs - rhs) <= 2e-6 * abs(lhs)


@pytest.mark.parametrize("name", ["t2d", "t3d", "c0"])
def test_ray_terms_match_oracle(pkg, name):
    case, d, mask, M, c0 = case_data(name)
    gpu = pkg.from_case(case)
    gpu.set_data(d.cuda())
    gpu.set_metal_mask(mask.cuda(), "ray")
    pay, F = gpu.ray_terms(c0.cuda())
    O = oracle_of(case)
    _, _, po, fo = O.ray_model(c0.double().numpy(), d.double().numpy(), mask.numpy(), np.arange(case.geo.n_rays))
    pg = pay.cpu().double().numpy().reshape(-1, 4)
    keep = ~near_tie(case.geo).reshape(-1)
    assert rel_l2(pg[keep, :2], po[keep, :2]) < 1e-5            # B~
    assert rel_l2(pg[keep, :2] + pg[keep, 2:], po[keep, 2:]) < 1e-5  # B^ = B~ + D
    assert rel_l2(pg[keep, 2:], po[keep, 2:] - po[keep, :2]) < 1e-4  # D directly
    metal = mask.numpy().reshape(-1).astype(bool)
    assert np.all(pg[metal, 2:] == 0.0)                         # Eq. 11: p = q on the trace
    assert F == pytest.approx(fo.sum(), rel=1e-5)


@pytest.mark.parametrize("name", ["t2d", "t3d", "c0"])
def test_iterations_match_oracle(pkg, name):
    case, d, mask, M, c0 = case_data(name)
    gpu = pkg.from_case(case)
    O = oracle_of(case)
    Z, _ = gpu.info()
    assert Z == pytest.approx(O.normaliser(), rel=1e-6)
    gpu.set_data(d.cuda())
    gpu.set_metal_mask(mask.cuda(), "ray")
    c = c0.clone().cuda()
    hist = gpu.iterate(c, 10)
    c_ref, h_ref, sk_ref = O.iterate(c0.double().numpy(), d.double().numpy(), mask.numpy(), n_iter=10)
    assert rel_l2(c.cpu().numpy(), c_ref) < 1e-4
    np.testing.assert_allclose(hist, h_ref, rtol=1e-5)
    assert np.all(np.diff(hist) < 0)
    assert gpu.info()[1] == sk_ref


def test_metal_mask_from_metal_image(pkg):
    case, d, mask, M, c0 = case_data("c0")
    gpu = pkg.from_case(case)
    gpu.set_metal_mask(M.cuda(), "voxel")
    mg = gpu.metal_mask().cpu().numpy()
    T, mo = oracle_of(case).metal_trace(M.double().numpy(), case.metal_threshold)
    sure = np.abs(T - case.metal_threshold) > 1e-5 * max(T.max(), 1.0)
    assert mo.sum() > 100
    assert np.array_equal(mg[sure], mo[sure])
    # a host metal image gives the same mask
    gpu.set_metal_mask(M.clone(), "voxel")
    assert np.array_equal(gpu.metal_mask().cpu().numpy(), mg)


def test_metal_trace_values_do_not_matter_bitwise(pkg):
    # Eq. 11: data on the metal trace is never used, so the iterates are bitwise equal
    case, d, mask, M, c0 = case_data("t3d")
    gpu = pkg.from_case(case)
    gpu.set_metal_mask(mask.cuda(), "ray")
    out = []
    for dd in (d, torch.where(mask.bool()[None], torch.full_like(d, 7.0e5), d)):
        gpu.set_data(dd.cuda())
        c = c0.clone().cuda()
        h = gpu.iterate(c, 3)
        out.append((c.cpu(), h))
    assert torch.equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_deterministic_and_host_buffers(pkg):
    case, d, mask, M, c0 = case_data("t3d")
    gpu = pkg.from_case(case)
    gpu.set_data(d.cuda())
    gpu.set_metal_mask(mask.cuda(), "ray")
    c1 = c0.clone().cuda()
    h1 = gpu.iterate(c1, 4)
    c2 = c0.clone().cuda()
    h2 = gpu.iterate(c2, 4)
    assert torch.equal(c1, c2) and np.array_equal(h1, h2)
    # host tensors through the same entry points
    gpu.set_data(d.clone())
    gpu.set_metal_mask(mask.clone(), "ray")
    ch = c0.clone()
    hh = gpu.iterate(ch, 4)
    assert torch.equal(ch, c1.cpu()) and np.array_equal(hh, h1)


def test_all_rays_metal_changes_nothing(pkg):
    case, d, mask, M, c0 = case_data("t2d")
    gpu = pkg.from_case(case)
    gpu.set_data(d.cuda())
    gpu.set_metal_mask(torch.ones_like(mask).cuda(), "ray")
    c = c0.clone().cuda()
    hist = gpu.iterate(c, 2)
    assert np.all(hist == 0.0)
    assert torch.equal(c.cpu(), c0)


def test_zero_iterations_and_errors(pkg):
    case, d, mask, M, c0 = case_data("t2d")
    gpu = pkg.from_case(case)
    c = c0.clone().cuda()
    with pytest.raises(pkg.DeamError) as e:
        gpu.iterate(c, 1)                      # no data yet
    assert e.value.code == pkg.DEAM_ERR_STATE
    gpu.set_data(d.cuda())
    assert gpu.iterate(c, 0).size == 0 and torch.equal(c.cpu(), c0)
    with pytest.raises(ValueError):
        gpu.iterate(c[:, :5].contiguous(), 1)  # wrong shape caught in the binding


def test_host_pointers_to_device_only_arguments_are_rejected(pkg):
    # a host buffer where device memory is required is an argument error caught
    # on the host; the context stays usable afterwards
    import ctypes as C
    case, d, mask, M, c0 = case_data("t2d")
    gpu = pkg.from_case(case)
    gpu.set_data(d.cuda())
    gpu.set_metal_mask(mask.cuda(), "ray")
    L = pkg.lib()
    host_c = c0.contiguous()
    l_dev = torch.empty(gpu.ray_shape + (2,), device="cuda")
    rc = L.deam_forward(gpu._h, C.c_void_p(host_c.data_ptr()), C.c_void_p(l_dev.data_ptr()), None, None)
    assert rc == pkg.DEAM_ERR_ARG and b"device memory" in L.deam_last_error()
    host_l = torch.empty(gpu.ray_shape + (2,))
    rc = L.deam_forward(gpu._h, C.c_void_p(c0.cuda().data_ptr()), C.c_void_p(host_l.data_ptr()), None, None)
    assert rc == pkg.DEAM_ERR_ARG
    host_m = torch.empty(gpu.ray_shape, dtype=torch.uint8)
    assert L.deam_get_metal_mask(gpu._h, C.c_void_p(host_m.data_ptr()), None) == pkg.DEAM_ERR_ARG
    assert gpu.objective(c0.cuda()) > 0          # still usable


def test_checkpoint_and_resume_is_bitwise(pkg):
    # the image is the whole state of an iteration: six iterations in one call
    # equal three, a copy of the image, and three more
    case, d, mask, M, c0 = case_data("t3d")
    gpu = pkg.from_case(case)
    gpu.set_data(d.cuda())
    gpu.set_metal_mask(mask.cuda(), "ray")
    a = c0.clone().cuda()
    ha = gpu.iterate(a, 6)
    b = c0.clone().cuda()
    hb1 = gpu.iterate(b, 3)
    saved = b.cpu().clone()
    b2 = saved.cuda()
    hb2 = gpu.iterate(b2, 3)
    assert torch.equal(a, b2)
    np.testing.assert_array_equal(ha, np.concatenate([hb1, hb2]))


def test_allocation_failure_is_reported(pkg):
    # a context whose ray table alone exceeds the device's memory: the first
    # refused allocation ends deam_init with DEAM_ERR_OOM (no further requests),
    # and the device stays usable
    case = synth.make_case("t2d")
    geo = case.geo.replace(n_views=2_000_000, views_per_rotation=2_000_000, n_channels=40_000,
                           channel_pitch=5e-5)   # ray table 1.3 TB
    with pytest.raises(pkg.DeamError) as e:
        pkg.Deam(geo, case.I0, case.mu)
    assert e.value.code == pkg.DEAM_ERR_OOM
    case, d, mask, M, c0 = case_data("t2d")
    gpu = pkg.from_case(case)
    gpu.set_data(d.cuda())
    assert gpu.objective(c0.cuda()) > 0


# Cuts of the two helical benchmark scans small enough for whole oracle runs:
# the 256x256x32 case at one rotation (1160 views) and the 512x512x64 volume,
# detector and spectra at a quarter rotation (290 views).
FULL_SCALE_CUTS = {"c1_one_rotation": ("c1", 1160), "c2_quarter_rotation": ("c2s", 290)}


@pytest.mark.parametrize("cut", sorted(FULL_SCALE_CUTS))
def test_ten_iterations_at_full_scale_cut(pkg, cut, record_property, capsys):
    # The parity bar at the benchmark volumes and detectors: the image
    # after 10 iterations to rel-L2 1e-4 and the objective history to 1e-5
    # against the full oracle run (paper Sec. 2.3), plus every per-ray output on
    # seeded sampled rays to 1e-5; the errors are printed as the precision
    # report's rows for these sizes
    import dataclasses
    name, views = FULL_SCALE_CUTS[cut]
    case = synth.make_case(name)
    case = dataclasses.replace(case, geo=case.geo.replace(n_views=views))
    geo = case.geo
    dev = torch.device("cuda")
    d, metal = synth.measure(case, device=dev, seed=1)
    truth, _ = synth.voxelize(case, device=dev)
    mask = (metal >= case.metal_threshold).to(torch.uint8)
    c0 = synth.initial_image(case, truth).to(dev)
    del truth, metal
    gpu = pkg.from_case(case)
    gpu.set_data(d)
    gpu.set_metal_mask(mask, "ray")
    O = oracle_of(case)
    rays = np.sort(np.random.default_rng(17).choice(geo.n_rays, size=20000, replace=False))
    per_view = geo.n_rows * geo.n_channels
    v_of, k_of = rays // per_view, rays % geo.n_channels
    beta = geo.start_angle + 2 * math.pi * v_of / geo.views_per_rotation
    gam = (k_of - (geo.n_channels - 1) / 2 + geo.channel_offset) * geo.channel_pitch
    rays = rays[np.abs(np.abs(np.cos(beta + gam)) - np.abs(np.sin(beta + gam))) >= 1e-6]
    sel = torch.from_numpy(rays).to(dev)
    cn, dn, mn = c0.cpu().double().numpy(), d.cpu().double().numpy(), mask.cpu().numpy()
    lo_, go_, po, _ = O.ray_model(cn, dn, mn, rays)
    l, g = gpu.forward(c0, want_l=True, want_g=True)
    lg = l.reshape(-1, 2)[sel].cpu().double().numpy()
    gg = g.reshape(2, -1)[:, sel].cpu().double().numpy().T
    pay, F0 = gpu.ray_terms(c0)
    pg = pay.reshape(-1, 4)[sel].cpu().double().numpy()
    del l, g, pay
    c = c0.clone()
    hist = gpu.iterate(c, 10)
    c_ref, h_ref, _ = O.iterate(cn, dn, mn, n_iter=10)
    errs = {
        "line_integrals": rel_l2(lg, lo_),
        "expected_counts": rel_l2(gg, go_),
        "B_tilde": rel_l2(pg[:, :2], po[:, :2]),
        "B_hat": rel_l2(pg[:, :2] + pg[:, 2:], po[:, 2:]),
        "D": rel_l2(pg[:, 2:], po[:, 2:] - po[:, :2]),
        "objective": abs(F0 - h_ref[0]) / h_ref[0],
        "objective_history_max": float(np.max(np.abs(hist - h_ref) / h_ref)),
        "image_after_10": rel_l2(c.cpu().numpy(), c_ref),
    }
    for key, v in errs.items():
        record_property(f"{cut}_{key}", v)
    with capsys.disabled():
        print(f"\nprecision vs FP64 oracle [{cut}]: " + ", ".join(f"{k_}={v:.2e}" for k_, v in errs.items()))
    assert max(errs[x] for x in ("line_integrals", "expected_counts", "B_tilde", "B_hat")) < 1e-5
    assert errs["D"] < 1e-4
    assert errs["objective"] < 1e-5 and errs["objective_history_max"] < 1e-5
    assert errs["image_after_10"] < 1e-4
    assert np.all(np.diff(hist) < 0)


def test_single_voxel_closed_form_on_gpu(pkg):
    # one voxel, one ray, one bin: c' - c* = (1 - mu.L/Z)(c - c*) with Z = (mu1+mu2) L
    geo = synth.Geometry(1, 1, 1, 1, 2.0, 3.0, 4.0, 0.0, 0.0, 0.0, 570.0, 1040.0, 1, 8, 0.0, 0.0, 0.0,
                         1, 1.0, 1, 0.01, 0.0, 0.0)
    mu = np.array([[0.031], [0.013]])
    I0 = np.array([[2e5], [2e5]])
    gpu = pkg.Deam(geo, I0, mu)
    L = 2.0
    cstar = np.array([0.8, 0.3])
    cin = np.array([1.1, 0.45])
    dval = 2e5 * math.exp(-L * mu[:, 0] @ cstar)
    gpu.set_data(torch.full((2, 1, 1, 1), dval, dtype=torch.float32).cuda())
    c = torch.tensor(cin, dtype=torch.float32).reshape(1, 1, 1, 2).cuda()
    gpu.iterate(c, 1)
    Z = (0.031 + 0.013) * L
    want = cin - (L / Z) * (mu[:, 0] @ (cin - cstar))
    np.testing.assert_allclose(c.cpu().double().numpy().reshape(2), want, rtol=0, atol=2e-6)


def test_c1_full_size_sampled_views(pkg):
    # Full-size 256x256x32 helical case (3480 views x 16 x 672): forward on sampled
    # views and backprojection of rays restricted to a view subset, against the
    # oracle on those views only.
    case = synth.make_case("c1")
    geo = case.geo
    gpu = pkg.from_case(case)
    O = oracle_of(case)
    x = synth.random_image(geo, 8).float()
    l, _ = gpu.forward(x.cuda())
    v0, v1 = 1700, 1712
    lo = O.forward(x.double().numpy(), v0, v1)[v0:v1]
    keep = ~near_tie(geo, np.arange(v0, v1))
    assert rel_l2(l[v0:v1].cpu().double().numpy()[keep], lo[keep]) < 1e-5
    y = torch.zeros(gpu.ray_shape + (2,))
    gen = torch.Generator().manual_seed(9)
    y[v0:v1] = torch.rand((v1 - v0,) + gpu.ray_shape[1:] + (2,), generator=gen)
    img = gpu.backproject(y.cuda())
    ref = O.adjoint(y.double().numpy(), v0, v1)
    assert rel_l2(img.cpu().double().numpy(), ref) < 1e-5


def test_c2_full_size_bench_configuration(pkg):
    # The benchmark's own workload (512x512x64, 5800 views x 16 x 816, 2 x 120
    # bins, steel hips, noisy counts) in the launch configuration bench.py times
    # (same context, 13-slice slabs, one-wave forward grid): per-ray terms on
    # seeded sampled rays and the forward on sampled views against the oracle,
    # the adjoint on a view subset against the oracle's, and, at full size, the
    # fused c-step against its own backprojected sums plus a decrease of F.
    dev = torch.device("cuda")
    case = synth.make_case("c2")
    geo = case.geo
    d, metal = synth.measure(case, device=dev, seed=1)
    truth, _ = synth.voxelize(case, device=dev)
    mask = (metal >= case.metal_threshold).to(torch.uint8)
    c0 = synth.initial_image(case, truth).to(dev)
    del truth, metal
    gpu = pkg.from_case(case)
    gpu.set_data(d)
    gpu.set_metal_mask(mask, "ray")
    O = oracle_of(case)
    rays = np.sort(np.random.default_rng(21).choice(geo.n_rays, size=4096, replace=False))
    per_view = geo.n_rows * geo.n_channels
    v_of = rays // per_view
    k_of = rays % geo.n_channels
    beta = geo.start_angle + 2 * math.pi * v_of / geo.views_per_rotation
    gam = (k_of - (geo.n_channels - 1) / 2 + geo.channel_offset) * geo.channel_pitch
    ok = np.abs(np.abs(np.cos(beta + gam)) - np.abs(np.sin(beta + gam))) >= 1e-6
    rays = rays[ok]
    dn = d.cpu().double().numpy()
    _, _, po, _ = O.ray_model(c0.cpu().double().numpy(), dn, mask.cpu().numpy(), rays)
    del dn
    pay, F0 = gpu.ray_terms(c0)
    pg = pay.reshape(-1, 4)[torch.from_numpy(rays).to(dev)].cpu().double().numpy()
    assert rel_l2(pg[:, :2], po[:, :2]) < 1e-5
    assert rel_l2(pg[:, :2] + pg[:, 2:], po[:, 2:]) < 1e-5
    del pay
    v0, v1 = 2900, 2906
    x = synth.random_image(geo, 8).float()
    l, _ = gpu.forward(x.to(dev))
    lo = O.forward(x.double().numpy(), v0, v1)[v0:v1]
    keep = ~near_tie(geo, np.arange(v0, v1))
    assert rel_l2(l[v0:v1].cpu().double().numpy()[keep], lo[keep]) < 1e-5
    y = torch.zeros(gpu.ray_shape + (2,))
    y[v0:v1] = torch.rand((v1 - v0,) + gpu.ray_shape[1:] + (2,), generator=torch.Generator().manual_seed(9))
    img = gpu.backproject(y.to(dev))
    ref = O.adjoint(y.double().numpy(), v0, v1)
    assert rel_l2(img.cpu().double().numpy(), ref) < 1e-5
    del l, y, img
    sums, F, Z = gpu.backprojected_sums(c0)
    c1 = c0.clone()
    hist = gpu.iterate(c1, 1)
    assert hist[0] == pytest.approx(F, rel=1e-12)
    b, dl = sums[..., :2].double(), sums[..., 2:].double()
    upd = (b > 0) & (dl / b.clamp_min(1e-300) > -1)
    step = torch.where(upd, -torch.log1p(dl / torch.where(upd, b, torch.ones_like(b))) / Z, torch.zeros_like(b))
    expect = c0.double() + step
    # the ratio is formed in FP32: where 1 + delta/b~ is tiny, log1p amplifies
    # its rounding, so those few voxels are left out of the strict comparison
    well = ~upd | (1 + dl / b.clamp_min(1e-300) >= 1e-2)
    assert float(well.double().mean()) > 0.9999
    err = (c1.double() - expect).abs()[well]
    assert float(err.max()) <= 1e-6 * float(expect.abs().max()) + 1e-7
    assert gpu.objective(c1) < F0


@pytest.mark.parametrize("name", ["c0", "t3d"])
def test_precision_report(pkg, name, record_property, capsys):
    # Error of every output of the path against the FP64 oracle on the same
    # inputs (FP32 sampling, compensated FP32 spectral sums, FP64 objective
    # reduction): printed and recorded, and held to the parity tolerances.
    case, d, mask, M, c0 = case_data(name)
    gpu = pkg.from_case(case)
    gpu.set_data(d.cuda())
    gpu.set_metal_mask(mask.cuda(), "ray")
    O = oracle_of(case)
    keep = ~near_tie(case.geo)
    l, g = gpu.forward(c0.cuda(), want_l=True, want_g=True)
    lo = O.forward(c0.double().numpy())
    go = O.expected(lo)
    pay, F = gpu.ray_terms(c0.cuda())
    _, _, po, fo = O.ray_model(c0.double().numpy(), d.double().numpy(), mask.numpy(), np.arange(case.geo.n_rays))
    pg = pay.cpu().double().numpy().reshape(-1, 4)
    k = keep.reshape(-1)
    c = c0.clone().cuda()
    hist = gpu.iterate(c, 10)
    c_ref, h_ref, _ = O.iterate(c0.double().numpy(), d.double().numpy(), mask.numpy(), n_iter=10)
    errs = {
        "line_integrals": rel_l2(l.cpu().numpy()[keep], lo[keep]),
        "expected_counts": rel_l2(g.cpu().numpy()[:, keep], go[:, keep]),
        "B_tilde": rel_l2(pg[k, :2], po[k, :2]),
        "B_hat": rel_l2(pg[k, :2] + pg[k, 2:], po[k, 2:]),
        "objective": abs(F - fo.sum()) / fo.sum(),
        "objective_history_max": float(np.max(np.abs(hist - h_ref) / h_ref)),
        "image_after_10": rel_l2(c.cpu().numpy(), c_ref),
    }
    for key, v in errs.items():
        record_property(f"{name}_{key}", v)
    with capsys.disabled():
        print(f"\nprecision vs FP64 oracle [{name}]: " + ", ".join(f"{k_}={v:.2e}" for k_, v in errs.items()))
    assert max(errs[x] for x in ("line_integrals", "expected_counts", "B_tilde", "B_hat")) < 1e-5
    assert errs["objective"] < 1e-5 and errs["objective_history_max"] < 1e-5
    assert errs["image_after_10"] < 1e-4


def test_per_spectrum_traces_match_oracle(pkg):
    # separate traces T_L, T_H (Sec. 2.1): parity with the oracle, and the
    # low-kVp data on T_L never matters (bitwise)
    case, d, mask, M, c0 = case_data("t3d")
    m = mask.bool()
    gen = torch.Generator().manual_seed(3)
    mH = m & (torch.rand(m.shape, generator=gen) < 0.5)
    per = torch.stack([m, mH])
    gpu = pkg.from_case(case)
    gpu.set_data(d.cuda())
    gpu.set_metal_mask(per.cuda(), "per_spectrum")
    O = oracle_of(case)
    bits = O.mask_bits(per.numpy())
    assert np.array_equal(gpu.metal_mask().cpu().numpy(), bits) and set(np.unique(bits)) == {0, 1, 3}
    c = c0.clone().cuda()
    hist = gpu.iterate(c, 5)
    c_ref, h_ref, _ = O.iterate(c0.double().numpy(), d.double().numpy(), per.numpy(), n_iter=5)
    assert rel_l2(c.cpu().numpy(), c_ref) < 1e-4
    np.testing.assert_allclose(hist, h_ref, rtol=1e-5)
    d2 = d.clone()
    d2[0][m] = 3.0e5
    gpu.set_data(d2.cuda())
    c2 = c0.clone().cuda()
    h2 = gpu.iterate(c2, 5)
    assert torch.equal(c2, c) and np.array_equal(h2, hist)


def test_basis_images_match_oracle(pkg):
    # VMI mu(x, E) = mu_1(E) c_1 + mu_2(E) c_2 and the spectrum-weighted images (Sec. 3)
    import oracle
    case, d, mask, M, c0 = case_data("c0")
    gpu = pkg.from_case(case)
    coef = np.array([[0.02, 0.05], [1.0, 0.0], [-0.3, 2.0]])
    out = gpu.basis_images(c0.cuda(), coef)
    assert rel_l2(out.cpu().numpy(), oracle.basis_images(c0.double().numpy(), coef)) < 1e-6
    # a pure basis-1 image shows mu_1(E) everywhere at a bin centre
    ones = torch.zeros_like(c0)
    ones[..., 0] = 1.0
    e = 40
    vmi = gpu.vmi(ones.cuda(), [case.energies[e]]).cpu().numpy()
    np.testing.assert_allclose(vmi, case.mu[0, e], rtol=1e-6)
    kvp = gpu.kvp_images(c0.cuda()).cpu().numpy()
    w = case.I0 / case.I0.sum(1, keepdims=True)
    ref = oracle.basis_images(c0.double().numpy(), np.stack([w @ case.mu[0], w @ case.mu[1]], 1))
    assert kvp.shape == (2,) + tuple(c0.shape[:3]) and rel_l2(kvp, ref) < 1e-6


@pytest.mark.parametrize("variant", ["single_row_anisotropic", "odd_rows_offset_centre"])
def test_helical_edge_geometries_match_oracle(pkg, variant):
    # helical scans off the beaten path, element-wise against the oracle:
    # a single detector row over a multi-slice volume with dy != dx (the
    # backprojector's single-row slab and the anisotropic in-plane ratios), and
    # an odd row count with a row offset, a volume centre off the axis and
    # dz below the slice a row covers (one ragged 13-slice slab over an 11-slice volume)
    import dataclasses
    case = synth.make_case("t3d")
    g = case.geo
    if variant == "single_row_anisotropic":
        geo = g.replace(n_rows=1, dy=g.dx * 1.3, feed=2.0, z_start=-3.0, n_views=200)
    else:
        geo = g.replace(n_rows=5, row_offset=0.35, cx=7.0, cy=-4.0, cz=1.5, dz=2.0)
    case = dataclasses.replace(case, geo=geo)
    d, metal = synth.measure(case, seed=3)
    truth, _ = synth.voxelize(case)
    mask = (metal >= case.metal_threshold).to(torch.uint8)
    c0 = synth.initial_image(case, truth)
    gpu = pkg.from_case(case)
    O = oracle_of(case)
    keep = ~near_tie(geo)
    l, _ = gpu.forward(c0.cuda())
    lo = O.forward(c0.double().numpy())
    assert rel_l2(l.cpu().double().numpy()[keep], lo[keep]) < 1e-5
    y = synth.random_rays(geo, 4).float()
    assert rel_l2(gpu.backproject(y.cuda()).cpu().double().numpy(), O.adjoint(y.double().numpy())) < 1e-5
    gpu.set_data(d.cuda())
    gpu.set_metal_mask(mask.cuda(), "ray")
    c = c0.clone().cuda()
    hist = gpu.iterate(c, 5)
    c_ref, h_ref, _ = O.iterate(c0.double().numpy(), d.double().numpy(), mask.numpy(), n_iter=5)
    assert rel_l2(c.cpu().numpy(), c_ref) < 1e-4
    np.testing.assert_allclose(hist, h_ref, rtol=1e-5)
