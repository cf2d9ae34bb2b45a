"""Pins of the oracle's MAR-DEAM arithmetic (Eqs. 5, 8-11 and the c-step)
against closed forms and invariants that hold independently of the oracle."""
import math

import numpy as np
import pytest

import synth


def _single_voxel_geo(dx=2.0):
    # one 1x1x1 voxel, one view, one row, one channel: the central ray of view 0
    # runs along -x through the voxel centre, so h = dx
    return synth.Geometry(1, 1, 1, 1, dx, 3.0, 4.0, 0.0, 0.0, 0.0, 570.0, 1040.0, 1, 8, 0.0, 0.0, 0.0,
                          1, 1.0, 1, 0.01, 0.0, 0.0)


def test_monoenergetic_closed_form(oracle_lib):
    # mu_i(E) constant in E: g = (sum_E I0(E) b(k)) exp(-mu . l) and S_i = mu_i g (Eq. 8)
    import oracle
    case = synth.make_case("t2d")
    nE = 5
    I0 = np.array([[1e4, 2e4, 0.0, 5e3, 1e3], [3e4, 0.0, 1e4, 1e4, 2e4]])
    mu = np.array([[0.02] * nE, [0.05] * nE])
    bow = np.linspace(0.5, 1.0, case.geo.n_channels)
    O = oracle.Oracle(case.geo, I0, mu, bowtie=bow)
    l = synth.random_rays(case.geo, 1).numpy() * 50.0
    g = O.expected(l)
    ex = np.exp(-(0.02 * l[..., 0] + 0.05 * l[..., 1])) * bow[None, None, :]
    np.testing.assert_allclose(g[0], I0[0].sum() * ex, rtol=1e-13)
    np.testing.assert_allclose(g[1], I0[1].sum() * ex, rtol=1e-13)


def test_single_bin_and_payload(oracle_lib):
    # One energy bin: g = I0 e^{-mu.l}; the payload of a non-metal ray is
    # B~_i = sum_j mu_i g_j and B^_i = sum_j mu_i d~_j (the p-step ratio d~/g of
    # Eq. 10 times S_ij = mu_i g_j); on a metal ray B^ = B~ (p = q, Eq. 11).
    import oracle
    case = synth.make_case("t2d")
    geo = case.geo
    I0 = np.array([[7e4], [3e4]])
    mu = np.array([[0.021], [0.047]])
    O = oracle.Oracle(geo, I0, mu)
    c = synth.random_image(geo, 4).numpy() * 0.5
    rng = np.random.default_rng(0)
    d = rng.uniform(10, 5e4, size=(2,) + O.ray_shape)
    d[0, 0, 0, :5] = -3.0    # negative counts are clamped to zero
    mask = np.zeros(O.ray_shape, np.uint8)
    mask[3, 0, 10:20] = 1
    rays = np.arange(geo.n_rays)
    l, g, pay, f = O.ray_model(c, d, mask, rays)
    ex = np.exp(-(l @ mu[:, 0]))
    np.testing.assert_allclose(g, ex[:, None] * I0[:, 0][None, :], rtol=1e-13)
    dt = np.maximum(d.reshape(2, -1).T, 0.0)
    m = mask.reshape(-1).astype(bool)
    Bt = np.outer(g.sum(1), mu[:, 0])
    Bh = np.outer(np.where(m, g.sum(1), dt.sum(1)), mu[:, 0])
    np.testing.assert_allclose(pay[:, :2], Bt, rtol=1e-13)
    np.testing.assert_allclose(pay[:, 2:], Bh, rtol=1e-13)
    # Eq. (5) per ray, 0 ln 0 = 0, metal rays excluded
    term = np.where(dt > 0, dt * np.log(np.where(dt > 0, dt, 1.0) / g) - dt + g, g)
    np.testing.assert_allclose(f, np.where(m, 0.0, term.sum(1)), rtol=1e-12)
    assert O.objective(c, d, mask) == pytest.approx(f.sum(), rel=1e-12)


@pytest.mark.parametrize("mu2", [0.0, 0.013])
def test_single_voxel_update_closed_form(oracle_lib, mu2):
    # One voxel, one ray of length L = dx, one energy bin, both spectra equal:
    # d = I0 exp(-L mu.c*), g = I0 exp(-L mu.c), so ln(b^_i / b~_i) = ln(d / g)
    # = L mu.(c - c*) for each component i with mu_i > 0, and the c-step gives
    # c_i' = c_i - (L / Z) mu.(c - c*) with Z = (mu_1 + mu_2) L.  A component
    # with mu_i = 0 has b~_i = 0 and is left unchanged.
    import oracle
    geo = _single_voxel_geo()
    L = geo.dx
    mu = np.array([[0.031], [mu2]])
    I0 = np.array([[2e5], [2e5]])
    O = oracle.Oracle(geo, I0, mu)
    cstar = np.array([0.8, 0.3])
    c = np.array([1.1, 0.45]).reshape(O.img_shape)
    dval = 2e5 * math.exp(-L * (mu[:, 0] @ cstar))
    d = np.full((2,) + O.ray_shape, dval)
    Z = O.normaliser()
    assert Z == pytest.approx((0.031 + mu2) * L, rel=1e-14)
    c1, hist, skipped = O.iterate(c, d, None, n_iter=1)
    s = (L / Z) * (mu[:, 0] @ (c.reshape(2) - cstar))
    want = c.reshape(2) - s
    if mu2 == 0.0:
        want[1] = c.reshape(2)[1]
        assert skipped == 1
        # Z = mu_1 L: the first component converges in one step
        assert want[0] == pytest.approx(cstar[0], abs=1e-12)
    np.testing.assert_allclose(c1.reshape(2), want, rtol=0, atol=1e-12)
    g = 2e5 * math.exp(-L * (mu[:, 0] @ c.reshape(2)))
    assert hist[0] == pytest.approx(2 * (dval * math.log(dval / g) - dval + g), rel=1e-10)


def _noisy_case(name, seed=0):
    case = synth.make_case(name, seed)
    d, metal = synth.measure(case, seed=seed + 1)
    truth, M = synth.voxelize(case)
    mask = (metal >= case.metal_threshold).numpy().astype(np.uint8)
    c0 = synth.initial_image(case, truth).double().numpy()
    return case, d.double().numpy(), mask, c0, truth.numpy(), M.numpy()


@pytest.mark.parametrize("name", ["t2d", "t3d"])
def test_noiseless_fixed_point_and_zero_objective(oracle_lib, name):
    # Data generated by the model at c is reproduced exactly: F(c) = 0 and the
    # c-step leaves c unchanged (b^ = b~ everywhere).
    import oracle
    case, _, mask, c0, _, _ = _noisy_case(name)
    O = oracle.from_case(case)
    d = O.expected(O.forward(c0))
    assert abs(O.objective(c0, d, mask)) < 1e-9 * d.sum()
    c1, _, _ = O.iterate(c0, d, mask, n_iter=1)
    np.testing.assert_allclose(c1, c0, rtol=0, atol=1e-12)


@pytest.mark.parametrize("name", ["t2d", "t3d"])
def test_objective_decreases_monotonically(oracle_lib, name):
    import oracle
    case, d, mask, c0, _, _ = _noisy_case(name)
    O = oracle.from_case(case)
    _, hist, _ = O.iterate(c0, d, mask, n_iter=8)
    assert np.all(hist >= 0)
    assert np.all(np.diff(hist) < 0), hist
    # without the metal trace (t = infinity) the plain DEAM objective decreases too
    _, hist0, _ = O.iterate(c0, d, np.zeros_like(mask), n_iter=4)
    assert np.all(np.diff(hist0) < 0)
    assert hist0[0] > hist[0]   # metal rays add data misfit


def test_metal_ray_values_are_ignored(oracle_lib):
    # Eq. (11): on rays with T(y) >= t the measurement is never used, so any
    # values there give the same iterates.
    import oracle
    case, d, mask, c0, _, _ = _noisy_case("t3d")
    O = oracle.from_case(case)
    assert mask.sum() > 100
    d2 = d.copy()
    rng = np.random.default_rng(7)
    m = mask.astype(bool)
    d2[0][m] = rng.uniform(-100, 1e6, size=m.sum())
    d2[1][m] = 0.0
    oracle.lib().or_set_threads(1)
    try:
        ca, ha, _ = O.iterate(c0, d, mask, n_iter=3)
        cb, hb, _ = O.iterate(c0, d2, mask, n_iter=3)
    finally:
        oracle.lib().or_set_threads(0)
    assert np.array_equal(ca, cb) and np.array_equal(ha, hb)
    # ... and changing a non-metal ray does change them
    d3 = d.copy()
    idx = np.argwhere(~m & (d[0] < 0.5 * d[0].max()))[0]   # a non-metal ray through the body
    d3[0][tuple(idx)] *= 1.5
    cc, _, _ = O.iterate(c0, d3, mask, n_iter=1)
    assert not np.array_equal(cc, O.iterate(c0, d, mask, n_iter=1)[0])


def test_voxels_seen_only_by_metal_rays_stay_fixed(oracle_lib):
    # If every ray through a voxel is a metal-trace ray then b^ = b~ there and the
    # c-step leaves the voxel unchanged (the paper's remark that MAR-DEAM cannot
    # reconstruct the metal region without a penalty term).
    import oracle
    case, d, _, c0, _, _ = _noisy_case("t2d")
    O = oracle.from_case(case)
    M = np.zeros(O.img_shape[:3])
    M[0, 20:24, 30:33] = 1.0
    T, mask = O.metal_trace(M, 1e-12)
    c1, _, _ = O.iterate(c0, d, mask, n_iter=2)
    region = M.astype(bool)
    np.testing.assert_allclose(c1[region], c0[region], rtol=0, atol=1e-13)
    assert np.abs(c1[~region] - c0[~region]).max() > 1e-4


def test_metal_trace_threshold(oracle_lib):
    # T = A M is the metal path length (mm); it approaches the exact metal chord
    # and T(y) = t counts as metal ("T(y) < t" is what keeps the data).
    import oracle
    case, _, _, _, _, M = _noisy_case("c0")
    O = oracle.from_case(case)
    T, mask = O.metal_trace(M, case.metal_threshold)
    _, metal = synth.measure(case, noiseless=True)
    metal = metal.numpy()
    hit = metal > 1.0
    assert np.abs(T[hit] - metal[hit]).mean() < 0.1 * metal[hit].mean()
    assert np.array_equal(mask.astype(bool), T >= case.metal_threshold)
    assert set(np.unique(mask)) <= {0, 3}        # one system operator: both spectra's bits
    t_exact = float(T[hit][0])
    _, m2 = O.metal_trace(M, t_exact)
    assert m2.reshape(-1)[np.flatnonzero(hit.reshape(-1))[0]] == 3
    _, m3 = O.metal_trace(M, np.inf)
    assert m3.sum() == 0


def test_gradient_matches_central_differences(oracle_lib):
    # dF/dc_i(x) = b^_i(x) - b~_i(x); checked with central differences at a
    # relative step of 1e-3 on 16 random (voxel, component) pairs.
    import oracle
    case, d, mask, c0, _, _ = _noisy_case("t3d")
    O = oracle.from_case(case)
    grad = O.gradient(c0, d, mask)
    rng = np.random.default_rng(3)
    flat = c0.reshape(-1)
    seen = np.flatnonzero(np.abs(grad.reshape(-1)) > 1e-3 * np.abs(grad).max())
    picks = rng.choice(seen, size=16, replace=False)
    for p in picks:
        h = 1e-3 * max(abs(flat[p]), 0.1)
        cp, cm = flat.copy(), flat.copy()
        cp[p] += h
        cm[p] -= h
        fd = (O.objective(cp.reshape(c0.shape), d, mask) - O.objective(cm.reshape(c0.shape), d, mask)) / (2 * h)
        assert fd == pytest.approx(grad.reshape(-1)[p], rel=2e-4, abs=1e-6 * np.abs(grad).max())


def test_backprojected_sums_are_adjoint_of_payload(oracle_lib):
    # b~ = A^T B~ and b^ = A^T B^ with the per-ray payload (derivation of the
    # c-step: the energy sums factor per ray)
    import oracle
    case, d, mask, c0, _, _ = _noisy_case("t3d")
    O = oracle.from_case(case)
    bt, bh, F = O.backprojected_sums(c0, d, mask)
    _, _, pay, f = O.ray_model(c0, d, mask, np.arange(case.geo.n_rays))
    pay = pay.reshape(O.ray_shape + (4,))
    np.testing.assert_allclose(bt, O.adjoint(pay[..., :2]), rtol=1e-11, atol=1e-9)
    np.testing.assert_allclose(bh, O.adjoint(pay[..., 2:]), rtol=1e-11, atol=1e-9)
    assert F == pytest.approx(f.sum(), rel=1e-12)


def test_per_spectrum_traces(oracle_lib):
    # Sec. 2.1: with different traces T_L, T_H the substitution p = q applies per
    # spectrum.  Data of spectrum j on its own trace is never used; data of the
    # other spectrum on those rays is.  Equal traces reproduce the joint mask.
    import oracle
    case, d, mask, c0, _, _ = _noisy_case("t3d")
    O = oracle.from_case(case)
    m = mask.astype(bool)
    rng = np.random.default_rng(11)
    mL = m.copy()
    mH = m & (rng.random(m.shape) < 0.5)          # a smaller high-kVp trace
    per = np.stack([mL, mH])
    ca, ha, _ = O.iterate(c0, d, per, n_iter=2)
    cj, hj, _ = O.iterate(c0, d, np.stack([m, m]), n_iter=2)
    cb, hb, _ = O.iterate(c0, d, mask, n_iter=2)
    np.testing.assert_allclose(cj, cb, rtol=0, atol=1e-13)
    d2 = d.copy()
    d2[0][mL] = rng.uniform(0, 1e6, size=mL.sum())  # low-kVp data on T_L: ignored
    c2, h2, _ = O.iterate(c0, d2, per, n_iter=2)
    np.testing.assert_allclose(c2, ca, rtol=0, atol=1e-13)
    np.testing.assert_allclose(h2, ha, rtol=1e-14)
    d3 = d.copy()
    only_L = mL & ~mH
    d3[1][only_L] *= 1.3                             # high-kVp data there is used
    c3, _, _ = O.iterate(c0, d3, per, n_iter=1)
    assert np.abs(c3 - O.iterate(c0, d, per, n_iter=1)[0]).max() > 1e-6
    assert ha[0] > hb[0]                             # fewer excluded rays: more data misfit
