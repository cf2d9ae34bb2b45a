"""Pins of the oracle's regularised MAR-DEAM (Eqs. 6-7): the penalty function,
the penalty sum, and the c-step with De Pierro's separable surrogate."""
import math

import numpy as np
import pytest

import synth


def test_phi_closed_forms(oracle_lib):
    import oracle
    for delta in (0.5, 2.0):
        assert oracle.phi(0.0, delta) == 0.0
        for u in (0.3, 1.7, 9.0):
            a = u / delta
            assert oracle.phi(u, delta) == pytest.approx(delta**2 * (a - math.log1p(a)), rel=1e-14)
            assert oracle.phi(-u, delta) == oracle.phi(u, delta)
        # quadratic near 0, linear (slope delta) far away, convex in between
        assert oracle.phi(1e-4, delta) == pytest.approx(0.5e-8, rel=1e-3)
        assert oracle.phi(1e6, delta) / 1e6 == pytest.approx(delta, rel=1e-4)
        us = np.linspace(-5, 5, 101)
        v = np.array([oracle.phi(u, delta) for u in us])
        assert np.all(v[:-2] + v[2:] - 2 * v[1:-1] >= -1e-15)


def test_penalty_of_two_voxels(oracle_lib):
    # two voxels along x: each ordered pair once, weight 1/dx: R = lambda 2 (1/dx) phi(a - b)
    import oracle
    geo = synth.Geometry(1, 2, 1, 1, 1.5, 1.0, 1.0, 0.0, 0.0, 0.0, 570.0, 1040.0, 1, 8, 0.0, 0.0, 0.0,
                         1, 1.0, 1, 0.01, 0.0, 0.0)
    O = oracle.Oracle(geo, np.ones((2, 1)), np.full((2, 1), 0.02))
    c = np.array([[[[0.7, 0.1], [1.2, 0.4]]]])
    lam, delta = 0.3, 0.8
    want = lam * 2 / 1.5 * (oracle.phi(-0.5, delta) + oracle.phi(-0.3, delta))
    assert O.penalty(c, lam, delta) == pytest.approx(want, rel=1e-14)
    # a 3x3x3 uniform-spacing cube: 26 neighbours of the centre at distances 1, sqrt2, sqrt3
    geo3 = geo.replace(nx=3, ny=3, nz=3, dx=1.0)
    O3 = oracle.Oracle(geo3, np.ones((2, 1)), np.full((2, 1), 0.02))
    c3 = np.zeros((3, 3, 3, 2))
    c3[1, 1, 1, 0] = 1.0
    # only pairs touching the centre differ: 2 x (6/1 + 12/sqrt2 + 8/sqrt3) phi(1)
    want3 = 2 * (6 + 12 / math.sqrt(2) + 8 / math.sqrt(3)) * oracle.phi(1.0, 1.0)
    assert O3.penalty(c3, 1.0, 1.0) == pytest.approx(want3, rel=1e-13)


def _case(name):
    case = synth.make_case(name)
    d, metal = synth.measure(case, seed=1)
    truth, _ = synth.voxelize(case)
    mask = (metal >= case.metal_threshold).numpy().astype(np.uint8)
    c0 = synth.initial_image(case, truth).double().numpy()
    return case, d.double().numpy(), mask, c0


def test_lambda_zero_is_plain_deam(oracle_lib):
    import oracle
    case, d, mask, c0 = _case("t3d")
    O = oracle.from_case(case)
    c1, h1, _ = O.iterate(c0, d, mask, n_iter=2)
    c2, h2, hR, _ = O.iterate_reg(c0, d, mask, n_iter=2, lam=0.0, delta=1.0)
    np.testing.assert_allclose(c2, c1, rtol=0, atol=1e-12)
    np.testing.assert_allclose(h2, h1, rtol=1e-13)
    assert np.all(hR == 0.0)


@pytest.mark.parametrize("name,lam,delta", [("t2d", 2e3, 0.05), ("t3d", 5e3, 0.02)])
def test_penalised_objective_decreases(oracle_lib, name, lam, delta):
    import oracle
    case, d, mask, c0 = _case(name)
    O = oracle.from_case(case)
    c, hF, hR, _ = O.iterate_reg(c0, d, mask, n_iter=6, lam=lam, delta=delta)
    tot = hF + hR
    assert np.all(np.diff(tot) < 0), tot
    assert hR[0] > 1e-3 * hF[0]                  # the penalty is not negligible here
    # the data-only surrogate step would not decrease F + R as reliably: the
    # penalty changes the result
    c_plain, _, _ = O.iterate(c0, d, mask, n_iter=6)
    assert np.abs(c - c_plain).max() > 1e-4


def test_penalty_moves_voxels_seen_only_by_metal_rays(oracle_lib):
    # Sec. 3: without data the metal region keeps its initial value; the penalty
    # term updates it gradually.  With every ray on the trace the data term is
    # neutral: a uniform image is a fixed point and a step edge is smoothed with
    # R decreasing at every iteration.
    import oracle
    case, d, mask, c0 = _case("t2d")
    O = oracle.from_case(case)
    allm = np.full_like(mask, 3)
    uni = np.zeros_like(c0)
    uni[..., 0] = 0.9
    u1, _, _, _ = O.iterate_reg(uni, d, allm, n_iter=2, lam=10.0, delta=0.1)
    np.testing.assert_allclose(u1, uni, rtol=0, atol=1e-13)
    step = uni.copy()
    step[:, :, : step.shape[2] // 2, 0] = 0.3
    s1, _, hR, _ = O.iterate_reg(step, d, allm, n_iter=4, lam=10.0, delta=0.1)
    assert np.all(np.diff(hR) < 0)
    edge = step.shape[2] // 2
    assert s1[0, 10, edge - 1, 0] > 0.3 and s1[0, 10, edge, 0] < 0.9
