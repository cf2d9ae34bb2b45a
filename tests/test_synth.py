"""Checks of the synthetic scanner/phantom generator (not of the method)."""
import math

import numpy as np
import torch

import synth


def test_chord_through_sphere_and_cylinder():
    o = synth.Obj("ellipsoid", (1.0, 2.0, 3.0), (5.0, 5.0, 5.0), 0.3)
    p = torch.tensor([[-100.0, 2.0, 3.0]], dtype=torch.float64)
    u = torch.tensor([[200.0, 0.0, 0.0]], dtype=torch.float64)
    L = synth.chord(o, p[:, 0], p[:, 1], p[:, 2], u[:, 0], u[:, 1], u[:, 2]) * 200.0
    assert abs(float(L) - 10.0) < 1e-12
    cyl = synth.Obj("cylinder", (0.0, 0.0, 0.0), (3.0, 3.0, 4.0), 0.0)
    # perpendicular through the axis: 2r; along the axis: the full length 2c
    L1 = synth.chord(cyl, p[:, 0] * 0 - 50, p[:, 1] * 0, p[:, 2] * 0, u[:, 0], u[:, 1], u[:, 2]) * 200.0
    assert abs(float(L1) - 6.0) < 1e-12
    Lz = synth.chord(cyl, torch.zeros(1, dtype=torch.float64), torch.zeros(1, dtype=torch.float64),
                     torch.full((1,), -50.0, dtype=torch.float64), torch.zeros(1, dtype=torch.float64),
                     torch.zeros(1, dtype=torch.float64), torch.full((1,), 100.0, dtype=torch.float64)) * 100.0
    assert abs(float(Lz) - 8.0) < 1e-12


def test_spectra_and_attenuation():
    E = synth.energy_grid(1.0)
    assert len(E) == 120 and E[0] == 20.5 and E[-1] == 139.5
    s90 = synth.spectrum(E, 90.0, 2.5, 1e5)
    assert abs(s90.sum() - 1e5) < 1e-6 and np.all(s90[E > 90] == 0) and np.count_nonzero(s90) == 70
    for m in ("polystyrene", "cacl2", "titanium", "steel"):
        mu = synth.attenuation(m, E)
        assert np.all(mu > 0) and np.all(np.diff(mu) < 0)
    mu = synth.attenuation("polystyrene", np.array([60.0]))
    assert abs(mu[0] - 0.0196) < 1e-12


def test_geometry_conventions():
    case = synth.make_case("c1")
    g = case.geo
    assert (g.n_views, g.n_rows, g.n_channels) == (3480, 16, 672)
    assert abs(g.feed - 6.0) < 1e-12
    s, u = synth.ray_endpoints(g, torch.tensor([0, g.views_per_rotation]))
    assert abs(float(s[1, 2] - s[0, 2]) - g.feed) < 1e-12
    # rays point from the source towards the isocentre side
    assert float((s[0, :2] * u[0, 0, 0, :2]).sum()) < 0
    c2 = synth.make_case("c2").geo
    assert (c2.nx, c2.nz, c2.n_views, c2.n_channels) == (512, 64, 5800, 816)
    assert c2.n_rays == 75_724_800


def test_measure_is_seeded_and_metal_marks_trace():
    case = synth.make_case("t2d")
    d1, m1 = synth.measure(case, seed=3)
    d2, m2 = synth.measure(case, seed=3)
    assert torch.equal(d1, d2) and torch.equal(m1, m2)
    assert (m1 >= case.metal_threshold).sum() > 0
    dn, _ = synth.measure(case, noiseless=True)
    assert float(dn.max()) <= 1e5 * 1.0000001
