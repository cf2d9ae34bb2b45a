"""Pins of the oracle's system operator h(x, y) (Eq. 8) against facts that do not
come from the oracle: hand-worked weights, exact chord lengths, brute-force
transposition and the adjoint identity."""
import math
import os

import numpy as np
import pytest
import torch

import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "joseph_worked.txt")


def _val(s):
    if s.startswith("atan:"):
        return math.atan(float(s[5:]))
    if s.startswith("sqrt:"):
        return math.sqrt(float(s[5:]))
    if s == "pi/2":
        return math.pi / 2
    return float(s)


def _load_golden():
    examples, cur = [], None
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        key, _, rest = line.partition(" ")
        if key == "example":
            cur = {"name": rest, "taps": []}
            examples.append(cur)
        elif key == "geometry":
            kv = dict(p.split("=") for p in rest.split())
            ints = {"kind", "nx", "ny", "nz", "n_views", "views_per_rotation", "n_rows", "n_channels"}
            cur["geo"] = synth.Geometry(**{k: (int(v) if k in ints else _val(v)) for k, v in kv.items()})
        elif key == "L":
            cur["L"] = _val(rest)
        elif key == "tap":
            ix, iy, iz, f = rest.split()
            cur["taps"].append((int(ix), int(iy), int(iz), float(f)))
    return examples


def _oracle(geo, nE=1):
    import oracle
    I0 = np.ones((2, nE))
    mu = np.full((2, nE), 0.02)
    return oracle.Oracle(geo, I0, mu)


@pytest.mark.parametrize("ex", _load_golden(), ids=lambda e: e["name"])
def test_hand_worked_weights(oracle_lib, ex):
    geo = ex["geo"]
    O = _oracle(geo)
    idx, w = O.taps(0, 0, 0)
    dense = np.zeros(geo.n_voxels)
    np.add.at(dense, idx, w)
    want = np.zeros(geo.n_voxels)
    for ix, iy, iz, f in ex["taps"]:
        want[(iz * geo.ny + iy) * geo.nx + ix] += ex["L"] * f
    np.testing.assert_allclose(dense, want, rtol=0, atol=1e-12)


def _box_geo(nx=7, ny=5, nz=3, **kw):
    base = dict(kind=1, nx=nx, ny=ny, nz=nz, dx=2.0, dy=3.0, dz=1.5, cx=0.0, cy=0.0, cz=0.0,
                sid=570.0, sdd=1040.0, n_views=1, views_per_rotation=8, start_angle=0.0, feed=0.0,
                z_start=0.0, n_rows=1, row_pitch=1.0, n_channels=1, channel_pitch=0.01,
                channel_offset=0.0, row_offset=0.0)
    base.update(kw)
    return synth.Geometry(**base)


def test_axis_aligned_ray_through_voxel_centres(oracle_lib):
    # Central ray of view 0 runs along -x at y = z = 0, i.e. through the centres
    # of the voxels (ix, 2, 1): the line integral is dx * sum of those values.
    geo = _box_geo()
    O = _oracle(geo)
    c = synth.random_image(geo, 3).numpy()
    l = O.forward(c)[0, 0, 0]
    np.testing.assert_allclose(l, geo.dx * c[1, 2, :, :].sum(axis=0), rtol=1e-14)
    # rotated by 90 degrees: along -y through (3, iy, 1), spacing dy
    geo2 = _box_geo(start_angle=math.pi / 2)
    l2 = _oracle(geo2).forward(c)[0, 0, 0]
    np.testing.assert_allclose(l2, geo2.dy * c[1, :, 3, :].sum(axis=0), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("beta,gamma_ch,row,nx,ny", [(0.3, 2, 1, 9, 41), (2.0, -3, 0, 41, 9),
                                                    (4.1, 1, 2, 41, 9), (3.3, 0, 0, 9, 41)])
def test_partition_of_unity(oracle_lib, beta, gamma_ch, row, nx, ny):
    _check_partition_of_unity(beta, gamma_ch, row, nx, ny)


def test_partition_of_unity_random_rays(oracle_lib):
    # the same property over random view angles, channels, rows and box shapes
    hyp = pytest.importorskip("hypothesis")
    st = hyp.strategies

    @hyp.settings(max_examples=40, deadline=None, derandomize=True)
    @hyp.given(beta=st.floats(0.0, 2 * math.pi), gamma_ch=st.integers(-3, 3), row=st.integers(0, 2),
               short=st.integers(5, 11))
    def check(beta, gamma_ch, row, short):
        # the box is long across the ray's dominant axis so every sample is interior
        ang = beta + gamma_ch * 0.002
        x_dominant = abs(math.cos(ang)) >= abs(math.sin(ang))
        nx, ny = (short, 41) if x_dominant else (41, short)
        if abs(abs(math.cos(ang)) - abs(math.sin(ang))) < 0.2:
            return  # near 45 degrees neither box shape keeps every sample interior
        _check_partition_of_unity(beta, gamma_ch, row, nx, ny)

    check()


def _check_partition_of_unity(beta, gamma_ch, row, nx, ny):
    # For a uniform image every interior sample's weights sum to L, so the line
    # integral of a uniform box is L times the number of planes, i.e. the exact
    # length of the ray between the first and last voxel-centre planes plus one
    # plane spacing.  The box is wide across the ray so every sample is interior.
    geo = _box_geo(nx=nx, ny=ny, nz=40, dx=1.0, dy=1.0, dz=1.0, start_angle=beta,
                   n_channels=7, channel_pitch=0.002, n_rows=3, row_pitch=2.0)
    O = _oracle(geo)
    c = np.zeros(O.img_shape)
    c[..., 0] = 1.0
    c[..., 1] = 2.5
    k = gamma_ch + 3
    l = O.forward(c)[0, row, k]
    ang = beta + (k - 3) * geo.channel_pitch
    u = np.array([-geo.sdd * math.cos(ang), -geo.sdd * math.sin(ang), (row - 1) * 2.0])
    s = np.array([geo.sid * math.cos(beta), geo.sid * math.sin(beta), 0.0])
    ax = 0 if abs(u[0]) >= abs(u[1]) else 1
    n, d = (geo.nx, geo.dx) if ax == 0 else (geo.ny, geo.dy)
    L = d * np.linalg.norm(u) / abs(u[ax])
    # count planes whose sample has all four taps inside (the sample lies in
    # the convex hull of voxel centres)
    cnt = 0
    for p in range(n):
        P = (p - (n - 1) / 2) * d
        t = (P - s[ax]) / u[ax]
        q = s[1 - ax] + t * u[1 - ax]
        z = s[2] + t * u[2]
        other = geo.ny if ax == 0 else geo.nx
        if abs(q) <= (other - 1) / 2 and abs(z) <= (geo.nz - 1) / 2 * geo.dz:
            cnt += 1
    assert cnt == n
    np.testing.assert_allclose(l, [L * cnt, 2.5 * L * cnt], rtol=1e-13)


def _sphere_case(n, fov=60.0, nz=None, helical=False):
    nz = n if nz is None else nz
    d = fov / n
    geo = synth.Geometry(1 if helical else 0, n, n, nz, d, d, fov / nz, 0.0, 0.0, 0.0, 570.0, 1040.0,
                         24, 24, 0.17, 6.0 if helical else 0.0, -6.0 if helical else 0.0,
                         5 if helical else 1, 6.0, 41, synth.fan_pitch(fov / 2, 570.0, 41), 0.3,
                         0.0)
    return geo


@pytest.mark.parametrize("helical", [False, True])
def test_chord_lengths_converge_under_refinement(oracle_lib, helical):
    # Projections of a voxelised ellipsoid (2D: elliptic cylinder) approach the
    # exact chord lengths as the voxels shrink: the error must fall roughly
    # in proportion to the voxel size.
    obj = synth.Obj("ellipsoid" if helical else "cylinder", (4.0, -3.0, 1.5), (17.0, 11.0, 14.0 if helical else 1e3),
                    0.6, c1=1.0)
    errs = []
    for n in (16, 32, 64):
        geo = _sphere_case(n, nz=(n // 2 if helical else 1), helical=helical)
        case = synth.Case("sphere", geo, np.array([60.0]), np.ones((2, 1)), np.full((2, 1), 0.02),
                          np.zeros(1), [obj], (1.0, 1.0))
        c, _ = synth.voxelize(case, ss=4)
        O = _oracle(geo)
        l = O.forward(c.double().numpy())[..., 0]
        s, u = synth.ray_endpoints(geo, torch.arange(geo.n_views))
        ux, uy, uz = u[..., 0], u[..., 1], u[..., 2]
        px = s[:, 0][:, None, None].expand_as(ux)
        py = s[:, 1][:, None, None].expand_as(ux)
        pz = s[:, 2][:, None, None].expand_as(ux)
        exact = (synth.chord(obj, px, py, pz, ux, uy, uz) * torch.sqrt(ux**2 + uy**2 + uz**2)).numpy()
        errs.append(np.sqrt(np.mean((l - exact) ** 2)) / np.sqrt(np.mean(exact**2)))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 0.04
    assert errs[0] / errs[2] > 2.5


def test_explicit_matrix_transpose(oracle_lib):
    # Build H column by column from forward projections of unit images and row
    # by row from backprojections of unit rays: the two must be transposes.
    geo = synth.Geometry(1, 5, 4, 3, 7.0, 8.0, 5.0, 1.0, -2.0, 0.5, 570.0, 1040.0, 6, 4, 0.2, 9.0, -6.0,
                         2, 9.0, 5, 0.02, 0.1, 0.3)
    O = _oracle(geo)
    nv, nr = geo.n_voxels, geo.n_rays
    Hf = np.zeros((nr, nv))
    for x in range(nv):
        c = np.zeros(O.img_shape)
        c.reshape(-1, 2)[x, 0] = 1.0
        Hf[:, x] = O.forward(c)[..., 0].reshape(-1)
    Ha = np.zeros((nr, nv))
    for y in range(nr):
        yy = np.zeros(O.ray_shape + (2,))
        yy.reshape(-1, 2)[y, 1] = 1.0
        Ha[y, :] = O.adjoint(yy)[..., 1].reshape(-1)
    assert np.count_nonzero(Hf) > 50
    np.testing.assert_allclose(Hf, Ha, rtol=0, atol=1e-15)


def test_adjoint_identity(oracle_lib):
    case = synth.make_case("t3d")
    O = _oracle(case.geo)
    x = synth.random_image(case.geo, 11).numpy()
    y = synth.random_rays(case.geo, 12).numpy()
    lhs = np.sum(O.forward(x) * y)
    rhs = np.sum(x * O.adjoint(y))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_view_subsets_partition(oracle_lib):
    # Backprojection is additive over views: partial sums over disjoint view
    # ranges add up to the whole (the basis of a view-sharded multi-GPU run).
    case = synth.make_case("t3d")
    O = _oracle(case.geo)
    y = synth.random_rays(case.geo, 5).numpy()
    full = O.adjoint(y)
    V = case.geo.n_views
    parts = O.adjoint(y, 0, V // 3) + O.adjoint(y, V // 3, V)
    np.testing.assert_allclose(parts, full, rtol=1e-12, atol=1e-12)


def test_normaliser_single_ray(oracle_lib):
    # Z = max_E (mu1 + mu2)(E) * max_y sum_x h(x, y); for one axis-aligned ray
    # through a 7-voxel row the row sum is 7 * dx.
    geo = _box_geo()
    import oracle
    E = 3
    I0 = np.array([[1.0, 2.0, 0.0], [0.0, 1.0, 1.0]])
    mu = np.array([[0.05, 0.03, 0.2], [0.01, 0.02, 0.04]])
    O = oracle.Oracle(geo, I0, mu)
    assert O.normaliser() == pytest.approx(max(0.06, 0.05, 0.24) * 7 * geo.dx, rel=1e-14)
    # a bin where both spectra are empty is ignored
    I0[:, 2] = 0.0
    assert oracle.Oracle(geo, I0, mu).normaliser() == pytest.approx(0.06 * 7 * geo.dx, rel=1e-14)
