"""Seeded synthetic CT inputs for MAR-DEAM: scanner geometry, spectra, attenuation
tables, phantoms, analytic (noisy) measurements, metal images and ray masks.

This module simulates the scanner and the object.  It holds none of the
reconstruction method's arithmetic: no Joseph projector, no spectral sums of the
forward model of Eq. (8) on a voxel grid, no I-divergence, no image update.
Both the FP64 CPU oracle and the CUDA path receive the arrays produced here,
so they always see identical inputs.

Measurements are generated from exact chord lengths through continuous
ellipsoids and finite elliptic cylinders (three materials: two basis materials
plus a metal that the two-basis model cannot represent), summed over energy and
sampled with Poisson (and, optionally, Gaussian electronic) noise.  Because the
data does not come from the voxel model, there is no inverse crime.

Geometry convention (third-generation helical CT, curved detector), shared by
every consumer as an interface, not as code:
  * view v: source angle beta_v = start_angle + 2*pi*v/views_per_rotation,
    source s_v = (sid*cos beta_v, sid*sin beta_v, z_start + feed*v/views_per_rotation);
  * channel k: fan angle gamma_k = (k - (K-1)/2 + channel_offset) * channel_pitch;
  * row r: height w_r = (r - (R-1)/2 + row_offset) * row_pitch (mm at the detector);
  * ray (v, r, k) runs from s_v along u = (sdd*d_k, w_r) with the in-plane unit
    vector d_k = -(cos(beta_v + gamma_k), sin(beta_v + gamma_k));
  * voxel (ix, iy, iz) has its centre at
    (cx + (ix-(nx-1)/2)*dx, cy + (iy-(ny-1)/2)*dy, cz + (iz-(nz-1)/2)*dz).
Image arrays are [nz][ny][nx] with the two basis components interleaved last;
ray arrays are [views][rows][channels].
"""
from __future__ import annotations

import dataclasses
import math
from dataclasses import dataclass, field

import numpy as np
import torch

FAN2D = 0
HELICAL = 1


@dataclass
class Geometry:
    kind: int
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float
    cx: float
    cy: float
    cz: float
    sid: float
    sdd: float
    n_views: int
    views_per_rotation: int
    start_angle: float
    feed: float          # table feed per rotation, mm
    z_start: float       # source z at view 0, mm
    n_rows: int
    row_pitch: float     # mm at the detector
    n_channels: int
    channel_pitch: float  # rad
    channel_offset: float = 0.0
    row_offset: float = 0.0

    @property
    def n_rays(self) -> int:
        return self.n_views * self.n_rows * self.n_channels

    @property
    def n_voxels(self) -> int:
        return self.nx * self.ny * self.nz

    def replace(self, **kw) -> "Geometry":
        return dataclasses.replace(self, **kw)


# ----------------------------------------------------------------------------
# Attenuation tables: a two-term parametric model (photoelectric ~ E^-3 plus
# Klein-Nishina Compton scattering).  NIST tables are not available offline, so
# each material is described by its photoelectric and Compton parts at 60 keV.
# ----------------------------------------------------------------------------
_E_REF = 60.0


def klein_nishina(E_keV: np.ndarray) -> np.ndarray:
    """Total Klein-Nishina cross-section per electron (units of 2*pi*r_e^2)."""
    k = np.asarray(E_keV, dtype=np.float64) / 510.998950
    l2k = np.log1p(2.0 * k)
    return ((1.0 + k) / k**2 * (2.0 * (1.0 + k) / (1.0 + 2.0 * k) - l2k / k)
            + l2k / (2.0 * k) - (1.0 + 3.0 * k) / (1.0 + 2.0 * k) ** 2)


# (photoelectric part, Compton part) of mu at 60 keV, in 1/mm
MATERIALS = {
    "polystyrene": (0.0008, 0.0188),   # basis 1
    "cacl2": (0.0170, 0.0230),         # basis 2 (CaCl2 solution)
    "aluminium": (0.0400, 0.0350),     # spectrum filter
    "titanium": (0.1700, 0.0550),
    "steel": (0.8400, 0.1100),
}


def attenuation(material: str, E_keV: np.ndarray) -> np.ndarray:
    """Linear attenuation mu(E) in 1/mm of a named material (float64)."""
    photo, compton = MATERIALS[material]
    E = np.asarray(E_keV, dtype=np.float64)
    return photo * (_E_REF / E) ** 3 + compton * klein_nishina(E) / klein_nishina(np.array([_E_REF]))[0]


def energy_grid(bin_keV: float, e_lo: float = 20.0, e_hi: float = 140.0) -> np.ndarray:
    """Centres of equal-width energy bins covering [e_lo, e_hi] keV."""
    n = int(round((e_hi - e_lo) / bin_keV))
    return e_lo + (np.arange(n) + 0.5) * bin_keV


def spectrum(E_keV: np.ndarray, kvp: float, al_mm: float, i0_total: float) -> np.ndarray:
    """Kramers bremsstrahlung (kVp - E) filtered by aluminium, normalised so the
    bins sum to i0_total counts per ray.  Bins above kVp are zero."""
    E = np.asarray(E_keV, dtype=np.float64)
    phi = np.clip(kvp - E, 0.0, None) * np.exp(-attenuation("aluminium", E) * al_mm)
    return phi * (i0_total / phi.sum())


# ----------------------------------------------------------------------------
# Phantom objects.  Each object adds a constant density vector over its region:
# (c1, c2) for the basis components and m for metal (a fraction of full density
# of the case's metal).  Overlaps add, so an insert is written as a difference
# from the surrounding material.
# ----------------------------------------------------------------------------
@dataclass
class Obj:
    kind: str                  # "ellipsoid" | "cylinder" (finite, axis along z)
    centre: tuple              # (x, y, z) mm
    axes: tuple                # semi-axes (a, b, c) mm; for a cylinder c = half length
    phi: float                 # rotation about z, rad
    c1: float = 0.0
    c2: float = 0.0
    metal: float = 0.0


def _ray_frame(o: Obj, px, py, pz, ux, uy, uz):
    """Express points/directions in the object's frame scaled to a unit shape."""
    cp, sp = math.cos(o.phi), math.sin(o.phi)
    X = px - o.centre[0]
    Y = py - o.centre[1]
    Z = pz - o.centre[2]
    xr = (cp * X + sp * Y) / o.axes[0]
    yr = (-sp * X + cp * Y) / o.axes[1]
    zr = Z / o.axes[2]
    vx = (cp * ux + sp * uy) / o.axes[0]
    vy = (-sp * ux + cp * uy) / o.axes[1]
    vz = uz / o.axes[2]
    return xr, yr, zr, vx, vy, vz


def chord(o: Obj, px, py, pz, ux, uy, uz):
    """Length (in units of |u|, i.e. a parameter interval) of the line p + t*u
    inside the object.  Multiply by |u| for mm."""
    xr, yr, zr, vx, vy, vz = _ray_frame(o, px, py, pz, ux, uy, uz)
    if o.kind == "ellipsoid":
        A = vx * vx + vy * vy + vz * vz
        B = 2.0 * (xr * vx + yr * vy + zr * vz)
        C = xr * xr + yr * yr + zr * zr - 1.0
        disc = B * B - 4.0 * A * C
        return torch.sqrt(torch.clamp(disc, min=0.0)) / A
    # finite elliptic cylinder: |(xr, yr)| <= 1 and |zr| <= 1
    A = vx * vx + vy * vy
    B = 2.0 * (xr * vx + yr * vy)
    C = xr * xr + yr * yr - 1.0
    disc = B * B - 4.0 * A * C
    sq = torch.sqrt(torch.clamp(disc, min=0.0))
    Asafe = torch.where(A > 0, A, torch.ones_like(A))
    t0 = (-B - sq) / (2.0 * Asafe)
    t1 = (-B + sq) / (2.0 * Asafe)
    inside_axial = (C <= 0)   # ray parallel to the axis: inside iff start point inside
    big = 1e30
    t0 = torch.where(A > 0, t0, torch.where(inside_axial, torch.full_like(t0, -big), torch.full_like(t0, big)))
    t1 = torch.where(A > 0, t1, torch.where(inside_axial, torch.full_like(t1, big), torch.full_like(t1, -big)))
    miss = (A > 0) & (disc <= 0)
    t0 = torch.where(miss, torch.full_like(t0, big), t0)
    t1 = torch.where(miss, torch.full_like(t1, -big), t1)
    vz_safe = torch.where(vz != 0, vz, torch.ones_like(vz))
    za = (-1.0 - zr) / vz_safe
    zb = (1.0 - zr) / vz_safe
    zlo = torch.where(vz != 0, torch.minimum(za, zb),
                      torch.where(zr.abs() <= 1.0, torch.full_like(za, -big), torch.full_like(za, big)))
    zhi = torch.where(vz != 0, torch.maximum(za, zb),
                      torch.where(zr.abs() <= 1.0, torch.full_like(za, big), torch.full_like(za, -big)))
    lo = torch.maximum(t0, zlo)
    hi = torch.minimum(t1, zhi)
    return torch.clamp(hi - lo, min=0.0)


def inside(o: Obj, x, y, z):
    """Indicator of points inside the object."""
    zero = torch.zeros_like(x)
    xr, yr, zr, _, _, _ = _ray_frame(o, x, y, z, zero, zero, zero)
    if o.kind == "ellipsoid":
        return (xr * xr + yr * yr + zr * zr <= 1.0)
    return (xr * xr + yr * yr <= 1.0) & (zr.abs() <= 1.0)


# ----------------------------------------------------------------------------
# Scanner rays (float64, any device)
# ----------------------------------------------------------------------------
def ray_endpoints(geo: Geometry, views: torch.Tensor, device=None):
    """Source positions [V,3] and ray vectors u [V,R,K,3] for the given views."""
    dev = device if device is not None else views.device
    v = views.to(dev, torch.float64)
    beta = geo.start_angle + 2.0 * math.pi * v / geo.views_per_rotation
    s = torch.stack([geo.sid * torch.cos(beta), geo.sid * torch.sin(beta),
                     geo.z_start + geo.feed * v / geo.views_per_rotation], dim=-1)
    k = torch.arange(geo.n_channels, device=dev, dtype=torch.float64)
    gam = (k - (geo.n_channels - 1) / 2.0 + geo.channel_offset) * geo.channel_pitch
    r = torch.arange(geo.n_rows, device=dev, dtype=torch.float64)
    w = (r - (geo.n_rows - 1) / 2.0 + geo.row_offset) * geo.row_pitch
    ang = beta[:, None] + gam[None, :]                      # [V,K]
    ux = (-geo.sdd * torch.cos(ang))[:, None, :].expand(-1, geo.n_rows, -1)
    uy = (-geo.sdd * torch.sin(ang))[:, None, :].expand(-1, geo.n_rows, -1)
    uz = w[None, :, None].expand(v.numel(), -1, geo.n_channels)
    return s, torch.stack([ux, uy, uz], dim=-1)


def voxel_centres(geo: Geometry, device="cpu"):
    x = geo.cx + (torch.arange(geo.nx, dtype=torch.float64, device=device) - (geo.nx - 1) / 2.0) * geo.dx
    y = geo.cy + (torch.arange(geo.ny, dtype=torch.float64, device=device) - (geo.ny - 1) / 2.0) * geo.dy
    z = geo.cz + (torch.arange(geo.nz, dtype=torch.float64, device=device) - (geo.nz - 1) / 2.0) * geo.dz
    return x, y, z


# ----------------------------------------------------------------------------
# Cases
# ----------------------------------------------------------------------------
@dataclass
class Case:
    name: str
    geo: Geometry
    energies: np.ndarray          # [nE] keV
    I0: np.ndarray                # [2][nE] counts per ray per bin (L = 0, H = 1)
    mu: np.ndarray                # [2][nE] 1/mm, basis materials
    mu_metal: np.ndarray          # [nE] 1/mm, the case's metal
    objects: list
    i0_total: tuple
    noise_sigma: float = 0.0
    n_iter: int = 10
    bowtie: np.ndarray | None = None
    extra: dict = field(default_factory=dict)

    @property
    def metal_threshold(self) -> float:
        """Default metal-trace threshold: half the smallest voxel edge (mm of metal)."""
        g = self.geo
        return 0.5 * min(g.dx, g.dy, g.dz if g.nz > 1 else g.dx)


def fan_pitch(r_fov: float, sid: float, n_channels: int) -> float:
    """Channel pitch (rad) whose fan covers a field of view of radius r_fov."""
    return 2.0 * math.asin(r_fov / sid) * 1.02 / n_channels


def _spectra(bin_keV, i0):
    E = energy_grid(bin_keV)
    I0 = np.stack([spectrum(E, 90.0, 2.5, i0), spectrum(E, 140.0, 6.0, i0)])
    mu = np.stack([attenuation("polystyrene", E), attenuation("cacl2", E)])
    return E, I0, mu


def _body(rng, a, b, half_len, n_inserts, r_lo, r_hi, z_span, metal_objs, ellipsoids=True):
    objs = [Obj("cylinder", (0.0, 0.0, 0.0), (a, b, half_len), 0.0, c1=1.0, c2=0.02)]
    mats = [(-0.08, 0.00), (-0.1, 0.45), (-0.3, 0.30), (-0.5, 0.55), (-0.05, 0.15), (0.02, 0.08)]
    placed = []
    tries = 0
    while len(placed) < n_inserts and tries < 1000:
        tries += 1
        r = rng.uniform(r_lo, r_hi)
        x = rng.uniform(-a + r + 5, a - r - 5)
        y = rng.uniform(-b + r + 5, b - r - 5)
        if (x / (a - r - 5)) ** 2 + (y / (b - r - 5)) ** 2 > 1.0:
            continue
        if any(math.hypot(x - px, y - py) < r + pr + 3 for px, py, pr in placed):
            continue
        if any(math.hypot(x - m.centre[0], y - m.centre[1]) < r + m.axes[0] + 4 for m in metal_objs):
            continue
        placed.append((x, y, r))
        d1, d2 = mats[len(placed) % len(mats)]
        if ellipsoids:
            zc = rng.uniform(-z_span, z_span)
            objs.append(Obj("ellipsoid", (x, y, zc), (r, r * rng.uniform(0.7, 1.0), rng.uniform(0.8, 2.0) * r),
                            rng.uniform(0, math.pi), c1=d1, c2=d2))
        else:
            objs.append(Obj("cylinder", (x, y, 0.0), (r, r * rng.uniform(0.7, 1.0), half_len),
                            rng.uniform(0, math.pi), c1=d1, c2=d2))
    for m in metal_objs:   # metal displaces tissue
        objs.append(dataclasses.replace(m, c1=-1.0, c2=-0.02, metal=0.0))
        objs.append(m)
    return objs


def make_case(name: str, seed: int = 0) -> Case:
    """Seeded case description (cheap; no rays are generated here).

    c0:   2D fan-beam slice, 128x128 pixels of 250/128 mm, 360 views x 256 channels,
          SID 570 / SDD 1040 mm, 90 and 140 kVp at 1 keV bins, I0 = 1e5, 6 mm Ti disk.
    c1:   3D helical 256x256x32 (0.98 x 0.98 x 1.5 mm), 16 x 672 curved detector,
          1160 views/rotation, pitch 0.5, 3 rotations, 2 keV bins, I0 = 2e5, Ti rod.
    c2:   3D helical 512x512x64 (0.98 x 0.98 x 0.75 mm), 16 x 816, 1160 views/rotation,
          pitch 0.6, 5 rotations, 1 keV bins, I0 = 1e5 + sigma 5 electronic noise,
          bilateral stainless-steel hip inserts.
    c2s:  c2 cut to one rotation (1160 views): a profiling-sized case of the same kernels.
    t2d / t3d: small cases of the same kinds for oracle parity (ragged sizes).
    """
    rng = np.random.default_rng(seed)
    if name in ("c0", "t2d"):
        n, K, V = (128, 256, 360) if name == "c0" else (50, 70, 64)
        fov = 250.0 if name == "c0" else 240.0
        dx = fov / n
        geo = Geometry(FAN2D, n, n, 1, dx, dx, 1.0, 0.0, 0.0, 0.0, 570.0, 1040.0,
                       V, V, 0.1, 0.0, 0.0, 1, 1.0, K,
                       fan_pitch(fov / 2.0, 570.0, K), 0.25, 0.0)
        E, I0, mu = _spectra(1.0, 1e5)
        ti = Obj("cylinder", (35.0, -20.0, 0.0), (3.0, 3.0, 1e3), 0.0, metal=1.0)
        objs = _body(rng, 105.0, 80.0, 1e3, 5, 6.0, 16.0, 0.0, [ti], ellipsoids=False)
        return Case(name, geo, E, I0, mu, attenuation("titanium", E), objs, (1e5, 1e5), 0.0, 10)
    if name in ("c1", "t3d"):
        if name == "c1":
            nx, ny, nz, dz, R, K, vpr, rot = 256, 256, 32, 1.5, 16, 672, 1160, 3
            dx = 0.98
        else:
            nx, ny, nz, dz, R, K, vpr, rot = 46, 40, 11, 3.0, 6, 64, 96, 2.5
            dx = 5.2
        row_iso = 0.75 if name == "c1" else 2.4
        fov = nx * dx
        pitch = 0.5
        feed = pitch * R * row_iso
        V = int(round(vpr * rot))
        travel = feed * V / vpr
        geo = Geometry(HELICAL, nx, ny, nz, dx, dx, dz, 0.0, 0.0, 0.0, 570.0, 1040.0,
                       V, vpr, 0.3, feed, -travel / 2.0, R, row_iso * 1040.0 / 570.0, K,
                       fan_pitch(fov / 2.0, 570.0, K), 0.25, 0.0)
        E, I0, mu = _spectra(2.0 if name == "c1" else 4.0, 2e5)
        ti = Obj("cylinder", (30.0, 25.0, 0.0), (4.0, 4.0, 1e3), 0.0, metal=1.0)
        zs = nz * dz / 2.0
        a, b = 0.85 * fov / 2.0, 0.65 * fov / 2.0
        objs = _body(rng, a, b, 1e3, 6, 0.05 * fov, 0.12 * fov, zs * 0.6, [ti], ellipsoids=True)
        return Case(name, geo, E, I0, mu, attenuation("titanium", E), objs, (2e5, 2e5), 0.0, 20)
    if name in ("c2", "c2s"):
        # c2s: the same scan cut to one rotation (profiling-sized)
        nx, ny, nz, dz, R, K, vpr, rot = 512, 512, 64, 0.75, 16, 816, 1160, 5 if name == "c2" else 1
        dx = 0.98
        row_iso = 0.75
        fov = nx * dx
        feed = 0.6 * R * row_iso
        V = vpr * rot
        travel = feed * V / vpr
        geo = Geometry(HELICAL, nx, ny, nz, dx, dx, dz, 0.0, 0.0, 0.0, 570.0, 1040.0,
                       V, vpr, 0.3, feed, -travel / 2.0, R, row_iso * 1040.0 / 570.0, K,
                       fan_pitch(fov / 2.0, 570.0, K), 0.25, 0.0)
        E, I0, mu = _spectra(1.0, 1e5)
        hips = [Obj("ellipsoid", (-85.0, 5.0, 4.0), (14.0, 14.0, 14.0), 0.0, metal=1.0),
                Obj("ellipsoid", (85.0, 5.0, -2.0), (14.0, 14.0, 14.0), 0.0, metal=1.0),
                Obj("cylinder", (-95.0, -8.0, 0.0), (6.0, 8.0, 60.0), 0.4, metal=1.0),
                Obj("cylinder", (95.0, -8.0, 0.0), (6.0, 8.0, 60.0), -0.4, metal=1.0)]
        a, b = 200.0, 140.0
        objs = _body(rng, a, b, 1e3, 8, 10.0, 28.0, 12.0, hips, ellipsoids=True)
        return Case(name, geo, E, I0, mu, attenuation("steel", E), objs, (1e5, 1e5), 5.0, 50)
    raise ValueError(f"unknown case {name!r}")


def make_batch_cases(n: int = 24, seed: int = 7, small: bool = False) -> list:
    """Seeded scans of uneven size for batched reconstruction: half 2D fan slices
    (128^2 to 512^2 pixels), half 3D helical slabs (256^2 x 16 to 512^2 x 48
    voxels, 16 rows), 180 to 1160 views per rotation, 1 to 3 titanium or steel
    inserts each.  small=True scales every scan down (for parity tests)."""
    rng = np.random.default_rng(seed)
    cases = []
    for i in range(n):
        metal_name = "titanium" if rng.random() < 0.5 else "steel"
        if i % 2 == 0:   # 2D slice
            npx = int(rng.choice([128, 192, 256, 320, 384, 448, 512]))
            V = int(rng.integers(180, 1161))
            if small:
                npx, V = max(24, npx // 8), max(24, V // 12)
            fov = float(rng.uniform(240.0, 320.0))
            dx = fov / npx
            K = int(8 * round(1.6 * npx / 8))
            geo = Geometry(FAN2D, npx, npx, 1, dx, dx, 1.0, 0.0, 0.0, 0.0, 570.0, 1040.0,
                           V, V, float(rng.uniform(0, 6.28)), 0.0, 0.0, 1, 1.0, K,
                           fan_pitch(fov / 2.0, 570.0, K), 0.25, 0.0)
            E, I0, mu = _spectra(2.0, 1e5)
            half_len = 1e3
        else:            # 3D helical slab
            npx = int(rng.choice([256, 384, 512]))
            nz = int(rng.choice([16, 32, 48]))
            vpr = int(rng.integers(180, 1161))
            R, row_iso, dxy, dz = 16, 0.75, 0.98, float(rng.choice([0.75, 1.0, 1.5]))
            if small:
                npx, nz, vpr, R, dxy = max(24, npx // 8), max(6, nz // 4), max(24, vpr // 12), 4, 0.98 * 8
                row_iso = 0.75 * 4
            fov = npx * dxy
            K = int(8 * round((816 if not small else 56) / 8))
            feed = 0.8 * R * row_iso
            rot = max(1, int(math.ceil(nz * dz / feed)))
            V = vpr * rot
            travel = feed * V / vpr
            geo = Geometry(HELICAL, npx, npx, nz, dxy, dxy, dz, 0.0, 0.0, 0.0, 570.0, 1040.0,
                           V, vpr, float(rng.uniform(0, 6.28)), feed, -travel / 2.0, R,
                           row_iso * 1040.0 / 570.0, K, fan_pitch(fov / 2.0, 570.0, K), 0.25, 0.0)
            E, I0, mu = _spectra(2.0, 1e5)
            half_len = nz * dz
        a, b = 0.42 * geo.nx * geo.dx, 0.32 * geo.ny * geo.dy
        metals = []
        for m in range(int(rng.integers(1, 4))):
            for _ in range(100):
                x, y = rng.uniform(-0.6 * a, 0.6 * a), rng.uniform(-0.6 * b, 0.6 * b)
                rr = float(rng.uniform(2.0, 6.0))
                if all(math.hypot(x - o.centre[0], y - o.centre[1]) > rr + o.axes[0] + 3 for o in metals):
                    metals.append(Obj("cylinder", (x, y, 0.0), (rr, rr, half_len), 0.0, metal=1.0))
                    break
        objs = _body(rng, a, b, half_len, 4, 0.06 * a, 0.15 * a, 0.3 * half_len if geo.nz > 1 else 0.0,
                     metals, ellipsoids=geo.nz > 1)
        cases.append(Case(f"batch{i}", geo, E, I0, mu, attenuation(metal_name, E), objs, (1e5, 1e5), 0.0, 10))
    return cases


# ----------------------------------------------------------------------------
# Measurements
# ----------------------------------------------------------------------------
def _chords(case: Case, views: torch.Tensor, device):
    """Basis and metal path integrals (mm) for every ray of the given views."""
    geo = case.geo
    s, u = ray_endpoints(geo, views, device)
    ux, uy, uz = u[..., 0], u[..., 1], u[..., 2]
    px = s[:, 0][:, None, None].expand_as(ux)
    py = s[:, 1][:, None, None].expand_as(ux)
    pz = s[:, 2][:, None, None].expand_as(ux)
    un = torch.sqrt(ux * ux + uy * uy + uz * uz)
    l1 = torch.zeros_like(ux)
    l2 = torch.zeros_like(ux)
    lm = torch.zeros_like(ux)
    for o in case.objects:
        L = chord(o, px, py, pz, ux, uy, uz) * un
        if o.c1:
            l1 += o.c1 * L
        if o.c2:
            l2 += o.c2 * L
        if o.metal:
            lm += o.metal * L
    return l1, l2, lm


def measure(case: Case, device="cpu", seed: int = 1, noiseless: bool = False,
            views_per_chunk: int = 256, dtype=torch.float32):
    """Simulated counts d [2][V][R][K] (float32) and the analytic metal path
    length [V][R][K] (float32, mm).  Chunked over views to bound memory."""
    geo = case.geo
    dev = torch.device(device)
    d = torch.empty((2, geo.n_views, geo.n_rows, geo.n_channels), dtype=dtype, device=dev)
    metal = torch.empty((geo.n_views, geo.n_rows, geo.n_channels), dtype=torch.float32, device=dev)
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    bow = None
    if case.bowtie is not None:
        bow = torch.as_tensor(case.bowtie, dtype=torch.float64, device=dev)
    wdt = torch.float64 if dev.type == "cpu" else torch.float32
    mu = torch.as_tensor(case.mu, dtype=wdt, device=dev)
    mum = torch.as_tensor(case.mu_metal, dtype=wdt, device=dev)
    I0 = torch.as_tensor(case.I0, dtype=wdt, device=dev)
    for v0 in range(0, geo.n_views, views_per_chunk):
        v1 = min(geo.n_views, v0 + views_per_chunk)
        views = torch.arange(v0, v1, device=dev)
        l1, l2, lm = _chords(case, views, dev)
        metal[v0:v1] = lm.to(torch.float32)
        l1, l2, lm = l1.to(wdt), l2.to(wdt), lm.to(wdt)
        for j in range(2):
            g = torch.zeros_like(l1)
            for e in range(len(case.energies)):
                if case.I0[j, e] <= 0:
                    continue
                g += I0[j, e] * torch.exp(-(mu[0, e] * l1 + mu[1, e] * l2 + mum[e] * lm))
            if bow is not None:
                g = g * bow.to(wdt)[None, None, :]
            if noiseless:
                dj = g
            else:
                dj = torch.poisson(g, generator=gen)
                if case.noise_sigma > 0:
                    dj = dj + case.noise_sigma * torch.randn(dj.shape, generator=gen, device=dev, dtype=dj.dtype)
            d[j, v0:v1] = dj.to(dtype)
    return d, metal


def voxelize(case: Case, device="cpu", ss: int = 2, z_chunk: int = 8):
    """Supersampled truth (c1, c2) image [nz][ny][nx][2] (float32) and the metal
    image M [nz][ny][nx] (float32, fraction of each voxel that is metal)."""
    geo = case.geo
    dev = torch.device(device)
    x, y, z = voxel_centres(geo, dev)
    offs = (torch.arange(ss, dtype=torch.float64, device=dev) + 0.5) / ss - 0.5
    c = torch.zeros((geo.nz, geo.ny, geo.nx, 2), dtype=torch.float32, device=dev)
    M = torch.zeros((geo.nz, geo.ny, geo.nx), dtype=torch.float32, device=dev)
    ssz = ss if geo.nz > 1 else 1
    offz = offs if geo.nz > 1 else torch.zeros(1, dtype=torch.float64, device=dev)
    for z0 in range(0, geo.nz, z_chunk):
        z1 = min(geo.nz, z0 + z_chunk)
        acc = torch.zeros((z1 - z0, geo.ny, geo.nx, 3), dtype=torch.float64, device=dev)
        for oz in offz:
            for oy in offs:
                for ox in offs:
                    Z = (z[z0:z1] + oz * geo.dz)[:, None, None].expand(-1, geo.ny, geo.nx)
                    Y = (y + oy * geo.dy)[None, :, None].expand(z1 - z0, -1, geo.nx)
                    X = (x + ox * geo.dx)[None, None, :].expand(z1 - z0, geo.ny, -1)
                    for o in case.objects:
                        ins = inside(o, X, Y, Z).to(torch.float64)
                        if o.c1:
                            acc[..., 0] += o.c1 * ins
                        if o.c2:
                            acc[..., 1] += o.c2 * ins
                        if o.metal:
                            acc[..., 2] += o.metal * ins
        acc /= ss * ss * ssz
        c[z0:z1] = acc[..., :2].to(torch.float32)
        M[z0:z1] = acc[..., 2].to(torch.float32)
    return c, M


def initial_image(case: Case, truth: torch.Tensor, seed: int = 2) -> torch.Tensor:
    """A seeded starting image c^0: the body support filled with the soft-tissue
    basis vector, lightly perturbed.  (The paper initialises with NMAR + FBP +
    image-domain decomposition; here c^0 is simply an input.)"""
    gen = torch.Generator(device="cpu")
    gen.manual_seed(seed)
    support = (truth[..., 0] > 0.3).to(torch.float32).cpu()
    c0 = torch.zeros_like(truth, device="cpu")
    c0[..., 0] = 0.95 * support
    c0[..., 1] = 0.05 * support
    c0 += 0.01 * support[..., None] * torch.rand(c0.shape, generator=gen)
    return c0.to(truth.device)


def random_image(geo: Geometry, seed: int, device="cpu") -> torch.Tensor:
    gen = torch.Generator(device="cpu")
    gen.manual_seed(seed)
    return torch.rand((geo.nz, geo.ny, geo.nx, 2), generator=gen, dtype=torch.float64).to(device)


def random_rays(geo: Geometry, seed: int, device="cpu") -> torch.Tensor:
    gen = torch.Generator(device="cpu")
    gen.manual_seed(seed)
    return torch.rand((geo.n_views, geo.n_rows, geo.n_channels, 2), generator=gen,
                      dtype=torch.float64).to(device)
