"""ctypes binding of the FP64 CPU oracle (``deam_oracle.c``, ``mar_init_oracle.c``).

TEST INFRASTRUCTURE ONLY: the oracle is what the CUDA path is checked against.
Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It imports nothing from the CUDA path.

Arrays are numpy float64 (uint8 for masks, int64 for ray lists) in the layouts
documented in ``deam_oracle.c``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, f) for f in ("deam_oracle.c", "mar_init_oracle.c", "or_types.h")]
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


class Geometry(C.Structure):
    _fields_ = [("kind", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
                ("cx", C.c_double), ("cy", C.c_double), ("cz", C.c_double),
                ("sid", C.c_double), ("sdd", C.c_double),
                ("n_views", C.c_int), ("views_per_rotation", C.c_int),
                ("start_angle", C.c_double), ("feed", C.c_double), ("z_start", C.c_double),
                ("n_rows", C.c_int), ("row_pitch", C.c_double),
                ("n_channels", C.c_int), ("channel_pitch", C.c_double),
                ("channel_offset", C.c_double), ("row_offset", C.c_double)]


class Model(C.Structure):
    _fields_ = [("n_e", C.c_int), ("I0", C.POINTER(C.c_double)), ("mu", C.POINTER(C.c_double)),
                ("bowtie", C.POINTER(C.c_double))]


class MarParams(C.Structure):
    _fields_ = [("calib", C.c_double * 4), ("t_air", C.c_double), ("t_bone", C.c_double),
                ("soft_value", C.c_double), ("count_floor", C.c_double), ("eps", C.c_double),
                ("prior_spectrum", C.c_int), ("prior_smooth", C.c_int)]


class Tap(C.Structure):
    _fields_ = [("idx", C.c_long), ("w", C.c_double)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, no FMA contraction, no fast-math)."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= max(os.path.getmtime(f) for f in _SRCS)):
            return _LIB
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-o", tmp] + [f for f in _SRCS if f.endswith(".c")] + ["-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
        return _LIB


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        P = C.POINTER
        d, i, l = C.c_double, C.c_int, C.c_long
        pd, pu8, pi64 = P(C.c_double), P(C.c_uint8), P(C.c_int64)
        G, M = P(Geometry), P(Model)
        sig = {
            "or_max_taps": (i, [G]),
            "or_num_threads": (i, []),
            "or_set_threads": (None, [i]),
            "or_ray_taps": (i, [G, l, i, i, P(Tap)]),
            "or_forward": (None, [G, pd, pd, i, i]),
            "or_forward_rays": (None, [G, pd, pi64, l, pd]),
            "or_adjoint": (None, [G, pd, pd, i, i]),
            "or_expected": (None, [G, M, pd, pd, i, i]),
            "or_ray_model": (None, [G, M, pd, pd, pu8, pi64, l, pd, pd, pd, pd]),
            "or_objective": (d, [G, M, pd, pd, pu8]),
            "or_backprojected_sums": (d, [G, M, pd, pd, pu8, pd, pd, i, i]),
            "or_normaliser": (d, [G, M]),
            "or_metal_trace": (None, [G, pd, d, pd, pu8]),
            "or_iterate": (l, [G, M, pd, pd, pu8, i, pd, d, i, i, i]),
            "or_gradient": (None, [G, M, pd, pd, pu8, pd]),
            "or_phi": (d, [d, d]),
            "or_penalty": (d, [G, pd, d, d]),
            "or_iterate_reg": (l, [G, M, pd, pd, pu8, i, pd, pd, d, i, d, d]),
            "or_log_sinogram": (None, [G, M, pd, d, pd]),
            "or_complete_trace": (None, [G, pd, pd, pu8, i, d, pd]),
            "or_ramp_filter": (None, [G, pd, pd]),
            "or_fbp_backproject": (None, [G, pd, pd]),
            "or_fbp": (None, [G, pd, pd]),
            "or_fbp_backproject_at": (None, [G, pd, pi64, l, pd]),
            "or_prior": (None, [l, pd, d, d, d, pd]),
            "or_smooth_inplane": (None, [i, i, i, pd, i]),
            "or_decompose": (None, [l, pd, pd, pd, pd]),
            "or_mar_init": (None, [G, M, pd, pu8, P(MarParams), pd, pd, pd, pd, pd]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _p(a, ctype=C.c_double):
    return a.ctypes.data_as(C.POINTER(ctype))


def _f64(a):
    a = np.asarray(a)
    if hasattr(a, "numpy"):
        a = a.numpy()
    return np.ascontiguousarray(a, dtype=np.float64)


def _np(a):
    try:
        import torch
        if isinstance(a, torch.Tensor):
            return a.detach().cpu().numpy()
    except ImportError:  # pragma: no cover
        pass
    return np.asarray(a)


def geometry(geo) -> Geometry:
    """Oracle geometry struct from any object with the synth.Geometry fields."""
    return Geometry(geo.kind, geo.nx, geo.ny, geo.nz, geo.dx, geo.dy, geo.dz, geo.cx, geo.cy, geo.cz,
                    geo.sid, geo.sdd, geo.n_views, geo.views_per_rotation, geo.start_angle, geo.feed,
                    geo.z_start, geo.n_rows, geo.row_pitch, geo.n_channels, geo.channel_pitch,
                    geo.channel_offset, geo.row_offset)


class Oracle:
    """FP64 MAR-DEAM on the CPU for one scan geometry and spectral model."""

    def __init__(self, geo, I0, mu, bowtie=None):
        self.geo = geo
        self.g = geometry(geo)
        self.I0 = _f64(_np(I0))
        self.mu = _f64(_np(mu))
        assert self.I0.shape == self.mu.shape and self.I0.shape[0] == 2
        self.bowtie = None if bowtie is None else _f64(_np(bowtie))
        self.m = Model(self.I0.shape[1], _p(self.I0), _p(self.mu),
                       _p(self.bowtie) if self.bowtie is not None else C.POINTER(C.c_double)())
        self.L = lib()

    # shapes
    @property
    def img_shape(self):
        return (self.geo.nz, self.geo.ny, self.geo.nx, 2)

    @property
    def ray_shape(self):
        return (self.geo.n_views, self.geo.n_rows, self.geo.n_channels)

    def taps(self, v, r, k):
        n = self.L.or_max_taps(C.byref(self.g))
        T = (Tap * n)()
        nt = self.L.or_ray_taps(C.byref(self.g), v, r, k, T)
        return np.array([T[i].idx for i in range(nt)], dtype=np.int64), np.array([T[i].w for i in range(nt)])

    def forward(self, c, v0=0, v1=None):
        c = _f64(_np(c)).reshape(self.img_shape)
        v1 = self.geo.n_views if v1 is None else v1
        out = np.zeros(self.ray_shape + (2,))
        self.L.or_forward(C.byref(self.g), _p(c), _p(out), v0, v1)
        return out

    def forward_rays(self, c, rays):
        c = _f64(_np(c)).reshape(self.img_shape)
        rays = np.ascontiguousarray(_np(rays), dtype=np.int64)
        out = np.zeros((rays.size, 2))
        self.L.or_forward_rays(C.byref(self.g), _p(c), _p(rays, C.c_int64), rays.size, _p(out))
        return out

    def adjoint(self, y, v0=0, v1=None):
        y = _f64(_np(y)).reshape(self.ray_shape + (2,))
        v1 = self.geo.n_views if v1 is None else v1
        out = np.zeros(self.img_shape)
        self.L.or_adjoint(C.byref(self.g), _p(y), _p(out), v0, v1)
        return out

    def expected(self, l):
        l = _f64(_np(l)).reshape(self.ray_shape + (2,))
        out = np.zeros((2,) + self.ray_shape)
        self.L.or_expected(C.byref(self.g), C.byref(self.m), _p(l), _p(out), 0, self.geo.n_views)
        return out

    def _dm(self, d, mask):
        d = _f64(_np(d)).reshape((2,) + self.ray_shape)
        return d, self.mask_bits(mask)

    def mask_bits(self, mask):
        """Metal mask in the oracle's encoding (bit j: on the trace of spectrum j)
        from None (no metal), a [V,R,K] mask (nonzero: both spectra) or a
        per-spectrum [2,V,R,K] mask."""
        if mask is None:
            return np.zeros(self.ray_shape, dtype=np.uint8)
        m = _np(mask)
        if m.shape == (2,) + self.ray_shape:
            return np.ascontiguousarray((m[0] != 0) * 1 + (m[1] != 0) * 2, dtype=np.uint8)
        return np.ascontiguousarray((m.reshape(self.ray_shape) != 0) * 3, dtype=np.uint8)

    def ray_model(self, c, d, mask, rays):
        """Per-ray l [n,2], g [n,2], payload [n,4] = (B~1, B~2, B^1, B^2), f [n]."""
        c = _f64(_np(c)).reshape(self.img_shape)
        d, mask = self._dm(d, mask)
        rays = np.ascontiguousarray(_np(rays), dtype=np.int64)
        n = rays.size
        l, g, pay, f = np.zeros((n, 2)), np.zeros((n, 2)), np.zeros((n, 4)), np.zeros(n)
        self.L.or_ray_model(C.byref(self.g), C.byref(self.m), _p(c), _p(d), _p(mask, C.c_uint8),
                            _p(rays, C.c_int64), n, _p(l), _p(g), _p(pay), _p(f))
        return l, g, pay, f

    def objective(self, c, d, mask=None):
        c = _f64(_np(c)).reshape(self.img_shape)
        d, mask = self._dm(d, mask)
        return self.L.or_objective(C.byref(self.g), C.byref(self.m), _p(c), _p(d), _p(mask, C.c_uint8))

    def backprojected_sums(self, c, d, mask=None, v0=0, v1=None):
        """(b~, b^, F) with b~, b^ of shape [nz,ny,nx,2]."""
        c = _f64(_np(c)).reshape(self.img_shape)
        d, mask = self._dm(d, mask)
        v1 = self.geo.n_views if v1 is None else v1
        bt, bh = np.zeros(self.img_shape), np.zeros(self.img_shape)
        F = self.L.or_backprojected_sums(C.byref(self.g), C.byref(self.m), _p(c), _p(d),
                                         _p(mask, C.c_uint8), _p(bt), _p(bh), v0, v1)
        return bt, bh, F

    def normaliser(self):
        return self.L.or_normaliser(C.byref(self.g), C.byref(self.m))

    def metal_trace(self, M, t):
        M = _f64(_np(M)).reshape(self.img_shape[:3])
        T = np.zeros(self.ray_shape)
        mask = np.zeros(self.ray_shape, dtype=np.uint8)
        self.L.or_metal_trace(C.byref(self.g), _p(M), float(t), _p(T), _p(mask, C.c_uint8))
        return T, mask

    def iterate(self, c, d, mask=None, n_iter=1, Z=0.0, clamp_nonneg=False, v0=0, v1=None):
        """Returns (c_new, hist, skipped)."""
        c = _f64(_np(c)).reshape(self.img_shape).copy()
        d, mask = self._dm(d, mask)
        v1 = self.geo.n_views if v1 is None else v1
        hist = np.zeros(max(n_iter, 1))
        skipped = self.L.or_iterate(C.byref(self.g), C.byref(self.m), _p(c), _p(d), _p(mask, C.c_uint8),
                                    n_iter, _p(hist), float(Z), int(clamp_nonneg), v0, v1)
        return c, hist[:n_iter], skipped

    def penalty(self, c, lam, delta):
        """R(c) of Eqs. (6)-(7) (26 neighbours, w = 1/distance, convex phi reading)."""
        c = _f64(_np(c)).reshape(self.img_shape)
        return self.L.or_penalty(C.byref(self.g), _p(c), float(lam), float(delta))

    def iterate_reg(self, c, d, mask=None, n_iter=1, lam=0.0, delta=1.0, Z=0.0, clamp_nonneg=False):
        """Regularised MAR-DEAM: returns (c_new, hist_F, hist_R, skipped)."""
        c = _f64(_np(c)).reshape(self.img_shape).copy()
        d, mask = self._dm(d, mask)
        hF, hR = np.zeros(max(n_iter, 1)), np.zeros(max(n_iter, 1))
        sk = self.L.or_iterate_reg(C.byref(self.g), C.byref(self.m), _p(c), _p(d), _p(mask, C.c_uint8), n_iter,
                                   _p(hF), _p(hR), float(Z), int(clamp_nonneg), float(lam), float(delta))
        return c, hF[:n_iter], hR[:n_iter], sk

    def gradient(self, c, d, mask=None):
        c = _f64(_np(c)).reshape(self.img_shape)
        d, mask = self._dm(d, mask)
        out = np.zeros(self.img_shape)
        self.L.or_gradient(C.byref(self.g), C.byref(self.m), _p(c), _p(d), _p(mask, C.c_uint8), _p(out))
        return out

    # ---- MAR initialisation (Sec. 2.2, Eq. 4) ----
    def log_sinogram(self, d, floor_counts=1.0):
        d = _f64(_np(d)).reshape((2,) + self.ray_shape)
        out = np.zeros((2,) + self.ray_shape)
        self.L.or_log_sinogram(C.byref(self.g), C.byref(self.m), _p(d), float(floor_counts), _p(out))
        return out

    def complete_trace(self, p, mask, bit, prior_proj=None, eps=1e-3):
        """NMAR (prior_proj given) or LI (None) completion of one sinogram [V,R,K]
        across the rays with mask bit `bit` set (mask in the oracle's bit encoding)."""
        p = _f64(_np(p)).reshape(self.ray_shape)
        mk = np.ascontiguousarray(_np(mask).reshape(self.ray_shape), dtype=np.uint8)
        pr = None if prior_proj is None else _f64(_np(prior_proj)).reshape(self.ray_shape)
        out = np.zeros(self.ray_shape)
        self.L.or_complete_trace(C.byref(self.g), _p(p), _p(pr) if pr is not None else C.POINTER(C.c_double)(),
                                 _p(mk, C.c_uint8), int(bit), float(eps), _p(out))
        return out

    def ramp_filter(self, p):
        p = _f64(_np(p)).reshape(self.ray_shape)
        out = np.zeros(self.ray_shape)
        self.L.or_ramp_filter(C.byref(self.g), _p(p), _p(out))
        return out

    def fbp_backproject(self, q):
        q = _f64(_np(q)).reshape(self.ray_shape)
        out = np.zeros(self.img_shape[:3])
        self.L.or_fbp_backproject(C.byref(self.g), _p(q), _p(out))
        return out

    def fbp_backproject_at(self, q, voxels):
        """FBP backprojection of the filtered sinogram q [V,R,K] at the listed
        voxel indices (iz*ny*nx + iy*nx + ix) only."""
        q = _f64(_np(q)).reshape(self.ray_shape)
        vox = np.ascontiguousarray(_np(voxels), dtype=np.int64)
        out = np.zeros(vox.size)
        self.L.or_fbp_backproject_at(C.byref(self.g), _p(q), _p(vox, C.c_int64), vox.size, _p(out))
        return out

    def fbp(self, p):
        p = _f64(_np(p)).reshape(self.ray_shape)
        out = np.zeros(self.img_shape[:3])
        self.L.or_fbp(C.byref(self.g), _p(p), _p(out))
        return out

    def mar_init(self, d, mask, calib, t_air, t_bone, soft_value, count_floor=1.0, eps=1e-3,
                 prior_spectrum=1, prior=None, prior_smooth=1):
        """(c [nz,ny,nx,2], prior, mu_L, mu_H) of the MAR initialisation; `prior`
        (optional) replaces the thresholded prior image."""
        d, mk = self._dm(d, mask)
        P = MarParams((C.c_double * 4)(*[float(x) for x in np.asarray(calib).reshape(4)]), float(t_air),
                      float(t_bone), float(soft_value), float(count_floor), float(eps), int(prior_spectrum),
                      int(prior_smooth))
        shp = self.img_shape[:3]
        pin = None if prior is None else _f64(_np(prior)).reshape(shp)
        c = np.zeros(self.img_shape)
        po, mL, mH = np.zeros(shp), np.zeros(shp), np.zeros(shp)
        self.L.or_mar_init(C.byref(self.g), C.byref(self.m), _p(d), _p(mk, C.c_uint8), C.byref(P),
                           _p(pin) if pin is not None else C.POINTER(C.c_double)(), _p(c), _p(po), _p(mL), _p(mH))
        return c, po, mL, mH


def smooth_inplane(f, passes=1):
    """n passes of the in-plane [1,2,1]/4 x [1,2,1]/4 smoothing (edges replicated)
    of an image [nz, ny, nx]."""
    f = _f64(_np(f)).copy()
    nz, ny, nx = f.shape
    lib().or_smooth_inplane(nx, ny, nz, _p(f), int(passes))
    return f


def prior_image(f, t_air, t_bone, soft_value):
    """Thresholded prior of a single-energy FBP image f (Sec. 2.2)."""
    f = _f64(_np(f))
    out = np.zeros_like(f)
    lib().or_prior(f.size, _p(f), float(t_air), float(t_bone), float(soft_value), _p(out))
    return out


def decompose(mu_L, mu_H, calib):
    """Eq. (4) with constant calibrated weights calib = (mu~_1L, mu~_2L, mu~_1H, mu~_2H)."""
    mL, mH = _f64(_np(mu_L)), _f64(_np(mu_H))
    cal = np.ascontiguousarray(np.asarray(calib, dtype=np.float64).reshape(4))
    out = np.zeros(mL.shape + (2,))
    lib().or_decompose(mL.size, _p(mL), _p(mH), _p(cal), _p(out))
    return out


def phi(u, delta):
    """phi(u) = delta^2 (|u|/delta - log(1 + |u|/delta)) (the convex reading of Eq. 7)."""
    return lib().or_phi(float(u), float(delta))


def basis_images(c, coef):
    """out[e] = coef[e, 0] c_1 + coef[e, 1] c_2 (the VMI mu(x, E) = mu_1(E) c_1(x) +
    mu_2(E) c_2(x) of Sec. 3 when coef = (mu_1(E), mu_2(E))), float64."""
    c = _f64(_np(c))
    coef = np.asarray(coef, dtype=np.float64).reshape(-1, 2)
    return np.stack([a * c[..., 0] + b * c[..., 1] for a, b in coef])


def from_case(case) -> Oracle:
    return Oracle(case.geo, case.I0, case.mu, case.bowtie)
