"""GB300 (sm_103a) MAR-DEAM: Python binding of libdeam.so.

Argument marshalling only: every step of the reconstruction runs in the CUDA
kernels behind the C ABI declared in ``include/deam.h``.  PyTorch provides device
memory and streams.  The binding refuses to run without the compiled library
(there is no CPU fallback); build it with ``paper_2202_00116_gb300.build.build()``.

Method: MAR-DEAM of Ge et al., "A Metal Artifact Reduction Scheme For Accurate
Iterative Dual-Energy CT Algorithms" (arXiv 2202.00116), Sec. 2.3: DEAM
iterations on the I-divergence of Eq. (5) with the polyenergetic model of Eq. (8)
and the metal-trace substitution of Eqs. (2)-(3) and (11).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# DEAM_LIB_PATH selects another build of the same library (the bounds-checked
# libdeam_checked.so); the default is the in-tree libdeam.so
LIB_PATH = os.environ.get("DEAM_LIB_PATH") or os.path.join(_HERE, "libdeam.so")

DEAM_OK, DEAM_ERR_ARG, DEAM_ERR_CUDA, DEAM_ERR_OOM, DEAM_ERR_STATE, DEAM_ERR_TIMEOUT, DEAM_ERR_NUMERIC = range(7)
FAN2D, HELICAL = 0, 1
MASK_VOXEL_IMAGE, MASK_RAY, MASK_RAY_PER_SPECTRUM = 0, 1, 2


class deam_geometry(C.Structure):
    _fields_ = [("kind", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
                ("cx", C.c_double), ("cy", C.c_double), ("cz", C.c_double),
                ("sid", C.c_double), ("sdd", C.c_double),
                ("n_views", C.c_int), ("views_per_rotation", C.c_int),
                ("start_angle", C.c_double), ("feed", C.c_double), ("z_start", C.c_double),
                ("n_rows", C.c_int), ("row_pitch", C.c_double),
                ("n_channels", C.c_int), ("channel_pitch", C.c_double),
                ("channel_offset", C.c_double), ("row_offset", C.c_double)]


class deam_spectra(C.Structure):
    _fields_ = [("n_e", C.c_int), ("energy_keV", C.POINTER(C.c_double)), ("I0", C.POINTER(C.c_double)),
                ("bowtie", C.POINTER(C.c_double))]


class deam_basis(C.Structure):
    _fields_ = [("n_e", C.c_int), ("mu", C.POINTER(C.c_double))]


class deam_options(C.Structure):
    _fields_ = [("metal_threshold", C.c_double), ("Z", C.c_double), ("penalty_lambda", C.c_double),
                ("penalty_delta", C.c_double), ("clamp_nonneg", C.c_int), ("precision", C.c_int),
                ("reserved", C.c_int * 6)]


class deam_mar_params(C.Structure):
    _fields_ = [("calib", C.c_double * 4), ("t_air", C.c_double), ("t_bone", C.c_double),
                ("soft_value", C.c_double), ("count_floor", C.c_double), ("eps", C.c_double),
                ("prior_spectrum", C.c_int), ("prior_smooth", C.c_int), ("reserved", C.c_int * 6)]


class DeamError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"deam error {code}: {msg}")
        self.code = code


_lib = None
EXPORTS = ["deam_init", "deam_set_data", "deam_set_metal_mask", "deam_get_metal_mask", "deam_forward",
           "deam_backproject", "deam_ray_terms", "deam_iterate", "deam_objective", "deam_info",
           "deam_gradient", "deam_backprojected_sums", "deam_penalty", "deam_basis_images", "deam_vmi",
           "deam_kvp_images", "deam_count_samples",
           "deam_profile", "deam_kernel_times", "deam_l1_bandwidth", "deam_bounds_checked", "deam_bounds_inject", "deam_log_sinogram", "deam_complete_trace", "deam_fbp",
           "deam_mar_init", "deam_batch_create",
           "deam_batch_iterate", "deam_batch_info", "deam_batch_destroy", "deam_objective_noalloc",
           "deam_destroy", "deam_last_error"]


def lib():
    """Load libdeam.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2202_00116_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        vp, i, pd = C.c_void_p, C.c_int, C.POINTER(C.c_double)
        sig = {
            "deam_init": [C.POINTER(deam_geometry), C.POINTER(deam_spectra), C.POINTER(deam_basis),
                          C.POINTER(deam_options), C.POINTER(vp)],
            "deam_set_data": [vp, vp, vp],
            "deam_set_metal_mask": [vp, vp, i, vp],
            "deam_get_metal_mask": [vp, vp, vp],
            "deam_forward": [vp, vp, vp, vp, vp],
            "deam_backproject": [vp, vp, vp, vp],
            "deam_ray_terms": [vp, vp, vp, pd, vp],
            "deam_iterate": [vp, vp, i, pd, vp],
            "deam_objective": [vp, vp, pd, vp],
            "deam_info": [vp, pd, C.POINTER(C.c_longlong)],
            "deam_gradient": [vp, vp, vp, pd, vp],
            "deam_backprojected_sums": [vp, vp, vp, pd, pd, vp],
            "deam_basis_images": [vp, vp, pd, i, vp, vp],
            "deam_vmi": [vp, vp, pd, i, vp, vp],
            "deam_kvp_images": [vp, vp, vp, vp],
            "deam_penalty": [vp, vp, pd, vp],
            "deam_count_samples": [vp, C.POINTER(C.c_longlong), vp],
            "deam_profile": [vp, i],
            "deam_l1_bandwidth": [pd, vp],
            "deam_bounds_checked": [],
            "deam_bounds_inject": [vp, vp],
            "deam_kernel_times": [vp, pd, C.POINTER(C.c_longlong), i],
            "deam_log_sinogram": [vp, C.c_double, vp, vp],
            "deam_complete_trace": [vp, vp, vp, i, C.c_double, vp, vp],
            "deam_fbp": [vp, vp, i, vp, vp],
            "deam_mar_init": [vp, C.POINTER(deam_mar_params), vp, vp, vp, vp, vp],
            "deam_objective_noalloc": [C.POINTER(deam_geometry), C.POINTER(deam_spectra), C.POINTER(deam_basis),
                                       vp, vp, vp, vp, vp],
            "deam_batch_create": [C.POINTER(vp), i, i, C.POINTER(vp)],
            "deam_batch_iterate": [vp, C.POINTER(vp), i, pd, vp],
            "deam_batch_info": [vp, C.POINTER(C.c_int), C.POINTER(C.c_float), C.POINTER(C.c_int),
                                C.POINTER(C.c_int), C.POINTER(C.c_float), C.POINTER(C.c_float)],
            "deam_batch_destroy": [vp],
            "deam_destroy": [vp],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_int
        L.deam_last_error.argtypes = []
        L.deam_last_error.restype = C.c_char_p
        _lib = L
    return _lib


def _check(rc):
    if rc != DEAM_OK:
        raise DeamError(rc, lib().deam_last_error().decode(errors="replace"))


class Deam:
    """One scan: geometry + spectra + basis tables on a CUDA device.

    Tensors are torch tensors: images float32 [nz, ny, nx, 2]; ray pairs float32
    [V, R, K, 2]; data float32 [2, V, R, K]; masks uint8 [V, R, K].
    """

    def __init__(self, geo, I0, mu, bowtie=None, energies=None, metal_threshold=0.0, Z=0.0,
                 clamp_nonneg=False, penalty_lambda=0.0, penalty_delta=1.0, precision="mixed", device=None):
        import torch
        self.torch = torch
        if device is None:
            device = torch.cuda.current_device() if torch.cuda.is_available() else 0
        self.device = torch.device("cuda", device)
        self.geo = geo
        self._g = deam_geometry(int(geo.kind), geo.nx, geo.ny, geo.nz, geo.dx, geo.dy, geo.dz, geo.cx, geo.cy,
                                geo.cz, geo.sid, geo.sdd, geo.n_views, geo.views_per_rotation, geo.start_angle,
                                geo.feed, geo.z_start, geo.n_rows, geo.row_pitch, geo.n_channels,
                                geo.channel_pitch, geo.channel_offset, geo.row_offset)
        self._I0 = np.ascontiguousarray(np.asarray(I0, dtype=np.float64))
        self._mu = np.ascontiguousarray(np.asarray(mu, dtype=np.float64))
        nE = self._I0.shape[1]
        P = C.POINTER(C.c_double)
        self._bow = None if bowtie is None else np.ascontiguousarray(np.asarray(bowtie, dtype=np.float64))
        self._E = None if energies is None else np.ascontiguousarray(np.asarray(energies, dtype=np.float64))
        sp = deam_spectra(nE, self._E.ctypes.data_as(P) if self._E is not None else P(),
                          self._I0.ctypes.data_as(P), self._bow.ctypes.data_as(P) if self._bow is not None else P())
        ba = deam_basis(self._mu.shape[1], self._mu.ctypes.data_as(P))
        if precision not in ("mixed", "fp32"):
            raise ValueError("precision is 'mixed' (compensated FP32 sums, FP64 objective) or 'fp32'")
        op = deam_options(float(metal_threshold), float(Z), float(penalty_lambda), float(penalty_delta),
                          int(bool(clamp_nonneg)), 1 if precision == "fp32" else 0)
        h = C.c_void_p()
        self._h = None
        if torch.cuda.is_available():
            with torch.cuda.device(self.device):
                _check(lib().deam_init(C.byref(self._g), C.byref(sp), C.byref(ba), C.byref(op), C.byref(h)))
        else:  # host-side validation still runs; without a device the call then fails
            _check(lib().deam_init(C.byref(self._g), C.byref(sp), C.byref(ba), C.byref(op), C.byref(h)))
        self._h = h

    # -- helpers --
    @property
    def ray_shape(self):
        return (self.geo.n_views, self.geo.n_rows, self.geo.n_channels)

    @property
    def img_shape(self):
        return (self.geo.nz, self.geo.ny, self.geo.nx, 2)

    def _stream(self):
        return C.c_void_p(self.torch.cuda.current_stream(self.device).cuda_stream)

    def _arg(self, t, shape, dtype, host_ok=False):
        torch = self.torch
        if not isinstance(t, torch.Tensor):
            raise TypeError("expected a torch tensor")
        if tuple(t.shape) != tuple(shape) or t.dtype != dtype or not t.is_contiguous():
            raise ValueError(f"expected contiguous {dtype} tensor of shape {tuple(shape)}, got "
                             f"{t.dtype} {tuple(t.shape)}")
        if t.is_cuda:
            if t.device != self.device:
                raise ValueError(f"tensor on {t.device}, context on {self.device}")
        elif not host_ok:
            raise ValueError("expected a CUDA tensor")
        return C.c_void_p(t.data_ptr())

    # -- API --
    def set_data(self, d):
        """Measured counts d [2, V, R, K] (CUDA or host tensor); stored as max(d, 0)."""
        _check(lib().deam_set_data(self._h, self._arg(d, (2,) + self.ray_shape, self.torch.float32, True),
                                   self._stream()))
        if not d.is_cuda:
            self.torch.cuda.current_stream(self.device).synchronize()

    def set_metal_mask(self, m, kind="ray"):
        """kind='ray': uint8 [V, R, K] (nonzero: both spectra); kind='per_spectrum':
        bool/uint8 [2, V, R, K] traces (T_L, T_H), packed into bits 0 and 1;
        kind='voxel': float32 metal image [nz, ny, nx]."""
        torch = self.torch
        if kind == "per_spectrum":
            if tuple(m.shape) != (2,) + self.ray_shape:
                raise ValueError(f"expected a mask of shape {(2,) + self.ray_shape}")
            m = ((m[0] != 0).to(torch.uint8) + 2 * (m[1] != 0).to(torch.uint8)).contiguous()
            p = self._arg(m, self.ray_shape, torch.uint8, True)
            k = MASK_RAY_PER_SPECTRUM
        elif kind == "ray":
            p = self._arg(m, self.ray_shape, torch.uint8, True)
            k = MASK_RAY
        else:
            p = self._arg(m, self.img_shape[:3], torch.float32, True)
            k = MASK_VOXEL_IMAGE
        _check(lib().deam_set_metal_mask(self._h, p, k, self._stream()))
        if not m.is_cuda:
            torch.cuda.current_stream(self.device).synchronize()

    def metal_mask(self):
        out = self.torch.empty(self.ray_shape, dtype=self.torch.uint8, device=self.device)
        _check(lib().deam_get_metal_mask(self._h, C.c_void_p(out.data_ptr()), self._stream()))
        return out

    def forward(self, c, want_l=True, want_g=False):
        """Line integrals l [V, R, K, 2] and/or expected counts g [2, V, R, K]."""
        torch = self.torch
        l = torch.empty(self.ray_shape + (2,), dtype=torch.float32, device=self.device) if want_l else None
        g = torch.empty((2,) + self.ray_shape, dtype=torch.float32, device=self.device) if want_g else None
        _check(lib().deam_forward(self._h, self._arg(c, self.img_shape, torch.float32),
                                  C.c_void_p(l.data_ptr()) if l is not None else None,
                                  C.c_void_p(g.data_ptr()) if g is not None else None, self._stream()))
        return l, g

    def backproject(self, y, out=None):
        torch = self.torch
        if out is None:
            out = torch.empty(self.img_shape, dtype=torch.float32, device=self.device)
        _check(lib().deam_backproject(self._h, self._arg(y, self.ray_shape + (2,), torch.float32),
                                      self._arg(out, self.img_shape, torch.float32), self._stream()))
        return out

    def ray_terms(self, c):
        """(payload [V, R, K, 4] = (B~1, B~2, D1, D2), F)."""
        torch = self.torch
        pay = torch.empty(self.ray_shape + (4,), dtype=torch.float32, device=self.device)
        F = C.c_double()
        _check(lib().deam_ray_terms(self._h, self._arg(c, self.img_shape, torch.float32),
                                    C.c_void_p(pay.data_ptr()), C.byref(F), self._stream()))
        return pay, F.value

    def iterate(self, c, n_iter):
        """n_iter MAR-DEAM iterations in place on c (CUDA or host tensor); returns
        the objective history F(c^k), k = 0..n_iter-1, as a numpy array."""
        hist = np.zeros(max(n_iter, 1), dtype=np.float64)
        _check(lib().deam_iterate(self._h, self._arg(c, self.img_shape, self.torch.float32, True), int(n_iter),
                                  hist.ctypes.data_as(C.POINTER(C.c_double)), self._stream()))
        return hist[:n_iter]

    def objective(self, c):
        F = C.c_double()
        _check(lib().deam_objective(self._h, self._arg(c, self.img_shape, self.torch.float32), C.byref(F),
                                    self._stream()))
        return F.value

    def gradient(self, c, out=None):
        """(dF/dc float32 [nz, ny, nx, 2], F(c)): the gradient of the objective,
        b^ - b~, from one recomputation of the per-ray terms and one gather
        backprojection."""
        torch = self.torch
        if out is None:
            out = torch.empty(self.img_shape, dtype=torch.float32, device=self.device)
        F = C.c_double()
        _check(lib().deam_gradient(self._h, self._arg(c, self.img_shape, torch.float32),
                                   self._arg(out, self.img_shape, torch.float32), C.byref(F), self._stream()))
        return out, F.value

    def backprojected_sums(self, c, out=None):
        """(sums float32 [nz, ny, nx, 4] = (b~1, b~2, delta1, delta2), F(c), Z):
        the c-step's backprojected sums at c without the update; delta = dF/dc."""
        torch = self.torch
        if out is None:
            out = torch.empty(self.img_shape[:3] + (4,), dtype=torch.float32, device=self.device)
        F, Z = C.c_double(), C.c_double()
        _check(lib().deam_backprojected_sums(self._h, self._arg(c, self.img_shape, torch.float32),
                                             self._arg(out, self.img_shape[:3] + (4,), torch.float32),
                                             C.byref(F), C.byref(Z), self._stream()))
        return out, F.value, Z.value

    def penalty(self, c):
        """R(c) of Eqs. (6)-(7) with the context's lambda and delta."""
        R = C.c_double()
        _check(lib().deam_penalty(self._h, self._arg(c, self.img_shape, self.torch.float32), C.byref(R),
                                  self._stream()))
        return R.value

    # -- MAR initialisation (Sec. 2.2, Eq. 4) --
    def log_sinogram(self, count_floor=1.0):
        """Line-integral sinograms p [2, V, R, K] = ln(I0_j / max(d~_j, count_floor))."""
        torch = self.torch
        p = torch.empty((2,) + self.ray_shape, dtype=torch.float32, device=self.device)
        _check(lib().deam_log_sinogram(self._h, float(count_floor), C.c_void_p(p.data_ptr()), self._stream()))
        return p

    def complete_trace(self, p, spectrum, prior_proj=None, eps=1e-3, out=None):
        """Trace completion of one sinogram [V, R, K] over spectrum's trace: NMAR
        with the prior's projection, else linear interpolation."""
        torch = self.torch
        if out is None:
            out = torch.empty(self.ray_shape, dtype=torch.float32, device=self.device)
        pp = C.c_void_p(None) if prior_proj is None else self._arg(prior_proj, self.ray_shape, torch.float32)
        _check(lib().deam_complete_trace(self._h, self._arg(p, self.ray_shape, torch.float32), pp, int(spectrum),
                                         float(eps), self._arg(out, self.ray_shape, torch.float32), self._stream()))
        return out

    def fbp(self, p):
        """FBP image(s) [n, nz, ny, nx] (1/mm) of line-integral sinogram(s) [n, V, R, K]
        or [V, R, K] (n = 1, 2)."""
        torch = self.torch
        single = p.dim() == 3
        pp = p.unsqueeze(0) if single else p
        n = pp.shape[0]
        img = torch.empty((n,) + self.img_shape[:3], dtype=torch.float32, device=self.device)
        _check(lib().deam_fbp(self._h, self._arg(pp.contiguous(), (n,) + self.ray_shape, torch.float32), n,
                              C.c_void_p(img.data_ptr()), self._stream()))
        return img[0] if single else img

    def mar_init(self, calib, t_air, t_bone, soft_value, count_floor=1.0, eps=1e-3, prior_spectrum=1,
                 prior=None, prior_smooth=1):
        """(c^0 [nz, ny, nx, 2], prior [nz, ny, nx], mu [2, nz, ny, nx]): NMAR-corrected
        FBP images of both spectra split by Eq. (4) with calib = (mu~_1L, mu~_2L,
        mu~_1H, mu~_2H); `prior` replaces the thresholded prior image."""
        torch = self.torch
        P = deam_mar_params((C.c_double * 4)(*[float(x) for x in np.asarray(calib, dtype=np.float64).reshape(4)]),
                            float(t_air), float(t_bone), float(soft_value), float(count_floor), float(eps),
                            int(prior_spectrum), int(prior_smooth))
        c = torch.empty(self.img_shape, dtype=torch.float32, device=self.device)
        pr = torch.empty(self.img_shape[:3], dtype=torch.float32, device=self.device)
        mu = torch.empty((2,) + self.img_shape[:3], dtype=torch.float32, device=self.device)
        pin = C.c_void_p(None) if prior is None else self._arg(prior, self.img_shape[:3], torch.float32)
        _check(lib().deam_mar_init(self._h, C.byref(P), pin, C.c_void_p(c.data_ptr()), C.c_void_p(pr.data_ptr()),
                                   C.c_void_p(mu.data_ptr()), self._stream()))
        return c, pr, mu

    def basis_images(self, c, coef):
        """out[e] = coef[e, 0] c_1 + coef[e, 1] c_2, float32 [n, nz, ny, nx]."""
        torch = self.torch
        coef = np.ascontiguousarray(np.asarray(coef, dtype=np.float64).reshape(-1, 2))
        out = torch.empty((coef.shape[0],) + self.img_shape[:3], dtype=torch.float32, device=self.device)
        _check(lib().deam_basis_images(self._h, self._arg(c, self.img_shape, torch.float32),
                                       coef.ctypes.data_as(C.POINTER(C.c_double)), coef.shape[0],
                                       C.c_void_p(out.data_ptr()), self._stream()))
        return out

    def vmi(self, c, energies_keV):
        """Virtual monoenergetic images mu(x, E) = mu_1(E) c_1 + mu_2(E) c_2 (1/mm) at the
        given energies (deam_vmi), float32 [n, nz, ny, nx]."""
        torch = self.torch
        E = np.ascontiguousarray(np.asarray(energies_keV, dtype=np.float64).reshape(-1))
        out = torch.empty((E.size,) + self.img_shape[:3], dtype=torch.float32, device=self.device)
        _check(lib().deam_vmi(self._h, self._arg(c, self.img_shape, torch.float32),
                              E.ctypes.data_as(C.POINTER(C.c_double)), int(E.size), C.c_void_p(out.data_ptr()),
                              self._stream()))
        return out

    def kvp_images(self, c):
        """The two spectrum-weighted averages of the VMIs (low, high kVp), float32
        [2, nz, ny, nx] (deam_kvp_images)."""
        torch = self.torch
        out = torch.empty((2,) + self.img_shape[:3], dtype=torch.float32, device=self.device)
        _check(lib().deam_kvp_images(self._h, self._arg(c, self.img_shape, torch.float32),
                                     C.c_void_p(out.data_ptr()), self._stream()))
        return out

    def info(self):
        Z = C.c_double()
        sk = C.c_longlong()
        _check(lib().deam_info(self._h, C.byref(Z), C.byref(sk)))
        return Z.value, sk.value

    def count_samples(self):
        """Joseph samples of one projection (the work unit of ray-samples/s)."""
        n = C.c_longlong()
        _check(lib().deam_count_samples(self._h, C.byref(n), self._stream()))
        return n.value

    def profile(self, enable=True):
        _check(lib().deam_profile(self._h, int(bool(enable))))

    def kernel_times(self, reset=False):
        """Accumulated (ms[4], launches[4]) of deam_iterate's stages: layout,
        forward + epilogue, objective reduction, backprojection + update."""
        ms = (C.c_double * 4)()
        n = (C.c_longlong * 4)()
        _check(lib().deam_kernel_times(self._h, ms, n, int(bool(reset))))
        return list(ms), list(n)

    def close(self):
        """Release the context (raises DeamError while a live DeamBatch holds it)."""
        if getattr(self, "_h", None):
            _check(lib().deam_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def from_case(case, **kw) -> Deam:
    return Deam(case.geo, case.I0, case.mu, bowtie=case.bowtie, energies=case.energies, **kw)


def l1_bandwidth():
    """Measured L1 data-path (shared-memory load) throughput of the current
    device in bytes/s (deam_l1_bandwidth)."""
    import torch
    v = C.c_double()
    _check(lib().deam_l1_bandwidth(C.byref(v), C.c_void_p(torch.cuda.current_stream().cuda_stream)))
    return v.value


def calibrate_decomposition(scans, roi):
    """Calibrated weights (mu~_1L, mu~_2L, mu~_1H, mu~_2H) of Eq. (4) from
    calibration scans: `scans` is a list of (deam, (c1, c2)) pairs, each a
    context holding the counts of a calibration phantom whose ROI (boolean
    [nz, ny, nx] tensor) has basis densities (c1, c2).  Each scan's two FBP
    images are averaged over the ROI and mu_j = mu~_1j c1 + mu~_2j c2 is solved
    by least squares over the scans (at least two with independent (c1, c2))."""
    A, b = [], []
    for dm, cc in scans:
        mu = dm.fbp(dm.log_sinogram()).cpu().double().numpy()
        r = np.asarray(roi.cpu() if hasattr(roi, "cpu") else roi, dtype=bool)
        b.append([float(mu[j][r].mean()) for j in range(2)])
        A.append([float(cc[0]), float(cc[1])])
    A, b = np.asarray(A), np.asarray(b)
    sol = np.linalg.lstsq(A, b, rcond=None)[0]   # [[m1L, m1H], [m2L, m2H]]
    return np.array([sol[0, 0], sol[1, 0], sol[0, 1], sol[1, 1]])


def objective_noalloc(geo, I0, mu, c, d, mask, F, bowtie=None, mask_kind="bits"):
    """deam_objective_noalloc: F(c) into the device double tensor F without any
    device allocation (see include/deam.h).  c, d, mask (or None), F are CUDA
    tensors owned by the caller; the call is enqueued on the current stream.
    mask_kind="bits": the mask holds the per-spectrum bits as
    Deam.metal_mask() returns them (bit 0 low kVp, bit 1 high kVp) and is
    passed as it is; "ray": nonzero means both spectra, converted here to
    bits (a new tensor: callers that cannot allocate pass bits)."""
    import torch
    g = deam_geometry(int(geo.kind), geo.nx, geo.ny, geo.nz, geo.dx, geo.dy, geo.dz, geo.cx, geo.cy, geo.cz,
                      geo.sid, geo.sdd, geo.n_views, geo.views_per_rotation, geo.start_angle, geo.feed,
                      geo.z_start, geo.n_rows, geo.row_pitch, geo.n_channels, geo.channel_pitch,
                      geo.channel_offset, geo.row_offset)
    I0 = np.ascontiguousarray(np.asarray(I0, dtype=np.float64))
    mu = np.ascontiguousarray(np.asarray(mu, dtype=np.float64))
    P = C.POINTER(C.c_double)
    bow = None if bowtie is None else np.ascontiguousarray(np.asarray(bowtie, dtype=np.float64))
    sp = deam_spectra(I0.shape[1], P(), I0.ctypes.data_as(P), bow.ctypes.data_as(P) if bow is not None else P())
    ba = deam_basis(mu.shape[1], mu.ctypes.data_as(P))
    for t, dt in ((c, torch.float32), (d, torch.float32), (F, torch.float64)):
        if not (t.is_cuda and t.dtype == dt and t.is_contiguous()):
            raise ValueError("c, d (float32) and F (float64) must be contiguous CUDA tensors")
    if mask is not None and not (mask.is_cuda and mask.dtype == torch.uint8 and mask.is_contiguous()):
        raise ValueError("mask must be a contiguous uint8 CUDA tensor or None")
    if mask_kind not in ("bits", "ray"):
        raise ValueError("mask_kind is 'bits' or 'ray'")
    if mask is not None and mask_kind == "ray":
        mask = (mask != 0).to(torch.uint8) * 3
    stream = C.c_void_p(torch.cuda.current_stream(c.device).cuda_stream)
    _check(lib().deam_objective_noalloc(C.byref(g), C.byref(sp), C.byref(ba), C.c_void_p(c.data_ptr()),
                                        C.c_void_p(d.data_ptr()),
                                        C.c_void_p(mask.data_ptr()) if mask is not None else None,
                                        C.c_void_p(F.data_ptr()), stream))


class DeamBatch:
    """Several scans (Deam contexts with data set) iterated together: one
    persistent launch per stage over all scans, replayed from a CUDA graph,
    tile shapes picked by timing on the first iterate (autotune=True)."""

    def __init__(self, scans, autotune=True, plan=None):
        """autotune=True: shapes and plan picked by timing on the first iterate;
        False: the persistent plan with default shapes; plan="per_scan" forces
        every scan's own kernels on graph branches (no tuning)."""
        import torch
        self.torch = torch
        self.scans = list(scans)
        arr = (C.c_void_p * len(self.scans))(*[s._h for s in self.scans])
        h = C.c_void_p()
        mode = 2 if plan == "per_scan" else int(bool(autotune))
        _check(lib().deam_batch_create(arr, len(self.scans), mode, C.byref(h)))
        self._h = h

    def iterate(self, images, n_iter):
        """n_iter iterations in place on the CUDA images (one per scan); returns
        the objective histories as a numpy array [n_scans, n_iter]."""
        if len(images) != len(self.scans):
            raise ValueError("one image per scan")
        ptrs = (C.c_void_p * len(images))(*[s._arg(c, s.img_shape, self.torch.float32)
                                            for s, c in zip(self.scans, images)])
        hist = np.zeros((len(images), max(n_iter, 1)), dtype=np.float64)
        stream = self.scans[0]._stream()
        _check(lib().deam_batch_iterate(self._h, ptrs, int(n_iter), hist.ctypes.data_as(C.POINTER(C.c_double)),
                                        stream))
        return hist[:, :n_iter]

    def info(self):
        plan = C.c_int()
        pm = (C.c_float * 2)()
        f = (C.c_int * 2)()
        b = (C.c_int * 9)()
        fm = (C.c_float * 3)()
        bm = (C.c_float * 6)()
        _check(lib().deam_batch_info(self._h, C.byref(plan), pm, f, b, fm, bm))
        bwd = [{"slab": b[3 * c], "tile": (b[3 * c + 1], b[3 * c + 2])} for c in range(3) if b[3 * c] > 0]
        return {"plan": ["persistent", "per-scan graph branches"][plan.value], "forward_tile": (32, f[0], f[1]),
                "backprojection": bwd,
                "tuning_ms": {"plans": list(pm), "forward": list(fm), "backprojection": [x for x in bm if x > 0]}}

    def close(self):
        if getattr(self, "_h", None):
            lib().deam_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def i_divergence(c, deam: Deam):
    """F(c) (Eq. 5 over rays off the metal trace) as a float64 torch scalar that
    autograd can differentiate with respect to the image c: the backward pass
    calls deam_gradient (per-ray terms recomputed, not stored)."""
    return _idiv_function().apply(c, deam)


_IDIV = None


def _idiv_function():
    global _IDIV
    if _IDIV is None:
        import torch

        class IDivergence(torch.autograd.Function):
            @staticmethod
            def forward(ctx, c, deam):
                ctx.save_for_backward(c)
                ctx.deam = deam
                return torch.tensor(deam.objective(c.detach()), dtype=torch.float64, device=c.device)

            @staticmethod
            def backward(ctx, grad_out):
                (c,) = ctx.saved_tensors
                g, _ = ctx.deam.gradient(c.detach())
                return (g * grad_out.to(g.dtype)), None

        _IDIV = IDivergence
    return _IDIV
