"""The C-ABI library builds, loads without a GPU, exports every entry point
declared in include/deam.h and validates arguments on the host before touching
the device."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libdeam():
    from paper_2202_00116_gb300 import build
    build.build()
    import paper_2202_00116_gb300 as pkg
    return pkg


def declared_functions():
    text = open(os.path.join(ROOT, "include", "deam.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(deam_\w+)\s*\(", text, flags=re.M)))


def test_every_declared_symbol_is_exported(libdeam):
    names = declared_functions()
    assert len(names) >= 12, names
    L = C.CDLL(libdeam.LIB_PATH)
    for n in names:
        assert hasattr(L, n), f"{n} declared in deam.h but not exported"
    assert set(names) == set(libdeam.EXPORTS)


def _geo(**kw):
    import synth
    g = synth.make_case("t2d").geo
    return g.replace(**kw)


@pytest.mark.parametrize("bad", [dict(nx=0), dict(dx=-1.0), dict(sdd=100.0), dict(n_views=0),
                                 dict(channel_pitch=0.0), dict(kind=7), dict(n_rows=2),
                                 dict(dx=30.0), dict(channel_pitch=0.1)])
def test_invalid_geometry_is_rejected_on_the_host(libdeam, bad):
    import synth
    case = synth.make_case("t2d")
    with pytest.raises(libdeam.DeamError) as e:
        libdeam.Deam(_geo(**bad), case.I0, case.mu)
    assert e.value.code == libdeam.DEAM_ERR_ARG


def test_invalid_tables_are_rejected_on_the_host(libdeam):
    import numpy as np
    import synth
    case = synth.make_case("t2d")
    for I0, mu in [(-case.I0, case.mu), (case.I0, -case.mu), (np.zeros_like(case.I0), case.mu),
                   (case.I0[:, :10], case.mu), (np.zeros((2, 300)), np.zeros((2, 300)))]:
        with pytest.raises(libdeam.DeamError) as e:
            libdeam.Deam(case.geo, I0, mu)
        assert e.value.code == libdeam.DEAM_ERR_ARG
    bow = np.ones(case.geo.n_channels)
    bow[3] = 0.0
    with pytest.raises(libdeam.DeamError):
        libdeam.Deam(case.geo, case.I0, case.mu, bowtie=bow)


def test_null_context_calls_fail_cleanly(libdeam):
    L = libdeam.lib()
    assert L.deam_iterate(None, None, 1, None, None) == libdeam.DEAM_ERR_ARG
    assert L.deam_destroy(None) == libdeam.DEAM_OK
    assert b"null" in L.deam_last_error()


def test_every_context_entry_point_rejects_a_null_context(libdeam):
    # host-side argument checks run before any device call, so they are
    # exercised here without a GPU
    L = libdeam.lib()
    P = libdeam.deam_mar_params()
    calls = [
        lambda: L.deam_set_data(None, None, None),
        lambda: L.deam_forward(None, None, None, None, None),
        lambda: L.deam_backproject(None, None, None, None),
        lambda: L.deam_ray_terms(None, None, None, None, None),
        lambda: L.deam_objective(None, None, None, None),
        lambda: L.deam_gradient(None, None, None, None, None),
        lambda: L.deam_backprojected_sums(None, None, None, None, None, None),
        lambda: L.deam_penalty(None, None, None, None),
        lambda: L.deam_log_sinogram(None, 1.0, None, None),
        lambda: L.deam_complete_trace(None, None, None, 0, 1e-3, None, None),
        lambda: L.deam_fbp(None, None, 1, None, None),
        lambda: L.deam_mar_init(None, C.byref(P), None, None, None, None, None),
        lambda: L.deam_vmi(None, None, None, 1, None, None),
        lambda: L.deam_kvp_images(None, None, None, None),
    ]
    for call in calls:
        assert call() == libdeam.DEAM_ERR_ARG
        assert b"null" in L.deam_last_error().lower()


def test_l1_probe_rejects_a_null_output(libdeam):
    assert libdeam.lib().deam_l1_bandwidth(None, None) == libdeam.DEAM_ERR_ARG


def test_batch_create_rejects_an_unknown_plan_mode(libdeam):
    h = C.c_void_p()
    arr = (C.c_void_p * 1)(None)
    assert libdeam.lib().deam_batch_create(arr, 1, 3, C.byref(h)) == libdeam.DEAM_ERR_ARG


def test_binding_fails_loudly_without_the_library(libdeam, monkeypatch, tmp_path):
    # no CPU fallback: with the compiled library missing, the binding raises
    monkeypatch.setattr(libdeam, "LIB_PATH", str(tmp_path / "missing" / "libdeam.so"))
    monkeypatch.setattr(libdeam, "_lib", None)
    import synth
    case = synth.make_case("t2d")
    with pytest.raises(RuntimeError, match="missing"):
        libdeam.Deam(case.geo, case.I0, case.mu)


def test_bounds_checked_build_exports_the_same_api(libdeam):
    # the -DDEAM_BOUNDS_CHECK build compiles (no GPU needed), exports every
    # declared entry point and says so; the default build says it is not one
    from paper_2202_00116_gb300 import build
    path = build.build(bounds_check=True)
    Lc = C.CDLL(path)
    for n in declared_functions():
        assert hasattr(Lc, n), n
    Lc.deam_bounds_checked.restype = C.c_int
    assert Lc.deam_bounds_checked() == 1
    assert libdeam.lib().deam_bounds_checked() == 0
    Lc.deam_bounds_inject.argtypes = [C.c_void_p, C.c_void_p]
    assert Lc.deam_bounds_inject(None, None) == libdeam.DEAM_ERR_ARG       # null context, on the host
