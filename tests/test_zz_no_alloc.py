"""deam_objective_noalloc: the objective for callers that cannot allocate device
memory (code whose device memory belongs to another allocator or a fixed arena,
or a latency-bound loop where cudaMalloc/cudaFree would synchronise the device;
such callers cannot create a context).  It must give the same F(c) as the
context-based deam_objective and as the FP64 oracle, within the objective
tolerance of the parity tests (relative 1e-5), on two calls in a row through
the C ABI -- the second call reuses the static scratch the first one left
behind -- and it must not change the device's free memory.

This file is collected last so that a run stopping at the first failure has
already run every other test."""
import dataclasses

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


def _case(name, **geo_changes):
    case = synth.make_case(name)
    if geo_changes:
        case = dataclasses.replace(case, geo=case.geo.replace(**geo_changes))
    d, metal = synth.measure(case, seed=1)
    truth, _ = synth.voxelize(case)
    mask = (metal >= case.metal_threshold).to(torch.uint8)
    c = synth.initial_image(case, truth)
    return case, d, mask, c


# t2d: fan-beam slice with a quarter-channel detector offset; t3d: helical with
# the same offset; the last case adds a row offset as well
CASES = [("t2d", {}), ("t3d", {}), ("c0", {}), ("t3d", {"row_offset": 0.3, "channel_offset": -0.4})]


@pytest.mark.parametrize("name,changes", CASES)
def test_objective_noalloc_matches_context_and_oracle(pkg, name, changes):
    import oracle
    case, d, mask, c = _case(name, **changes)
    ctx = pkg.from_case(case)
    ctx.set_data(d.cuda())
    ctx.set_metal_mask(mask.cuda(), "ray")
    F_ref = ctx.objective(c.cuda())
    bits = ctx.metal_mask()          # per-spectrum bits, as the context holds them
    ctx.close()
    F_or = oracle.from_case(case).objective(c.double().numpy(), d.double().numpy(), mask.numpy())

    cd, dd = c.cuda(), d.cuda()
    F = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    for _ in range(2):
        F.fill_(float("nan"))
        pkg.objective_noalloc(case.geo, case.I0, case.mu, cd, dd, bits, F)
        torch.cuda.synchronize()
        assert F.item() == pytest.approx(F_ref, rel=1e-5)
        assert F.item() == pytest.approx(F_or, rel=1e-5)
    # a 0/1 mask converted by the binding gives the same value
    pkg.objective_noalloc(case.geo, case.I0, case.mu, cd, dd, mask.cuda(), F, mask_kind="ray")
    torch.cuda.synchronize()
    assert F.item() == pytest.approx(F_ref, rel=1e-5)
    # without a mask every ray counts
    pkg.objective_noalloc(case.geo, case.I0, case.mu, cd, dd, None, F)
    torch.cuda.synchronize()
    assert F.item() > F_ref


def test_objective_noalloc_per_spectrum_bits(pkg):
    # separate traces T_L, T_H (Sec. 2.1): bit j leaves out only spectrum j's term
    import oracle
    case, d, mask, c = _case("t3d")
    m = mask.bool()
    mH = m & (torch.rand(m.shape, generator=torch.Generator().manual_seed(3)) < 0.5)
    per = torch.stack([m, mH])
    ctx = pkg.from_case(case)
    ctx.set_data(d.cuda())
    ctx.set_metal_mask(per.cuda(), "per_spectrum")
    F_ref = ctx.objective(c.cuda())
    bits = ctx.metal_mask()
    ctx.close()
    F_or = oracle.from_case(case).objective(c.double().numpy(), d.double().numpy(), per.numpy())
    F = torch.zeros(1, dtype=torch.float64, device="cuda")
    pkg.objective_noalloc(case.geo, case.I0, case.mu, c.cuda(), d.cuda(), bits, F)
    torch.cuda.synchronize()
    assert F.item() == pytest.approx(F_ref, rel=1e-5) and F.item() == pytest.approx(F_or, rel=1e-5)


def test_objective_noalloc_allocates_nothing(pkg):
    case, d, mask, c = _case("t3d")
    cd, dd = c.cuda(), d.cuda()
    bits = (mask != 0).to(torch.uint8).cuda() * 3
    F = torch.zeros(1, dtype=torch.float64, device="cuda")
    pkg.objective_noalloc(case.geo, case.I0, case.mu, cd, dd, bits, F)   # set-up on this device
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(5):
        pkg.objective_noalloc(case.geo, case.I0, case.mu, cd, dd, bits, F)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_objective_noalloc_rejects_oversized_scans(pkg):
    case = synth.make_case("t2d")
    # 600000 views x 1 row x 256 channels = 153.6e6 rays > 134217728: rejected on the host
    geo = case.geo.replace(n_views=600_000, views_per_rotation=600_000, n_channels=256)
    dummy = torch.zeros(4, device="cuda")
    F = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.DeamError) as e:
        pkg.objective_noalloc(geo, case.I0, case.mu, dummy, dummy, None, F)
    assert e.value.code == pkg.DEAM_ERR_ARG
    assert "134217728" in str(e.value)


def test_objective_noalloc_refuses_what_the_context_refuses(pkg):
    # a volume reaching past the source circle: deam_init refuses it, and so
    # does the context-free entry point (no silently wrong F)
    case = synth.make_case("t2d")
    geo = case.geo.replace(cx=450.0)
    with pytest.raises(pkg.DeamError) as e:
        pkg.Deam(geo, case.I0, case.mu)
    assert e.value.code == pkg.DEAM_ERR_ARG
    dummy = torch.zeros(4, device="cuda")
    F = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.DeamError) as e:
        pkg.objective_noalloc(geo, case.I0, case.mu, dummy, dummy, None, F)
    assert e.value.code == pkg.DEAM_ERR_ARG and "source circle" in str(e.value)


def test_objective_noalloc_rejects_host_buffers(pkg):
    # called through the C ABI directly (the binding refuses host tensors
    # itself): a host buffer is an argument error, not a device fault
    import ctypes as C
    case = synth.make_case("t2d")
    g = case.geo
    geo = pkg.deam_geometry(int(g.kind), g.nx, g.ny, g.nz, g.dx, g.dy, g.dz, g.cx, g.cy, g.cz, g.sid, g.sdd,
                            g.n_views, g.views_per_rotation, g.start_angle, g.feed, g.z_start, g.n_rows,
                            g.row_pitch, g.n_channels, g.channel_pitch, g.channel_offset, g.row_offset)
    I0 = np.ascontiguousarray(case.I0, dtype=np.float64)
    mu = np.ascontiguousarray(case.mu, dtype=np.float64)
    P = C.POINTER(C.c_double)
    sp = pkg.deam_spectra(I0.shape[1], P(), I0.ctypes.data_as(P), P())
    ba = pkg.deam_basis(mu.shape[1], mu.ctypes.data_as(P))
    c_host = torch.zeros((g.nz, g.ny, g.nx, 2))
    d_dev = torch.zeros((2, g.n_views, g.n_rows, g.n_channels), device="cuda")
    F = torch.zeros(1, dtype=torch.float64, device="cuda")
    rc = pkg.lib().deam_objective_noalloc(C.byref(geo), C.byref(sp), C.byref(ba), C.c_void_p(c_host.data_ptr()),
                                          C.c_void_p(d_dev.data_ptr()), None, C.c_void_p(F.data_ptr()), None)
    assert rc == pkg.DEAM_ERR_ARG and b"device memory" in pkg.lib().deam_last_error()
