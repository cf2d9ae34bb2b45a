"""The bounds-checked build (-DDEAM_BOUNDS_CHECK, libdeam_checked.so) on the GPU:
with every index in range it gives the default build's iterates, and a fault
record written from the host (deam_bounds_inject; no device fault is made) is
read back by the next entry point as DEAM_ERR_ARG, after which the context
works again.  Run in a child process that loads the checked library."""
import os
import subprocess
import sys

import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
pytestmark = pytest.mark.gpu

CHILD = r"""
import sys, numpy as np, torch
sys.path.insert(0, {root!r})
import synth, paper_2202_00116_gb300 as pkg
assert pkg.lib().deam_bounds_checked() == 1
case = synth.make_case("t3d")
d, metal = synth.measure(case, seed=1)
truth, _ = synth.voxelize(case)
mask = (metal >= case.metal_threshold).to(torch.uint8)
c = synth.initial_image(case, truth).cuda()
g = pkg.from_case(case)
g.set_data(d.cuda())
g.set_metal_mask(mask.cuda(), "ray")
h = g.iterate(c, 3)
np.save({out!r}, np.concatenate([c.cpu().double().numpy().ravel(), h]))
import ctypes as C
assert pkg.lib().deam_bounds_inject(g._h, None) == 0
try:
    g.objective(c)
    raise SystemExit("the injected fault record was not reported")
except pkg.DeamError as e:
    assert e.code == pkg.DEAM_ERR_ARG and "site 99" in str(e), e
assert g.objective(c) > 0      # cleared: the context works again
print("checked ok")
"""


def test_bounds_checked_build_on_gpu(tmp_path):
    assert torch.cuda.is_available()
    from paper_2202_00116_gb300 import build
    path = build.build(bounds_check=True)
    build.build()
    out = str(tmp_path / "checked.npy")
    env = dict(os.environ, DEAM_LIB_PATH=path)
    r = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT, out=out)], env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0 and "checked ok" in r.stdout, r.stdout + r.stderr
    import numpy as np
    import synth
    import paper_2202_00116_gb300 as pkg
    case = synth.make_case("t3d")
    d, metal = synth.measure(case, seed=1)
    truth, _ = synth.voxelize(case)
    mask = (metal >= case.metal_threshold).to(torch.uint8)
    c = synth.initial_image(case, truth).cuda()
    g = pkg.from_case(case)
    g.set_data(d.cuda())
    g.set_metal_mask(mask.cuda(), "ray")
    h = g.iterate(c, 3)
    ref = np.concatenate([c.cpu().double().numpy().ravel(), h])
    got = np.load(out)
    n = c.numel()
    assert np.linalg.norm(got[:n] - ref[:n]) <= 1e-6 * np.linalg.norm(ref[:n])
    np.testing.assert_allclose(got[n:], ref[n:], rtol=1e-9)
