"""Multi-process paths on CPU with the gloo backend (world size 2).

* The benchmark's reference arm under torchrun: rank 0 alone runs and prints
  one JSON line, the other rank exits 0.
* The max-over-ranks reduction the GPU arm applies to its timings.
* The view-sharded form of one MAR-DEAM iteration: each rank backprojects the
  spectral sums of its half of the views, one all-reduce (sum) of b~, b^ and F
  gives exactly the single-process sums, and the c-step applied to them
  reproduces the oracle's iteration."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _init(rank, world, port):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)


def _max_worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    _init(rank, world, port)
    import bench
    v = bench.reduce_max(dist, 10.0 + rank, "cpu")
    out[rank] = v
    dist.destroy_process_group()


def test_reduce_max_over_ranks():
    port = _free_port()
    out = mp.Manager().dict()
    mp.spawn(_max_worker, args=(2, port, out), nprocs=2, join=True)
    assert dict(out) == {0: 11.0, 1: 11.0}


def _shard_worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    _init(rank, world, port)
    import oracle
    import synth
    case = synth.make_case("t3d")
    d, metal = synth.measure(case, seed=1)
    truth, _ = synth.voxelize(case)
    mask = (metal >= case.metal_threshold).numpy().astype(np.uint8)
    c0 = synth.initial_image(case, truth).double().numpy()
    O = oracle.from_case(case)
    V = case.geo.n_views
    v0, v1 = (0, V // 2) if rank == 0 else (V // 2, V)
    bt, bh, F = O.backprojected_sums(c0, d.double().numpy(), mask, v0, v1)
    t = torch.from_numpy(np.concatenate([bt.ravel(), bh.ravel(), [F]]))
    dist.all_reduce(t, op=dist.ReduceOp.SUM)     # the one exchange step of a view-sharded iteration
    out[rank] = t.numpy().copy()
    dist.destroy_process_group()


def test_view_sharded_iteration_matches_single_process(oracle_lib):
    import oracle
    import synth
    port = _free_port()
    out = mp.Manager().dict()
    mp.spawn(_shard_worker, args=(2, port, out), nprocs=2, join=True)
    assert np.array_equal(out[0], out[1])
    case = synth.make_case("t3d")
    d, metal = synth.measure(case, seed=1)
    truth, _ = synth.voxelize(case)
    mask = (metal >= case.metal_threshold).numpy().astype(np.uint8)
    c0 = synth.initial_image(case, truth).double().numpy()
    O = oracle.from_case(case)
    bt, bh, F = O.backprojected_sums(c0, d.double().numpy(), mask)
    n = bt.size
    red = out[0]
    np.testing.assert_allclose(red[:n], bt.ravel(), rtol=1e-12, atol=1e-9)
    np.testing.assert_allclose(red[n:2 * n], bh.ravel(), rtol=1e-12, atol=1e-9)
    assert red[-1] == pytest.approx(F, rel=1e-12)
    # c-step on the reduced sums = the oracle's own iteration
    Z = O.normaliser()
    bts, bhs = red[:n], red[n:2 * n]
    ok = (bts > 0) & (bhs > 0)
    c1 = c0.ravel().copy()
    c1[ok] -= np.log(bhs[ok] / bts[ok]) / Z
    c_ref, h_ref, _ = O.iterate(c0, d.double().numpy(), mask, n_iter=1)
    np.testing.assert_allclose(c1, c_ref.ravel(), rtol=0, atol=1e-12)
    assert h_ref[0] == pytest.approx(red[-1], rel=1e-12)


def test_reference_arm_under_torchrun(oracle_lib):
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", f"--master-port={port}", os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--config", "t2d", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="", OMP_NUM_THREADS="2")
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "it/s"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0
    # the same config object as the GPU arm's line (bench.workload_config)
    sys.path.insert(0, ROOT)
    import bench
    import synth
    args = type("A", (), {"config": "t2d"})()
    assert line["config"] == bench.workload_config(args, synth.make_case("t2d"), 2)
