"""The multi-process path on CPU (world size 2, gloo): the bench's max-over-ranks
helpers, frame sharding by global frame index (results equal to one process over
the union of the frames) and the reference arm under torchrun (rank 0 alone
prints one line, every rank exits 0)."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    bench.barrier(world)
    mx = bench.dist_max(float(10 + rank), world)
    # replicas: rank r decodes frames [r B, (r + 1) B) of one seeded workload (oracle, CPU)
    import oracle
    from paper_2102_11089_gb300 import workloads as wl
    c, v, m = wl.regular_code(96, 3, 6, 1)
    B = 16
    lam = wl.seeded_llrs(96, world * B, wl.sigma2_from_ebn0(1.5, 0.5), 3).astype(np.float64)
    mine = lam[rank * B:(rank + 1) * B]
    o = oracle.decode(c, v, m, 96, llr=mine, schedule="me-lmd-cirbp", max_updates=5 * len(c), n_p=8, n_g=8,
                      frame_offset=rank * B, want_trace=True)
    t = torch.from_numpy(np.concatenate([o["updates"].astype(np.float64), o["hard"].sum(1).astype(np.float64)]))
    parts = [torch.zeros_like(t) for _ in range(world)]
    dist.all_gather(parts, t)
    q.put((rank, mx, [p.numpy() for p in parts]))
    dist.destroy_process_group()


def test_two_gloo_ranks_max_and_sharding():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert all(mx == 11.0 for _, mx, _ in res)
    gathered = res[0][2]
    import oracle
    from paper_2102_11089_gb300 import workloads as wl
    c, v, m = wl.regular_code(96, 3, 6, 1)
    lam = wl.seeded_llrs(96, 32, wl.sigma2_from_ebn0(1.5, 0.5), 3).astype(np.float64)
    o = oracle.decode(c, v, m, 96, llr=lam, schedule="me-lmd-cirbp", max_updates=5 * len(c), n_p=8, n_g=8)
    want = np.concatenate([o["updates"].astype(np.float64), o["hard"].sum(1).astype(np.float64)])
    got_upd = np.concatenate([g[:16] for g in gathered])
    got_err = np.concatenate([g[16:] for g in gathered])
    assert np.array_equal(got_upd, want[:32]) and np.array_equal(got_err, want[32:])


def test_reference_arm_under_torchrun_two_ranks():
    env = dict(os.environ, OMP_NUM_THREADS="1")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0", "--cpu-seconds", "0.3"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
