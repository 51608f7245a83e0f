"""Multi-process (gloo, world size 2, CPU) checks of the replica-run host logic and of
bench.py's reference arm under torchrun (rank 0 prints, the other rank exits 0)."""
import json
import os
import socket
import subprocess
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    from paper_0908_4421_gb300.replicas import Group
    g = Group(backend="gloo")
    g.barrier()
    out[rank] = (g.max(10.0 + rank), g.sum(1.0), g.rank, g.world)
    g.close()


def test_group_max_and_sum_gloo():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == (11.0, 2.0, 0, 2)
    assert res[1] == (11.0, 2.0, 1, 2)


def test_single_process_group_is_noop(monkeypatch):
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    from paper_0908_4421_gb300.replicas import Group
    g = Group()
    assert (g.rank, g.world) == (0, 1)
    assert g.max(3.5) == 3.5
    g.barrier()
    g.close()


def test_bench_reference_arm_under_torchrun():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3",
           "--workload", "tiny-40x40x30-5mm-5beam", "--cpu-budget-s", "1"]
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == "time-to-plan" and d["unit"] == "s"
    assert d["n_gpus"] == 2 and d["cpu_baseline"]["kind"] == "oracle" and d["value"] > 0
    assert d["e2e"] == {"value": d["value"], "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
