"""Plans allocate from the library's stream-ordered pool, which keeps the memory of destroyed
plans for later ones (no mapping of new memory per plan_create); imrt_trim_memory hands it
back to the system. Run in a fresh process: plans other tests keep alive would leave the pool
partly used, and a new plan could then fit into their freed space without growing it."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

BODY = r"""
import json, torch
from paper_0908_4421_gb300 import Options, Plan, phantom, trim_memory
case = phantom.random_case(7, m=200_000, n=2000, density=0.05)
def free():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]
out = {}
with Plan.from_case(case, Options()):
    pass  # the first plan also makes the context's one-time reservations (kernel code, local memory)
trim_memory(0)
out["start"] = free()
with Plan.from_case(case, Options()) as p:
    out["held"] = p.info()["device_bytes"]
    out["alive"] = free()
out["destroyed"] = free()
with Plan.from_case(case, Options()):
    out["second"] = free()
trim_memory(0)
out["trimmed"] = free()
print(json.dumps(out))
"""


def test_pool_keeps_memory_until_trimmed():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    env = dict(os.environ, PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, "-c", BODY], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    f = json.loads(r.stdout.strip().splitlines()[-1])
    held = f["held"]
    assert held > 100 << 20
    assert f["start"] - f["alive"] >= 0.9 * held
    assert f["start"] - f["destroyed"] >= 0.9 * held      # the destroyed plan's memory stays in the pool
    assert f["second"] >= f["destroyed"] - (held >> 3)    # a plan of the same shape reuses it
    assert f["trimmed"] >= f["start"] - (held >> 3)       # trimming hands it back
