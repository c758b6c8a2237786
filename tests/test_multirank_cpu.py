"""Multi-rank aggregation of bench.py on the CPU: two gloo ranks on
127.0.0.1.  Each rank reports a different time; both get the slowest one,
and the whole-job rate counts every rank's units over it.  The reference arm
does no work and prints nothing on a rank other than 0."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


RANK_SCRIPT = r"""
import json, os, sys
sys.path.insert(0, sys.argv[1])
import torch.distributed as dist
import bench
dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%s" % sys.argv[2],
                        rank=int(sys.argv[3]), world_size=2)
mine = [12.5, 20.0][int(sys.argv[3])]
ms = bench.max_over_ranks(mine, "cpu")
print(json.dumps({"rank": int(sys.argv[3]), "ms": ms,
                  "rate": bench.whole_job_rate(64 * 100, dist.get_world_size(), ms)}))
dist.destroy_process_group()
"""


def test_max_over_ranks_with_two_gloo_ranks():
    pytest.importorskip("torch")
    port = _free_port()
    procs = [subprocess.Popen([sys.executable, "-c", RANK_SCRIPT, ROOT, str(port), str(r)],
                              stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)
             for r in range(2)]
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err
        outs.append(json.loads(out.strip().splitlines()[-1]))
    for o in outs:
        assert o["ms"] == 20.0
        assert o["rate"] == pytest.approx(64 * 100 * 2 / 0.020)


def test_single_rank_keeps_its_own_time():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.25, "cpu") == 7.25
    assert bench.whole_job_rate(640, 1, 10.0) == pytest.approx(64000.0)


def test_reference_arm_is_silent_off_rank_zero():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "1"], env=env, capture_output=True, text=True,
                       timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
