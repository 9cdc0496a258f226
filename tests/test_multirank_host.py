"""The N > 1 path of bench.py on the CPU: two gloo ranks (127.0.0.1) run the replica
aggregation. Replicas image independent specimens (no data-path collective); the only
exchange is the max-over-ranks step time, and value = ranks x pixels / that time."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_CHILD = r"""
import json, os, sys
sys.path.insert(0, sys.argv[1])
import torch.distributed as dist
import bench
rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
dist.init_process_group("gloo", rank=rank, world_size=world)
t = bench.max_over_ranks([100.0, 130.0][rank], world, dist, device="cpu")
w = bench.replica_workload(rank)
ph = w.phonons[1]
print(json.dumps({"rank": rank, "t": t, "sig": float(ph.x[:64].sum() + ph.y[:64].sum()),
                  "pixels": w.n_pixels}))
dist.destroy_process_group()
"""


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_share_the_slowest_time_and_image_distinct_replicas():
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", _CHILD, ROOT], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=240)
        assert p.returncode == 0, err[-2000:]
        outs.append(json.loads(out.strip().splitlines()[-1]))
    outs.sort(key=lambda r: r["rank"])
    assert [r["t"] for r in outs] == [130.0, 130.0]
    assert outs[0]["sig"] != outs[1]["sig"]          # independent phonon seeds per rank
    assert outs[0]["pixels"] == outs[1]["pixels"] == 128 * 128
