"""bench.py's multi-rank path on CPU: two gloo ranks on 127.0.0.1 agree on the
max-over-ranks step time, each evaluates its own seeded inputs (rank 0 the
sweep recipe itself), deterministically, with the same problem sizes."""
import json
import os
import socket
import subprocess
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks():
    port = free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                   LOCAL_RANK=str(rank))
        procs.append(subprocess.Popen([sys.executable, os.path.join(HERE, "_multirank_worker.py")], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=180)
        assert p.returncode == 0, e[-2000:]
        outs.append(json.loads(o.strip().splitlines()[-1]))
    outs.sort(key=lambda d: d["rank"])
    assert [d["ms"] for d in outs] == [13.0, 13.0]
    assert all(d["deterministic"] for d in outs)
    assert outs[0]["digest"] != outs[1]["digest"]
    assert outs[0]["npair"] == outs[1]["npair"] == 16 and outs[0]["naux"] == outs[1]["naux"] == 8
    # rank 0 evaluates exactly the sweep recipe
    sys.path.insert(0, os.path.dirname(HERE))
    from paper_2210_03192_gb300 import workloads as W
    p0 = W.sweep_class(2, 1, 3, 3, 16, 8)
    assert np.isclose(outs[0]["digest"], float(p0.orb.xyz.sum() + p0.orb.exps.sum() + p0.aux.exps.sum()))
