"""The host-driven iteration loop (FH_HOST_LOOP=1, for profilers that cannot
look inside graphs with conditional nodes) runs the same kernels with the same
arguments as the graph's while node, chunk by chunk, so a solve must give the
same iteration counts, residuals and fields bit for bit.  The variable is read
once per process, so the host-loop solve runs in a child process."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from gpu_util import cuda_or_skip

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

CHILD = r"""
import json, sys
import numpy as np
sys.path.insert(0, {root!r})
from paper_1004_1122_gb300 import fh, microstructure as micro
out = []
phase = micro.rsa_disks(135, 0.3, 4, 9, seed=7)
for precision in ("fp64", "fp32_refined"):
    L = micro.isotropic_table([1.0, 50.0], 2)
    with fh.Solver(phase, L, precision=precision) as s:
        x, col, info = s.solve([1.0, 0.0], tol=1e-7, method="cg", max_iter=5000)
        out.append({{"iters": info["iters"], "rel": info["rel_res_true"], "col": [float(c) for c in col],
                    "x": np.asarray(x.cpu().numpy()).tobytes().hex()}})
cells = [micro.rsa_disks(n, 0.3, 3, 8, seed=9 + n) for n in (81, 135, 81)]
tabs = [micro.isotropic_table([1.0, 20.0], 2) for _ in cells]
with fh.Batch(cells, tabs, nloads=2, precision="fp32_refined") as bt:
    Leff, st, it, info = bt.solve(np.eye(2), tol=1e-7, method="cg", max_iter=5000)
    out.append({{"Leff": np.asarray(Leff).tolist(), "iters": np.asarray(it).tolist(), "st": np.asarray(st).tolist()}})
print(json.dumps(out))
"""


def _run(host_loop):
    env = dict(os.environ)
    env.pop("FH_HOST_LOOP", None)
    if host_loop:
        env["FH_HOST_LOOP"] = "1"
    r = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT)], env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_host_loop_gives_the_graph_loops_iterates():
    cuda_or_skip()
    graph, host = _run(False), _run(True)
    for g, h in zip(graph[:2], host[:2]):
        assert g["iters"] == h["iters"] and g["rel"] == h["rel"] and g["col"] == h["col"], (g, h)
        assert g["x"] == h["x"]
    assert graph[2] == host[2]
    assert np.all(np.asarray(graph[2]["st"]) == 0)
