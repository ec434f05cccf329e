"""The fast-math build (libmanta_fast.so: FMA contraction, approximate
division and square root, flush-to-zero) against the oracle: over 600 steps
of the tiny workload every vehicle's position within 1e-4 m and speed within
1e-4 m/s, the same vehicles on the same edges and lanes, and exactly the same
link entry and exit counts."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import nets
from oracle import oracle as O
from paper_2007_03614_b300 import synth
from paper_2007_03614_b300.build import LIB_FAST, build

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RUN = r"""
import sys, json
import numpy as np
sys.path[:0] = [{root!r}, {tests!r}]
import nets
from paper_2007_03614_b300 import manta, synth
net = synth.tiny_network()
tr = synth.tiny_trips(net)
g = manta.Sim(net)
nets.load(g, tr)
g.step({steps})
s = g.snapshot()
ec = g.edge_counters(0)
np.savez({out!r}, **{{k: s[k] for k in s}}, entries=ec["entries"], exits=ec["exits"])
print(json.dumps(g.stats()))
"""


@pytest.mark.parametrize("steps", [600])
def test_fast_math_build_within_tolerance(tmp_path, steps):
    build()
    assert os.path.exists(LIB_FAST)
    out = str(tmp_path / "fast.npz")
    code = RUN.format(root=ROOT, tests=os.path.join(ROOT, "tests"), steps=steps, out=out)
    env = dict(os.environ, MANTA_LIBRARY=LIB_FAST)
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    fast = np.load(out)
    net = synth.tiny_network()
    tr = synth.tiny_trips(net)
    o = O.OracleSim(net)
    nets.load(o, tr)
    o.step(steps)
    so = o.snapshot()
    eo = o.edge_counters(0)
    assert np.array_equal(so["id"], fast["id"]), "different vehicles on the network"
    for key in ("edge", "lane", "route_pos"):
        bad = np.nonzero(so[key] != fast[key])[0]
        assert bad.size == 0, f"{key} differs first at vehicle {so['id'][bad[0]]}"
    dx = np.abs(so["x"].astype(np.float64) - fast["x"])
    dv = np.abs(so["v"].astype(np.float64) - fast["v"])
    assert dx.max() <= 1e-4, (float(dx.max()), int(so["id"][np.argmax(dx)]))
    assert dv.max() <= 1e-4, (float(dv.max()), int(so["id"][np.argmax(dv)]))
    assert np.array_equal(eo["entries"], fast["entries"])
    assert np.array_equal(eo["exits"], fast["exits"])
    st = json.loads(r.stdout.strip().splitlines()[-1])
    assert st["vehicle_updates"] == o.stats()["vehicle_updates"]
