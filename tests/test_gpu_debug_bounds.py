"""Debug build with device-side bounds checks (GPU only). The library is rebuilt with
SBSE_DEBUG_BOUNDS (libsbse_dbg.so) and the hot path is run on an 80^3 system in the mixed mode
(lane-pair FFT sweeps, staged z sweep, tensor-core cleaning and contractions) and on 16^3 in FP64:
no index may be recorded out of range, and the debug build reports itself as such. Runs in a child
process, since the binding loads one library per process."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import json, os, sys
import numpy as np
sys.path.insert(0, os.environ["SBSE_ROOT"])
from paper_2205_06690_gb300 import build
build.build(debug_bounds=True)
import sbse_inputs as si
from paper_2205_06690_gb300 import binding as B
out = {}
B.load()
out["enabled"], _ = B.sbse_debug_bounds()
for N, prec, name in ((80, B.SBSE_MIXED, "mixed80"), (16, B.SBSE_FP64, "fp64_16")):
    p = si.model_system.Preset(f"db{N}", N=N, box=0.25 * N if N > 32 else 8.0, n_wells=6, seed=N, n_occ=6, n_o=3,
                               n_c=4)
    s = si.make_system(p)
    prm = B.TDHParams(n_s=4, n_steps=12, clean_every=4, dt=0.05, gamma=0.1, alpha=1e-4, seed=5)
    with B.Context(0, prec) as c:
        c.set_grid(N, p.box, s.v_loc)
        c.set_orbitals(p.n_occ, p.n_o, p.n_c, s.phi, s.eps, 0.5)
        pairs = [(i, j) for i in range(3) for j in range(i, 3)]
        W = c.apply_W(prm, pairs, copy_out=True)
        c.build_A(copy_out=False)
        ev = c.spectrum(4)
    out[name] = {"fault": B.sbse_debug_bounds()[1], "finite": bool(np.all(np.isfinite(W)) and np.all(np.isfinite(ev)))}
print("RESULT " + json.dumps(out))
'''


def test_debug_build_records_no_out_of_range_index():
    env = dict(os.environ, SBSE_DEBUG_BOUNDS="1", SBSE_ROOT=ROOT)
    r = subprocess.run([sys.executable, "-c", CHILD], env=env, cwd=ROOT, capture_output=True, text=True,
                       timeout=1200)
    assert r.returncode == 0, r.stderr[-3000:]
    line = [x for x in r.stdout.splitlines() if x.startswith("RESULT ")][-1]
    res = json.loads(line[len("RESULT "):])
    assert res["enabled"] is True
    for name in ("mixed80", "fp64_16"):
        assert res[name]["finite"]
        assert res[name]["fault"] == 0, f"{name}: out-of-range index recorded, code {res[name]['fault']:#x}"
