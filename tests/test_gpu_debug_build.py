"""The bounds-checked debug build (libsrw_debug.so, -DSRW_DEBUG_CHECKS) on the
ragged edge cases.

In the debug build every SRW_CHECK index check in the folds and the
reduction is compiled in, and a canary block follows the batched partial
sums.  Run in a fresh process with SRW_LIB=debug, the ragged workloads (no
size a multiple of a tile), a single point, the 7Be and solar sets in every
precision must raise no check (no SRW_ECHECK) and give the release build's
values.
"""

import json
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import json, sys
sys.path.insert(0, %r)
sys.path.insert(0, %r)
import numpy as np
import workloads
from test_gpu_edges import small_workload, _asimov
import paper_2607_00488_gb300 as srw
assert srw.LIB_PATH.endswith("libsrw_debug.so" if %r == "debug" else "libsrw.so"), srw.LIB_PATH
out = {}
cases = [("ragged", small_workload(), None), ("ragged2", small_workload(n_t=65, n_rec=300, seed=1), None),
         ("be7", workloads.be7_line_workload(), "be7_line_256")]
for name, wl, cname in cases:
    counts = workloads.load_counts(cname) if cname else _asimov(wl)
    th = np.concatenate([np.zeros((1, 5), np.float32), workloads.theta_box(131, 3, eps_max=0.02, mu_max=0.4)])
    with srw.Likelihood(wl, counts) as lk:
        for p in ("fp32", "bf16", "bf16x3", "fp16x3"):
            out[name + "/" + p] = lk.loglik(th, srw.PRECISIONS[p]).tolist()
        out[name + "/single"] = lk.loglik(th[3:4], srw.SRW_FP32).tolist()
print(json.dumps(out))
"""


def _run(lib):
    env = dict(os.environ, SRW_LIB=lib)
    code = SCRIPT % (ROOT, os.path.join(ROOT, "tests"), lib)
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_debug_build_raises_no_check_and_matches_release():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    dbg = _run("debug")  # any failed check raises SrwError(SRW_ECHECK) in the child
    rel = _run("release")
    assert dbg.keys() == rel.keys()
    for k in dbg:
        np.testing.assert_array_equal(np.asarray(dbg[k]), np.asarray(rel[k]), err_msg=k)
