"""The TMA-staged step's bounded mbarrier wait (GPU, host-side fault injection).

With QUAPI_FAULT=tma_tx set when a context is created, CTA 0 of every TMA step
arms its first tile's mbarrier with 16 bytes more than the tile's copies
deliver.  The copies complete normally; the barrier's phase never does, so the
wait runs out after QUAPI_WAIT_MS, the CTA records the error flag, waits
(bounded) for its other copies and returns, and the call reports
QUAPI_ERR_TIMEOUT.  Nothing faults, traps or hangs: the test then checks that a
context created without the injection still propagates correctly in the same
process.  It runs in a subprocess so that the environment stays local to it.
"""

import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_SCRIPT = r"""
import os, sys, time
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_1205_6872_gb300 import quapi as q, workloads as wl
p = wl.spin_boson_L6()
L, steps = 8, [0, 12]   # memory length 8: 4^7 fibers of the FP32 full layout, TMA-staged (lo_size 256)
os.environ["QUAPI_FAULT"] = "tma_tx"
bad = q.quapi_setup(p.s, p.H, p.jkind, p.ja, p.wc, p.beta, p.dt, L, q.quapi_opts_init(precision=32))
del os.environ["QUAPI_FAULT"]
good = q.quapi_setup(p.s, p.H, p.jkind, p.ja, p.wc, p.beta, p.dt, L, q.quapi_opts_init(precision=32))
t0 = time.time()
try:
    q.quapi_propagate(bad, p.rho0, steps, 2)
    print("NO_ERROR")
except q.QuapiError as e:
    print("STATUS", e.status)
print("SECONDS", time.time() - t0)
r = q.quapi_propagate(good, p.rho0, steps, 2)
print("TRACE", float(np.trace(r[1]).real))
# the faulty context is still usable as a context: its next call reports the same expiry, no CUDA error
try:
    q.quapi_propagate(bad, p.rho0, steps, 2)
    print("AGAIN NO_ERROR")
except q.QuapiError as e:
    print("AGAIN", e.status)
q.quapi_destroy(bad)
q.quapi_destroy(good)
"""


def test_tma_step_bounded_wait_reports_timeout(tmp_path):
    script = tmp_path / "tma_wait_case.py"
    script.write_text(_SCRIPT)
    env = dict(os.environ, QUAPI_WAIT_MS="20")
    env.pop("QUAPI_FAULT", None)
    out = subprocess.run([sys.executable, str(script), ROOT], env=env, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    assert "STATUS 4" in out.stdout, out.stdout          # QUAPI_ERR_TIMEOUT
    assert "AGAIN 4" in out.stdout, out.stdout
    trace = float(out.stdout.split("TRACE")[1].split()[0])
    assert abs(trace - 1.0) < 1e-5
