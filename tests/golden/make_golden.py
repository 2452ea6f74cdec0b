"""Write the stored oracle results used by the GPU parity tests at full size.

Calls only ``oracle`` (and the seeded input generators); nothing here touches
the CUDA path.  Usage:  python tests/golden/make_golden.py <workload> [...]
Each workload writes tests/golden/<workload>.json holding rho (FP64, STRANG
end-point treatment) at the listed steps, the eta vector the oracle used, and
the wall time the oracle took.
"""

from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from oracle.eta import Spectral  # noqa: E402
from paper_1205_6872_gb300 import workloads as wl  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))

STEPS = {
    "spin_boson_L6": list(range(0, 101)),
    "biased_L12": list(range(0, 31)) + list(range(40, 401, 10)),
    "three_level_L8": list(range(0, 21)) + list(range(30, 301, 10)),
    "spin_boson_L14": list(range(0, 17)) + [50, 100, 200, 300, 500, 750, 1000],
    "quantum_dot_L11": list(range(0, 21)) + list(range(50, 1001, 50)),
}


def _c(a):
    a = np.asarray(a, dtype=np.complex128)
    return [[float(z.real), float(z.imag)] for z in a.reshape(-1)]


def run_single(name: str):
    p = wl.CONFIGS[name]()
    spec = Spectral(p.jkind, p.ja, p.wc)
    t0 = time.time()
    run = oracle.OracleRun(p.s, p.H, spec, p.beta, p.dt, p.L)
    eta = oracle.pack_eta(run.eta)
    rho = run.run(p.rho0, STEPS[name])
    wall = time.time() - t0
    out = dict(workload=name, M=p.M, L=p.L, N=p.N, endpoint="strang",
               steps=sorted(rho), eta=_c(eta),
               rho={str(k): _c(v) for k, v in sorted(rho.items())},
               oracle_wall_s=wall, oracle_threads=os.environ.get("OMP_NUM_THREADS", "all"))
    with open(os.path.join(HERE, f"{name}.json"), "w") as fh:
        json.dump(out, fh)
    print(f"{name}: {wall:.1f} s")


def run_batched():
    probs = wl.batched_256()
    t0 = time.time()
    res = []
    for i, p in enumerate(probs):
        spec = Spectral(p.jkind, p.ja, p.wc)
        run = oracle.OracleRun(p.s, p.H, spec, p.beta, p.dt, p.L)
        rho = run.run(p.rho0, [p.N])
        res.append(dict(index=i, L=p.L, eta=_c(oracle.pack_eta(run.eta)), rho=_c(rho[p.N])))
    wall = time.time() - t0
    with open(os.path.join(HERE, "batched_256.json"), "w") as fh:
        json.dump(dict(workload="batched_256", N=probs[0].N, instances=res, oracle_wall_s=wall), fh)
    print(f"batched_256: {wall:.1f} s")


def run_pulse_sweep(n=64, L=11, N=200):
    """The paper's pulse-area sweep (Sec. III model, justFinalPoint): rho(t_N) of each instance."""
    probs = wl.pulse_area_sweep(n=n, L=L, N=N)
    t0 = time.time()
    res = []
    for i, p in enumerate(probs):
        spec = Spectral(p.jkind, p.ja, p.wc)
        run = oracle.OracleRun(p.s, p.H, spec, p.beta, p.dt, p.L)
        rho = run.run(p.rho0, [p.N])
        res.append(dict(index=i, omega=float(p.H[0, 1].real * 2.0), eta=_c(oracle.pack_eta(run.eta)),
                        rho=_c(rho[p.N])))
    wall = time.time() - t0
    name = f"pulse_area_sweep_{n}"
    with open(os.path.join(HERE, f"{name}.json"), "w") as fh:
        json.dump(dict(workload=name, L=L, N=N, instances=res, oracle_wall_s=wall,
                       oracle_threads=os.environ.get("OMP_NUM_THREADS", "all")), fh)
    print(f"{name}: {wall:.1f} s")


if __name__ == "__main__":
    for name in sys.argv[1:]:
        if name == "pulse_area_sweep_64":
            run_pulse_sweep()
        elif name == "batched_256":
            run_batched()
        else:
            run_single(name)
