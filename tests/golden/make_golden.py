"""Write oracle-computed expected values that take the oracle minutes.

Calls only the CPU oracle (oracle/) on the seeded inputs of
paper_2301_05726_gb300.synth; nothing here comes from the CUDA path.
Usage: python tests/golden/make_golden.py [name ...]
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from paper_2301_05726_gb300 import synth  # noqa: E402
from oracle import Oracle  # noqa: E402


def write(name, header, rows):
    path = os.path.join(HERE, name)
    with open(path, "w") as f:
        for line in header:
            f.write(f"# {line}\n")
        for r in rows:
            f.write(" ".join(repr(float(x)) if isinstance(x, (float, np.floating)) else str(x) for x in r) + "\n")
    print("wrote", path)


def energy_gradient(cfg, n_factors=None):
    prob = synth.config_problem(cfg)
    if n_factors:
        prob = prob.prefix(n_factors)
    o = Oracle(prob)
    t = time.time()
    keys, amps, cnt = o.apply()
    E, n2 = o.energy(keys, amps)
    E2, g = o.gradient()
    assert E2 == E
    name = f"cfg{cfg}" + (f"_prefix{n_factors}" if n_factors else "")
    write(f"{name}_energy_gradient.txt",
          [f"oracle E and dE/dtheta for {prob.name} (seeded synthetic problem), eps={prob.eps}",
           f"n_det={len(keys)} norm2={n2!r} rotations={cnt['rotations']} oracle_seconds={time.time() - t:.1f}",
           "line 1: E; then one line per factor: k dE/dtheta_k"],
          [[E]] + [[k, g[k]] for k in range(len(g))])


JOBS = {
    "cfg1": lambda: energy_gradient(1),
    "cfg2": lambda: energy_gradient(2),
    "cfg3_prefix60": lambda: energy_gradient(3, 60),
}

if __name__ == "__main__":
    names = sys.argv[1:] or list(JOBS)
    for n in names:
        JOBS[n]()
