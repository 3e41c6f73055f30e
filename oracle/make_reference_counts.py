"""Run the oracle's GMRES(W) policy iteration (Alg. 2) to completion on the paper-scale dense
workload (S=10^4, A=8, Dirichlet(0.1) rows stored in FP32, gamma=0.99, alpha=0.1, W=30,
tol=1e-8) and store its outer/inner iteration counts and per-phase seconds in
oracle/reference_counts.json.

The benchmark's CPU baseline times a bounded sample of the same computation (one outer
iteration and one Bellman sweep) and scales it to a whole solve with these counts.
Test infrastructure: calls only oracle/ (and the shared seeded generator).
"""
from __future__ import annotations

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import mdp_synth  # noqa: E402
import oracle  # noqa: E402


def main():
    syn = mdp_synth.config(2)
    m = oracle.from_synth(syn)
    t0 = time.perf_counter()
    b = oracle.bellman(m, syn.g[0] * 0.0)
    t_sweep = time.perf_counter() - t0
    t0 = time.perf_counter()
    r = oracle.gmres_policy_iteration(m, alpha=0.1, W=30, tol=1e-8)
    t_all = time.perf_counter() - t0
    out = {
        "config2": {
            "workload": "dense Dirichlet(0.1), S=10000, A=8, FP32 P, gamma=0.99, alpha=0.1, W=30, tol=1e-8",
            "status": r.status, "outer": r.outer, "inner": r.inner, "restarts": r.restarts,
            "sweeps": r.sweeps, "residual": r.residual, "history": r.history,
            "seconds_total": t_all, "seconds_one_sweep": t_sweep,
            "cores": os.cpu_count(),
        }
    }
    path = os.path.join(HERE, "reference_counts.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out))
    del b


if __name__ == "__main__":
    main()
