"""Write tests/golden/oracle_256x128_N32_K6.json with the CPU oracle only.

For each of the three seeded initial conditions of the 256x128, N = 32,
K = 6, Krylov-cap-192 workload: the r^k history, dim S^k, the smallest kept
residual ratio |R_jj|/||a_j|| per iteration (the conditioning of the
Householder basis), the error eps against the serial fine solution
(Eq. errorDef), ||q_N^K||, and 64 entries of q_N^K at fixed seeded indices.
Run: python tests/golden/make_oracle_reference.py   (about 6 minutes, CPU)
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import workloads as W  # noqa: E402


def main():
    wl = W.workload_medium()
    p = wl.problem
    idx = np.sort(np.random.default_rng(12345).choice(p.d, size=64, replace=False))
    out = {"workload": wl.name, "K": wl.K, "krylov_cap": wl.krylov_cap, "eta": 1e-10,
           "sample_indices": idx.tolist(), "ics": {}}
    for name, f in wl.ics:
        q0 = f().ravel()
        r = oracle.parareal(p, q0, wl.K, cap=wl.krylov_cap)
        qs = oracle.serial_fine(p, q0)
        minratio = [float(np.min(r["ratio"][k][r["kept"][k] == 1])) for k in range(wl.K)]
        out["ics"][name] = {
            "r": [float(x) for x in r["r"]], "rank": [int(x) for x in r["rank"]],
            "min_kept_ratio": minratio, "eps": oracle.rel_error(r["q"][-1], qs[-1]),
            "qN_norm": float(np.linalg.norm(r["q"][-1])), "qN_sample": r["q"][-1][idx].tolist(),
            "qseq_sample": qs[-1][idx].tolist(), "qseq_norm": float(np.linalg.norm(qs[-1])),
        }
        print(name, out["ics"][name]["r"], out["ics"][name]["eps"], flush=True)
    with open(os.path.join(HERE, "oracle_256x128_N32_K6.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
