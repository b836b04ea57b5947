"""Write the oracle reference of the 256x128 workload with the CPU oracle only.

tests/golden/oracle_256x128_N32_K6.json -- for each of the three seeded
initial conditions of the 256x128, N = 32, K = 6, Krylov-cap-192 workload:
the r^k history, dim S^k, the smallest kept residual ratio |R_jj|/||a_j|| per
iteration (the conditioning of the Householder basis), the error eps against
the serial fine solution (Eq. errorDef), ||q_N^K||, 64 entries of q_N^K and
of the serial fine solution at fixed seeded indices, and the oracle's own
spread: the relative l2 change of q_N^K (and the change of eps) when every
entry of the initial value moves by one unit in the last place (random
direction, two seeds) -- how well the method's result is determined in FP64
arithmetic at all -- and the same for the initial value rounded to FP32.
tests/golden/oracle_256x128_N32_K6_qN.npz -- q_N^K of every initial value in
full (float64), for element-by-element comparison.
Run: python tests/golden/make_oracle_reference.py   (about 10 minutes on 8 cores)
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
    oracle.set_threads(os.cpu_count() or 1)   # the results do not depend on it
    wl = W.workload_medium()
    p = wl.problem
    idx = np.sort(np.random.default_rng(12345).choice(p.d, size=64, replace=False))
    out = {"workload": wl.name, "K": wl.K, "krylov_cap": wl.krylov_cap, "eta": 1e-10,
           "sample_indices": idx.tolist(), "ics": {}}
    full = {}
    for name, f in wl.ics:
        q0 = f().ravel()
        r = oracle.parareal(p, q0, wl.K, cap=wl.krylov_cap)
        qs = oracle.serial_fine(p, q0)
        qN = r["q"][-1]
        eps = oracle.rel_error(qN, qs[-1])
        minratio = [float(np.min(r["ratio"][k][r["kept"][k] == 1])) for k in range(wl.K)]
        spread = []
        for seed in (7, 8):
            sgn = np.random.default_rng(seed).choice([-1.0, 1.0], size=q0.size)
            q1 = np.nextafter(q0, q0 + sgn)
            r1 = oracle.parareal(p, q1, wl.K, cap=wl.krylov_cap)
            qs1 = oracle.serial_fine(p, q1)
            spread.append({"seed": seed,
                           "qN_rel_l2": float(np.linalg.norm(r1["q"][-1] - qN) / np.linalg.norm(qN)),
                           "eps_shift": abs(oracle.rel_error(r1["q"][-1], qs1[-1]) - eps),
                           "rank_equal": bool(np.array_equal(r1["rank"], r["rank"]))})
        # the spread at FP32 input precision: the same solve from the initial
        # value rounded to FP32 (what a solve with FP32 tendencies sees first)
        q32 = q0.astype(np.float32).astype(np.float64)
        r32 = oracle.parareal(p, q32, wl.K, cap=wl.krylov_cap)
        qs32 = oracle.serial_fine(p, q32)
        spread32 = {"qN_rel_l2": float(np.linalg.norm(r32["q"][-1] - qN) / np.linalg.norm(qN)),
                    "eps_shift": abs(oracle.rel_error(r32["q"][-1], qs32[-1]) - eps)}
        full[name] = qN
        out["ics"][name] = {
            "r": [float(x) for x in r["r"]], "rank": [int(x) for x in r["rank"]],
            "min_kept_ratio": minratio, "eps": eps,
            "qN_norm": float(np.linalg.norm(qN)), "qN_sample": qN[idx].tolist(),
            "qseq_sample": qs[-1][idx].tolist(), "qseq_norm": float(np.linalg.norm(qs[-1])),
            "spread_1ulp": spread, "spread_fp32_input": spread32,
        }
        print(name, out["ics"][name]["r"], eps, spread, flush=True)
    with open(os.path.join(HERE, "oracle_256x128_N32_K6.json"), "w") as fh:
        json.dump(out, fh, indent=1)
    np.savez_compressed(os.path.join(HERE, "oracle_256x128_N32_K6_qN.npz"), **full)


if __name__ == "__main__":
    main()
