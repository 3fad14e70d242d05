"""Step-ratio sweep for the MOCCA step-preconditioner (Sec. 2: lambda "must be tuned").

Runs the FP64 oracle on a named synthetic workload for a log grid of lambda
(half decades) and prints D_TPL after a fixed number of iterations for each;
the lambda with the smallest final D_TPL among the runs that stayed finite is
the tuned value.  Test and benchmark infrastructure: it calls only the oracle
and the input generator.

    python oracle/tune_lambda.py small_64 200 -8 -4
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import oracle  # noqa: E402
from paper_1801_06263_gb300 import inputs  # noqa: E402


def measured_counts(w):
    cbar = oracle.counts(w.geom, w.spectra, w.f_true)
    return cbar if w.noise_seed is None else inputs.poisson_counts(cbar, w.noise_seed)


def sweep(name: str, n_iters: int, e_lo: float, e_hi: float):
    w = inputs.workload(name)
    c = measured_counts(w)
    rows = []
    for e in np.arange(e_lo, e_hi + 1e-9, 0.5):
        lam = float(10.0 ** e)
        try:
            st, hist = oracle.mocca(w.geom, w.spectra, c, n_iters, lam)
            d = float(hist[-1])
        except np.linalg.LinAlgError:
            d = float("inf")
        if not np.isfinite(d):
            d = float("inf")
        rows.append({"lambda": lam, "dtpl_final": d})
        print(json.dumps(rows[-1]), flush=True)
    best = min(rows, key=lambda r: r["dtpl_final"])
    return best, rows


if __name__ == "__main__":
    name = sys.argv[1] if len(sys.argv) > 1 else "small_64"
    n_it = int(sys.argv[2]) if len(sys.argv) > 2 else 200
    lo = float(sys.argv[3]) if len(sys.argv) > 3 else -8.0
    hi = float(sys.argv[4]) if len(sys.argv) > 4 else -4.0
    best, _ = sweep(name, n_it, lo, hi)
    print(json.dumps({"workload": name, "iterations": n_it, "best": best}))
