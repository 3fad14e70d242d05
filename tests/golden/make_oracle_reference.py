"""Write the FP64 oracle's material maps after a full reconstruction of a named
workload (calls only the oracle and the input generator).

    python tests/golden/make_oracle_reference.py medium_256 500 OUT.npz

The output holds x (float64 [P, 3]), the D_TPL history, the counts' seed and
lambda; the GPU parity check for full-length solves compares against it.
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1801_06263_gb300 import inputs  # noqa: E402

LAMBDA = {"small_64": 1e-7, "medium_256": 10.0 ** -7.5}


def main(name, n_iters, out):
    w = inputs.workload(name)
    sp = w.spectra
    s32 = inputs.Spectra(sp.energies, sp.s.astype(np.float32).astype(np.float64),
                         sp.N.astype(np.float32).astype(np.float64), sp.mu.astype(np.float32).astype(np.float64))
    c = inputs.poisson_counts(oracle.counts(w.geom, s32, w.f_true), w.noise_seed).astype(np.float32)
    st, hist = oracle.mocca(w.geom, s32, c.astype(np.float64), n_iters, LAMBDA[name])
    np.savez_compressed(out, x=st.x, dtpl=hist, lam=LAMBDA[name], n_iters=n_iters, noise_seed=w.noise_seed)


if __name__ == "__main__":
    main(sys.argv[1], int(sys.argv[2]), sys.argv[3])
