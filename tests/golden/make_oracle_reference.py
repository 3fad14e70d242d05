"""Write the FP64 oracle's material maps after a reconstruction of a named
workload (calls only the oracle and the input generator).

    python tests/golden/make_oracle_reference.py medium_256 500 OUT.npz
    python tests/golden/make_oracle_reference.py large_512 100 OUT.npz --f32 --keep 20

The output holds x (float64 [P, 3]; with --f32 rounded to float32, which is
far below the 1e-4 relative tolerance the GPU is held to), the D_TPL history,
the counts' seed, lambda and the oracle's seconds per iteration and thread
count on the machine that wrote it; --keep k also stores the maps after k
iterations as x_k.  The GPU parity checks for long solves compare against it.
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1801_06263_gb300 import inputs  # noqa: E402

LAMBDA = {"small_64": 1e-7, "medium_256": 10.0 ** -7.5, "large_512": 10.0 ** -8.5}


def main(name, n_iters, out, f32=False, keep=()):
    w = inputs.workload(name)
    sp = w.spectra
    s32 = inputs.Spectra(sp.energies, sp.s.astype(np.float32).astype(np.float64),
                         sp.N.astype(np.float32).astype(np.float64), sp.mu.astype(np.float32).astype(np.float64))
    c = inputs.poisson_counts(oracle.counts(w.geom, s32, w.f_true), w.noise_seed).astype(np.float32)
    c64 = c.astype(np.float64)
    lam = LAMBDA[name]
    st, hist, extra, done = None, [], {}, 0
    t0 = time.perf_counter()
    for stop in sorted(set(k for k in keep if 0 < k < n_iters)) + [n_iters]:
        st, h = oracle.mocca(w.geom, s32, c64, stop - done, lam, st)
        hist.append(h)
        done = stop
        if stop != n_iters:
            extra[f"x_{stop}"] = st.x.astype(np.float32) if f32 else st.x.copy()
        print(f"{name}: {done} iterations, {time.perf_counter() - t0:.1f} s", flush=True)
    sec = (time.perf_counter() - t0) / n_iters
    x = st.x.astype(np.float32) if f32 else st.x
    np.savez_compressed(out, x=x, dtpl=np.concatenate(hist), lam=lam, n_iters=n_iters, noise_seed=w.noise_seed,
                        oracle_s_per_iteration=sec, oracle_threads=oracle.max_threads(), **extra)


if __name__ == "__main__":
    args = sys.argv[1:]
    f32 = "--f32" in args
    keep = []
    if "--keep" in args:
        i = args.index("--keep")
        keep = [int(v) for v in args[i + 1].split(",")]
        del args[i:i + 2]
    args = [a for a in args if a != "--f32"]
    main(args[0], int(args[1]), args[2], f32=f32, keep=keep)
