"""A full-length reconstruction at 256 x 256 against the FP64 oracle.

The oracle's maps after 500 MOCCA iterations on medium_256 (256 x 256 pixels,
512 views x 512 bins, seeded Poisson counts) are stored in
tests/golden/oracle_medium_256_500.npz, written by
tests/golden/make_oracle_reference.py from the oracle alone.  The GPU solve runs
the same 500 iterations from the same counts; every material map must agree to
1e-4 relative L2; the Gd map, the smallest and noisiest of the three, has its
error printed on its own.
"""
import os

import numpy as np
import pytest

from paper_1801_06263_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_medium_256_500.npz")


def test_medium_256_500_iterations_match_oracle(orc):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_06263_gb300 import Reconstructor
    ref = np.load(GOLDEN)
    w = inputs.workload("medium_256")
    assert int(ref["noise_seed"]) == w.noise_seed
    sp = w.spectra
    s32 = inputs.Spectra(sp.energies, sp.s.astype(np.float32).astype(np.float64),
                         sp.N.astype(np.float32).astype(np.float64), sp.mu.astype(np.float32).astype(np.float64))
    c = inputs.poisson_counts(orc.counts(w.geom, s32, w.f_true), w.noise_seed).astype(np.float32)
    n_it, lam = int(ref["n_iters"]), float(ref["lam"])
    R = Reconstructor(w.geom, sp, lam)
    R.set_counts(torch.tensor(c, device="cuda"))
    R.step(n_it)
    x = R.maps().cpu().double().numpy()[:, :3]
    d = R.dtpl(1)
    R.close()
    rel = np.linalg.norm(x - ref["x"], axis=0) / np.linalg.norm(ref["x"], axis=0)
    print(f"\nrel L2 after {n_it} iterations: PMMA {rel[0]:.3e}  Al {rel[1]:.3e}  Gd {rel[2]:.3e}")
    assert np.all(rel < 1e-4), rel
    assert abs(d - ref["dtpl"][-1]) <= 1e-5 * abs(ref["dtpl"][-1])
