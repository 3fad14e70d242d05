"""Which step-preconditioner converges fastest (Sec. 3, Fig. 3), under each reading.

The paper reports, on noiseless data (its "inverse crime" setting), that the
m-block-diagonal SPC converges faster than mu-PC and that the diagonal SPC of
Pock and Chambolle fails for every step ratio lambda.  The MOCCA step and mu-PC
are both details the paper leaves to Barber et al. 2016, so this study runs each
candidate reading on the same noiseless small_64 data (64 x 64 pixels, 128 x 128
rays, counts c = c^(f_true) from the FP64 oracle), 2000 iterations as in Sec. 3,
each with its own best lambda on a quarter-decade grid (1e-11 .. 1e1, best =
smallest final D_TPL among the runs that stay finite):

  block          m-block SPC, curvature = the clipped per-ray Hessian (model 0)
  block_gn       m-block SPC, Gauss-Newton curvature sum_w c_w a_w a_w^T (model 2)
  block_sep      m-block SPC, separable W = diag(c) (model 3)
  mu_pc          mu-PC, Euclidean inner product over the energy grid (spc = 2)
  mu_pc_phi      mu-PC, inner product weighted by the detected spectrum
                 sum_w N_w s_w(E) (the curves transformed by the caller, spc = 1)
  diagonal       the diagonal SPC in the original basis (spc = 1)

It prints D_TPL at the maps and the Gd relative error after 100, 200, 1000 and
2000 iterations for each, and asserts the orderings that hold under these
readings: every form of the block SPC beats the diagonal SPC by orders of
magnitude (the paper's finding), and mu-PC (either inner product) reaches a
lower D_TPL than the block SPC (the opposite of the paper's Fig. 3 ordering,
which none of the readings here reproduces).
"""
import numpy as np
import pytest

from paper_1801_06263_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MARKS = (100, 200, 1000, 2000)
GRID = 10.0 ** np.arange(-11.0, 1.01, 0.25)


def _sp32(sp):
    return inputs.Spectra(sp.energies, sp.s.astype(np.float32).astype(np.float64),
                          sp.N.astype(np.float32).astype(np.float64), sp.mu.astype(np.float32).astype(np.float64))


def _run(w, c, lam, model, spc, mu, M):
    from paper_1801_06263_gb300 import OsscirError, Reconstructor
    R = Reconstructor(w.geom, w.spectra, lam, model=model, spc=spc, mu=mu)
    R.set_counts(c)
    rows, done = [], 0
    for m in MARKS:
        R.step(m - done)
        done = m
        try:
            d = R.dtpl(0)
        except OsscirError:
            d = np.inf
        x = R.maps().cpu().double().numpy()[:, :3]
        if M is not None:   # maps of a caller-transformed basis back to the original one
            x = x @ M.T
        gd = np.linalg.norm(x[:, 2] - w.f_true[:, 2]) / np.linalg.norm(w.f_true[:, 2])
        rows.append((d, gd if np.isfinite(gd) else np.inf))
        if not np.isfinite(d):
            rows += [(np.inf, np.inf)] * (len(MARKS) - len(rows))
            break
    R.close()
    return rows


def test_preconditioner_readings(orc):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    w = inputs.workload("small_64")
    sp = w.spectra
    c = torch.tensor(orc.counts(w.geom, _sp32(sp), w.f_true).astype(np.float32), device="cuda")
    phi = (sp.N[:, None, :] * sp.s).sum(axis=2).mean(axis=0)   # detected photons per energy bin
    mu_phi, M_phi = orc.mu_pc(sp.mu.astype(np.float32).astype(np.float64), weights=phi)
    methods = {"block": (0, 0, None, None), "block_gn": (2, 0, None, None), "block_sep": (3, 0, None, None),
               "mu_pc": (0, 2, None, None), "mu_pc_phi": (0, 1, mu_phi, M_phi), "diagonal": (0, 1, None, None)}
    best = {}
    for name, (model, spc, mu, M) in methods.items():
        runs = [(lam, _run(w, c, float(lam), model, spc, mu, M)) for lam in GRID]
        lam, rows = min(runs, key=lambda r: r[1][-1][0])
        best[name] = (lam, rows)
    print("\nnoiseless small_64, D_TPL at the maps / Gd rel. error after " + ", ".join(map(str, MARKS)) + " iterations")
    for name, (lam, rows) in best.items():
        cells = "  ".join(f"{d:9.3e} / {gd:8.2e}" for d, gd in rows)
        print(f"{name:10s} lambda {lam:8.2e}  {cells}")
    final = {k: v[1][-1][0] for k, v in best.items()}
    for name in ("block", "block_gn", "block_sep"):
        assert final[name] < 1e-2 * final["diagonal"], (name, final)
    assert final["mu_pc"] < final["block"] and final["mu_pc_phi"] < final["block"], final
