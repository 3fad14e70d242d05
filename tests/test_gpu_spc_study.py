"""Which step-preconditioner converges fastest (Sec. 3, Fig. 3), under each reading.

The paper reports, on noiseless data (its "inverse crime" setting), that the
m-block-diagonal SPC converges faster than mu-PC and that the diagonal SPC of
Pock and Chambolle fails for every step ratio lambda.  The MOCCA local quadratic
and mu-PC are both details the paper leaves to Barber et al. 2016, so this
study runs every pairing of a preconditioner with a curvature reading on the
same noiseless small_64 data (64 x 64 pixels, 128 x 128 rays, counts c =
c^(f_true) from the FP64 oracle), 2000 iterations as in Sec. 3, each with its
own best lambda on a quarter-decade grid (1e-11 .. 1e1; best = smallest final
D_TPL among the runs that stay finite):

  preconditioners  block      m-block SPC (spc = 0)
                   mu_pc      mu-PC, Euclidean inner product over the energy grid (spc = 2)
                   mu_pc_phi  mu-PC, inner product weighted by the detected spectrum
                              sum_w N_w s_w(E) (curves transformed by the caller, spc = 1)
                   diagonal   the diagonal SPC in the original basis (spc = 1)
  curvatures       hessian    the per-ray Hessian with its negative eigenvalues removed (model 0)
                   gauss_newton  its first term alone, sum_w c_w a_w a_w^T (model 2)
                   separable  W = diag(c) on the window line integrals (model 3)

It prints D_TPL at the maps and the Gd relative error after 100, 200, 1000 and
2000 iterations for each pairing, and asserts what holds: the diagonal SPC is
orders of magnitude behind the block SPC under every reading (the paper's
finding); with the separable and Gauss-Newton curvatures the block SPC beats
both forms of mu-PC (the paper's Fig. 3 ordering), while with the clipped
Hessian it does not.
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


def _run(w, c, lam, model, spc, mu, M):   # noqa: PLR0913
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
    precs = {"block": (0, None, None), "mu_pc": (2, None, None), "mu_pc_phi": (1, mu_phi, M_phi),
             "diagonal": (1, None, None)}
    curvs = {"hessian": 0, "gauss_newton": 2, "separable": 3}
    best = {}
    for cname, model in curvs.items():
        for pname, (spc, mu, M) in precs.items():
            runs = [(lam, _run(w, c, float(lam), model, spc, mu, M)) for lam in GRID]
            lam, rows = min(runs, key=lambda r: r[1][-1][0])
            best[(pname, cname)] = (lam, rows)
    print("\nnoiseless small_64, D_TPL at the maps / Gd rel. error after " + ", ".join(map(str, MARKS)) + " iterations")
    for (pname, cname), (lam, rows) in best.items():
        cells = "  ".join(f"{d:9.3e} / {gd:8.2e}" for d, gd in rows)
        print(f"{pname:10s} {cname:12s} lambda {lam:8.2e}  {cells}")
    final = {k: v[1][-1][0] for k, v in best.items()}
    for cname in curvs:
        assert final[("block", cname)] < 1e-2 * final[("diagonal", cname)], (cname, final)
    for cname in ("separable", "gauss_newton"):
        for pname in ("mu_pc", "mu_pc_phi"):
            assert final[("block", cname)] < final[(pname, cname)], (cname, pname, final)
    assert final[("mu_pc", "hessian")] < final[("block", "hessian")], final
