"""Batched form: many solves of different sizes advanced by one launch per
kernel per iteration.

Each solve's iterates, dual, D_TPL and iteration count must equal, bit for bit,
what its own context gives alone (the batched kernels run the same per-ray and
per-pixel arithmetic), for every launch configuration and after autotuning.
The solves cover every back-projection view-group count (8, 4, 2 and 1 thread
groups per pixel), the box-constrained and zero-curvature variants, and the
diagonal SPC and the exp counts model; one plain solve is also checked against
the FP64 oracle.
"""
import numpy as np
import pytest

from paper_1801_06263_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# (n, pixel_mm, views, bins, lambda, options)
SOLVES = [
    (64, 0.5, 128, 128, 1e-7, {}),
    (48, 0.5, 90, 80, 1e-7, {"box": ((0.0, 0.0, 0.0), (1.5, 1.5, 0.05))}),
    (40, 0.6, 60, 72, 3e-8, {"model": 1}),
    (368, 0.1, 24, 64, 1e-7, {}),            # 135,424 pixels: 4 view groups
    (730, 0.05, 8, 16, 1e-7, {}),            # 532,900 pixels: 2 view groups
    (20, 0.9, 1, 9, 1e-7, {}),               # one view: 1 view group
    (33, 0.5, 45, 50, 1e-7, {"spc": 1}),     # diagonal SPC
    (36, 0.5, 50, 60, 1e-7, {"counts_model": 1}),   # the exp counts model
]


def _make(n, px, views, bins, lam, opts, seed):
    from paper_1801_06263_gb300 import Reconstructor
    g = inputs.make_geometry(n, px, views, bins)
    sp = inputs.make_spectra(g.n_bins, 1e5)
    R = Reconstructor(g, sp, lam, **opts)
    f = inputs.disk_phantom(g, radius_mm=0.4 * n * px, insert_mm=0.06 * n * px)
    f4 = torch.zeros((g.n_pixels, 4), device="cuda")
    f4[:, :3] = torch.tensor(f, device="cuda")
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    c = torch.poisson(R.simulate(f4), generator=gen).contiguous()
    R.set_counts(c)
    return R, c, (g, sp)


def _result(R):
    from paper_1801_06263_gb300 import _lib
    x, xbar, y, it = R.get_state()
    torch.cuda.synchronize()
    try:
        d = R.dtpl(1)
    except _lib.OsscirError as e:       # a diverged solve must diverge identically
        assert e.status == _lib.OSSCIR_E_DIVERGED
        d = float("nan")
    return x.cpu().numpy(), xbar.cpu().numpy(), y.cpu().numpy(), it, d


def _same(a, b):
    assert a[3] == b[3]
    for u, v in zip(a[:3], b[:3]):
        assert np.array_equal(u, v, equal_nan=True)
    assert a[4] == b[4] or (np.isnan(a[4]) and np.isnan(b[4]))


@pytest.fixture(scope="module")
def solves():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    out = [_make(*s, seed=10 + i) for i, s in enumerate(SOLVES)]
    yield out
    for R, _, _ in out:
        R.close()


def _plain(solves, n_it):
    ref = []
    for R, c, _ in solves:
        R.set_counts(c)
        R.step(n_it)
        ref.append(_result(R))
    return ref


def test_batch_equals_plain(solves):
    from paper_1801_06263_gb300 import Batch
    n_it = 12
    ref = _plain(solves, n_it)
    for R, c, _ in solves:
        R.set_counts(c)
    assert all(np.isfinite(r[4]) for r in ref)
    B = Batch([R for R, _, _ in solves])
    B.step(n_it)
    for (R, _, _), r in zip(solves, ref):
        _same(_result(R), r)
    ms = B.last_kernel_ms()
    assert all(m > 0 for m in ms)
    B.close()


CONFIGS = [
    dict(proj_views=1, proj_grid=0, proj_order=1, ray_grid=0, ray_order=2, bp_tile_x=4, bp_grid=0, bp_order=1,
         branches=2),
    dict(proj_views=8, proj_grid=152, proj_order=2, ray_grid=300, ray_order=0, bp_tile_x=32, bp_grid=304,
         bp_order=2, branches=4),
    dict(proj_views=2, proj_grid=7, proj_order=0, ray_grid=5, ray_order=1, bp_tile_x=16, bp_grid=3, bp_order=0,
         branches=1),
]


@pytest.mark.parametrize("ci", range(len(CONFIGS)))
def test_every_configuration_gives_the_same_iterates(solves, ci):
    from paper_1801_06263_gb300 import Batch
    n_it = 5
    ref = _plain(solves, n_it)
    for R, c, _ in solves:
        R.set_counts(c)
    B = Batch([R for R, _, _ in reversed(solves)])   # order in the batch does not matter either
    B.config = CONFIGS[ci]
    assert B.config == CONFIGS[ci]
    B.step(n_it)
    for (R, _, _), r in zip(solves, ref):
        _same(_result(R), r)
    B.close()


def test_autotune_keeps_state_and_results(solves):
    from paper_1801_06263_gb300 import Batch, _lib
    n_it = 6
    ref = _plain(solves, n_it)
    for R, c, _ in solves:
        R.set_counts(c)
        R.step(2)            # the batch starts mid-solve
    B = Batch([R for R, _, _ in solves], autotune=True)
    cfg = B.config
    assert cfg["proj_views"] in (1, 2, 4, 8) and cfg["bp_tile_x"] in (2, 4, 8, 16, 32)
    B.step(n_it - 2)
    for (R, _, _), r in zip(solves, ref):
        _same(_result(R), r)
    assert cfg["branches"] in (1, 2, 4)
    with pytest.raises(_lib.OsscirError):
        B.config = dict(cfg, proj_views=3)
    with pytest.raises(_lib.OsscirError):
        B.config = dict(cfg, branches=3)
    B.close()


def test_batched_solve_matches_oracle(orc, solves):
    from paper_1801_06263_gb300 import Batch
    R, c, (g, sp) = solves[0]
    R.set_counts(c)
    B = Batch([R])
    B.step(40)
    x = R.maps().cpu().double().numpy()[:, :3]
    B.close()
    s32 = inputs.Spectra(sp.energies, sp.s.astype(np.float32).astype(np.float64),
                         sp.N.astype(np.float32).astype(np.float64), sp.mu.astype(np.float32).astype(np.float64))
    st, _ = orc.mocca(g, s32, c.cpu().double().numpy(), 40, 1e-7)
    rel = np.linalg.norm(x - st.x, axis=0) / np.linalg.norm(st.x, axis=0)
    assert np.all(rel < 1e-4), rel
