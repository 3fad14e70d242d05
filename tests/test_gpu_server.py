"""Served form: continuous batching of reconstruction requests.

A request's result must not depend on what else runs: each result equals the
plain per-solve path bit for bit, alone and in a mix of different geometries.
Also checks admission under the memory budget and slot count, context reuse,
poll timeouts, unknown tickets, oversized requests and divergence reporting.
"""
import time

import numpy as np
import pytest

from paper_1801_06263_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _problem(n, views, bins, seed, photons=1e5):
    g = inputs.make_geometry(n, 0.5, views, bins)
    sp = inputs.make_spectra(g.n_bins, photons)
    f = inputs.disk_phantom(g, radius_mm=0.4 * n * 0.5, insert_mm=0.06 * n * 0.5)
    return g, sp, f, seed


def _counts(g, sp, f, seed):
    from paper_1801_06263_gb300 import Reconstructor
    R = Reconstructor(g, sp, 1e-7)
    f4 = torch.zeros((g.n_pixels, 4), device="cuda")
    f4[:, :3] = torch.tensor(f, device="cuda")
    chat = R.simulate(f4)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    c = torch.poisson(chat, generator=gen).cpu().numpy().astype(np.float32)
    R.close()
    return c


def _plain(g, sp, c, lam, n_it):
    from paper_1801_06263_gb300 import Reconstructor
    R = Reconstructor(g, sp, lam)
    R.set_counts(torch.tensor(c, device="cuda"))
    R.step(n_it)
    x = R.maps().cpu().numpy()
    R.close()
    return x


@pytest.fixture(scope="module")
def problems():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    out = []
    for (n, v, b, seed) in [(64, 128, 128, 1), (48, 96, 80, 2), (64, 128, 128, 3)]:
        g, sp, f, s = _problem(n, v, b, seed)
        out.append((g, sp, _counts(g, sp, f, s)))
    return out


def _submit(L, srv, g, sp, c, lam, n_it):
    return L.osscir_submit(srv, g, sp.s, sp.N, sp.mu, lam, c, n_it)


def test_served_results_equal_plain_alone_and_in_a_mix(problems):
    from paper_1801_06263_gb300 import _lib as L
    lam, n_it = 1e-7, 40
    plain = [_plain(g, sp, c, lam, n_it) for g, sp, c in problems]
    srv = L.osscir_server_create(8 << 30, 4)
    try:
        # alone
        alone = []
        for g, sp, c in problems:
            t = _submit(L, srv, g, sp, c, lam, n_it)
            out = np.zeros((g.n_pixels, 4), np.float32)
            rc, st = L.osscir_poll(srv, t, -1, out)
            assert rc == 0 and st.status == 0 and st.iterations == n_it
            alone.append(out)
        # in a mix: all submitted before any is collected, plus repeats
        tickets = [(_submit(L, srv, g, sp, c, lam, n_it), i) for rep in range(2)
                   for i, (g, sp, c) in enumerate(problems)]
        for t, i in tickets:
            out = np.zeros((problems[i][0].n_pixels, 4), np.float32)
            rc, st = L.osscir_poll(srv, t, -1, out)
            assert rc == 0
            assert np.array_equal(out[:, :3], plain[i][:, :3])
            assert np.array_equal(out[:, :3], alone[i][:, :3])
            assert st.latency_ms >= st.queue_ms >= 0.0 and st.gpu_ms > 0.0
    finally:
        L.osscir_server_destroy(srv)


def test_admission_respects_budget_and_slots(problems):
    from paper_1801_06263_gb300 import _lib as L
    g, sp, c = problems[0]
    g2, sp2, c2 = problems[1]
    sizes = []
    for pb in problems[:2]:
        probe = L.osscir_server_create(8 << 30, 1)
        try:
            rc, _ = L.osscir_poll(probe, _submit(L, probe, *pb, 1e-7, 1), -1)
            assert rc == 0
            sizes.append(L.osscir_server_info(probe)[2])
        finally:
            L.osscir_server_destroy(probe)
    # a budget that holds a context of either configuration but not both: the two
    # configurations must run one after the other, each reusing its cached context
    budget = max(sizes) + min(sizes) // 2
    srv = L.osscir_server_create(budget, 4)
    try:
        ts = [_submit(L, srv, *(problems[i % 2]), 1e-7, 60) for i in range(4)]
        peak = 0
        for _ in range(5000):
            r, q, b = L.osscir_server_info(srv)
            peak = max(peak, r)
            assert b <= budget
            if r == 0 and q == 0:
                break
            time.sleep(0.001)
        for t in ts:
            rc, st = L.osscir_poll(srv, t, -1)
            assert rc == 0
        assert peak == 1
        assert 0 < L.osscir_server_info(srv)[2] <= budget
    finally:
        L.osscir_server_destroy(srv)


def test_busy_timeout_notfound_and_divergence(problems):
    from paper_1801_06263_gb300 import _lib as L
    g, sp, c = problems[0]
    tiny = L.osscir_server_create(1 << 20, 2)
    try:
        with pytest.raises(L.OsscirError) as e:
            _submit(L, tiny, g, sp, c, 1e-7, 10)
        assert e.value.status == L.OSSCIR_E_BUSY
    finally:
        L.osscir_server_destroy(tiny)
    srv = L.osscir_server_create(4 << 30, 2)
    try:
        rc, _ = L.osscir_poll(srv, 12345, 0)
        assert rc == L.OSSCIR_E_NOTFOUND
        t = _submit(L, srv, g, sp, c, 1e-7, 3000)
        rc, _ = L.osscir_poll(srv, t, 0)
        assert rc == L.OSSCIR_E_TIMEOUT
        rc, st = L.osscir_poll(srv, t, -1)
        assert rc == 0
        with pytest.raises(L.OsscirError):
            _submit(L, srv, g, sp, -c, 1e-7, 10)
        # far too large a step ratio: MOCCA diverges and the request says so
        t = _submit(L, srv, g, sp, c, 1.0, 200)
        rc, st = L.osscir_poll(srv, t, -1)
        assert rc == L.OSSCIR_E_DIVERGED and st.status == L.OSSCIR_E_DIVERGED
    finally:
        L.osscir_server_destroy(srv)
