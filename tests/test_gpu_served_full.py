"""The served form at the full size of the mixed request stream that the
benchmark times: 16 requests of 128x128 to 512x512 images, 90-1024 views,
1e4-1e6 photons per ray and 200-500 iterations each (inputs.served_requests),
submitted at once to a server with the benchmark's 150 GB budget and 4 slots,
so that requests of different geometries share batches and streams while
others join and leave.

Each request's maps must equal, bit for bit, what the plain per-solve path
(osscir_reconstruct on a context of its own) returns.  The plain path is
checked against the FP64 oracle at 64x64, 256x256 and 512x512 elsewhere.
"""
import numpy as np
import pytest

from paper_1801_06263_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_full_served_stream_equals_plain():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_06263_gb300 import Reconstructor, _lib
    reqs = inputs.served_requests(16, seed=3000)
    assert {w.geom.n for w in reqs} <= {128, 192, 256, 384, 512}
    lams = [inputs.step_ratio(w.geom.n, w.photons_per_ray) for w in reqs]
    counts, plain = [], []
    for w, lam in zip(reqs, lams):
        R = Reconstructor(w.geom, w.spectra, lam)
        f4 = torch.zeros((w.geom.n_pixels, 4), dtype=torch.float32, device="cuda")
        f4[:, :3] = torch.tensor(w.f_true, dtype=torch.float32, device="cuda")
        c = _lib.osscir_poisson_noise(R.simulate(f4), w.noise_seed).cpu()
        out = torch.empty((w.geom.n_pixels, 4), dtype=torch.float32)
        _lib.osscir_reconstruct(R.handle, c, w.n_iters, out)
        R.close()
        counts.append(c.numpy())
        plain.append(out.numpy())
    srv = _lib.osscir_server_create(150 << 30, 4)
    try:
        tickets = [_lib.osscir_submit(srv, w.geom, w.spectra.s, w.spectra.N, w.spectra.mu, lam, c, w.n_iters)
                   for w, lam, c in zip(reqs, lams, counts)]
        for t, w, ref in zip(tickets, reqs, plain):
            maps = np.zeros((w.geom.n_pixels, 4), dtype=np.float32)
            rc, st = _lib.osscir_poll(srv, t, -1, maps)
            assert rc == 0
            assert np.array_equal(maps.view(np.uint32), ref.view(np.uint32))
    finally:
        _lib.osscir_server_destroy(srv)
