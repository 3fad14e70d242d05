"""The batched form at the full size of the 64-solve mixed batch that the
benchmark times (image sides 128-512, 90-720 views, 1e4-1e6 photons per ray,
each solve with its own phantom, noise seed and step ratio; inputs.batch_workloads).

Every solve's state after two iterations of the batch (the default launch
configuration, then the autotuned one) must equal, bit for bit, the state its
own context reaches alone.  The plain per-solve path is checked against the
FP64 oracle at 64x64, 256x256 and 512x512 elsewhere, so this carries the
oracle parity over to the batch at its benchmarked size.
"""
import numpy as np
import pytest

from paper_1801_06263_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N_IT = 2


def _state(R):
    x, xbar, y, it = R.get_state()
    torch.cuda.synchronize()
    return x.cpu().numpy(), xbar.cpu().numpy(), y.cpu().numpy(), it


def _same(a, b):
    assert a[3] == b[3]
    for u, v in zip(a[:3], b[:3]):
        assert np.array_equal(u.view(np.uint32), v.view(np.uint32))


@pytest.fixture(scope="module")
def batch64():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_06263_gb300 import Reconstructor, _lib
    ws = inputs.batch_workloads(64)
    recs, counts = [], []
    for w in ws:
        R = Reconstructor(w.geom, w.spectra, inputs.step_ratio(w.geom.n, w.photons_per_ray))
        f4 = torch.zeros((w.geom.n_pixels, 4), dtype=torch.float32, device="cuda")
        f4[:, :3] = torch.tensor(w.f_true, dtype=torch.float32, device="cuda")
        c = _lib.osscir_poisson_noise(R.simulate(f4), w.noise_seed)
        recs.append(R)
        counts.append(c)
    ref = []
    for R, c in zip(recs, counts):   # each solve alone
        R.set_counts(c)
        R.step(N_IT)
        ref.append(_state(R))
    yield ws, recs, counts, ref
    for R in recs:
        R.close()


def test_full_batch_default_configuration_equals_plain(batch64):
    from paper_1801_06263_gb300 import Batch
    ws, recs, counts, ref = batch64
    assert len(ws) == 64 and {w.geom.n for w in ws} == {128, 192, 256, 384, 512}
    for R, c in zip(recs, counts):
        R.set_counts(c)
    B = Batch(recs)
    B.step(N_IT)
    for R, r in zip(recs, ref):
        _same(_state(R), r)
    B.close()


def test_full_batch_autotuned_equals_plain(batch64):
    from paper_1801_06263_gb300 import Batch
    ws, recs, counts, ref = batch64
    for R, c in zip(recs, counts):
        R.set_counts(c)
    B = Batch(recs, autotune=True)   # the tuner restores every solve's state after its trials
    B.step(N_IT)
    for R, r in zip(recs, ref):
        _same(_state(R), r)
    B.close()
