"""Pins for the oracle's projector X (Eq. fullModel's X_{l,k}: length of ray l in pixel k).

The oracle uses Siddon's incremental method; these tests tie it to an
independent brute-force Liang-Barsky clip of every ray against every pixel,
to the closed-form chord of a ray through the image square and through a
disk, and to the adjoint identity <X x, y> = <x, X^T y>.
"""
import math

import numpy as np
import pytest

from paper_1801_06263_gb300 import inputs

GEOMS = [
    inputs.make_geometry(8, 0.5, 12, 10),
    # odd bin count: the centre ray of view 0 runs exactly along a row boundary
    inputs.make_geometry(8, 0.5, 4, 9),
    # short scan, wide fan, non-dyadic pixel size
    inputs.make_geometry(12, 0.3, 9, 20, sid_mm=100.0, sdd_mm=180.0, arc_deg=200.0,
                         start_deg=17.0),
]


def _endpoints(geom, v, b):
    th = math.radians(geom.start_deg + v * geom.arc_deg / geom.n_views)
    c, s = math.cos(th), math.sin(th)
    u = (b - 0.5 * (geom.n_bins - 1)) * geom.bin_mm
    S = np.array([geom.sid_mm * c, geom.sid_mm * s])
    D = np.array([(geom.sid_mm - geom.sdd_mm) * c - u * s, (geom.sid_mm - geom.sdd_mm) * s + u * c])
    return S, D


def _clip_lengths(geom, S, D):
    """Liang-Barsky clip of segment S->D against every pixel square.  A ray
    parallel to an axis is inside a slab iff lo <= coordinate < hi."""
    n, h = geom.n, geom.pixel_mm
    x0 = -0.5 * n * h
    lo = x0 + np.arange(n) * h
    hi = x0 + (np.arange(n) + 1) * h
    d = D - S
    out = np.zeros(n * n)
    for iy in range(n):
        for ix in range(n):
            t0, t1 = 0.0, 1.0
            ok = True
            for axis, (a, bnd) in enumerate(((lo[ix], hi[ix]), (lo[iy], hi[iy]))):
                if d[axis] == 0.0:
                    if not (a <= S[axis] < bnd):
                        ok = False
                    continue
                ta = (a - S[axis]) / d[axis]
                tb = (bnd - S[axis]) / d[axis]
                t0 = max(t0, min(ta, tb))
                t1 = min(t1, max(ta, tb))
            if ok and t1 > t0:
                out[iy * n + ix] = (t1 - t0) * float(np.hypot(d[0], d[1]))
    return out


@pytest.mark.parametrize("gi", range(len(GEOMS)))
def test_siddon_matches_bruteforce_clip(orc, gi):
    geom = GEOMS[gi]
    thr = 1e-9 * geom.pixel_mm
    for v in range(geom.n_views):
        for b in range(geom.n_bins):
            S, D = _endpoints(geom, v, b)
            So, Do = orc.ray_endpoints(geom, v, b)
            np.testing.assert_allclose(So, S, rtol=0, atol=1e-12)
            np.testing.assert_allclose(Do, D, rtol=0, atol=1e-12)
            ref = _clip_lengths(geom, S, D)
            pix, ln = orc.siddon(geom, v, b)
            want = np.flatnonzero(ref > thr)
            assert sorted(pix.tolist()) == want.tolist(), (v, b)
            got = np.zeros_like(ref)
            got[pix] = ln
            np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12 * geom.pixel_mm)


def test_aligned_ray_uses_closed_low_side(orc):
    geom = GEOMS[1]                       # 9 bins: bin 4 is the centre ray
    pix, ln = orc.siddon(geom, 0, 4)      # view 0: the ray runs along y = 0
    rows = sorted(set((pix // geom.n).tolist()))
    assert rows == [geom.n // 2]          # the row whose low side is y = 0
    assert abs(ln.sum() - geom.n * geom.pixel_mm) < 1e-12


@pytest.mark.parametrize("gi", range(len(GEOMS)))
def test_ray_sum_is_chord_through_image(orc, gi):
    geom = GEOMS[gi]
    ones = np.ones(geom.n_pixels)
    g = orc.forward(geom, ones)
    half = 0.5 * geom.n * geom.pixel_mm
    for l in range(geom.n_rays):
        S, D = _endpoints(geom, l // geom.n_bins, l % geom.n_bins)
        d = D - S
        t0, t1 = 0.0, 1.0
        for a in range(2):
            if d[a] == 0.0:
                continue
            ta, tb = (-half - S[a]) / d[a], (half - S[a]) / d[a]
            t0, t1 = max(t0, min(ta, tb)), min(t1, max(ta, tb))
        chord = max(0.0, t1 - t0) * float(np.hypot(*d))
        assert abs(g[l] - chord) <= 1e-11 * max(1.0, chord)


def test_disk_line_integrals_converge(orc):
    """A rasterised unit disk projects to 2 sqrt(R^2 - d^2); the error of the
    supersampled rasterisation shrinks with the pixel size."""
    R, cx, cy, fov = 3.0, 0.3, -0.2, 12.0
    errs = []
    for n in (16, 32, 64):
        geom = inputs.make_geometry(n, fov / n, 8, 24, bin_mm=0.6)
        f = inputs.rasterize(geom, [inputs.Ellipse(cx, cy, R, R, (1.0, 0.0, 0.0))])[:, 0]
        g = orc.forward(geom, f)
        e = []
        for l in range(geom.n_rays):
            S, D = _endpoints(geom, l // geom.n_bins, l % geom.n_bins)
            u = (D - S) / np.hypot(*(D - S))
            dist = abs((cx - S[0]) * u[1] - (cy - S[1]) * u[0])
            if dist < R - 2 * geom.pixel_mm:
                e.append(abs(g[l] - 2 * math.sqrt(R * R - dist * dist)))
        errs.append(float(np.mean(e)))
    # first order in the pixel size h = fov / n: the error halves as n doubles
    assert 0.4 < errs[1] / errs[0] < 0.6 and 0.4 < errs[2] / errs[1] < 0.6, errs
    assert errs[2] < 0.2 * fov / 64, errs


@pytest.mark.parametrize("gi", range(len(GEOMS)))
def test_adjoint_identity(orc, gi):
    geom = GEOMS[gi]
    x, _ = inputs.random_state(geom, 11)
    rng = np.random.default_rng(12)
    y = rng.normal(size=(geom.n_rays, 3))
    lhs = float(np.sum(orc.forward(geom, x) * y))
    rhs = float(np.sum(x * orc.backproject(geom, y)))
    assert abs(lhs - rhs) <= 1e-13 * (abs(lhs) + abs(rhs) + 1e-300) * 10
    assert abs(lhs - rhs) <= 1e-12 * np.sum(np.abs(orc.forward(geom, np.abs(x)) * np.abs(y)))
