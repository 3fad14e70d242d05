"""Seeded synthetic inputs for three-material spectral CT (no reconstruction arithmetic).

This module builds everything a reconstruction takes as *input*: the fan-beam
geometry, the energy grid, parametric attenuation curves for the PMMA / Al / Gd
basis, the normalised window responses s_{w,l,i} and incident photon numbers
N_{w,l} of Eq. (fullModel), and rasterised phantom maps f_{k,m}.  It contains
none of the method's arithmetic (no projection, no counts model, no objective,
no MOCCA step): the expected counts of a phantom are produced either by the
FP64 oracle (tests) or by the library's own forward model (benchmarks), and
only the Poisson draw on top of them lives here.

Physics stand-ins (the paper's calibrated spectra and tabulated attenuation
data are not available, Sec. 3):
  * energies E_i = 20, 21, ..., 120 keV (1 keV bins);
  * mu_m(E) = a_m (E/30)^-3 J_m(E) + b_m sigma_KN(E)/sigma_KN(30 keV), with the
    textbook Klein-Nishina total cross-section and a Gd K-edge jump J = j_K for
    E >= 50.2 keV (Eq. matdecomp expresses mu as a sum of material terms);
  * a Kramers-like 120 kVp spectrum filtered by 1 mm Al, with seeded jitter;
  * four overlapping windows 20-40-50-65-120 keV whose inner edges are
    jittered per detector bin (the per-pixel response variation of Sec. 3)
    with Gaussian (sigma = 5 keV) roll-off;
  * the five-window variant (Sec. 1 recalls an earlier simulation with five
    ideal windows, sharp edges and no overlap, without giving the edges): the
    same layout with 65-120 keV split at 80 keV, 20-40-50-65-80-120 keV;
  * s_{w,b,i} normalised so that sum_i s = 1 (Eq. fullModel), and
    N_{w,b} = N0 * sum_i Phi_i R_{w,b}(E_i).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

N_WINDOWS = 4
N_MATERIALS = 3
MATERIALS = ("PMMA", "Al", "Gd")

# Synthetic material constants (1/mm per unit density fraction).
MU_A = {"PMMA": 0.012, "Al": 0.25, "Gd": 30.0}
MU_B = {"PMMA": 0.022, "Al": 0.06, "Gd": 0.3}
GD_K_EDGE_KEV = 50.2
GD_K_JUMP = 5.0
WINDOW_EDGES_KEV = (20.0, 40.0, 50.0, 65.0, 120.0)
WINDOW_EDGES_5_KEV = (20.0, 40.0, 50.0, 65.0, 80.0, 120.0)
WINDOW_ROLLOFF_KEV = 5.0
KVP = 120.0
FILTER_AL_MM = 1.0


@dataclasses.dataclass(frozen=True)
class Geometry:
    """2-D fan-beam geometry with a flat detector.

    Image: n x n square pixels of side pixel_mm centred on the rotation axis;
    pixel k = iy*n + ix covers [X0 + ix h, X0 + (ix+1) h) x [Y0 + iy h, ...)
    with X0 = Y0 = -n h / 2.  View v has source angle
    start_deg + v * arc_deg / n_views (counter-clockwise), the source at radius
    sid_mm, the detector a line at distance sdd_mm from the source, bin b
    centred at u_b = (b - (n_bins - 1)/2) * bin_mm.  Ray l = v * n_bins + b.
    """

    n: int
    pixel_mm: float
    n_views: int
    n_bins: int
    bin_mm: float
    sid_mm: float = 500.0
    sdd_mm: float = 1000.0
    arc_deg: float = 360.0
    start_deg: float = 0.0

    @property
    def n_pixels(self) -> int:
        return self.n * self.n

    @property
    def n_rays(self) -> int:
        return self.n_views * self.n_bins

    def as_tuple(self):
        return (self.n, self.pixel_mm, self.n_views, self.arc_deg, self.start_deg,
                self.n_bins, self.bin_mm, self.sid_mm, self.sdd_mm)


def default_bin_mm(n: int, pixel_mm: float, n_bins: int, sid_mm: float = 500.0,
                   sdd_mm: float = 1000.0) -> float:
    """Detector pitch such that the fan covers 1.1x the image circumradius."""
    r_c = n * pixel_mm * math.sqrt(2.0) / 2.0
    return 1.1 * (2.0 * r_c * sdd_mm / sid_mm) / n_bins


def make_geometry(n: int, pixel_mm: float, n_views: int, n_bins: int, *,
                  sid_mm: float = 500.0, sdd_mm: float = 1000.0,
                  arc_deg: float = 360.0, start_deg: float = 0.0,
                  bin_mm: float | None = None) -> Geometry:
    if bin_mm is None:
        bin_mm = default_bin_mm(n, pixel_mm, n_bins, sid_mm, sdd_mm)
    return Geometry(n=n, pixel_mm=pixel_mm, n_views=n_views, n_bins=n_bins,
                    bin_mm=bin_mm, sid_mm=sid_mm, sdd_mm=sdd_mm,
                    arc_deg=arc_deg, start_deg=start_deg)


# --------------------------------------------------------------------------- physics tables

def energies_keV(e_lo: float = 20.0, e_hi: float = 120.0, step: float = 1.0) -> np.ndarray:
    return np.arange(e_lo, e_hi + 0.5 * step, step, dtype=np.float64)


def klein_nishina_total(E_keV: np.ndarray) -> np.ndarray:
    """Klein-Nishina total cross-section per electron, in units of 2 pi r_e^2."""
    eps = np.asarray(E_keV, dtype=np.float64) / 511.0
    l = np.log1p(2.0 * eps)
    return ((1.0 + eps) / eps**2 * (2.0 * (1.0 + eps) / (1.0 + 2.0 * eps) - l / eps)
            + l / (2.0 * eps) - (1.0 + 3.0 * eps) / (1.0 + 2.0 * eps) ** 2)


def mu_curves(E_keV: np.ndarray, materials=MATERIALS) -> np.ndarray:
    """Attenuation table mu[m, i] in 1/mm per unit density fraction."""
    E = np.asarray(E_keV, dtype=np.float64)
    kn = klein_nishina_total(E) / klein_nishina_total(np.array([30.0]))[0]
    pe = (E / 30.0) ** -3
    rows = []
    for m in materials:
        jump = np.where(E >= GD_K_EDGE_KEV, GD_K_JUMP, 1.0) if m == "Gd" else 1.0
        rows.append(MU_A[m] * pe * jump + MU_B[m] * kn)
    return np.stack(rows)


def source_spectrum(E_keV: np.ndarray, seed: int = 7) -> np.ndarray:
    """Seeded Kramers-like spectrum Phi_i (sums to 1), 1 mm Al filtration."""
    E = np.asarray(E_keV, dtype=np.float64)
    rng = np.random.default_rng(seed)
    mu_al = mu_curves(E, ("Al",))[0]
    phi = np.clip(KVP - E, 0.0, None) / E * np.exp(-mu_al * FILTER_AL_MM)
    phi = phi * (1.0 + 0.05 * rng.uniform(-1.0, 1.0, size=E.shape))
    return phi / phi.sum()


def _erf(x):
    return np.vectorize(math.erf, otypes=[np.float64])(x)


def window_edges(n_windows: int = N_WINDOWS) -> tuple:
    """Nominal window edges (keV) of the four- or five-window layout."""
    if n_windows == 4:
        return WINDOW_EDGES_KEV
    if n_windows == 5:
        return WINDOW_EDGES_5_KEV
    raise ValueError("4 or 5 windows")


def window_responses(E_keV: np.ndarray, n_bins: int, seed: int = 7, ideal: bool = False,
                     n_windows: int = N_WINDOWS) -> np.ndarray:
    """R[b, i, w]: window responses with per-bin jittered inner edges and Gaussian
    roll-off; ideal=True gives sharp windows [lo, hi) (the last one closed) with
    the nominal edges in every bin, so each energy falls in exactly one window
    (the ideal, non-overlapping photon-counting response the paper contrasts with
    its realistic overlapping windows, Sec. 1)."""
    E = np.asarray(E_keV, dtype=np.float64)
    edges0 = window_edges(n_windows)
    if ideal:
        R = np.zeros((n_bins, E.size, n_windows))
        for w in range(n_windows):
            lo, hi = edges0[w], edges0[w + 1]
            inside = (E >= lo) & ((E < hi) if w < n_windows - 1 else (E <= hi))
            R[:, inside, w] = 1.0
        return R
    rng = np.random.default_rng(seed + 1)
    edges = np.tile(np.asarray(edges0), (n_bins, 1))
    edges[:, 1:-1] += rng.uniform(-1.0, 1.0, size=(n_bins, len(edges0) - 2))
    sq = math.sqrt(2.0) * WINDOW_ROLLOFF_KEV
    R = np.empty((n_bins, E.size, n_windows))
    for w in range(n_windows):
        lo = edges[:, w][:, None]
        hi = edges[:, w + 1][:, None]
        R[:, :, w] = 0.5 * (_erf((E[None, :] - lo) / sq) - _erf((E[None, :] - hi) / sq))
    return R


@dataclasses.dataclass
class Spectra:
    energies: np.ndarray   # [nE] keV
    s: np.ndarray          # [n_bins, nE, W], sum over energies = 1 per (bin, window)
    N: np.ndarray          # [n_bins, W] incident photons per window
    mu: np.ndarray         # [3, nE] 1/mm

    @property
    def n_energies(self) -> int:
        return int(self.energies.size)


def make_spectra(n_bins: int, photons_per_ray: float, *, seed: int = 7,
                 E_keV: np.ndarray | None = None, ideal_windows: bool = False,
                 n_windows: int = N_WINDOWS) -> Spectra:
    E = energies_keV() if E_keV is None else np.asarray(E_keV, dtype=np.float64)
    phi = source_spectrum(E, seed)
    R = window_responses(E, n_bins, seed, ideal=ideal_windows, n_windows=n_windows)
    weighted = phi[None, :, None] * R                  # [b, i, w]
    tot = weighted.sum(axis=1)                         # [b, w]
    s = weighted / tot[:, None, :]
    N = photons_per_ray * tot
    return Spectra(energies=E, s=s, N=N, mu=mu_curves(E))


# --------------------------------------------------------------------------- phantoms

@dataclasses.dataclass(frozen=True)
class Ellipse:
    cx: float
    cy: float
    ax: float
    ay: float
    values: tuple          # (f_PMMA, f_Al, f_Gd) assigned inside (later shapes overwrite)


def rasterize(geom: Geometry, shapes, supersample: int = 4) -> np.ndarray:
    """Pixel maps f[k, m] by supersampled point coverage (area fraction)."""
    n, h = geom.n, geom.pixel_mm
    x0 = -n * h / 2.0
    sub = (np.arange(supersample) + 0.5) / supersample
    xs = x0 + (np.arange(n)[:, None] + sub[None, :]).reshape(-1) * h    # n*ss
    X, Y = np.meshgrid(xs, xs, indexing="xy")                             # [y, x]
    acc = np.zeros((n * supersample, n * supersample, N_MATERIALS))
    for e in shapes:
        inside = ((X - e.cx) / e.ax) ** 2 + ((Y - e.cy) / e.ay) ** 2 <= 1.0
        acc[inside] = np.asarray(e.values, dtype=np.float64)
    f = acc.reshape(n, supersample, n, supersample, N_MATERIALS).mean(axis=(1, 3))
    return f.reshape(n * n, N_MATERIALS)


def disk_phantom(geom: Geometry, radius_mm: float = 14.0, gd_levels=(0.001, 0.01),
                 insert_mm: float = 2.0) -> np.ndarray:
    """PMMA disk with two Al inserts (replacing PMMA) and two Gd inserts (in PMMA)."""
    shapes = [Ellipse(0.0, 0.0, radius_mm, radius_mm, (1.0, 0.0, 0.0))]
    rr = radius_mm / 2.0
    shapes.append(Ellipse(rr, 0.0, insert_mm, insert_mm, (0.0, 1.0, 0.0)))
    shapes.append(Ellipse(-rr, 0.0, insert_mm, insert_mm, (0.0, 1.0, 0.0)))
    shapes.append(Ellipse(0.0, rr, insert_mm, insert_mm, (1.0, 0.0, gd_levels[0])))
    shapes.append(Ellipse(0.0, -rr, insert_mm, insert_mm, (1.0, 0.0, gd_levels[1])))
    return rasterize(geom, shapes)


def ellipse_phantom(geom: Geometry, seed: int, n_al: int = 4,
                    gd_levels=(0.001, 0.002, 0.005, 0.01, 0.015, 0.02),
                    r_min_mm: float = 2.0, r_max_mm: float = 6.0) -> np.ndarray:
    """PMMA ellipse (semi-axes 0.42 n h, 0.34 n h) with Al and Gd inserts placed by
    seeded rejection sampling (non-overlapping, inside the body)."""
    rng = np.random.default_rng(seed)
    nh = geom.n * geom.pixel_mm
    ax, ay = 0.42 * nh, 0.34 * nh
    r_max = min(r_max_mm, 0.12 * min(ax, ay))
    r_min = min(r_min_mm, 0.5 * r_max)
    body = Ellipse(0.0, 0.0, ax, ay, (1.0, 0.0, 0.0))
    kinds = [("Al", None)] * n_al + [("Gd", g) for g in gd_levels]
    placed = []
    for kind, level in kinds:
        for _ in range(10000):
            r = rng.uniform(r_min, r_max)
            cx = rng.uniform(-ax, ax)
            cy = rng.uniform(-ay, ay)
            if (abs(cx) + r) ** 2 / ax**2 + (abs(cy) + r) ** 2 / ay**2 > 0.8:
                continue
            if any((cx - p[0]) ** 2 + (cy - p[1]) ** 2 < (r + p[2] + 1.0) ** 2 for p in placed):
                continue
            placed.append((cx, cy, r, kind, level))
            break
        else:
            raise RuntimeError("could not place insert")
    shapes = [body]
    for cx, cy, r, kind, level in placed:
        vals = (0.0, 1.0, 0.0) if kind == "Al" else (1.0, 0.0, level)
        shapes.append(Ellipse(cx, cy, r, r, vals))
    return rasterize(geom, shapes)


def poisson_counts(cbar: np.ndarray, seed: int) -> np.ndarray:
    """Seeded Poisson draw of measured counts from expected counts."""
    rng = np.random.default_rng(seed)
    return rng.poisson(np.asarray(cbar, dtype=np.float64)).astype(np.float64)


# --------------------------------------------------------------------------- named workloads

@dataclasses.dataclass
class Workload:
    name: str
    geom: Geometry
    spectra: Spectra
    f_true: np.ndarray          # [P, 3]
    photons_per_ray: float
    noise_seed: int | None      # None: noiseless (expected counts used as data)
    n_iters: int


def workload(name: str) -> Workload:
    """Named synthetic workloads.

    small_64:  64x64 (0.5 mm), 128 views x 128 bins, disk phantom, 1e5 photons, 200 iterations
    medium_256: 256x256 (0.5 mm), 512 views x 512 bins, ellipse phantom (4 Al, 6 Gd), 1e5, 500
    large_512: 512x512 (0.5 mm), 1024 views x 1024 bins, ellipse phantom, 1e6, 1000
    tiny_16:   16x16 (0.5 mm), 32 views x 24 bins, disk phantom (noiseless), for pins
    """
    if name == "small_64":
        g = make_geometry(64, 0.5, 128, 128)
        return Workload(name, g, make_spectra(g.n_bins, 1e5), disk_phantom(g), 1e5, 2000, 200)
    if name == "medium_256":
        g = make_geometry(256, 0.5, 512, 512)
        return Workload(name, g, make_spectra(g.n_bins, 1e5), ellipse_phantom(g, 1001), 1e5,
                        2001, 500)
    if name == "large_512":
        g = make_geometry(512, 0.5, 1024, 1024)
        return Workload(name, g, make_spectra(g.n_bins, 1e6), ellipse_phantom(g, 1002), 1e6,
                        2002, 1000)
    if name == "tiny_16":
        g = make_geometry(16, 0.5, 32, 24)
        f = disk_phantom(g, radius_mm=3.2, insert_mm=0.8, gd_levels=(0.003, 0.006))
        return Workload(name, g, make_spectra(g.n_bins, 1e5), f, 1e5, None, 2000)
    raise KeyError(name)


def step_ratio(n: int, photons_per_ray: float) -> float:
    """Step ratio lambda for a solve of size n and dose: the values tuned with the
    oracle (1e-7 at 64 x 64 / 1e5, 10^-7.5 at 256 x 256 / 1e5, 10^-8.5 at
    512 x 512 / 1e6) follow roughly 10^-7.5 (256 / n) (1e5 / N0)^(1/2); half of
    that keeps every size and dose of the batched workloads inside the stable range."""
    return 0.5 * 10.0 ** -7.5 * (256.0 / n) * (1e5 / photons_per_ray) ** 0.5


def batch_workloads(n_solves: int = 64, seed: int = 4000) -> list:
    """Independent reconstructions of uneven sizes for the batched form: n from
    {128, 192, 256, 384, 512} (0.5 mm pixels), views uniform in [90, 720] with as
    many detector bins, dose log-uniform in [1e4, 1e6] photons per ray, and
    their own ellipse phantom (seed 1000 + i) and noise seed (2000 + i)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_solves):
        n = int(rng.choice([128, 192, 256, 384, 512]))
        views = int(rng.integers(90, 721))
        photons = float(10.0 ** rng.uniform(4.0, 6.0))
        g = make_geometry(n, 0.5, views, views)
        out.append(Workload(f"batch_{i}", g, make_spectra(views, photons), ellipse_phantom(g, 1000 + i),
                            photons, 2000 + i, 500))
    return out


def served_requests(n_requests: int = 16, seed: int = 3000) -> list:
    """A stream of mixed reconstruction requests for the served form: n from
    {128, 192, 256, 384, 512} (0.5 mm pixels), views uniform in [90, 1024] with
    as many detector bins, dose log-uniform in [1e4, 1e6] photons per ray,
    iterations uniform in [200, 500], their own ellipse phantom and noise seed."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_requests):
        n = int(rng.choice([128, 192, 256, 384, 512]))
        views = int(rng.integers(90, 1025))
        photons = float(10.0 ** rng.uniform(4.0, 6.0))
        iters = int(rng.integers(200, 501))
        g = make_geometry(n, 0.5, views, views)
        out.append(Workload(f"request_{i}", g, make_spectra(views, photons), ellipse_phantom(g, seed + 100 + i),
                            photons, seed + 200 + i, iters))
    return out


def random_state(geom: Geometry, seed: int, scale: float = 1.0):
    """Seeded random image (float [P,3]) and dual (float [L,4]) for projector tests."""
    rng = np.random.default_rng(seed)
    return (scale * rng.uniform(-1.0, 1.0, size=(geom.n_pixels, 3)),
            scale * rng.uniform(-1.0, 1.0, size=(geom.n_rays, 4)))
