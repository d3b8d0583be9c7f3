"""Seeded synthetic inputs for explicit f-x poststack depth migration.

This module only *generates inputs*: acquisition geometry, frequency band,
velocity models, reflectivity and simple zero-offset sections.  It holds none
of the migration method's arithmetic (no transform to frequency, no operator
design, no extrapolation, no imaging), so that the CUDA library and the CPU
oracle can both consume it without sharing any of the method's code.

The paper migrates the SEG/EAGE salt zero-offset section (Sec. IV, Figs. 4-5),
which is not available here.  The workloads below stand in for it: a point
diffractor in constant velocity, a single spike, and seeded layered media with
dipping interfaces and a smoothed high-velocity lens (strong lateral
variation, the case Sec. II and Sec. III single out for f-x extrapolation).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Workload", "DIFFRACTOR_128", "LAYERED_LENS_2048", "LARGE_8192",
    "band_bins", "ricker", "diffractor_section", "spike_section",
    "layered_lens_model", "normal_incidence_section", "batched_lines",
    "Workload3d", "DIFFRACTOR_3D", "LAYERED_LENS_3D", "diffractor_section_3d", "spike_section_3d",
    "layered_lens_model_3d", "normal_incidence_section_3d",
]


@dataclasses.dataclass(frozen=True)
class Workload:
    """Sizes and physical constants of one 2-D migration problem.

    Frequencies f_j = j / (nt * dt) with f_lo <= f_j <= f_hi (DC and Nyquist
    excluded) form the band that is migrated.  ``L`` is the operator
    half-length (2L+1 taps, the N of Eq. 1), ``nk`` the number of wavenumber
    samples in the operator table, ``theta_deg`` the design dip.
    """
    name: str
    nx: int
    dx: float
    nt: int
    dt: float
    nz: int
    dz: float
    f_lo: float
    f_hi: float
    L: int
    nk: int = 1024
    theta_deg: float = 65.0
    seed: int = 0

    @property
    def band(self) -> tuple[int, int]:
        return band_bins(self.nt, self.dt, self.f_lo, self.f_hi)

    @property
    def i0(self) -> int:
        return self.band[0]

    @property
    def nw(self) -> int:
        return self.band[1]

    @property
    def points(self) -> int:
        """Extrapolated points x frequencies of one full migration."""
        return self.nx * self.nz * self.nw


def band_bins(nt: int, dt: float, f_lo: float, f_hi: float) -> tuple[int, int]:
    """First bin and bin count of f_lo <= j/(nt*dt) <= f_hi, 1 <= j < nt/2."""
    df = 1.0 / (nt * dt)
    j0 = max(1, int(math.ceil(f_lo / df - 1e-9)))
    j1 = min((nt - 1) // 2, int(math.floor(f_hi / df + 1e-9)))
    if j1 < j0:
        return j0, 0
    return j0, j1 - j0 + 1


# Point diffractor in constant velocity, 128 traces.
DIFFRACTOR_128 = Workload("diffractor_128", nx=128, dx=10.0, nt=256, dt=0.004,
                          nz=100, dz=5.0, f_lo=5.0, f_hi=60.0, L=12, seed=0)
# Layered medium with dipping interfaces and a lens, 2048 traces x 800 depths.
LAYERED_LENS_2048 = Workload("layered_lens_2048", nx=2048, dx=12.5, nt=2000, dt=0.002,
                             nz=800, dz=5.0, f_lo=5.0, f_hi=60.0, L=12, seed=1)
# Large line, 8192 traces x 2000 depths, 35-tap operators.
LARGE_8192 = Workload("large_8192", nx=8192, dx=6.25, nt=4000, dt=0.002,
                      nz=2000, dz=4.0, f_lo=5.0, f_hi=80.0, L=17, seed=3)


def ricker(t: np.ndarray, fp: float = 25.0) -> np.ndarray:
    """Zero-phase Ricker wavelet (1 - 2 pi^2 fp^2 t^2) exp(-pi^2 fp^2 t^2)."""
    a = (math.pi * fp * t) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


def diffractor_section(w: Workload, x0: float = 640.0, z0: float = 300.0,
                       v: float = 2000.0, fp: float = 25.0) -> np.ndarray:
    """Zero-offset section [nx][nt] (float64) of one point diffractor.

    Exploding-reflector geometry: the event at trace x arrives at the two-way
    time 2 sqrt(z0^2 + (x - x0)^2) / v, with a 25 Hz Ricker wavelet and unit
    amplitude (no spreading).
    """
    x = np.arange(w.nx) * w.dx
    t = np.arange(w.nt) * w.dt
    tx = 2.0 * np.sqrt(z0 * z0 + (x - x0) ** 2) / v
    return ricker(t[None, :] - tx[:, None], fp)


def spike_section(w: Workload, ix: int, it: int) -> np.ndarray:
    """Section [nx][nt] that is zero except d[ix][it] = 1."""
    d = np.zeros((w.nx, w.nt))
    d[ix, it] = 1.0
    return d


def _gaussian_smooth(a: np.ndarray, sigma: float) -> np.ndarray:
    """Separable Gaussian blur (reflecting edges), radius 4 sigma."""
    r = int(math.ceil(4 * sigma))
    k = np.exp(-0.5 * (np.arange(-r, r + 1) / sigma) ** 2)
    k /= k.sum()
    out = a
    for axis in (0, 1):
        pad = [(0, 0), (0, 0)]
        pad[axis] = (r, r)
        p = np.pad(out, pad, mode="reflect")
        acc = np.zeros_like(out)
        for i in range(2 * r + 1):
            sl = [slice(None), slice(None)]
            sl[axis] = slice(i, i + out.shape[axis])
            acc += k[i] * p[tuple(sl)]
        out = acc
    return out


def layered_lens_model(w: Workload, seed: int | None = None, n_interfaces: int = 8,
                       v_top: float = 1500.0, v_range=(1800.0, 4200.0),
                       v_lens: float = 4500.0, lens: bool = True):
    """Seeded medium velocity v[nz][nx] (float64, m/s) and reflectivity.

    Eight interfaces z_j(x) = z0_j + tan(alpha_j) (x - X/2) with
    z0_j ~ U(0.05, 0.95) Z and alpha_j ~ U(-20, 20) degrees; the layer index at
    (x, z) counts the interfaces above z.  Layer 0 has v_top, the layers below
    draw U(1800, 4200) m/s.  A lens (ellipse, centre x in the middle half,
    z in 30-60 % of Z, semi-axes X/8 and Z/10) is blended toward 4500 m/s
    through its Gaussian-smoothed (sigma = 5 samples) indicator, and the model
    is clipped to [1500, 4500].  Reflectivity is +-1 (seeded) at every cell
    where the layer index changes from the row above.
    """
    rng = np.random.default_rng(w.seed if seed is None else seed)
    X, Z = w.nx * w.dx, w.nz * w.dz
    x = np.arange(w.nx) * w.dx
    z = np.arange(w.nz) * w.dz
    z0 = rng.uniform(0.05, 0.95, n_interfaces) * Z
    alpha = np.radians(rng.uniform(-20.0, 20.0, n_interfaces))
    vl = np.concatenate([[v_top], rng.uniform(v_range[0], v_range[1], n_interfaces)])
    zi = z0[:, None] + np.tan(alpha)[:, None] * (x[None, :] - X / 2)     # [ni][nx]
    layer = (zi[None, :, :] <= z[:, None, None]).sum(axis=1)           # [nz][nx]
    v = vl[layer]
    if lens:
        cx = rng.uniform(0.25, 0.75) * X
        cz = rng.uniform(0.30, 0.60) * Z
        ind = (((x[None, :] - cx) / (X / 8)) ** 2 + ((z[:, None] - cz) / (Z / 10)) ** 2 <= 1.0)
        s = _gaussian_smooth(ind.astype(np.float64), 5.0)
        v = v + s * (v_lens - v)
    v = np.clip(v, v_top, v_lens)
    change = np.zeros_like(layer, dtype=bool)
    change[1:] = layer[1:] != layer[:-1]
    refl = np.where(change, rng.choice([-1.0, 1.0], size=layer.shape), 0.0)
    return v, refl


def normal_incidence_section(w: Workload, v: np.ndarray, refl: np.ndarray,
                             seed: int | None = None, fp: float = 25.0,
                             noise: float = 0.01) -> np.ndarray:
    """Zero-offset section [nx][nt] from vertical two-way times.

    Each trace is the sum of Ricker wavelets r(t - T(x, z)) weighted by the
    reflectivity, with T(x, z) = 2 sum_{z' < z} dz / v(x, z') the vertical
    two-way time, plus Gaussian noise of ``noise`` times the section rms.
    This is a cheap stand-in with the spectrum, amplitudes and event density of
    the layered models; it carries no dips or diffractions.
    """
    rng = np.random.default_rng((w.seed if seed is None else seed) + 7919)
    T = 2.0 * np.concatenate([np.zeros((1, w.nx)), np.cumsum(w.dz / v, axis=0)[:-1]], axis=0)
    t = np.arange(w.nt) * w.dt
    d = np.zeros((w.nx, w.nt))
    iz, ix = np.nonzero(refl)
    half = int(math.ceil(0.08 / w.dt))
    for zz, xx in zip(iz, ix):
        c = T[zz, xx]
        k0 = max(0, int(c / w.dt) - half)
        k1 = min(w.nt, int(c / w.dt) + half + 1)
        if k0 < k1:
            d[xx, k0:k1] += refl[zz, xx] * ricker(t[k0:k1] - c, fp)
    rms = math.sqrt(float(np.mean(d * d))) or 1.0
    d += rng.normal(0.0, noise * rms, d.shape)
    return d


def batched_lines(n_lines: int = 64, seed0: int = 1000):
    """Workloads of the batched-lines case: uneven Nx, Nz, band and L."""
    out = []
    for i in range(n_lines):
        rng = np.random.default_rng(seed0 + i)
        nx = int(rng.integers(512, 8193))
        nz = int(rng.integers(200, 1501))
        f_hi = float(rng.integers(40, 81))
        L = int(rng.choice([8, 12, 17]))
        out.append(Workload(f"line_{i}", nx=nx, dx=12.5, nt=2000, dt=0.002, nz=nz,
                            dz=5.0, f_lo=5.0, f_hi=f_hi, L=L, seed=seed0 + i))
    return out


def mlp_init(seed: int = 2, hidden: int = 64, n_out: int = 26, input_scale: float = 8.0) -> "np.ndarray":
    """Seeded initial parameters of the operator network, flat in the order
    W1, b1, W2, b2, W3, b3, W4, b4 (each row-major, W[out][in]).  The scalar
    input lies in [0, 1]: W1 ~ N(0, input_scale^2) and b1 = -W1 c with
    c ~ U(0, 1), so the first-layer units bend at points spread over the
    input range; the other weights are N(0, 1/fan_in) and their biases zero.
    The draws are inputs shared by the network code and its oracle."""
    rng = np.random.default_rng(seed)
    W1 = rng.normal(0.0, input_scale, (hidden, 1))
    b1 = -W1[:, 0] * rng.uniform(0.0, 1.0, hidden)
    parts = [W1.ravel(), b1]
    for fan_in, fan_out in ((hidden, hidden), (hidden, hidden), (hidden, n_out)):
        parts.append(rng.normal(0.0, 1.0 / math.sqrt(fan_in), (fan_out, fan_in)).ravel())
        parts.append(np.zeros(fan_out))
    return np.concatenate(parts)


# ------------------------------------------------------------------ 3-D grids
@dataclasses.dataclass(frozen=True)
class Workload3d:
    """Sizes of one 3-D migration problem: nx x ny surface points with one
    spacing dx, nz depth rows of dz; the band, L (the 2-D operator's
    half-length: a (2L+1) x (2L+1) stencil) and the table as in Workload."""
    name: str
    nx: int
    ny: int
    dx: float
    nt: int
    dt: float
    nz: int
    dz: float
    f_lo: float
    f_hi: float
    L: int
    nk: int = 512
    theta_deg: float = 65.0
    seed: int = 0

    @property
    def band(self) -> tuple[int, int]:
        return band_bins(self.nt, self.dt, self.f_lo, self.f_hi)

    @property
    def i0(self) -> int:
        return self.band[0]

    @property
    def nw(self) -> int:
        return self.band[1]

    @property
    def points(self) -> int:
        return self.nx * self.ny * self.nz * self.nw


# Point diffractor in constant velocity on a 40 x 40 grid.
DIFFRACTOR_3D = Workload3d("diffractor_3d", nx=40, ny=40, dx=20.0, nt=256, dt=0.004, nz=40, dz=10.0,
                           f_lo=5.0, f_hi=40.0, L=6, nk=256, seed=0)
# Layered medium with dipping planes and a lens, 128 x 128 points x 150 depths.
LAYERED_LENS_3D = Workload3d("layered_lens_3d", nx=128, ny=128, dx=20.0, nt=512, dt=0.004, nz=150, dz=10.0,
                             f_lo=5.0, f_hi=40.0, L=6, nk=512, seed=5)


def diffractor_section_3d(w: Workload3d, x0: float, y0: float, z0: float, v: float,
                          fp: float = 25.0) -> np.ndarray:
    """Zero-offset section [ny][nx][nt] of one point diffractor (two-way time
    2 sqrt(z0^2 + r^2) / v, Ricker wavelet, unit amplitude)."""
    x = np.arange(w.nx) * w.dx
    y = np.arange(w.ny) * w.dx
    t = np.arange(w.nt) * w.dt
    r2 = (x[None, :] - x0) ** 2 + (y[:, None] - y0) ** 2
    tx = 2.0 * np.sqrt(z0 * z0 + r2) / v
    return ricker(t[None, None, :] - tx[:, :, None], fp)


def spike_section_3d(w: Workload3d, ix: int, iy: int, it: int) -> np.ndarray:
    """Section [ny][nx][nt] that is zero except d[iy][ix][it] = 1."""
    d = np.zeros((w.ny, w.nx, w.nt))
    d[iy, ix, it] = 1.0
    return d


def layered_lens_model_3d(w: Workload3d, n_interfaces: int = 6, v_top: float = 1500.0,
                          v_range=(1800.0, 4200.0), v_lens: float = 4500.0):
    """Seeded medium velocity v[nz][ny][nx] (float64, m/s) and reflectivity.

    Planar interfaces z_j(x, y) = z0_j + tan(a_j)(x - X/2) + tan(b_j)(y - Y/2)
    with z0_j ~ U(0.05, 0.95) Z and a_j, b_j ~ U(-15, 15) degrees; layer 0 has
    v_top, the layers below U(1800, 4200) m/s.  A lens (ellipsoid with
    semi-axes X/6, Y/6, Z/8, centre in the middle half laterally and 30-60 %
    of Z) is blended toward 4500 m/s through its Gaussian-smoothed (sigma = 2
    samples) indicator.  Reflectivity is +-1 where the layer index changes
    from the row above.
    """
    rng = np.random.default_rng(w.seed)
    X, Y, Z = w.nx * w.dx, w.ny * w.dx, w.nz * w.dz
    x = np.arange(w.nx) * w.dx
    y = np.arange(w.ny) * w.dx
    z = np.arange(w.nz) * w.dz
    z0 = rng.uniform(0.05, 0.95, n_interfaces) * Z
    ta = np.tan(np.radians(rng.uniform(-15.0, 15.0, n_interfaces)))
    tb = np.tan(np.radians(rng.uniform(-15.0, 15.0, n_interfaces)))
    vl = np.concatenate([[v_top], rng.uniform(v_range[0], v_range[1], n_interfaces)])
    zi = z0[:, None, None] + ta[:, None, None] * (x[None, None, :] - X / 2) + tb[:, None, None] * (y[None, :, None] - Y / 2)
    layer = np.zeros((w.nz, w.ny, w.nx), dtype=np.int64)
    for j in range(n_interfaces):
        layer += (zi[j][None, :, :] <= z[:, None, None])
    v = vl[layer]
    cx, cy, cz = rng.uniform(0.25, 0.75) * X, rng.uniform(0.25, 0.75) * Y, rng.uniform(0.3, 0.6) * Z
    ind = ((((x[None, None, :] - cx) / (X / 6)) ** 2 + ((y[None, :, None] - cy) / (Y / 6)) ** 2
            + ((z[:, None, None] - cz) / (Z / 8)) ** 2) <= 1.0).astype(np.float64)
    r = 8
    k = np.exp(-0.5 * (np.arange(-r, r + 1) / 2.0) ** 2)
    k /= k.sum()
    s = ind
    for axis in range(3):
        pad = [(0, 0)] * 3
        pad[axis] = (r, r)
        p = np.pad(s, pad, mode="reflect")
        acc = np.zeros_like(s)
        for i in range(2 * r + 1):
            sl = [slice(None)] * 3
            sl[axis] = slice(i, i + s.shape[axis])
            acc += k[i] * p[tuple(sl)]
        s = acc
    v = np.clip(v + s * (v_lens - v), v_top, v_lens)
    change = np.zeros_like(layer, dtype=bool)
    change[1:] = layer[1:] != layer[:-1]
    refl = np.where(change, rng.choice([-1.0, 1.0], size=layer.shape), 0.0)
    return v, refl


def normal_incidence_section_3d(w: Workload3d, v: np.ndarray, refl: np.ndarray, fp: float = 25.0,
                                noise: float = 0.01) -> np.ndarray:
    """Zero-offset section [ny][nx][nt] from vertical two-way times (as
    normal_incidence_section, trace by trace), plus Gaussian noise of
    ``noise`` times the section rms."""
    rng = np.random.default_rng(w.seed + 7919)
    T = 2.0 * np.concatenate([np.zeros((1, w.ny, w.nx)), np.cumsum(w.dz / v, axis=0)[:-1]], axis=0)
    t = np.arange(w.nt) * w.dt
    d = np.zeros((w.ny, w.nx, w.nt))
    half = int(math.ceil(0.08 / w.dt))
    iz, iy, ix = np.nonzero(refl)
    for zz, yy, xx in zip(iz, iy, ix):
        c = T[zz, yy, xx]
        k0 = max(0, int(c / w.dt) - half)
        k1 = min(w.nt, int(c / w.dt) + half + 1)
        if k0 < k1:
            d[yy, xx, k0:k1] += refl[zz, yy, xx] * ricker(t[k0:k1] - c, fp)
    rms = math.sqrt(float(np.mean(d * d))) or 1.0
    d += rng.normal(0.0, noise * rms, d.shape)
    return d
