"""FP64 CPU oracle for explicit f-x poststack depth migration.

TEST INFRASTRUCTURE ONLY.  This package is the slow, plainly written reference
that the CUDA library is checked against.  Only ``tests/``, the smoke check in
``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may import it; the
library never does.  It shares no code with the CUDA sources (the seeded
``workloads`` generators, which hold none of the method's arithmetic, are the
only thing both sides read).

Paper: Shawahna, Salam, Al-Mouhamed, "Seismic Imaging: An Overview and Parallel
Implementation of Poststack Depth Migration", arXiv 1912.05529.

Steps, in the order of Algorithm 1, and what each follows:

* ``band_dft``            Algorithm 1, time-to-frequency step;
                          Sec. III.  Naive DFT, e^{-i w t}, no scaling, band
                          bins only.
* ``design_operators``    Sec. II (design as an optimisation between short and
                          long filters), Sec. III (filters designed in advance
                          and stored).  Weighted least squares against the
                          one-way phase shift exp(i sqrt(k^2 - kx^2) dz), then
                          an amplitude guard so |H| <= 1 (Sec. II: the
                          recursion is unstable unless the design is accurate).
* ``lookup_index``        Sec. III per-point filter choice (C, fp32 index).
* ``step`` / ``migrate``  Eq. 1 and Algorithm 1's depth loop with the
                          depth row summed over frequencies (C, FP64).
* ``model``               exact adjoint of ``migrate``; used only to synthesise
                          test sections (conjugate-operator upward
                          extrapolation of a reflectivity).

Parity status: every function is pinned by a test in ``tests/test_oracle_*.py``
against closed forms, invariants, brute force or an independent library routine.
The comparison with the paper's own SEG/EAGE images is parity unpinned: the
paper's data and figures are not available.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fxo.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "libfxo.so")
_lib = None

__all__ = [
    "build", "band_dft", "omegas", "k_grid", "q_values", "design_operators",
    "response", "lookup_index", "slowness", "step", "adjoint_step", "migrate",
    "model", "band_to_time", "ricker_spectrum", "max_threads",
]


def build(force: bool = False) -> str:
    """Compile ``fxo.c`` into ``_build/libfxo.so`` (gcc, OpenMP, no FP contraction)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fcx-limited-range",
               "-fno-fast-math", "-std=c11", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        f, i, d = ctypes.c_float, ctypes.c_int, ctypes.c_void_p
        lib.fxo_lookup_index.argtypes = [f, f, i]
        lib.fxo_lookup_index.restype = i
        lib.fxo_slowness.argtypes = [f]
        lib.fxo_slowness.restype = f
        lib.fxo_max_threads.restype = i
        lib.fxo_step.argtypes = [i, i, i, i, d, d, d, d, d, i]
        lib.fxo_adjoint_step.argtypes = [i, i, i, i, d, d, d, d, d, i]
        lib.fxo_migrate.argtypes = [i, i, i, i, i, d, d, d, d, i, i, d, i]
        lib.fxo_migrate.restype = i
        lib.fxo_model.argtypes = [i, i, i, i, i, d, d, d, d, d, i]
        lib.fxo_model.restype = i
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def max_threads() -> int:
    """OpenMP threads the C oracle uses by default."""
    return int(_load().fxo_max_threads())


# ---------------------------------------------------------------- frequency axis
def omegas(i0: int, nw: int, nt: int, dt: float) -> np.ndarray:
    """Angular frequencies w_j = 2 pi (i0 + j) / (nt dt) of the band bins."""
    return 2.0 * math.pi * (i0 + np.arange(nw, dtype=np.float64)) / (nt * dt)


def band_dft(section: np.ndarray, i0: int, nw: int) -> np.ndarray:
    """t -> f along the time axis (Algorithm 1), band bins only.

    P[j][x] = sum_{t=0}^{nt-1} d[x][t] exp(-2 pi i (i0+j) t / nt): the forward
    DFT with the e^{-i w t} sign and no 1/nt scaling, evaluated directly as a
    sum (one matrix product) in FP64.  Returns [nw][nx] complex128.
    """
    d = np.asarray(section, dtype=np.float64)
    nt = d.shape[1]
    j = i0 + np.arange(nw, dtype=np.int64)
    t = np.arange(nt, dtype=np.int64)
    phase = (np.outer(t, j) % nt).astype(np.float64) * (2.0 * math.pi / nt)
    E = np.exp(-1j * phase)                      # [nt][nw]
    return np.ascontiguousarray((d @ E).T)


def band_to_time(P: np.ndarray, i0: int, nt: int) -> np.ndarray:
    """Inverse of ``band_dft`` for a band-limited spectrum: [nw][nx] -> [nx][nt].

    The real section whose DFT is P on the band bins and zero elsewhere
    (1/nt scaling, Hermitian extension); used only to synthesise test input.
    """
    nw, nx = P.shape
    spec = np.zeros((nx, nt // 2 + 1), dtype=np.complex128)
    spec[:, i0:i0 + nw] = P.T
    return np.fft.irfft(spec, n=nt, axis=1)


def ricker_spectrum(f: np.ndarray, fp: float = 25.0, dt: float = 1.0) -> np.ndarray:
    """Fourier transform of the zero-phase Ricker wavelet, divided by dt.

    R(f) = 2 f^2 / (sqrt(pi) fp^3) exp(-f^2 / fp^2); the DFT of the sampled,
    centred wavelet is R(f) / dt.
    """
    f = np.asarray(f, dtype=np.float64)
    return 2.0 * f * f / (math.sqrt(math.pi) * fp ** 3) * np.exp(-(f / fp) ** 2) / dt


# ------------------------------------------------------------------ operators
def k_grid(nk: int, k_max: float) -> tuple[np.ndarray, float]:
    """Table wavenumbers k_j = j dk, dk = k_max / (nk - 1)."""
    dk = k_max / (nk - 1) if nk > 1 else 0.0
    return np.arange(nk, dtype=np.float64) * dk, dk


def q_values(w: np.ndarray, dk: float) -> np.ndarray:
    """q_w = fl32(w / dk): the per-frequency factor of the table index."""
    return (np.asarray(w, dtype=np.float64) / dk).astype(np.float32)


def _basis(kx: np.ndarray, dx: float, L: int) -> np.ndarray:
    n = np.arange(L + 1)
    c = np.where(n == 0, 1.0, 2.0)
    return c[None, :] * np.cos(np.outer(kx * dx, n))


def response(h: np.ndarray, kx: np.ndarray, dx: float) -> np.ndarray:
    """Wavenumber response H(kx) = h0 + 2 sum_{n>=1} h_n cos(n kx dx) of
    symmetric taps h[..., 0..L] (the Fourier transform of Eq. 1's filter)."""
    h = np.asarray(h)
    return h @ _basis(np.asarray(kx, dtype=np.float64), dx, h.shape[-1] - 1).T


def design_at(k, dx: float, dz: float, L: int, theta_deg: float = 65.0, stop_weight: float = 1e-2,
              n_samples: int | None = None, guard_points: int = 4096, return_info: bool = False):
    """Weighted least-squares operators (Sec. II, Sec. III) at the wavenumbers k.

    For each k find symmetric taps h[0..L] whose response
    H(kx) = sum_n c_n h_n cos(n kx dx), c_0 = 1, c_n = 2, fits the one-way
    downward phase shift
        D(kx) = exp(+i sqrt(k^2 - kx^2) dz)   for kx <= k   (propagating)
        D(kx) = exp(-sqrt(kx^2 - k^2) dz)     for kx >  k   (evanescent)
    on M = max(256, 16(L+1)) samples kx_m = m pi / (dx (M-1)), with weight 1
    for kx <= k sin(theta) and ``stop_weight`` elsewhere.  Re and Im are fitted
    separately (the basis is real) by Householder QR of sqrt(W) A.  Then the
    amplitude guard: with G = max |H| over ``guard_points`` samples of
    [0, pi/dx], taps are scaled by 1/G when G > 1 (|H| <= 1 keeps the recursion
    of Eq. 1 stable).  Returns [len(k)][L+1] complex128 (and a dict of
    intermediates when ``return_info``).
    """
    k = np.atleast_1d(np.asarray(k, dtype=np.float64))
    M = n_samples or max(256, 16 * (L + 1))
    kx = np.arange(M, dtype=np.float64) * (math.pi / (dx * (M - 1)))
    A = _basis(kx, dx, L)                                      # [M][L+1]
    kz2 = k[:, None] ** 2 - kx[None, :] ** 2                   # [nk][M]
    D = np.where(kz2 >= 0.0,
                 np.exp(1j * np.sqrt(np.maximum(kz2, 0.0)) * dz),
                 np.exp(-np.sqrt(np.maximum(-kz2, 0.0)) * dz))
    W = np.where(kx[None, :] <= k[:, None] * math.sin(math.radians(theta_deg)), 1.0, stop_weight)
    sw = np.sqrt(W)
    B = sw[:, :, None] * A[None, :, :]                         # [nk][M][L+1]
    Q, R = np.linalg.qr(B)                                     # Householder, batched
    rhs = np.einsum("kml,km->kl", Q, sw * D.real) + 1j * np.einsum("kml,km->kl", Q, sw * D.imag)
    h_ls = np.linalg.solve(R, rhs.real[..., None])[..., 0] + 1j * np.linalg.solve(R, rhs.imag[..., None])[..., 0]
    kxd = np.arange(guard_points, dtype=np.float64) * (math.pi / (dx * (guard_points - 1)))
    G = np.abs(h_ls @ _basis(kxd, dx, L).T).max(axis=1)
    scale = np.where(G > 1.0, 1.0 / G, 1.0)
    h = h_ls * scale[:, None]
    if return_info:
        return h, {"k": k, "kx": kx, "A": A, "D": D, "W": W, "h_ls": h_ls, "G": G, "scale": scale,
                   "kx_guard": kxd}
    return h


def design_operators(nk: int, k_max: float, dx: float, dz: float, L: int,
                     theta_deg: float = 65.0, stop_weight: float = 1e-2,
                     n_samples: int | None = None, guard_points: int = 4096,
                     return_info: bool = False):
    """The operator table of Sec. III: ``design_at`` on the grid k_j = j dk,
    dk = k_max / (nk - 1).  Returns [nk][L+1] complex128 (and the
    intermediates, with "dk", when ``return_info``)."""
    k, dk = k_grid(nk, k_max)
    out = design_at(k, dx, dz, L, theta_deg, stop_weight, n_samples, guard_points, return_info)
    if return_info:
        out[1]["dk"] = dk
    return out


# ------------------------------------------------------------ lookup and steps
def lookup_index(q, s, nk: int) -> np.ndarray:
    """Table index rint_half_even(fl32(q s)) clamped to [0, nk-1] (C, fp32)."""
    lib = _load()
    q = np.broadcast_to(np.asarray(q, dtype=np.float32), np.broadcast(q, s).shape)
    s = np.broadcast_to(np.asarray(s, dtype=np.float32), q.shape)
    out = np.empty(q.shape, dtype=np.int64)
    for idx in np.ndindex(q.shape):
        out[idx] = lib.fxo_lookup_index(float(q[idx]), float(s[idx]), int(nk))
    return out


def slowness(v) -> np.ndarray:
    """fl32(1 / v) in IEEE fp32 (C)."""
    lib = _load()
    v = np.asarray(v, dtype=np.float32)
    out = np.empty(v.shape, dtype=np.float32)
    for idx in np.ndindex(v.shape):
        out[idx] = lib.fxo_slowness(float(v[idx]))
    return out


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def step(P: np.ndarray, vrow: np.ndarray, table: np.ndarray, q: np.ndarray,
         nthreads: int = 0) -> np.ndarray:
    """One Eq. 1 step of every line: [nw][nx] -> [nw][nx] (velocity row vrow)."""
    P = _c128(P)
    nw, nx = P.shape
    table = _c128(table)
    nk, L1 = table.shape
    out = np.empty_like(P)
    _load().fxo_step(nx, nw, L1 - 1, nk, _p(_f32(q)), _p(_f32(vrow)), _p(table), _p(P), _p(out), nthreads)
    return out


def adjoint_step(P: np.ndarray, vrow: np.ndarray, table: np.ndarray, q: np.ndarray,
                 nthreads: int = 0) -> np.ndarray:
    """Conjugate transpose of ``step`` with the same velocity row."""
    P = _c128(P)
    nw, nx = P.shape
    table = _c128(table)
    nk, L1 = table.shape
    out = np.empty_like(P)
    _load().fxo_adjoint_step(nx, nw, L1 - 1, nk, _p(_f32(q)), _p(_f32(vrow)), _p(table), _p(P), _p(out), nthreads)
    return out


def migrate(P0: np.ndarray, vel: np.ndarray, table: np.ndarray, q: np.ndarray,
            z_begin: int = 0, z_end: int | None = None, nthreads: int = 0):
    """Algorithm 1's depth loop: returns (P at depth z_end, image [nz][nx]).

    ``vel`` is the [nz][nx] migration velocity (the extrapolation velocity;
    exploding-reflector data use half the medium velocity).  Image rows outside
    [z_begin, z_end) are zero.
    """
    P = _c128(P0).copy()
    nw, nx = P.shape
    vel = _f32(vel)
    nz = vel.shape[0]
    z_end = nz if z_end is None else z_end
    table = _c128(table)
    nk, L1 = table.shape
    image = np.zeros((nz, nx), dtype=np.float64)
    rc = _load().fxo_migrate(nx, nz, nw, L1 - 1, nk, _p(_f32(q)), _p(vel), _p(table), _p(P),
                             int(z_begin), int(z_end), _p(image), nthreads)
    if rc != 0:
        raise MemoryError("oracle migrate: allocation failed")
    return P, image


def model(refl: np.ndarray, vel: np.ndarray, table: np.ndarray, q: np.ndarray,
          nthreads: int = 0) -> np.ndarray:
    """Exact adjoint of ``migrate`` (all rows): reflectivity [nz][nx] -> P0 [nw][nx]."""
    refl = np.ascontiguousarray(refl, dtype=np.float64)
    vel = _f32(vel)
    nz, nx = vel.shape
    table = _c128(table)
    nk, L1 = table.shape
    q = _f32(q)
    out = np.empty((q.shape[0], nx), dtype=np.complex128)
    rc = _load().fxo_model(nx, nz, q.shape[0], L1 - 1, nk, _p(q), _p(vel), _p(table), _p(refl), _p(out), nthreads)
    if rc != 0:
        raise MemoryError("oracle model: allocation failed")
    return out


# ------------------------------------------------- pointwise operators (no table)
def convolve_pointwise(P: np.ndarray, h: np.ndarray) -> np.ndarray:
    """Eq. 1 with its own operator at every output point:
    out[j][x] = h[j][x][0] P[j][x] + sum_{n=1}^{L} h[j][x][n] (P[j][x-n] + P[j][x+n]),
    P = 0 outside [0, nx).  P [nw][nx], h [nw][nx][L+1]; FP64."""
    P = np.asarray(P, dtype=np.complex128)
    h = np.asarray(h, dtype=np.complex128)
    nx = P.shape[1]
    L = h.shape[2] - 1
    Pp = np.pad(P, ((0, 0), (L, L)))
    out = h[:, :, 0] * P
    for n in range(1, L + 1):
        out = out + h[:, :, n] * (Pp[:, L - n:L - n + nx] + Pp[:, L + n:L + n + nx])
    return out


def migrate_pointwise(P0: np.ndarray, vel: np.ndarray, w: np.ndarray, taps_fn,
                      z_begin: int = 0, z_end: int | None = None):
    """Algorithm 1's depth loop with the operator of point (j, x, z) produced by
    ``taps_fn(w_pairs, s_pairs) -> [n][L+1]`` for frequency w_j and slowness
    s = fl32(1 / vel[z][x]) instead of a table row.  The function is called
    once per row on the distinct (w, s) pairs of that row.  Returns (P at
    depth z_end, image [nz][nx]) like ``migrate``; FP64 arithmetic."""
    P = np.asarray(P0, dtype=np.complex128).copy()
    vel = np.asarray(vel, dtype=np.float32)
    nz, nx = vel.shape
    w = np.asarray(w, dtype=np.float64)
    z_end = nz if z_end is None else z_end
    image = np.zeros((nz, nx), dtype=np.float64)
    for z in range(z_begin, z_end):
        image[z] = P.real.sum(axis=0)
        s = slowness(vel[z])
        su, inv = np.unique(s, return_inverse=True)
        h = np.asarray(taps_fn(np.repeat(w, su.size), np.tile(su, w.size)))   # pairs (w_j, su_u), j-major
        L1 = h.shape[1]
        hp = h.reshape(w.size, su.size, L1)[:, inv.ravel(), :]                  # [nw][nx][L+1]
        P = convolve_pointwise(P, hp)
    return P, image


def table_taps_fn(table: np.ndarray, q: np.ndarray, w: np.ndarray):
    """The table lookup of Sec. III as a ``taps_fn``: the row
    rint_half_even(fl32(q_j s)) clamped, q_j the table factor of frequency w_j."""
    table = np.asarray(table)
    w = np.asarray(w, dtype=np.float64)
    q = np.asarray(q, dtype=np.float32)

    def fn(wp, sp):
        j = np.searchsorted(w, wp)
        qs = (q[j] * np.asarray(sp, dtype=np.float32)).astype(np.float32)
        return table[np.clip(np.rint(qs).astype(np.int64), 0, table.shape[0] - 1)]
    return fn


def design_taps_fn(dx: float, dz: float, L: int, theta_deg: float = 65.0):
    """Least-squares operators designed at the exact wavenumber k = w s of every
    point (``design_at``): the continuous-velocity reference, free of table
    quantisation."""
    def fn(wp, sp):
        k = np.asarray(wp, dtype=np.float64) * np.asarray(sp, dtype=np.float32).astype(np.float64)
        ku, inv = np.unique(k, return_inverse=True)
        return design_at(ku, dx, dz, L, theta_deg)[inv.ravel()]
    return fn
