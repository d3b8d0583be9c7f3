"""FP64 CPU oracle for 3-D explicit f-x depth migration with 2-D extrapolators.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may use it.
It shares no code with the CUDA sources.

The paper (Sec. I and Sec. II) notes that explicit f-x migration extends to
3-D depth migration, where the extrapolator becomes a 2-D filter applied by a
2-D spatial convolution over the (x, y) surface grid, frequency by frequency.
This module writes that extension out plainly:

* ``design2d_at`` / ``design2d_operators``  the 2-D counterpart of the Sec. II
  / Sec. III design: a (2L+1) x (2L+1) operator with the symmetries of a
  square grid (h(i, j) = h(-i, j) = h(i, -j) = h(j, i)), fitted by weighted
  least squares to the one-way phase shift exp(i sqrt(k^2 - kx^2 - ky^2) dz)
  on samples of the octant 0 <= ky <= kx <= pi/dx, then the same amplitude
  guard as the 2-D design (|H| <= 1).
* ``orbits``   the unique taps (a, b), a >= b >= 0, and the grid offsets that
  share each one.
* ``step3d`` / ``migrate3d``  Eq. 1 with the sum over the 2-D stencil, the
  operator chosen per output point by the Sec. III table lookup, and the
  depth row of the image summed over frequencies (Algorithm 1).

Parity status: pinned in ``tests/test_oracle_fx3d.py`` (identity at dz = 0,
normal equations, phase accuracy along the axis and the diagonal against the
exact phase shift, amplitude guard, brute-force 2-D convolution with the
expanded stencil, plane-wave eigenvalue, the impulse response of a spike on a
hemisphere, a point diffractor focused at its position).
"""
from __future__ import annotations

import math

import numpy as np

from . import lookup_index, slowness

__all__ = ["orbits", "design2d_at", "design2d_operators", "response2d", "expand_stencil",
           "step3d", "migrate3d", "samples_per_axis"]


def orbits(L: int):
    """Unique taps p = (a, b), 0 <= b <= a <= L, ordered by a then b, and for
    each the list of offsets (i, j) in [-L, L]^2 that share it (the orbit of
    (a, b) under sign changes and the swap of i and j)."""
    out = []
    for a in range(L + 1):
        for b in range(a + 1):
            pts = set()
            for i, j in ((a, b), (b, a)):
                for si in (-1, 1):
                    for sj in (-1, 1):
                        pts.add((si * i, sj * j))
            out.append(((a, b), sorted(pts)))
    return out


def samples_per_axis(L: int) -> int:
    """Wavenumber samples per axis of the 2-D design, on [0, pi/dx]."""
    return max(48, 6 * (L + 1))


def _basis(kx: np.ndarray, ky: np.ndarray, dx: float, L: int) -> np.ndarray:
    """Real response of each unique tap: B[m, p] = sum over the orbit of p of
    cos(i kx dx) cos(j ky dx) (the stencil is even in i and in j)."""
    cols = []
    for (a, b), pts in orbits(L):
        col = np.zeros(kx.shape)
        for i, j in pts:
            col = col + np.cos(i * kx * dx) * np.cos(j * ky * dx)
        cols.append(col)
    return np.stack(cols, axis=-1)


def response2d(h: np.ndarray, kx, ky, dx: float) -> np.ndarray:
    """H(kx, ky) of the unique taps h[p] (complex), by the orbit basis."""
    L = int(round((math.sqrt(8 * len(h) + 1) - 3) / 2))
    kx = np.asarray(kx, dtype=np.float64)
    ky = np.asarray(ky, dtype=np.float64)
    return _basis(kx, ky, dx, L) @ np.asarray(h)


def _target(k: float, kr: np.ndarray, dz: float) -> np.ndarray:
    kz2 = k * k - kr * kr
    out = np.empty(kr.shape, dtype=np.complex128)
    prop = kz2 >= 0.0
    out[prop] = np.exp(1j * np.sqrt(kz2[prop]) * dz)
    out[~prop] = np.exp(-np.sqrt(-kz2[~prop]) * dz)
    return out


def design2d_at(k, dx: float, dz: float, L: int, theta_deg: float = 65.0, stop_weight: float = 1e-2,
                return_info: bool = False):
    """Unique taps [len(k)][(L+1)(L+2)/2] (complex128) of the 2-D operators at
    wavenumbers k.

    Samples: kx_m = m pi / (dx (M-1)), m = 0..M-1, M = samples_per_axis(L), on
    the octant ky <= kx (the response has the grid's symmetries, so the octant
    determines it); weight 1 where sqrt(kx^2 + ky^2) <= k sin(theta), the stop
    weight elsewhere; Re and Im of the target solved separately by least
    squares (QR, numpy lstsq).  Guard: G = max |H| over the octant samples of a
    4x finer grid; the taps are scaled by 1/G when G > 1.
    """
    k = np.atleast_1d(np.asarray(k, dtype=np.float64))
    M = samples_per_axis(L)
    g = np.arange(M) * (math.pi / (dx * (M - 1)))
    ii, jj = np.tril_indices(M)                      # ky index <= kx index
    kx, ky = g[ii], g[jj]
    kr = np.hypot(kx, ky)
    B = _basis(kx, ky, dx, L)
    Mg = 4 * M
    gg = np.arange(Mg) * (math.pi / (dx * (Mg - 1)))
    gi, gj = np.tril_indices(Mg)
    Bg = _basis(gg[gi], gg[gj], dx, L)
    sin_t = math.sin(math.radians(theta_deg))
    out = np.empty((len(k), B.shape[1]), dtype=np.complex128)
    guards = np.empty(len(k))
    for n, kk in enumerate(k):
        w = np.where(kr <= kk * sin_t, 1.0, stop_weight)
        sw = np.sqrt(w)
        D = _target(kk, kr, dz)
        A = B * sw[:, None]
        hr = np.linalg.lstsq(A, sw * D.real, rcond=None)[0]
        hi = np.linalg.lstsq(A, sw * D.imag, rcond=None)[0]
        h = hr + 1j * hi
        G = float(np.max(np.abs(Bg @ h)))
        guards[n] = G
        out[n] = h / G if G > 1.0 else h
    if return_info:
        return out, {"guard": guards, "samples": M}
    return out


def design2d_operators(nk: int, k_max: float, dx: float, dz: float, L: int, theta_deg: float = 65.0):
    """The 2-D operator table on k_j = j dk, dk = k_max / (nk - 1) (Sec. III's
    table, one entry per wavenumber): [nk][(L+1)(L+2)/2] complex128."""
    dk = k_max / (nk - 1) if nk > 1 else 0.0
    return design2d_at(np.arange(nk) * dk, dx, dz, L, theta_deg)


def expand_stencil(h: np.ndarray) -> np.ndarray:
    """The full (2L+1) x (2L+1) stencil s[i + L][j + L] of unique taps h."""
    L = int(round((math.sqrt(8 * len(h) + 1) - 3) / 2))
    s = np.zeros((2 * L + 1, 2 * L + 1), dtype=np.complex128)
    for p, (_, pts) in enumerate(orbits(L)):
        for i, j in pts:
            s[i + L, j + L] = h[p]
    return s


def _indices(q: float, s_plane: np.ndarray, nk: int) -> np.ndarray:
    """Sec. III table index of every point of a plane (the pinned fp32 lookup,
    evaluated once per distinct slowness value)."""
    vals, inv = np.unique(s_plane, return_inverse=True)
    idx = lookup_index(np.full(vals.shape, q, dtype=np.float32), vals, nk)
    return idx[inv].reshape(s_plane.shape)


def step3d(P: np.ndarray, vplane: np.ndarray, table: np.ndarray, q: np.ndarray) -> np.ndarray:
    """One depth step of every frequency plane: P [nw][ny][nx] -> [nw][ny][nx],
    out(y, x) = sum over the stencil of h_(y,x)(i, j) P(y + j, x + i), the
    operator of output (y, x) from its slowness fl32(1/v) and the frequency's
    q (P = 0 outside the grid)."""
    P = np.asarray(P, dtype=np.complex128)
    nw, ny, nx = P.shape
    nk, nu = table.shape
    L = int(round((math.sqrt(8 * nu + 1) - 3) / 2))
    s = slowness(vplane)
    orb = orbits(L)
    out = np.empty_like(P)
    for w in range(nw):
        idx = _indices(float(q[w]), s, nk)
        pad = np.zeros((ny + 2 * L, nx + 2 * L), dtype=np.complex128)
        pad[L:L + ny, L:L + nx] = P[w]
        acc = np.zeros((ny, nx), dtype=np.complex128)
        for p, (_, pts) in enumerate(orb):
            S = np.zeros((ny, nx), dtype=np.complex128)
            for i, j in pts:
                S += pad[L + j:L + j + ny, L + i:L + i + nx]
            acc += table[idx, p] * S
        out[w] = acc
    return out


def migrate3d(P0: np.ndarray, vel: np.ndarray, table: np.ndarray, q: np.ndarray,
              z_begin: int = 0, z_end: int | None = None):
    """Algorithm 1's depth loop in 3-D: returns (P at depth z_end, image
    [nz][ny][nx]).  Row k of the image is the sum over frequencies of Re P
    before step k; rows outside [z_begin, z_end) are zero.  ``vel`` is the
    [nz][ny][nx] migration velocity."""
    P = np.array(P0, dtype=np.complex128)
    nz = vel.shape[0]
    z_end = nz if z_end is None else z_end
    image = np.zeros((nz,) + P.shape[1:], dtype=np.float64)
    for z in range(z_begin, z_end):
        image[z] = P.real.sum(axis=0)
        P = step3d(P, vel[z], table, q)
    return P, image
