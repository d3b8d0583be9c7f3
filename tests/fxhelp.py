"""Shared helpers of the GPU parity tests: build seeded inputs, run the oracle
and the library on the same values, measure relative L2 errors."""
import math

import numpy as np

import oracle as O
import workloads as W

# Tolerances (FP32 GPU vs FP64 oracle on identical inputs).  Each step of
# Eq. 1 sums 2L+1 fp32 products (relative rounding ~1e-7 per step); over a few
# hundred steps the errors add like a random walk, a few 1e-6 on the
# wavefield.  The bars are the ones the method is held to.
TOL_SLICE = 1e-5      # wavefield P(., z_k, .) over all x and frequencies
TOL_IMAGE = 1e-4      # final image
TOL_T2F = 2e-6        # fp32 FFT against the FP64 DFT
TOL_DESIGN64 = 1e-10  # FP64 taps, Cholesky (GPU) vs QR (oracle)


def rel_l2(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def small_layered(nx=700, nz=120, nt=512, dt=0.004, L=12, seed=5, name="layered_700"):
    return W.Workload(name, nx=nx, dx=12.5, nt=nt, dt=dt, nz=nz, dz=5.0, f_lo=5.0, f_hi=60.0, L=L, seed=seed)


def problem(w, v_medium, section):
    """Oracle-side inputs of a workload: migration velocity (v/2), table, q, P0."""
    vm = (0.5 * np.asarray(v_medium)).astype(np.float32)
    om = O.omegas(w.i0, w.nw, w.nt, w.dt)
    k_max = float(om[-1] / float(vm.min()))
    table = O.design_operators(w.nk, k_max, w.dx, w.dz, w.L, w.theta_deg)
    _, dk = O.k_grid(w.nk, k_max)
    q = O.q_values(om, dk)
    P0 = O.band_dft(section, w.i0, w.nw)
    return dict(vm=vm, k_max=k_max, table=table, q=q, P0=P0)


def desc_of(fx, w, k_max):
    return fx.Desc(nx=w.nx, nz=w.nz, nt=w.nt, nw=w.nw, i0=w.i0, L=w.L, nk=w.nk, dx=w.dx, dz=w.dz,
                   dt=w.dt, theta_max_deg=w.theta_deg, k_max=k_max)


def max_abs_rel(a, b):
    """max |a - b| over the largest |b| (a localised error, e.g. at a seam
    between CTAs, that a global norm could hide)."""
    a = np.asarray(a)
    b = np.asarray(b)
    m = float(np.max(np.abs(b))) if b.size else 0.0
    return float(np.max(np.abs(a - b)) / (m if m > 0 else 1.0)) if a.size else 0.0


# per-element bars next to the norm bars: a slice element may deviate by 1e-4
# of the slice's largest value (the norm bar allows 1e-5 on average), an image
# pixel by 1e-3 of the image's largest value
TOL_SLICE_MAX = 1e-4
TOL_IMAGE_MAX = 1e-3


def modeled_problem(w, noise=0.01):
    """Parity input with dipping events: the layered lens model's reflectivity
    taken up to the surface with the oracle's conjugate operators (oracle.model,
    the exact adjoint of the depth loop: upward extrapolation with the
    conjugate table operators), shaped by the Ricker spectrum (25 Hz), plus
    complex Gaussian noise of `noise` times the data RMS (seeded)."""
    v, refl = W.layered_lens_model(w)
    vm = (0.5 * v).astype(np.float32)
    om = O.omegas(w.i0, w.nw, w.nt, w.dt)
    k_max = float(om[-1] / float(vm.min()))
    table = O.design_operators(w.nk, k_max, w.dx, w.dz, w.L, w.theta_deg)
    _, dk = O.k_grid(w.nk, k_max)
    q = O.q_values(om, dk)
    P0 = O.model(refl, vm, table, q)
    f = (w.i0 + np.arange(w.nw)) / (w.nt * w.dt)
    P0 = P0 * O.ricker_spectrum(f, 25.0, w.dt)[:, None]
    rng = np.random.default_rng(w.seed + 1000)
    rms = float(np.sqrt(np.mean(np.abs(P0) ** 2)))
    P0 = P0 + noise * rms * (rng.standard_normal(P0.shape) + 1j * rng.standard_normal(P0.shape)) / math.sqrt(2)
    return dict(vm=vm, k_max=k_max, table=table, q=q, P0=P0, refl=refl)


def layered_inputs(w):
    v, refl = W.layered_lens_model(w)
    d = W.normal_incidence_section(w, v, refl)
    return v, refl, d
