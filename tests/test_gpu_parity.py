"""GPU parity of every hot-path kernel against the FP64 oracle, through the C ABI.

Each kernel gets the oracle's own inputs (rounded to the fp32 the kernel
takes), so only the kernel's arithmetic is under test; the end-to-end test then
runs every GPU step from the raw section."""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W
from fxhelp import (TOL_DESIGN64, TOL_IMAGE, TOL_IMAGE_MAX, TOL_SLICE, TOL_SLICE_MAX, TOL_T2F, desc_of, max_abs_rel,
                    modeled_problem, layered_inputs, problem, rel_l2,
                    small_layered)

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def fx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_05529_gb300 import build
    build.build()
    import paper_1912_05529_gb300 as fx
    return fx


def _cuda(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


def run_gpu_migrate(fx, d, P0_32, vm, table32, launch=None, chunks=None):
    """Returns (slabs after each chunk, image) from the library."""
    slab = _cuda(P0_32, torch.complex64)
    vel = _cuda(vm, torch.float32)
    table = _cuda(table32, torch.complex64)
    nparts = fx.fxmig_num_partials(d, launch)
    partials = torch.full((nparts, d.nz, d.nx), float("nan"), dtype=torch.float32, device="cuda")
    ws = torch.zeros(fx.fxmig_workspace_bytes(d, fx.FXMIG_WS_MIGRATE), dtype=torch.uint8, device="cuda")
    image = torch.empty((d.nz, d.nx), dtype=torch.float32, device="cuda")
    bounds = chunks or [0, d.nz]
    slabs = []
    for zb, ze in zip(bounds[:-1], bounds[1:]):
        fx.fxmig_migrate_ex(d, launch, slab, vel, table, partials, zb, ze, ws)
        slabs.append(slab.cpu().numpy().copy())
    assert fx.fxmig_check(ws) == fx.FXMIG_OK
    fx.fxmig_image(d, partials, image)
    torch.cuda.synchronize()
    return slabs, image.cpu().numpy()


def test_design_matches_oracle(fx):
    for (dx, dz, L, kmax) in [(10.0, 5.0, 12, 2 * math.pi * 59.57 / 1000), (12.5, 5.0, 12, 0.503),
                              (6.25, 4.0, 17, 0.67), (12.5, 5.0, 8, 0.3), (12.5, 0.0, 4, 0.3)]:
        d = fx.Desc(nx=8, nz=1, nt=64, nw=1, i0=1, L=L, nk=1024, dx=dx, dz=dz, dt=0.004, theta_max_deg=65.0,
                    k_max=kmax)
        t32 = torch.empty((1024, L + 1), dtype=torch.complex64, device="cuda")
        t64 = torch.empty((1024, L + 1), dtype=torch.complex128, device="cuda")
        fx.fxmig_design_operators(d, t32, t64)
        ref = O.design_operators(1024, kmax, dx, dz, L, 65.0)
        g64 = t64.cpu().numpy()
        err = np.max(np.abs(g64 - ref)) / np.max(np.abs(ref))
        assert err < TOL_DESIGN64, (dx, dz, L, err)
        g32 = t32.cpu().numpy()
        assert np.max(np.abs(g32 - ref.astype(np.complex64))) <= 2 * 2 ** -24 * np.max(np.abs(ref)) + 1e-30


@pytest.mark.parametrize("nx,nt,i0,nw", [(128, 256, 6, 56), (37, 2000, 20, 221), (64, 4000, 40, 601),
                                         (5, 250, 1, 124), (33, 60, 2, 20), (16, 7 * 13 * 4, 3, 100)])
def test_t2f_matches_oracle_dft(fx, nx, nt, i0, nw):
    rng = np.random.default_rng(nt + nx)
    sec = rng.standard_normal((nx, nt)).astype(np.float32)
    d = fx.Desc(nx=nx, nz=1, nt=nt, nw=nw, i0=i0, L=4, nk=2, dx=10.0, dz=5.0, dt=0.004, theta_max_deg=65.0,
                k_max=0.1)
    slab = torch.empty((nw, nx), dtype=torch.complex64, device="cuda")
    ws = torch.empty(fx.fxmig_workspace_bytes(d, fx.FXMIG_WS_T2F), dtype=torch.uint8, device="cuda")
    fx.fxmig_t2f(d, _cuda(sec, torch.float32), slab, ws)
    ref = O.band_dft(sec.astype(np.float64), i0, nw)
    assert rel_l2(slab.cpu().numpy(), ref) < TOL_T2F * math.log2(nt)


# Persistent launches: automatic; one CTA per group; clusters of 2 with 2
# lines per group (no cut line), with 3 lines per group (the middle line cut
# between the two CTAs: halo one step behind, redundant outputs), with 7-8
# lines and two items per compute lane, and with one line per group (every
# line cut in half, two waves of CTAs); per-depth launches.
LAUNCHES = [None, dict(mode=1, cluster=1), dict(mode=1, cluster=2), dict(mode=1, cluster=2, groups=37),
            dict(mode=1, cluster=2, groups=15, warps=6), dict(mode=1, cluster=2, groups=112),
            dict(mode=1, cluster=1, groups=200), dict(mode=1, ctas_per_sm=2), dict(mode=1, ctas_per_sm=2, groups=56),
            dict(mode=2), dict(mode=2, groups=3)]


@pytest.fixture(scope="module")
def layered_case():
    w = small_layered()
    pr = modeled_problem(w)
    table32 = pr["table"].astype(np.complex64)
    P0_32 = pr["P0"].astype(np.complex64)
    chunks = [0, 1, 37, 80, w.nz]
    slabs, image = [], np.zeros((w.nz, w.nx))
    P = P0_32.astype(np.complex128)
    for zb, ze in zip(chunks[:-1], chunks[1:]):
        P, img = O.migrate(P, pr["vm"], table32.astype(np.complex128), pr["q"], zb, ze)
        slabs.append(P.copy())
        image[zb:ze] = img[zb:ze]
    return w, pr, table32, P0_32, chunks, slabs, image


@pytest.mark.parametrize("launch", LAUNCHES)
def test_migrate_matches_oracle_per_depth_slice(fx, layered_case, launch):
    w, pr, table32, P0_32, chunks, ref_slabs, ref_image = layered_case
    d = desc_of(fx, w, pr["k_max"])
    lc = fx.Launch(**launch) if launch else None
    slabs, image = run_gpu_migrate(fx, d, P0_32, pr["vm"], table32, lc, chunks)
    for s, r, ze in zip(slabs, ref_slabs, chunks[1:]):
        assert rel_l2(s, r) < TOL_SLICE, ze
        assert max_abs_rel(s, r) < TOL_SLICE_MAX, ze
    assert rel_l2(image, ref_image) < TOL_IMAGE
    assert max_abs_rel(image, ref_image) < TOL_IMAGE_MAX
    assert np.all(np.isfinite(image))


def test_split_equals_unsplit_and_deterministic(fx, layered_case):
    w, pr, table32, P0_32, chunks, _, _ = layered_case
    d = desc_of(fx, w, pr["k_max"])
    a_slabs, a_img = run_gpu_migrate(fx, d, P0_32, pr["vm"], table32, None, chunks)
    b_slabs, b_img = run_gpu_migrate(fx, d, P0_32, pr["vm"], table32, None, None)
    c_slabs, c_img = run_gpu_migrate(fx, d, P0_32, pr["vm"], table32, None, None)
    assert np.array_equal(a_slabs[-1], b_slabs[-1]) and np.array_equal(a_img, b_img)
    assert np.array_equal(b_slabs[-1], c_slabs[-1]) and np.array_equal(b_img, c_img)


def _tie_slowness(q, n):
    """A slowness s (fp32) with fl32(q s) = n + 1/2 exactly and fl32(1/fl32(1/s))
    = s (so the velocity fl32(1/s) maps back to s), searched around (n + 1/2)/q;
    None if none is found within 64 ulps."""
    q = np.float32(q)
    s0 = np.float32((n + 0.5) / float(q))
    cand = [s0]
    up = dn = s0
    for _ in range(64):
        up = np.nextafter(up, np.float32(np.inf))
        dn = np.nextafter(dn, np.float32(0))
        cand += [up, dn]
    for s in cand:
        if np.float32(q * s) == np.float32(n + 0.5):
            v = np.float32(np.float32(1) / s)
            if np.float32(np.float32(1) / v) == s:
                return s, v
    return None


def test_lookup_ties_match_oracle(fx):
    # Velocities chosen so that, on one frequency line, fl32(q s) is exactly
    # n + 1/2 at every trace (Sec. III nearest-entry lookup; round half to
    # even).  Every table row holds distinct random taps, so a lookup that
    # rounds a tie the other way (or takes the product in FP64) picks another
    # row and moves the output far outside the bar.
    nx, nz, nk, L = 96, 3, 256, 8
    w = W.Workload("ties", nx=nx, dx=12.5, nt=256, dt=0.004, nz=nz, dz=5.0, f_lo=10.0, f_hi=40.0, L=L, seed=3)
    om = O.omegas(w.i0, w.nw, w.nt, w.dt)
    k_max = float(om[-1] / 700.0)
    _, dk = O.k_grid(nk, k_max)
    q = O.q_values(om, dk)
    j = w.nw // 2
    rng = np.random.default_rng(21)
    vel = np.empty((nz, nx), np.float32)
    exact_ties = fp64_differs = 0
    for z in range(nz):
        for x in range(nx):
            for _ in range(1000):
                n = int(rng.integers(4, int(q[j] * (1.0 / 700.0)) - 4))
                r = _tie_slowness(q[j], n)
                if r is not None:
                    break
            assert r is not None
            s, v = r
            vel[z, x] = v
            exact_ties += 1
            fp64_differs += int(np.rint(float(q[j]) * float(s)) != np.rint(np.float32(q[j] * s)))
    s_all = O.slowness(vel)
    idx = O.lookup_index(np.float32(q[j]), s_all, nk)
    assert np.all(np.float32(q[j]) * s_all == np.floor(np.float32(q[j]) * s_all) + np.float32(0.5))
    assert np.all(idx % 2 == 0)  # ties go to the even neighbour
    table = (rng.standard_normal((nk, L + 1)) + 1j * rng.standard_normal((nk, L + 1))) * 0.1
    table[:, 0] += 0.5
    table32 = table.astype(np.complex64)
    P0 = (rng.standard_normal((w.nw, nx)) + 1j * rng.standard_normal((w.nw, nx))).astype(np.complex64)
    P_ref, img_ref = O.migrate(P0.astype(np.complex128), vel, table32.astype(np.complex128), q)
    d = fx.Desc(nx=nx, nz=nz, nt=w.nt, nw=w.nw, i0=w.i0, L=L, nk=nk, dx=w.dx, dz=w.dz, dt=w.dt,
                theta_max_deg=w.theta_deg, k_max=k_max)
    for launch in (None, dict(mode=1, cluster=2, groups=w.nw), dict(mode=2)):
        lc = fx.Launch(**launch) if launch else None
        slabs, image = run_gpu_migrate(fx, d, P0, vel, table32, lc)
        assert rel_l2(slabs[-1][j], P_ref[j]) < TOL_SLICE, launch
        assert max_abs_rel(slabs[-1][j], P_ref[j]) < TOL_SLICE_MAX, launch
        assert rel_l2(image, img_ref) < TOL_IMAGE, launch
    print(f"{exact_ties} exact ties, {fp64_differs} of them where an FP64 product would round differently")


@pytest.mark.parametrize("launch", [None, dict(mode=1, cluster=2), dict(mode=1, cluster=1),
                                    dict(mode=1, cluster=2, groups=15, warps=6), dict(mode=1, ctas_per_sm=2)])
def test_rough_velocity_every_output_queued(fx, launch):
    # A velocity drawn independently at every point (Sec. III: each point
    # takes its own table operator), so almost every output's operator differs
    # from its 8-point item's first one: the persistent form queues up to 7 of
    # every 8 outputs per step, and the queue is drained in many rounds by the
    # fixup warp and the compute warps that join it.  Every slice and the image
    # must still match the oracle.
    w = W.Workload("rough_700", nx=700, dx=12.5, nt=512, dt=0.004, nz=40, dz=5.0, f_lo=5.0, f_hi=60.0, L=12,
                   seed=8)
    rng = np.random.default_rng(8)
    v = rng.uniform(1500.0, 4000.0, size=(w.nz, w.nx)).astype(np.float32)
    section = rng.standard_normal((w.nx, w.nt)).astype(np.float32)
    pr = problem(w, v, section)
    s_all = O.slowness(pr["vm"])
    j = w.nw - 1
    idx = O.lookup_index(np.float32(pr["q"][j]), s_all, w.nk)
    first = np.repeat(idx[:, ::8], 8, axis=1)[:, : w.nx]
    assert np.mean(idx != first) > 0.75  # most outputs of the top line leave their item's operator
    table32 = pr["table"].astype(np.complex64)
    P0_32 = pr["P0"].astype(np.complex64)
    chunks = [0, 13, w.nz]
    ref_slabs, ref_image = [], np.zeros((w.nz, w.nx))
    P = P0_32.astype(np.complex128)
    for zb, ze in zip(chunks[:-1], chunks[1:]):
        P, img = O.migrate(P, pr["vm"], table32.astype(np.complex128), pr["q"], zb, ze)
        ref_slabs.append(P.copy())
        ref_image[zb:ze] = img[zb:ze]
    d = desc_of(fx, w, pr["k_max"])
    lc = fx.Launch(**launch) if launch else None
    slabs, image = run_gpu_migrate(fx, d, P0_32, pr["vm"], table32, lc, chunks)
    for sl, r, ze in zip(slabs, ref_slabs, chunks[1:]):
        assert rel_l2(sl, r) < TOL_SLICE, ze
        assert max_abs_rel(sl, r) < TOL_SLICE_MAX, ze
    assert rel_l2(image, ref_image) < TOL_IMAGE
    assert max_abs_rel(image, ref_image) < TOL_IMAGE_MAX


@pytest.mark.parametrize("L", [4, 8, 17, 20])
def test_other_filter_lengths(fx, L):
    w = small_layered(nx=300, nz=40, L=L, seed=9)
    pr = modeled_problem(w)
    table32 = pr["table"].astype(np.complex64)
    P0_32 = pr["P0"].astype(np.complex64)
    P, img = O.migrate(P0_32.astype(np.complex128), pr["vm"], table32.astype(np.complex128), pr["q"])
    d = desc_of(fx, w, pr["k_max"])
    for launch in (None, fx.Launch(mode=2)):
        slabs, image = run_gpu_migrate(fx, d, P0_32, pr["vm"], table32, launch)
        assert rel_l2(slabs[-1], P) < TOL_SLICE
        assert rel_l2(image, img) < TOL_IMAGE


def test_diffractor_end_to_end(fx):
    # Every GPU step from the raw section (design, t -> f, depth loop, imaging)
    # against every oracle step.
    w = W.DIFFRACTOR_128
    sec = W.diffractor_section(w)
    vm = np.full((w.nz, w.nx), 1000.0, np.float32)
    om = O.omegas(w.i0, w.nw, w.nt, w.dt)
    k_max = float(om[-1] / 1000.0)
    table = O.design_operators(w.nk, k_max, w.dx, w.dz, w.L, w.theta_deg)
    _, dk = O.k_grid(w.nk, k_max)
    _, ref_img = O.migrate(O.band_dft(sec, w.i0, w.nw), vm, table, O.q_values(om, dk))
    d = desc_of(fx, w, k_max)
    img = fx.migrate_section(d, torch.from_numpy(sec.astype(np.float32)), torch.from_numpy(vm))
    torch.cuda.synchronize()
    img = img.numpy()
    assert rel_l2(img, ref_img) < TOL_IMAGE
    iz, ix = np.unravel_index(np.argmax(np.abs(img)), img.shape)
    assert abs(ix - 64) <= 1 and abs(iz - 60) <= 1


@pytest.mark.parametrize("nx", [333, 514, 1021])
@pytest.mark.parametrize("launch", [None, dict(mode=1, cluster=2, groups=37),
                                    dict(mode=1, cluster=2, groups=37, precision=3), dict(mode=2)])
def test_migrate_widths_not_multiple_of_four(fx, nx, launch):
    # rows of nx % 4 != 0 floats are not 16-byte aligned in device memory:
    # the persistent form then converts velocity rows in shared memory
    w = small_layered(nx=nx, nz=30, name=f"layered_{nx}")
    pr = modeled_problem(w)
    table32 = pr["table"].astype(np.complex64)
    P0_32 = pr["P0"].astype(np.complex64)
    d = desc_of(fx, w, pr["k_max"])
    lc = fx.Launch(**launch) if launch else None
    slabs, image = run_gpu_migrate(fx, d, P0_32, pr["vm"], table32, lc)
    P_ref, img_ref = O.migrate(P0_32.astype(np.complex128), pr["vm"], table32.astype(np.complex128), pr["q"])
    tol_s, tol_i = (TOL_SLICE, TOL_IMAGE) if not (launch and launch.get("precision")) else (1e-2, 1e-2)
    assert rel_l2(slabs[-1], P_ref) < tol_s
    assert rel_l2(image, img_ref) < tol_i


@pytest.mark.parametrize("L,prec", [(8, "FP32"), (12, "FP32"), (17, "FP32"), (20, "FP32"),
                                    (12, "FP16_SPLIT"), (17, "FP16_SPLIT")])
def test_cut_lines(fx, L, prec):
    # 1000 traces, groups of about 3 lines over clusters of 2: the middle line
    # of a group is cut between the two CTAs (at chunk 62 of 125, so the cut
    # falls inside a warp's items), whose extra warps exchange the halo one
    # step behind and compute the L redundant outputs on the other side; odd
    # L, 16-bit storage, several depth ranges
    w = small_layered(nx=1000, nz=24, L=L, seed=11, name="layered_1000")
    pr = modeled_problem(w)
    table32 = pr["table"].astype(np.complex64)
    P0_32 = pr["P0"].astype(np.complex64)
    d = desc_of(fx, w, pr["k_max"])
    launch = fx.Launch(mode=1, cluster=2, groups=w.nw // 3, precision=getattr(fx, "FXMIG_PREC_" + prec))
    slabs, image = run_gpu_migrate(fx, d, P0_32, pr["vm"], table32, launch, [0, 9, w.nz])
    P_ref, img_ref = O.migrate(P0_32.astype(np.complex128), pr["vm"], table32.astype(np.complex128), pr["q"])
    tol_s, tol_i = (TOL_SLICE, TOL_IMAGE) if prec == "FP32" else (1e-2, 1e-2)
    assert rel_l2(slabs[-1], P_ref) < tol_s
    assert rel_l2(image, img_ref) < tol_i


@pytest.mark.parametrize("nx", [16, 40, 192])
@pytest.mark.parametrize("L,prec", [(4, "FP32"), (12, "FP32"), (17, "FP32"), (20, "FP32"),
                                    (12, "FP16_SPLIT"), (17, "FP16_SPLIT")])
def test_cut_lines_tiny_halves(fx, nx, L, prec):
    # One line per group: every line cut in half, halves of 1 chunk (16
    # traces), 2-3 chunks (40) and 12 chunks (192).  The halo (2L values) and
    # the redundant outputs (L) reach past the neighbour's half and past the
    # line ends, where the wavefield is zero.
    w = small_layered(nx=nx, nz=24, L=L, seed=17, name=f"layered_{nx}")
    pr = modeled_problem(w)
    table32 = pr["table"].astype(np.complex64)
    P0_32 = pr["P0"].astype(np.complex64)
    d = desc_of(fx, w, pr["k_max"])
    launch = fx.Launch(mode=1, cluster=2, groups=w.nw, precision=getattr(fx, "FXMIG_PREC_" + prec))
    try:
        fx.fxmig_num_partials(d, launch)
    except fx.FxmigError:
        pytest.skip("no plan for this shape (LT not compiled for 16-bit storage)")
    slabs, image = run_gpu_migrate(fx, d, P0_32, pr["vm"], table32, launch, [0, 7, w.nz])
    P_ref, img_ref = O.migrate(P0_32.astype(np.complex128), pr["vm"], table32.astype(np.complex128), pr["q"])
    tol_s, tol_i = (TOL_SLICE, TOL_IMAGE) if prec == "FP32" else (1e-2, 1e-2)
    assert rel_l2(slabs[-1], P_ref) < tol_s
    assert rel_l2(image, img_ref) < tol_i


def test_cut_lines_straddling_warps(fx):
    # 496 traces (62 chunks, not a multiple of 32) and groups of about 3
    # lines over clusters of 2: the segments of a CTA run across warp
    # boundaries and the cut falls at an odd chunk
    w = small_layered(nx=496, nz=20, L=12, seed=13, name="layered_496")
    pr = modeled_problem(w)
    table32 = pr["table"].astype(np.complex64)
    P0_32 = pr["P0"].astype(np.complex64)
    d = desc_of(fx, w, pr["k_max"])
    launch = fx.Launch(mode=1, cluster=2, groups=max(1, w.nw // 3))
    slabs, image = run_gpu_migrate(fx, d, P0_32, pr["vm"], table32, launch)
    P_ref, img_ref = O.migrate(P0_32.astype(np.complex128), pr["vm"], table32.astype(np.complex128), pr["q"])
    assert rel_l2(slabs[-1], P_ref) < TOL_SLICE
    assert rel_l2(image, img_ref) < TOL_IMAGE


def test_frequency_shards_on_device_sum_to_full_band(fx):
    # the ω-shard helper's per-rank path (shard_desc, the library's depth loop
    # and imaging on the rank's lines) for every rank of a 3-way split, summed
    # in rank order, against the full-band oracle
    from paper_1912_05529_gb300 import distributed as D
    w = small_layered(nx=300, nz=30, seed=23, name="layered_300")
    pr = modeled_problem(w)
    table32 = pr["table"].astype(np.complex64)
    P0_32 = pr["P0"].astype(np.complex64)
    d = desc_of(fx, w, pr["k_max"])
    _, img_ref = O.migrate(P0_32.astype(np.complex128), pr["vm"], table32.astype(np.complex128), pr["q"])
    vel, table = _cuda(pr["vm"], torch.float32), _cuda(table32, torch.complex64)
    total = torch.zeros((w.nz, w.nx), dtype=torch.float32, device="cuda")
    for rank in range(3):
        j0, n = D.frequency_block(w.nw, 3, rank)
        sd = D.shard_desc(d, 3, rank)
        assert sd.i0 == d.i0 + j0 and sd.nw == n and sd.k_max == d.k_max
        total += D._migrate_on_device(sd, _cuda(P0_32[j0:j0 + n], torch.complex64), vel, table)
    torch.cuda.synchronize()
    assert rel_l2(total.cpu().numpy(), img_ref) < TOL_IMAGE
