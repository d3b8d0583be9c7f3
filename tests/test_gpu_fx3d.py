"""3-D migration with 2-D extrapolators on the GPU against the FP64 oracle
(oracle/fx3d.py): the 2-D operator design, the depth steps (wavefield slices)
and the image, on ragged grids that span several 32 x 8 tiles, for several
operator half-lengths and frequency groupings; split depth ranges; edge
cases; velocity checks."""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W
from fxhelp import TOL_DESIGN64, TOL_IMAGE, TOL_SLICE, rel_l2

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


@pytest.fixture(scope="module")
def F():
    O.build()
    import oracle.fx3d as fx3d
    return fx3d


def _cuda(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


def _desc(fx, w, k_max, **kw):
    v = dict(nx=w.nx, ny=w.ny, nz=w.nz, nt=w.nt, nw=w.nw, i0=w.i0, L=w.L, nk=w.nk, dx=w.dx, dz=w.dz, dt=w.dt,
             theta_max_deg=w.theta_deg, k_max=k_max)
    v.update(kw)
    return fx.Desc3d(**v)


@pytest.mark.parametrize("L,dx,dz", [(2, 20.0, 10.0), (6, 20.0, 10.0), (6, 12.5, 5.0), (8, 25.0, 12.0)])
def test_design_matches_oracle(fx, F, L, dx, dz):
    nk, k_max = 24, 0.25
    d = fx.Desc3d(nx=8, ny=8, nz=4, nt=64, nw=4, i0=2, L=L, nk=nk, dx=dx, dz=dz, dt=0.004, theta_max_deg=65.0,
                  k_max=k_max)
    nu = fx.fxmig3d_num_taps(L)
    table = torch.empty((nk, nu), dtype=torch.complex64, device="cuda")
    table64 = torch.empty((nk, nu), dtype=torch.complex128, device="cuda")
    fx.fxmig3d_design_operators(d, table, table64)
    torch.cuda.synchronize()
    ref = F.design2d_operators(nk, k_max, dx, dz, L)
    assert rel_l2(table64.cpu().numpy(), ref) < TOL_DESIGN64
    assert rel_l2(table.cpu().numpy(), ref) < 1e-6


def _case(F, nx, ny, nz, L, seed=5, lens=True):
    w = W.Workload3d(f"grid_{nx}x{ny}", nx=nx, ny=ny, dx=20.0, nt=128, dt=0.004, nz=nz, dz=10.0, f_lo=5.0,
                     f_hi=40.0, L=L, nk=96, seed=seed)
    v, refl = W.layered_lens_model_3d(w)
    vm = (0.5 * v).astype(np.float32)
    if not lens:
        vm[:] = 1000.0
    sec = W.normal_incidence_section_3d(w, v, refl)
    om = O.omegas(w.i0, w.nw, w.nt, w.dt)
    k_max = float(om[-1] / float(vm.min()))
    table = F.design2d_operators(w.nk, k_max, w.dx, w.dz, w.L).astype(np.complex64)
    _, dk = O.k_grid(w.nk, k_max)
    q = O.q_values(om, dk)
    P0 = O.band_dft(sec.reshape(ny * nx, w.nt), w.i0, w.nw).reshape(w.nw, ny, nx).astype(np.complex64)
    return w, dict(vm=vm, k_max=k_max, table=table, q=q, P0=P0)


def _gpu(fx, d, pr, z_ranges, groups=0, slab=None):
    """Run the depth ranges in order; returns the slab after each range and the image."""
    npts = d.nx * d.ny
    if slab is None:
        slab = _cuda(pr["P0"], torch.complex64)
    partials = torch.full((fx.fxmig3d_num_partials(d), d.nz, d.ny, d.nx), float("nan"), dtype=torch.float32,
                          device="cuda")
    ws = torch.zeros(fx.fxmig3d_workspace_bytes(d), dtype=torch.uint8, device="cuda")
    vel = _cuda(pr["vm"], torch.float32)
    table = _cuda(pr["table"], torch.complex64)
    slabs = []
    for z0, z1 in z_ranges:
        fx.fxmig3d_migrate(d, slab, vel, table, partials, z0, z1, ws, groups=groups)
        assert fx.fxmig_check(ws) == fx.FXMIG_OK
        slabs.append(slab.cpu().numpy().reshape(d.nw, d.ny, d.nx))
    image = torch.empty((d.nz, d.ny, d.nx), dtype=torch.float32, device="cuda")
    fx.fxmig3d_image(d, partials, image)
    torch.cuda.synchronize()
    assert npts == d.nx * d.ny
    return slabs, image.cpu().numpy()


@pytest.mark.parametrize("nx,ny,L,groups", [(37, 29, 6, 0), (64, 17, 2, 1), (33, 40, 8, 3), (70, 9, 6, 0)])
def test_migrate_matches_oracle(fx, F, nx, ny, L, groups):
    nz = 14
    w, pr = _case(F, nx, ny, nz, L)
    d = _desc(fx, w, pr["k_max"])
    half = nz // 2
    slabs, image = _gpu(fx, d, pr, [(0, half), (half, nz)], groups=groups)
    P_half, img_half = F.migrate3d(pr["P0"].astype(np.complex128), pr["vm"], pr["table"].astype(np.complex128),
                                   pr["q"], 0, half)
    P_end, img_rest = F.migrate3d(P_half, pr["vm"], pr["table"].astype(np.complex128), pr["q"], half, nz)
    ref_img = img_half + img_rest
    for j in range(w.nw):
        assert rel_l2(slabs[0][j], P_half[j]) < TOL_SLICE, ("half", j)
        assert rel_l2(slabs[1][j], P_end[j]) < TOL_SLICE, ("end", j)
    assert rel_l2(image, ref_img) < TOL_IMAGE
    assert np.max(np.abs(image - ref_img)) < 1e-3 * np.max(np.abs(ref_img))


def test_split_groups_and_repeat_are_bitwise_equal(fx, F):
    w, pr = _case(F, 41, 23, 10, 6)
    d = _desc(fx, w, pr["k_max"])
    ref_slabs, ref_img = _gpu(fx, d, pr, [(0, 10)])
    for ranges, groups in (([(0, 3), (3, 10)], 0), ([(0, 10)], 1), ([(0, 10)], w.nw), ([(0, 10)], 0)):
        slabs, img = _gpu(fx, d, pr, ranges, groups=groups)
        assert np.array_equal(slabs[-1], ref_slabs[-1]), (ranges, groups)
        assert np.array_equal(img, ref_img), (ranges, groups)


@pytest.mark.parametrize("nx,ny", [(1, 1), (1, 12), (12, 1), (5, 3)])
def test_tiny_grids(fx, F, nx, ny):
    w, pr = _case(F, nx, ny, 6, 4, lens=False)
    d = _desc(fx, w, pr["k_max"])
    slabs, image = _gpu(fx, d, pr, [(0, 6)])
    P, ref = F.migrate3d(pr["P0"].astype(np.complex128), pr["vm"], pr["table"].astype(np.complex128), pr["q"])
    assert rel_l2(slabs[-1], P) < TOL_SLICE
    assert rel_l2(image, ref) < TOL_IMAGE


def test_outputs_stay_inside_their_buffers(fx, F):
    # canaries after the slab, the accumulator and the image are untouched
    w, pr = _case(F, 37, 11, 8, 6)
    d = _desc(fx, w, pr["k_max"])
    npts = d.nx * d.ny
    guard = 4096
    slab_buf = torch.full((d.nw * npts + guard,), complex(7.0, 7.0), dtype=torch.complex64, device="cuda")
    slab_buf[:d.nw * npts] = _cuda(pr["P0"].reshape(-1), torch.complex64)
    nparts = fx.fxmig3d_num_partials(d)
    acc_buf = torch.full((nparts * d.nz * npts + guard,), 7.0, dtype=torch.float32, device="cuda")
    img_buf = torch.full((d.nz * npts + guard,), 7.0, dtype=torch.float32, device="cuda")
    ws = torch.zeros(fx.fxmig3d_workspace_bytes(d), dtype=torch.uint8, device="cuda")
    fx.fxmig3d_migrate(d, slab_buf, _cuda(pr["vm"], torch.float32), _cuda(pr["table"], torch.complex64),
                       acc_buf[:nparts * d.nz * npts], 0, d.nz, ws)
    fx.fxmig3d_image(d, acc_buf[:nparts * d.nz * npts], img_buf)
    torch.cuda.synchronize()
    assert fx.fxmig_check(ws) == fx.FXMIG_OK
    assert bool((slab_buf[d.nw * npts:] == complex(7.0, 7.0)).all())
    assert bool((acc_buf[nparts * d.nz * npts:] == 7.0).all())
    assert bool((img_buf[d.nz * npts:] == 7.0).all())
    P, ref = F.migrate3d(pr["P0"].astype(np.complex128), pr["vm"], pr["table"].astype(np.complex128), pr["q"])
    assert rel_l2(img_buf[:d.nz * npts].cpu().numpy().reshape(ref.shape), ref) < TOL_IMAGE


def test_bad_velocity_is_reported(fx, F):
    w, pr = _case(F, 16, 16, 4, 4, lens=False)
    d = _desc(fx, w, pr["k_max"])
    for bad in (0.0, -1.0, float("nan"), float("inf")):
        vm = pr["vm"].copy()
        vm[2, 5, 7] = bad
        slab = _cuda(pr["P0"], torch.complex64)
        partials = torch.zeros((fx.fxmig3d_num_partials(d), d.nz, d.ny, d.nx), dtype=torch.float32, device="cuda")
        ws = torch.zeros(fx.fxmig3d_workspace_bytes(d), dtype=torch.uint8, device="cuda")
        fx.fxmig3d_migrate(d, slab, _cuda(vm, torch.float32), _cuda(pr["table"], torch.complex64), partials, 0,
                           d.nz, ws)
        assert fx.fxmig_check(ws) == fx.FXMIG_EVELOCITY, bad


def test_diffractor_focuses_on_the_gpu(fx, F):
    # the whole chain on the device (t->f of the flattened section, the 2-D
    # operator table, the depth steps, the image): the diffractor of the
    # oracle pin focuses at its grid point here too, and the image matches the
    # oracle's from the same inputs
    w = W.DIFFRACTOR_3D
    sec = W.diffractor_section_3d(w, 400.0, 400.0, 200.0, 2000.0).astype(np.float32)
    om = O.omegas(w.i0, w.nw, w.nt, w.dt)
    k_max = float(om[-1] / 1000.0)
    d = _desc(fx, w, k_max)
    d2 = fx.flat_desc(d)
    slab = torch.empty((w.nw, w.ny * w.nx), dtype=torch.complex64, device="cuda")
    ws_t = torch.zeros(fx.fxmig_workspace_bytes(d2, fx.FXMIG_WS_T2F), dtype=torch.uint8, device="cuda")
    fx.fxmig_t2f(d2, _cuda(sec.reshape(w.ny * w.nx, w.nt), torch.float32), slab, ws_t)
    table = torch.empty((w.nk, fx.fxmig3d_num_taps(w.L)), dtype=torch.complex64, device="cuda")
    fx.fxmig3d_design_operators(d, table)
    vm = np.full((w.nz, w.ny, w.nx), 1000.0, np.float32)
    partials = torch.zeros((fx.fxmig3d_num_partials(d), w.nz, w.ny, w.nx), dtype=torch.float32, device="cuda")
    ws = torch.zeros(fx.fxmig3d_workspace_bytes(d), dtype=torch.uint8, device="cuda")
    fx.fxmig3d_migrate(d, slab, _cuda(vm, torch.float32), table, partials, 0, w.nz, ws)
    image = torch.empty((w.nz, w.ny, w.nx), dtype=torch.float32, device="cuda")
    fx.fxmig3d_image(d, partials, image)
    torch.cuda.synchronize()
    assert fx.fxmig_check(ws) == fx.FXMIG_OK
    img = image.cpu().numpy()
    iz, iy, ix = np.unravel_index(np.argmax(np.abs(img)), img.shape)
    assert abs(ix - 20) <= 1 and abs(iy - 20) <= 1 and abs(iz - 20) <= 1, (ix, iy, iz)
    P0 = O.band_dft(sec.reshape(w.ny * w.nx, w.nt).astype(np.float64), w.i0, w.nw).reshape(w.nw, w.ny, w.nx)
    _, dk = O.k_grid(w.nk, k_max)
    ref_table = F.design2d_operators(w.nk, k_max, w.dx, w.dz, w.L)
    _, ref = F.migrate3d(P0, vm, ref_table, O.q_values(om, dk))
    assert rel_l2(img, ref) < 1e-4


def test_frequency_shards_on_device_sum_to_full_band(fx, F):
    # the frequency-shard helper's per-rank path for a 3-D description
    # (shard_desc, the library's depth steps and image on the rank's planes)
    # for every rank of a 3-way split, summed in rank order, against the
    # full-band oracle
    from paper_1912_05529_gb300 import distributed as D
    w, pr = _case(F, 35, 21, 10, 6)
    d = _desc(fx, w, pr["k_max"])
    _, img_ref = F.migrate3d(pr["P0"].astype(np.complex128), pr["vm"], pr["table"].astype(np.complex128), pr["q"])
    vel, table = _cuda(pr["vm"], torch.float32), _cuda(pr["table"], torch.complex64)
    total = torch.zeros((w.nz, w.ny, w.nx), dtype=torch.float32, device="cuda")
    for rank in range(3):
        j0, n = D.frequency_block(w.nw, 3, rank)
        sd = D.shard_desc(d, 3, rank)
        assert sd.i0 == d.i0 + j0 and sd.nw == n and sd.k_max == d.k_max and (sd.nx, sd.ny) == (d.nx, d.ny)
        total += D._migrate3d_on_device(sd, _cuda(pr["P0"][j0:j0 + n], torch.complex64), vel, table)
    torch.cuda.synchronize()
    assert rel_l2(total.cpu().numpy(), img_ref) < TOL_IMAGE
