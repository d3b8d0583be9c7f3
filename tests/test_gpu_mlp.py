"""GPU parity of the learned-operator path against the FP64 oracle, through the
C ABI: least-squares design at arbitrary k, network forward and gradient,
Adam step, training, migration with network operators, and what the trained
network gains over the table of Sec. III against a continuous-velocity
reference."""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W
from fxhelp import TOL_DESIGN64, rel_l2
from oracle import mlp as OM

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

# Split-BF16 network arithmetic (two BF16 terms per operand, three MMAs per
# product, FP32 accumulation): each operand keeps 16 significant bits
# (|v - hi - lo| <= 2^-17 |v|) and the dropped lo*lo term is below 2^-16
# relative, so a 64-term dot product carries a relative error of a few 2^-16
# (about 5e-5) of the sum of |terms|.  Through four layers and GELU (FP32
# erff) the outputs stay within about 1e-4 of the output scale.
TOL_MLP_FWD = 2e-4    # max |taps - oracle| / max |oracle taps|
TOL_MLP_GRAD = 1e-3   # rel-L2 of the whole gradient vector
TOL_MLP_LOSS = 1e-4   # relative loss


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


def _desc(fx, L=12, k_max=0.5, nx=64, nz=8, nt=256, dt=0.004, dx=12.5, dz=5.0):
    i0, nw = W.band_bins(nt, dt, 5.0, 60.0)
    return fx.Desc(nx=nx, nz=nz, nt=nt, nw=nw, i0=i0, L=L, nk=1024, dx=dx, dz=dz, dt=dt,
                   theta_max_deg=65.0, k_max=k_max)


def test_design_at_matches_oracle(fx, oracle_mod):
    d = _desc(fx, L=12, k_max=0.45)
    k = np.sort(np.random.default_rng(7).uniform(0.0, d.k_max, 301))
    taps = torch.empty((k.size, d.L + 1), dtype=torch.complex64, device="cuda")
    taps64 = torch.empty((k.size, d.L + 1), dtype=torch.complex128, device="cuda")
    fx.fxmig_design_at(d, _cuda(k, torch.float64), taps, taps64)
    torch.cuda.synchronize()
    ref = O.design_at(k, d.dx, d.dz, d.L)
    g64 = taps64.cpu().numpy()
    assert np.abs(g64 - ref).max() <= TOL_DESIGN64 * np.abs(ref).max()
    assert np.array_equal(taps.cpu().numpy(), g64.astype(np.complex64))


def test_mlp_forward_matches_oracle(fx):
    d = _desc(fx, L=12, k_max=0.5)
    v = W.mlp_init(3)
    k = np.random.default_rng(1).uniform(-0.05, 0.55, 1003)   # ragged, includes clipped inputs
    taps = torch.empty((k.size, d.L + 1), dtype=torch.complex64, device="cuda")
    fx.fxmig_mlp_taps(d, _cuda(v, torch.float32), _cuda(k, torch.float64), taps)
    torch.cuda.synchronize()
    # the oracle takes the same float32 parameters the kernel reads
    ref = OM.taps_at(v.astype(np.float32).astype(np.float64), k, d.k_max, d.L)
    err = np.abs(taps.cpu().numpy() - ref).max() / np.abs(ref).max()
    print(f"network forward: max err / max |taps| = {err:.3e}")
    assert err <= TOL_MLP_FWD


def _train_set(d, n, seed=2):
    k = np.random.default_rng(seed).uniform(0.0, d.k_max, n)
    return k, O.design_at(k, d.dx, d.dz, d.L)


def test_mlp_gradient_matches_oracle(fx):
    d = _desc(fx, L=12, k_max=0.5)
    v = W.mlp_init(3).astype(np.float32).astype(np.float64)
    k, t = _train_set(d, 1000)   # 15 full CTAs of 64 samples and a ragged one
    P = fx.fxmig_mlp_param_count(d.L)
    ws = torch.empty(fx.fxmig_mlp_train_ws_bytes(d.L, k.size), dtype=torch.uint8, device="cuda")
    grad = torch.empty(P, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    fx.fxmig_mlp_grad(d, _cuda(v, torch.float32), _cuda(k, torch.float64), _cuda(t, torch.complex64), grad, ws,
                      loss=loss)
    torch.cuda.synchronize()
    p = OM.unflatten(v, 64, 2 * (d.L + 1))
    t32 = t.astype(np.complex64)
    tgt = np.stack([t32.real, t32.imag], -1).reshape(k.size, -1).astype(np.float64)
    y, cache = OM.forward(p, (k / d.k_max).astype(np.float32).astype(np.float64))
    g_ref = OM.flatten(OM.backward(p, cache, y, tgt))
    l_ref = OM.loss(y, tgt)
    g = grad.cpu().numpy().astype(np.float64)
    e_g = rel_l2(g, g_ref)
    e_l = abs(float(loss.item()) - l_ref) / l_ref
    print(f"gradient rel-L2 {e_g:.3e}, loss rel {e_l:.3e}")
    assert e_g <= TOL_MLP_GRAD
    assert e_l <= TOL_MLP_LOSS
    # every parameter block, not only the largest
    o = 0
    for name in OM.PARAM_ORDER:
        sz = int(np.prod(OM.shapes(64, 2 * (d.L + 1))[name]))
        assert rel_l2(g[o:o + sz], g_ref[o:o + sz]) <= 10 * TOL_MLP_GRAD, name
        o += sz


def test_mlp_adam_step_matches_oracle(fx):
    d = _desc(fx, L=12, k_max=0.5)
    v = W.mlp_init(5).astype(np.float32)
    k, t = _train_set(d, 640)
    P = v.size
    ws = torch.empty(fx.fxmig_mlp_train_ws_bytes(d.L, k.size), dtype=torch.uint8, device="cuda")
    params = _cuda(v, torch.float32)
    m = torch.zeros(P, dtype=torch.float32, device="cuda")
    s = torch.zeros(P, dtype=torch.float32, device="cuda")
    kk, tt = _cuda(k, torch.float64), _cuda(t, torch.complex64)
    lr = 1e-3
    fx.fxmig_mlp_train(d, params, m, s, 0, 1, lr, lr, 0, kk, tt, ws)
    torch.cuda.synchronize()
    t32 = t.astype(np.complex64)
    tgt = np.stack([t32.real, t32.imag], -1).reshape(k.size, -1).astype(np.float64)
    p = OM.unflatten(v.astype(np.float64), 64, 2 * (d.L + 1))
    y, cache = OM.forward(p, (k / d.k_max).astype(np.float32).astype(np.float64))
    g = OM.flatten(OM.backward(p, cache, y, tgt))
    v1, m1, s1 = OM.adam_step(v.astype(np.float64), g, np.zeros(P), np.zeros(P), 1, lr)
    got = params.cpu().numpy().astype(np.float64)
    # first Adam step is lr * g / (|g| + eps): compare where the gradient is not negligible
    big = np.abs(g) > 1e-3 * np.abs(g).max()
    assert np.abs((got - v)[big] - (v1 - v)[big]).max() <= 1e-3 * lr
    # |update| <= lr, up to the fp32 rounding of the updated parameter
    assert np.all(np.abs(got - v) <= lr * (1 + 1e-5) + np.spacing(np.abs(v)).astype(np.float64))
    assert rel_l2(m.cpu().numpy(), m1) <= TOL_MLP_GRAD


def _train(fx, d, k, t, steps, lr_max=3e-3, lr_min=1e-5, seed=2):
    P = fx.fxmig_mlp_param_count(d.L)
    params = _cuda(W.mlp_init(seed, n_out=2 * (d.L + 1)), torch.float32)
    m = torch.zeros(P, dtype=torch.float32, device="cuda")
    s = torch.zeros(P, dtype=torch.float32, device="cuda")
    ws = torch.empty(fx.fxmig_mlp_train_ws_bytes(d.L, k.size), dtype=torch.uint8, device="cuda")
    loss = torch.empty(steps, dtype=torch.float32, device="cuda")
    fx.fxmig_mlp_train(d, params, m, s, 0, steps, lr_max, lr_min, steps, _cuda(k, torch.float64),
                       _cuda(t, torch.complex64), ws, loss=loss)
    torch.cuda.synchronize()
    return params, loss.cpu().numpy()


def test_mlp_training_converges_and_is_deterministic(fx):
    d = _desc(fx, L=12, k_max=0.5)
    k, t = _train_set(d, 2048)
    p1, l1 = _train(fx, d, k, t, 1500)
    p2, l2 = _train(fx, d, k, t, 1500)
    print(f"loss {l1[0]:.3e} -> {l1[-1]:.3e}")
    assert np.all(np.isfinite(l1))
    assert l1[-1] < 1e-2 * l1[0]
    assert torch.equal(p1, p2) and np.array_equal(l1, l2)


def _synthetic_network(L, seed=11):
    """A network whose operators stay close to the identity (stable over many
    depth steps) but vary with the input: small random output weights and a
    0.95 bias on Re h0."""
    v = W.mlp_init(seed, n_out=2 * (L + 1))
    p = OM.unflatten(v, 64, 2 * (L + 1))
    p["W4"] *= 0.02
    p["b4"][:] = 0.0
    p["b4"][0] = 0.95
    return OM.flatten(p).astype(np.float32).astype(np.float64)


def _layered(nx, nz, seed, lens=False, nt=256, dt=0.004):
    wl = W.Workload("layered", nx=nx, dx=12.5, nt=nt, dt=dt, nz=nz, dz=5.0, f_lo=5.0, f_hi=60.0, L=12, seed=seed)
    v, refl = W.layered_lens_model(wl, lens=lens)
    sec = W.normal_incidence_section(wl, v, refl)
    vm = (0.5 * v).astype(np.float32)
    w = O.omegas(wl.i0, wl.nw, wl.nt, wl.dt)
    return wl, vm, w, O.band_dft(sec, wl.i0, wl.nw)


def _gpu_mlp_migrate(fx, d, P0, vm, params, z_begin=0, z_end=None):
    z_end = d.nz if z_end is None else z_end
    slab = _cuda(P0.astype(np.complex64), torch.complex64)
    nparts = fx.fxmig_mlp_num_partials(d)
    partials = torch.zeros((nparts, d.nz, d.nx), dtype=torch.float32, device="cuda")
    ws = torch.empty(fx.fxmig_workspace_bytes(d, fx.FXMIG_WS_MLP_MIGRATE), dtype=torch.uint8, device="cuda")
    image = torch.empty((d.nz, d.nx), dtype=torch.float32, device="cuda")
    fx.fxmig_mlp_migrate(d, slab, _cuda(vm, torch.float32), params, partials, z_begin, z_end, ws)
    fx.fxmig_image(d, partials, image)
    assert fx.fxmig_check(ws) == 0
    return slab.cpu().numpy(), image.cpu().numpy()


def _desc_of(fx, wl, k_max):
    return fx.Desc(nx=wl.nx, nz=wl.nz, nt=wl.nt, nw=wl.nw, i0=wl.i0, L=wl.L, nk=wl.nk, dx=wl.dx, dz=wl.dz,
                   dt=wl.dt, theta_max_deg=wl.theta_deg, k_max=k_max)


@pytest.mark.parametrize("nx,nz,lens", [(200, 24, True), (300, 16, False), (203, 16, True)])
def test_mlp_migrate_matches_pointwise_oracle(fx, oracle_mod, nx, nz, lens):
    wl, vm, w, P0 = _layered(nx, nz, seed=21, lens=lens)
    k_max = float(w.max() / vm.min())
    d = _desc_of(fx, wl, k_max)
    v = _synthetic_network(d.L)
    P0_32 = P0.astype(np.complex64).astype(np.complex128)
    errs = []
    for z_end in (1, nz // 2, nz):
        P_g, img_g = _gpu_mlp_migrate(fx, d, P0, vm, _cuda(v, torch.float32), 0, z_end)
        P_o, img_o = O.migrate_pointwise(P0_32, vm, w, OM.taps_fn(v, k_max, d.L), 0, z_end)
        errs.append((z_end, rel_l2(P_g, P_o), rel_l2(img_g[:z_end], img_o[:z_end])))
    print("slab / image rel-L2 by depth:", errs)
    for z_end, e_slab, e_img in errs:
        assert e_slab <= 2e-5 * max(1, z_end) ** 0.5 * 5, (z_end, e_slab)
        assert e_img <= 1e-4, (z_end, e_img)


def test_mlp_migrate_split_equals_unsplit(fx):
    wl, vm, w, P0 = _layered(160, 20, seed=22, lens=True)
    k_max = float(w.max() / vm.min())
    d = _desc_of(fx, wl, k_max)
    params = _cuda(_synthetic_network(d.L), torch.float32)
    P_a, img_a = _gpu_mlp_migrate(fx, d, P0, vm, params)
    slab = _cuda(P0.astype(np.complex64), torch.complex64)
    nparts = fx.fxmig_mlp_num_partials(d)
    partials = torch.zeros((nparts, d.nz, d.nx), dtype=torch.float32, device="cuda")
    ws = torch.empty(fx.fxmig_workspace_bytes(d, fx.FXMIG_WS_MLP_MIGRATE), dtype=torch.uint8, device="cuda")
    for z0, z1 in ((0, 7), (7, 7), (7, 20)):
        fx.fxmig_mlp_migrate(d, slab, _cuda(vm, torch.float32), params, partials, z0, z1, ws)
    image = torch.empty((d.nz, d.nx), dtype=torch.float32, device="cuda")
    fx.fxmig_image(d, partials, image)
    torch.cuda.synchronize()
    assert np.array_equal(slab.cpu().numpy(), P_a) and np.array_equal(image.cpu().numpy(), img_a)


def _phase_error(h, k, dx, dz, theta_deg=65.0, n=256):
    """Per tap set: max over the design passband kx <= k sin(theta) of the
    phase error |arg(H(kx) / exp(i sqrt(k^2 - kx^2) dz))|."""
    kx = np.linspace(0.0, 1.0, n)[None, :] * (k[:, None] * math.sin(math.radians(theta_deg)))
    L = h.shape[1] - 1
    c = np.where(np.arange(L + 1) == 0, 1.0, 2.0)
    H = np.einsum("kn,kmn->km", h, c * np.cos(kx[:, :, None] * dx * np.arange(L + 1)))
    D = np.exp(1j * np.sqrt(np.maximum(k[:, None] ** 2 - kx ** 2, 0.0)) * dz)
    return np.abs(np.angle(H / D)).max(axis=1)


def test_learned_operators_gain_over_table(fx, oracle_mod):
    """Against the reference that designs the operator at every point's exact
    slowness (no quantisation), the network path beats the nearest-entry
    table of 1024 wavenumbers: smaller operator error and smaller image error."""
    wl, vm, w, P0 = _layered(256, 60, seed=23, lens=False)
    k_max = float(w.max() / vm.min())
    d = _desc_of(fx, wl, k_max)
    # training set: 8192 designed operators at k ~ U[0, k_max] (seeded)
    k_tr = np.random.default_rng(2).uniform(0.0, k_max, 8192)
    t_tr = torch.empty((k_tr.size, d.L + 1), dtype=torch.complex64, device="cuda")
    kk = _cuda(k_tr, torch.float64)
    fx.fxmig_design_at(d, kk, t_tr)
    params, loss = _train(fx, d, k_tr, t_tr.cpu().numpy(), 100000)
    print(f"training loss {loss[0]:.3e} -> {loss[-1]:.3e}")
    # operator error against the design at the exact wavenumber
    k_te = np.random.default_rng(3).uniform(0.02 * k_max, k_max, 4000)
    h_des = O.design_at(k_te, d.dx, d.dz, d.L)
    taps = torch.empty((k_te.size, d.L + 1), dtype=torch.complex64, device="cuda")
    fx.fxmig_mlp_taps(d, params, _cuda(k_te, torch.float64), taps)
    h_mlp = taps.cpu().numpy().astype(np.complex128)
    table = O.design_operators(d.nk, k_max, d.dx, d.dz, d.L)
    dk = k_max / (d.nk - 1)
    h_tab = table[np.clip(np.rint(k_te / dk).astype(int), 0, d.nk - 1)]
    e_op_mlp = np.sqrt(np.mean(np.abs(h_mlp - h_des) ** 2))
    e_op_tab = np.sqrt(np.mean(np.abs(h_tab - h_des) ** 2))
    pe_des = _phase_error(h_des, k_te, d.dx, d.dz)
    pe_mlp = np.abs(_phase_error(h_mlp, k_te, d.dx, d.dz) - pe_des)
    pe_tab = np.abs(_phase_error(h_tab, k_te, d.dx, d.dz) - pe_des)
    # images: table path and network path on the GPU against the continuous reference
    _, img_ref = O.migrate_pointwise(P0.astype(np.complex64).astype(np.complex128), vm, w,
                                     O.design_taps_fn(d.dx, d.dz, d.L))
    _, img_mlp = _gpu_mlp_migrate(fx, d, P0, vm, params)
    slab = _cuda(P0.astype(np.complex64), torch.complex64)
    nparts = fx.fxmig_num_partials(d)
    partials = torch.zeros((nparts, d.nz, d.nx), dtype=torch.float32, device="cuda")
    ws = torch.empty(fx.fxmig_workspace_bytes(d, fx.FXMIG_WS_MIGRATE), dtype=torch.uint8, device="cuda")
    tab_gpu = torch.empty((d.nk, d.L + 1), dtype=torch.complex64, device="cuda")
    fx.fxmig_design_operators(d, tab_gpu)
    fx.fxmig_migrate(d, slab, _cuda(vm, torch.float32), tab_gpu, partials, 0, d.nz, ws)
    img_tab = torch.empty((d.nz, d.nx), dtype=torch.float32, device="cuda")
    fx.fxmig_image(d, partials, img_tab)
    e_img_mlp = rel_l2(img_mlp, img_ref)
    e_img_tab = rel_l2(img_tab.cpu().numpy(), img_ref)
    print(f"operator rms error vs exact design: network {e_op_mlp:.3e}, table {e_op_tab:.3e}")
    print(f"excess passband phase error: network mean {pe_mlp.mean():.3e} max {pe_mlp.max():.3e}; "
          f"table mean {pe_tab.mean():.3e} max {pe_tab.max():.3e}")
    print(f"image rel-L2 vs continuous reference: network {e_img_mlp:.3e}, table {e_img_tab:.3e}")
    assert e_img_mlp <= 1e-2
    assert e_op_mlp < e_op_tab
    assert e_img_mlp < e_img_tab
