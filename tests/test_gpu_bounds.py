"""Out-of-bounds checks without a sanitizer: every buffer a call writes sits
between canary regions that must be intact afterwards; tiny and ragged
shapes (a few traces, three depth rows) match the FP64 oracle exactly as
the larger cases do."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from fxhelp import TOL_IMAGE, TOL_SLICE, desc_of, layered_inputs, problem, rel_l2

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

PAD = 1 << 16        # canary bytes before and after every buffer (keeps 256-byte alignment)
CANARY = 0xA5


@pytest.fixture(scope="module")
def fx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_05529_gb300 import build
    build.build()
    import paper_1912_05529_gb300 as fx
    return fx


class Guarded:
    """A device buffer of `nbytes` between two canary regions."""

    def __init__(self, nbytes, dtype, shape, init=None):
        self.raw = torch.full((PAD + nbytes + PAD,), CANARY, dtype=torch.uint8, device="cuda")
        self.t = self.raw[PAD:PAD + nbytes].view(dtype).view(shape)
        if init is not None:
            self.t.copy_(init)

    def intact(self):
        torch.cuda.synchronize()
        head, tail = self.raw[:PAD], self.raw[-PAD:]
        return bool((head == CANARY).all().item() and (tail == CANARY).all().item())


def _problem(nx, nz, L, seed=31):
    w = W.Workload(f"t{nx}", nx=nx, dx=12.5, nt=256, dt=0.004, nz=nz, dz=5.0, f_lo=5.0, f_hi=60.0, L=L, seed=seed)
    v, refl, sec = layered_inputs(w)
    return w, problem(w, v, sec)


def _guarded_migrate(fx, w, pr, launch):
    d = desc_of(fx, w, pr["k_max"])
    nparts = fx.fxmig_num_partials(d, launch)
    slab = Guarded(d.nw * d.nx * 8, torch.complex64, (d.nw, d.nx),
                   torch.from_numpy(pr["P0"].astype(np.complex64)).cuda())
    parts = Guarded(nparts * d.nz * d.nx * 4, torch.float32, (nparts, d.nz, d.nx))
    parts.t.zero_()
    image = Guarded(d.nz * d.nx * 4, torch.float32, (d.nz, d.nx))
    ws_bytes = fx.fxmig_workspace_bytes(d, fx.FXMIG_WS_MIGRATE)
    ws = Guarded(ws_bytes, torch.uint8, (ws_bytes,))
    vel = torch.from_numpy(pr["vm"]).cuda()
    table = torch.from_numpy(pr["table"].astype(np.complex64)).cuda()
    fx.fxmig_migrate_ex(d, launch, slab.t, vel, table, parts.t, 0, d.nz, ws.t)
    fx.fxmig_image(d, parts.t, image.t)
    assert fx.fxmig_check(ws.t) == fx.FXMIG_OK
    for name, g in (("slab", slab), ("partials", parts), ("image", image), ("workspace", ws)):
        assert g.intact(), name
    return slab.t.cpu().numpy(), image.t.cpu().numpy()


LAUNCHES = [None, dict(mode=1, cluster=1), dict(mode=1, ctas_per_sm=2), dict(mode=1, cluster=2),
            dict(mode=1, cluster=2, groups=19),
            dict(mode=1, cluster=2, groups=56, warps=1), dict(mode=1, precision=1),
            dict(mode=1, cluster=2, groups=19, precision=4), dict(mode=2)]


@pytest.mark.parametrize("nx,L", [(8, 4), (13, 8), (24, 12), (40, 12), (64, 17), (100, 12)])
@pytest.mark.parametrize("launch", LAUNCHES)
def test_tiny_shapes_canaries_and_parity(fx, nx, L, launch):
    w, pr = _problem(nx, 3, L)
    lc = fx.Launch(**launch) if launch else None
    try:
        fx.fxmig_num_partials(desc_of(fx, w, pr["k_max"]), lc)
    except fx.FxmigError:
        pytest.skip("no plan for this shape (segment narrower than the operator, or LT not compiled)")
    P, img = _guarded_migrate(fx, w, pr, lc)
    P_ref, img_ref = O.migrate(pr["P0"].astype(np.complex64).astype(np.complex128), pr["vm"],
                               pr["table"].astype(np.complex64).astype(np.complex128), pr["q"])
    tol_s, tol_i = (TOL_SLICE, TOL_IMAGE) if not (launch and launch.get("precision")) else (3e-2, 3e-2)
    assert rel_l2(P, P_ref) < tol_s
    assert rel_l2(img, img_ref) < tol_i


def test_batch_and_learned_canaries(fx):
    cases = [_problem(nx, nz, L, seed) for nx, nz, L, seed in ((37, 5, 8, 1), (130, 7, 12, 2), (64, 4, 12, 3))]
    # batch
    descs = [desc_of(fx, w, pr["k_max"]) for w, pr in cases]
    plan = fx.BatchPlan(cluster=1)
    nparts = fx.fxmig_batch_num_partials([fx.Line(d=d) for d in descs], plan)
    guards, lines = [], []
    for (w, pr), d, p in zip(cases, descs, nparts):
        slab = Guarded(d.nw * d.nx * 8, torch.complex64, (d.nw, d.nx),
                       torch.from_numpy(pr["P0"].astype(np.complex64)).cuda())
        parts = Guarded(p * d.nz * d.nx * 4, torch.float32, (p, d.nz, d.nx))
        parts.t.zero_()
        vel = torch.from_numpy(pr["vm"]).cuda()
        table = torch.from_numpy(pr["table"].astype(np.complex64)).cuda()
        guards += [slab, parts]
        lines.append((vel, table, fx.line_of(d, slab.t, vel, table, parts.t)))
    ws_bytes = fx.fxmig_batch_workspace_bytes([l[2] for l in lines])
    ws = Guarded(ws_bytes, torch.uint8, (ws_bytes,))
    fx.fxmig_migrate_batch([l[2] for l in lines], plan, ws.t)
    assert fx.fxmig_check(ws.t) == fx.FXMIG_OK
    assert all(g.intact() for g in guards + [ws])
    # learned operators
    (w, pr), d = cases[1], descs[1]
    params = torch.from_numpy(W.mlp_init(3, n_out=2 * (d.L + 1)).astype(np.float32)).cuda()
    slab = Guarded(d.nw * d.nx * 8, torch.complex64, (d.nw, d.nx),
                   torch.from_numpy(pr["P0"].astype(np.complex64)).cuda())
    p = fx.fxmig_mlp_num_partials(d)
    parts = Guarded(p * d.nz * d.nx * 4, torch.float32, (p, d.nz, d.nx))
    ws_bytes = fx.fxmig_workspace_bytes(d, fx.FXMIG_WS_MLP_MIGRATE)
    ws = Guarded(ws_bytes, torch.uint8, (ws_bytes,))
    fx.fxmig_mlp_migrate(d, slab.t, torch.from_numpy(pr["vm"]).cuda(), params, parts.t, 0, d.nz, ws.t)
    # an untrained network's operators are far from |H| <= 1: the wavefield may
    # grow beyond the image accumulator's range, which is reported, not hidden
    assert fx.fxmig_check(ws.t) in (fx.FXMIG_OK, fx.FXMIG_ERANGE)
    assert slab.intact() and parts.intact() and ws.intact()
