"""Device-side failure detection without a GPU fault: a bounded wait that
runs out is reported by fxmig_check and leaves the context usable; velocity
samples that are not finite and positive are reported by every form."""
import numpy as np
import pytest

import oracle as O
from fxhelp import TOL_IMAGE, desc_of, layered_inputs, problem, rel_l2, small_layered

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


@pytest.fixture(scope="module")
def case():
    w = small_layered(nx=256, nz=12, name="layered_256")
    v, refl, sec = layered_inputs(w)
    pr = problem(w, v, sec)
    return w, pr


def _migrate(fx, d, pr, vel, launch=None):
    slab = _cuda(pr["P0"].astype(np.complex64), torch.complex64)
    partials = torch.zeros((fx.fxmig_num_partials(d, launch), d.nz, d.nx), dtype=torch.float32, device="cuda")
    ws = torch.zeros(fx.fxmig_workspace_bytes(d, fx.FXMIG_WS_MIGRATE), dtype=torch.uint8, device="cuda")
    fx.fxmig_migrate_ex(d, launch, slab, _cuda(vel, torch.float32), _cuda(pr["table"], torch.complex64), partials,
                        0, d.nz, ws)
    return fx.fxmig_check(ws), slab, partials


def test_bounded_wait_timeout_is_reported_and_context_survives(fx, case):
    ws = torch.zeros(256, dtype=torch.uint8, device="cuda")
    fx.fxmig_selftest_timeout(ws, polls=1000)
    assert fx.fxmig_check(ws) == fx.FXMIG_ETIMEOUT
    # the same context keeps working: a migration right after is correct
    w, pr = case
    d = desc_of(fx, w, pr["k_max"])
    code, _, partials = _migrate(fx, d, pr, pr["vm"])
    assert code == fx.FXMIG_OK
    image = torch.empty((d.nz, d.nx), dtype=torch.float32, device="cuda")
    fx.fxmig_image(d, partials, image)
    _, img_ref = O.migrate(pr["P0"].astype(np.complex64).astype(np.complex128), pr["vm"],
                           pr["table"].astype(np.complex64).astype(np.complex128), pr["q"])
    assert rel_l2(image.cpu().numpy(), img_ref) < TOL_IMAGE


@pytest.mark.parametrize("bad", [0.0, -1500.0, float("nan"), float("inf")])
@pytest.mark.parametrize("launch", [None, dict(mode=1, cluster=2, precision=3), dict(mode=2)])
def test_bad_velocity_is_reported(fx, case, bad, launch):
    w, pr = case
    d = desc_of(fx, w, pr["k_max"])
    vel = pr["vm"].copy()
    vel[d.nz // 2, d.nx // 3] = bad
    lc = fx.Launch(**launch) if launch else None
    code, slab, _ = _migrate(fx, d, pr, vel, lc)
    assert code == fx.FXMIG_EVELOCITY
    # the status word is cleared by the next call
    code2, _, _ = _migrate(fx, d, pr, pr["vm"], lc)
    assert code2 == fx.FXMIG_OK


def test_bad_velocity_is_reported_by_batch_and_learned_forms(fx, case):
    w, pr = case
    d = desc_of(fx, w, pr["k_max"])
    vel = pr["vm"].copy()
    vel[3, 7] = float("nan")
    vel_t = _cuda(vel, torch.float32)
    table = _cuda(pr["table"], torch.complex64)
    # batch of one line
    slab = _cuda(pr["P0"].astype(np.complex64), torch.complex64)
    nparts = fx.fxmig_batch_num_partials([fx.Line(d=d)], None)
    parts = torch.zeros((nparts[0], d.nz, d.nx), dtype=torch.float32, device="cuda")
    lines = [fx.line_of(d, slab, vel_t, table, parts)]
    ws = torch.zeros(fx.fxmig_batch_workspace_bytes(lines), dtype=torch.uint8, device="cuda")
    fx.fxmig_migrate_batch(lines, None, ws)
    assert fx.fxmig_check(ws) == fx.FXMIG_EVELOCITY
    # learned operators (any network: the check is on the velocity)
    import workloads as W
    params = _cuda(W.mlp_init(3, n_out=2 * (d.L + 1)), torch.float32)
    slab = _cuda(pr["P0"].astype(np.complex64), torch.complex64)
    parts = torch.zeros((fx.fxmig_mlp_num_partials(d), d.nz, d.nx), dtype=torch.float32, device="cuda")
    ws = torch.zeros(fx.fxmig_workspace_bytes(d, fx.FXMIG_WS_MLP_MIGRATE), dtype=torch.uint8, device="cuda")
    fx.fxmig_mlp_migrate(d, slab, vel_t, params, parts, 0, d.nz, ws)
    assert fx.fxmig_check(ws) == fx.FXMIG_EVELOCITY
