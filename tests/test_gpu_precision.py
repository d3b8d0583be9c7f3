"""GPU forms with 16-bit storage (FP16 / BF16 wavefield lines and taps, FP32
arithmetic) against the FP64 oracle, with their errors stated; the
multi-wave persistent plan in FP32; and the 512-trace window of the large
8192-trace line (35-tap operators, 601 frequencies, 2000 depth steps)."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from fxhelp import TOL_IMAGE, TOL_SLICE, desc_of, layered_inputs, modeled_problem, problem, rel_l2, small_layered

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


def gpu_migrate(fx, d, P0_32, vm, table32, launch):
    slab = _cuda(P0_32, torch.complex64)
    nparts = fx.fxmig_num_partials(d, launch)
    partials = torch.full((nparts, d.nz, d.nx), float("nan"), dtype=torch.float32, device="cuda")
    ws = torch.zeros(fx.fxmig_workspace_bytes(d, fx.FXMIG_WS_MIGRATE), dtype=torch.uint8, device="cuda")
    image = torch.empty((d.nz, d.nx), dtype=torch.float32, device="cuda")
    fx.fxmig_migrate_ex(d, launch, slab, _cuda(vm, torch.float32), _cuda(table32, torch.complex64), partials, 0,
                        d.nz, ws)
    assert fx.fxmig_check(ws) == fx.FXMIG_OK
    fx.fxmig_image(d, partials, image)
    torch.cuda.synchronize()
    return slab.cpu().numpy(), image.cpu().numpy()


# The bar of the reduced-precision forms: image rel-L2 <= 1e-2 against the
# FP64 oracle.  Rounding the wavefield to 16 bits after every step adds a
# relative error of up to 2^-11 (FP16) or 2^-8 (BF16) per value and step, of
# random sign, so after n steps the wavefield error grows like sqrt(n) times
# that; unsplit taps add a systematic error of the same size per step that
# grows like n.  The hi/lo split makes the tap error negligible (about 2^-22 /
# 2^-16).  Only FP16 with split taps stays within the bar on every workload
# (hundreds to thousands of steps); the others are reported above the bar.
BAR = 1e-2
PREC_FORMS = ["FP16_SPLIT", "BF16_SPLIT", "FP16", "BF16"]
MEETS_BAR = {"FP16_SPLIT"}


@pytest.fixture(scope="module")
def layered_case():
    w = small_layered()
    pr = modeled_problem(w)
    table32 = pr["table"].astype(np.complex64)
    P0_32 = pr["P0"].astype(np.complex64)
    P, img = O.migrate(P0_32.astype(np.complex128), pr["vm"], table32.astype(np.complex128), pr["q"])
    return w, pr, table32, P0_32, P, img


@pytest.fixture(scope="module")
def split_error(fx, layered_case):
    w, pr, table32, P0_32, P_ref, img_ref = layered_case
    d = desc_of(fx, w, pr["k_max"])
    _, img = gpu_migrate(fx, d, P0_32, pr["vm"], table32, fx.Launch(mode=1, precision=fx.FXMIG_PREC_FP16_SPLIT))
    return rel_l2(img, img_ref)


@pytest.mark.parametrize("name", PREC_FORMS)
@pytest.mark.parametrize("launch", [dict(cluster=1), dict(cluster=2), dict(cluster=2, groups=37)])
def test_16bit_forms_against_oracle(fx, layered_case, split_error, name, launch):
    w, pr, table32, P0_32, P_ref, img_ref = layered_case
    d = desc_of(fx, w, pr["k_max"])
    prec = getattr(fx, "FXMIG_PREC_" + name)
    P, img = gpu_migrate(fx, d, P0_32, pr["vm"], table32, fx.Launch(mode=1, precision=prec, **launch))
    e_img, e_slab = rel_l2(img, img_ref), rel_l2(P, P_ref)
    print(f"{name} {launch}: image rel-L2 {e_img:.3e}, final slice rel-L2 {e_slab:.3e}")
    assert np.all(np.isfinite(img))
    if name in MEETS_BAR:
        assert e_img <= BAR
    else:
        # above the bar: no accuracy claim beyond the ordering of the forms
        assert e_img >= split_error


def test_split_taps_do_not_lose_accuracy(fx, layered_case):
    w, pr, table32, P0_32, P_ref, img_ref = layered_case
    d = desc_of(fx, w, pr["k_max"])
    for a, b in (("FP16_SPLIT", "FP16"), ("BF16_SPLIT", "BF16")):
        _, ia = gpu_migrate(fx, d, P0_32, pr["vm"], table32,
                            fx.Launch(mode=1, precision=getattr(fx, "FXMIG_PREC_" + a)))
        _, ib = gpu_migrate(fx, d, P0_32, pr["vm"], table32,
                            fx.Launch(mode=1, precision=getattr(fx, "FXMIG_PREC_" + b)))
        assert rel_l2(ia, img_ref) <= 1.05 * rel_l2(ib, img_ref), (a, b)


def test_multiwave_plan_matches_oracle(fx, oracle_mod):
    # 4096 traces x 401 frequencies, one line per cluster of 2 (half a line,
    # 256 chunks, per CTA): more CTAs than SMs, several waves
    w = W.Workload("wide", nx=4096, dx=12.5, nt=2000, dt=0.002, nz=6, dz=5.0, f_lo=5.0, f_hi=105.0, L=12, seed=9)
    pr = modeled_problem(w)
    d = desc_of(fx, w, pr["k_max"])
    launch = fx.Launch(mode=1, cluster=2, groups=d.nw)
    assert fx.fxmig_launch_shape(d, launch).waves > 1
    table32 = pr["table"].astype(np.complex64)
    P0_32 = pr["P0"].astype(np.complex64)
    P, img = gpu_migrate(fx, d, P0_32, pr["vm"], table32, launch)
    P_ref, img_ref = O.migrate(P0_32.astype(np.complex128), pr["vm"], table32.astype(np.complex128), pr["q"])
    assert rel_l2(P, P_ref) < TOL_SLICE
    assert rel_l2(img, img_ref) < TOL_IMAGE


@pytest.fixture(scope="module")
def large_window():
    """Traces [3840, 4352) of the 8192-trace line: its velocity and section
    (seeded model of the full line), migrated as a 512-trace problem."""
    w = W.LARGE_8192
    v, refl = W.layered_lens_model(w)
    sec = W.normal_incidence_section(w, v, refl)
    x0 = 3840
    ww = W.Workload("large_8192_window", nx=512, dx=w.dx, nt=w.nt, dt=w.dt, nz=w.nz, dz=w.dz, f_lo=w.f_lo,
                    f_hi=w.f_hi, L=w.L, seed=w.seed)
    pr = problem(ww, v[:, x0:x0 + 512], sec[x0:x0 + 512])
    table32 = pr["table"].astype(np.complex64)
    P0_32 = pr["P0"].astype(np.complex64)
    P, img = O.migrate(P0_32.astype(np.complex128), pr["vm"], table32.astype(np.complex128), pr["q"])
    return ww, pr, table32, P0_32, P, img


@pytest.mark.parametrize("name", ["FP32"] + PREC_FORMS)
def test_large_line_window_against_oracle(fx, large_window, name):
    ww, pr, table32, P0_32, P_ref, img_ref = large_window
    assert ww.nw == 601 and ww.L == 17
    d = desc_of(fx, ww, pr["k_max"])
    prec = getattr(fx, "FXMIG_PREC_" + name)
    P, img = gpu_migrate(fx, d, P0_32, pr["vm"], table32, fx.Launch(mode=1, precision=prec))
    e_img, e_slab = rel_l2(img, img_ref), rel_l2(P, P_ref)
    print(f"512-trace window, {name}: image rel-L2 {e_img:.3e}, final slice rel-L2 {e_slab:.3e}")
    assert np.all(np.isfinite(img))
    if name == "FP32":
        assert e_img < TOL_IMAGE
    elif name in MEETS_BAR:
        assert e_img <= BAR
