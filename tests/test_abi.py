"""The C ABI library builds for sm_103a, loads, exports every entry point that
include/fxmig.h declares, and rejects bad arguments on the host (no GPU needed:
none of these calls reaches a kernel)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fx():
    from paper_1912_05529_gb300 import build
    build.build()
    import paper_1912_05529_gb300 as fx
    fx.lib()
    return fx


def _declared():
    src = open(os.path.join(ROOT, "include", "fxmig.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|size_t|const char\s*\*)\s*\*?\s*(fxmig(?:3d)?_\w+)\s*\(", src, re.M)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("fxmig_design_operators", "fxmig_t2f", "fxmig_migrate", "fxmig_image", "fxmig3d_design_operators",
              "fxmig3d_migrate", "fxmig3d_image"):
        assert n in names


def test_library_exports_every_declared_symbol(fx):
    lib = fx.lib()
    for n in _declared():
        assert hasattr(lib, n), n


def test_version_and_strerror(fx):
    assert fx.fxmig_version() == 2
    for code in (0, -1, -2, -3, -4, -5):
        assert fx.fxmig_strerror(code) and fx.fxmig_strerror(code) != "unknown error"
    assert fx.fxmig_strerror(-99) == "unknown error"


def _desc(fx, **kw):
    d = fx.desc_for(nx=128, nz=100, nt=256, dx=10.0, dz=5.0, dt=0.004, f_lo=5.0, f_hi=60.0, L=12, v_min=1000.0)
    for k, v in kw.items():
        setattr(d, k, v)
    return d


def test_descriptor_band(fx):
    d = _desc(fx)
    assert (d.i0, d.nw) == (6, 56)


def test_workspace_sizes(fx):
    d = _desc(fx)
    assert fx.fxmig_workspace_bytes(d, fx.FXMIG_WS_T2F) >= 256 + 8 * d.nt
    assert fx.fxmig_workspace_bytes(d, fx.FXMIG_WS_MIGRATE) >= 256 + 16 * d.nk * (d.L + 1)
    assert fx.fxmig_workspace_bytes(d, 99) == 0
    assert fx.fxmig_workspace_bytes(_desc(fx, nx=0), fx.FXMIG_WS_T2F) == 0


@pytest.mark.parametrize("bad", [dict(nx=0), dict(nz=0), dict(nw=0), dict(i0=0), dict(i0=120),
                                 dict(L=21), dict(dx=0.0), dict(dt=-1.0), dict(k_max=float("nan")),
                                 dict(theta_max_deg=120.0)])
def test_invalid_descriptors_are_rejected(fx, bad):
    d = _desc(fx, **bad)
    lib = fx.lib()
    dummy = ctypes.c_void_p(256)
    assert lib.fxmig_design_operators(ctypes.byref(d), dummy, None, None) == fx.FXMIG_EINVAL
    assert lib.fxmig_t2f(ctypes.byref(d), dummy, dummy, dummy, 1 << 20, None) == fx.FXMIG_EINVAL
    assert lib.fxmig_migrate(ctypes.byref(d), dummy, dummy, dummy, dummy, 1, 0, 1, dummy, 1 << 30, None) \
        == fx.FXMIG_EINVAL
    assert lib.fxmig_image(ctypes.byref(d), dummy, 1, dummy, None) == fx.FXMIG_EINVAL
    assert lib.fxmig_num_partials(ctypes.byref(d), None) == fx.FXMIG_EINVAL


def test_null_and_misaligned_pointers(fx):
    d = _desc(fx)
    lib = fx.lib()
    ok = ctypes.c_void_p(1 << 20)
    big = 1 << 30
    assert lib.fxmig_design_operators(ctypes.byref(d), None, None, None) == fx.FXMIG_EINVAL
    assert lib.fxmig_t2f(ctypes.byref(d), None, ok, ok, big, None) == fx.FXMIG_EINVAL
    assert lib.fxmig_t2f(ctypes.byref(d), ok, ok, ctypes.c_void_p((1 << 20) + 8), big, None) == fx.FXMIG_EINVAL
    assert lib.fxmig_migrate(ctypes.byref(d), ok, None, ok, ok, 1000, 0, 1, ok, big, None) == fx.FXMIG_EINVAL
    assert lib.fxmig_migrate(ctypes.byref(d), ok, ok, ok, ctypes.c_void_p((1 << 20) + 4), 1000, 0, 1, ok, big,
                             None) == fx.FXMIG_EINVAL
    assert lib.fxmig_image(ctypes.byref(d), None, 1, ok, None) == fx.FXMIG_EINVAL
    assert lib.fxmig_check(None, None) == fx.FXMIG_EINVAL


def test_bad_depth_range_and_small_buffers(fx):
    d = _desc(fx)
    lib = fx.lib()
    ok = ctypes.c_void_p(1 << 20)
    big = 1 << 30
    for zb, ze in ((-1, 5), (5, 4), (0, 101)):
        assert lib.fxmig_migrate(ctypes.byref(d), ok, ok, ok, ok, 1000, zb, ze, ok, big, None) == fx.FXMIG_EINVAL
    need = fx.fxmig_workspace_bytes(d, fx.FXMIG_WS_MIGRATE)
    assert lib.fxmig_migrate(ctypes.byref(d), ok, ok, ok, ok, 1000, 0, 5, ok, need - 1, None) == fx.FXMIG_ENOSPC
    assert lib.fxmig_migrate(ctypes.byref(d), ok, ok, ok, ok, 0, 0, 5, ok, need, None) == fx.FXMIG_ENOSPC
    assert lib.fxmig_t2f(ctypes.byref(d), ok, ok, ok, 16, None) == fx.FXMIG_ENOSPC


def test_unsupported_fft_length(fx):
    d = _desc(fx, nt=2 * 17 * 19, i0=3, nw=10)
    lib = fx.lib()
    ok = ctypes.c_void_p(1 << 20)
    assert lib.fxmig_t2f(ctypes.byref(d), ok, ok, ok, 1 << 30, None) == fx.FXMIG_EINVAL


def test_invalid_launch_choices(fx):
    d = _desc(fx)
    assert fx.lib().fxmig_num_partials(ctypes.byref(d), ctypes.byref(fx.Launch(mode=7))) == fx.FXMIG_EINVAL
    assert fx.lib().fxmig_num_partials(ctypes.byref(d), ctypes.byref(fx.Launch(cluster=3))) == fx.FXMIG_EINVAL
    # warps counts compute warps, 1..12 (the edge warp of a cluster comes on top)
    for w in (1, 12):
        assert fx.lib().fxmig_num_partials(ctypes.byref(d), ctypes.byref(fx.Launch(mode=1, warps=w))) > 0
    assert fx.lib().fxmig_num_partials(ctypes.byref(d), ctypes.byref(fx.Launch(mode=1, warps=13))) == fx.FXMIG_EINVAL


def test_precision_choices(fx):
    lib = fx.lib()
    d = _desc(fx)
    npart = lambda **kw: lib.fxmig_num_partials(ctypes.byref(d), ctypes.byref(fx.Launch(**kw)))
    assert npart(precision=fx.FXMIG_PREC_FP16) > 0
    assert npart(precision=fx.FXMIG_PREC_BF16_SPLIT) > 0
    assert npart(precision=5) == fx.FXMIG_EINVAL
    assert npart(precision=-1) == fx.FXMIG_EINVAL
    # the per-depth form has no 16-bit storage form
    assert npart(mode=fx.FXMIG_MODE_PER_DEPTH, precision=fx.FXMIG_PREC_FP16) == fx.FXMIG_EINVAL
    # 16-bit forms are compiled for LT = 8, 12, 17 only
    d20 = _desc(fx, L=20)
    assert lib.fxmig_num_partials(ctypes.byref(d20), ctypes.byref(fx.Launch(precision=1))) == fx.FXMIG_EINVAL
    assert lib.fxmig_num_partials(ctypes.byref(d20), None) > 0


def test_large_problem_plans_several_waves(fx):
    # 8192 traces x 601 frequencies: half a line per CTA (clusters of 2, one
    # frequency per group, two items per lane), several waves of CTAs
    d = fx.desc_for(nx=8192, nz=2000, nt=4000, dx=6.25, dz=4.0, dt=0.002, f_lo=5.0, f_hi=80.0, L=17,
                    v_min=750.0)
    assert d.nw == 601
    for prec in (fx.FXMIG_PREC_FP32, fx.FXMIG_PREC_FP16):
        s = fx.fxmig_launch_shape(d, fx.Launch(precision=prec))
        assert s.cluster == 2 and s.groups == 601 and s.items_per_lane == 2 and s.waves > 1
        assert s.smem_bytes <= 227 * 1024
    assert fx.fxmig_num_partials(d) == 3


def test_bench_workload_shape(fx):
    # 2048 traces x 221 frequencies: 74 clusters of 2 over 152 SMs, groups of
    # 2 or 3 lines laid end to end and cut in half (one cut line per CTA), one
    # item per compute lane; on request, one whole line per CTA and two CTAs
    # per SM
    d = fx.desc_for(nx=2048, nz=800, nt=2000, dx=12.5, dz=5.0, dt=0.002, f_lo=5.0, f_hi=60.0, L=12,
                    v_min=750.0)
    s = fx.fxmig_launch_shape(d)
    assert (s.cluster, s.ctas_per_sm, s.items_per_lane, s.warps) == (2, 1, 1, 12)
    assert 2 * s.groups >= 140 and s.waves == 1 and s.smem_bytes <= 227 * 1024
    o = fx.fxmig_launch_shape(d, fx.Launch(ctas_per_sm=2))
    assert (o.cluster, o.ctas_per_sm, o.items_per_lane, o.warps) == (1, 2, 1, 8)
    assert o.groups == 221 and o.waves == 1
    assert 2 * o.smem_bytes <= 228 * 1024 - 2048
    pd = fx.fxmig_launch_shape(d, fx.Launch(mode=fx.FXMIG_MODE_PER_DEPTH))
    assert pd.mode == fx.FXMIG_MODE_PER_DEPTH and pd.ctas == 8 * pd.groups


def test_learned_operator_entry_points_reject_bad_arguments(fx):
    lib = fx.lib()
    d = _desc(fx)
    ok = ctypes.c_void_p(1 << 20)
    assert fx.fxmig_mlp_param_count(12) == 10138
    assert lib.fxmig_mlp_param_count(16) == fx.FXMIG_EINVAL
    assert lib.fxmig_mlp_train_ws_bytes(12, 0) == 0
    assert lib.fxmig_mlp_num_partials(ctypes.byref(_desc(fx, L=17))) == fx.FXMIG_EINVAL
    assert lib.fxmig_mlp_num_partials(ctypes.byref(d)) > 0
    assert lib.fxmig_design_at(ctypes.byref(d), ok, -1, ok, None, None) == fx.FXMIG_EINVAL
    assert lib.fxmig_design_at(ctypes.byref(d), None, 4, ok, None, None) == fx.FXMIG_EINVAL
    ws = fx.fxmig_mlp_train_ws_bytes(12, 100)
    assert lib.fxmig_mlp_train(ctypes.byref(d), None, ok, ok, 0, 1, 1e-3, 1e-3, 0, ok, ok, 100, None, ok, ws,
                               None) == fx.FXMIG_EINVAL
    assert lib.fxmig_mlp_train(ctypes.byref(d), ok, ok, ok, 0, 1, 1e-3, 1e-3, 0, ok, ok, 100, None, ok, ws - 1,
                               None) == fx.FXMIG_ENOSPC
    assert lib.fxmig_mlp_grad(ctypes.byref(d), ok, ok, ok, 0, ok, None, ok, ws, None) == fx.FXMIG_EINVAL
    need = fx.fxmig_workspace_bytes(d, fx.FXMIG_WS_MLP_MIGRATE)
    assert need > 0
    assert lib.fxmig_mlp_migrate(ctypes.byref(d), ok, ok, None, ok, 64, 0, 5, ok, need, None) == fx.FXMIG_EINVAL
    assert lib.fxmig_mlp_migrate(ctypes.byref(d), ok, ok, ok, ok, 64, 0, 5, ok, need - 1, None) == fx.FXMIG_ENOSPC


def test_batch_entry_points_reject_bad_arguments(fx):
    lib = fx.lib()
    d = _desc(fx)
    ok = ctypes.c_void_p(1 << 20)
    good = fx.Line(d=d, slab=ok, vel=ok, table=ok, partials=ok, z_begin=0, z_end=d.nz)
    arr = (fx.Line * 2)(good, good)
    out = (ctypes.c_int * 2)()
    assert lib.fxmig_batch_num_partials(arr, 2, None, out) == fx.FXMIG_OK and min(out) >= 1
    assert lib.fxmig_batch_num_partials(arr, 0, None, out) == fx.FXMIG_EINVAL
    bad_plan = fx.BatchPlan(cluster=3)
    assert lib.fxmig_batch_num_partials(arr, 2, ctypes.byref(bad_plan), out) == fx.FXMIG_EINVAL
    need = lib.fxmig_batch_workspace_bytes(arr, 2, 0)
    assert need > 0 and lib.fxmig_batch_workspace_bytes(arr, 2, 1) > need
    assert lib.fxmig_migrate_batch(arr, 2, None, None, need, None) == fx.FXMIG_EINVAL
    assert lib.fxmig_migrate_batch(arr, 2, None, ok, need - 1, None) == fx.FXMIG_ENOSPC
    assert lib.fxmig_migrate_batch(arr, 2, ctypes.byref(bad_plan), ok, need, None) == fx.FXMIG_EINVAL
    many = (fx.Line * 129)(*([good] * 129))
    assert lib.fxmig_batch_workspace_bytes(many, 129, 0) == 0
    nulled = fx.Line(d=d, slab=ok, vel=None, table=ok, partials=ok, z_begin=0, z_end=d.nz)
    arr2 = (fx.Line * 1)(nulled)
    assert lib.fxmig_migrate_batch(arr2, 1, None, ok, need, None) == fx.FXMIG_EINVAL
    plan = fx.BatchPlan()
    assert lib.fxmig_batch_autotune(arr, 2, ctypes.byref(plan), None, ok, need, None) == fx.FXMIG_ENOSPC


def test_selftest_rejects_bad_arguments(fx):
    lib = fx.lib()
    ok = ctypes.c_void_p(1 << 20)
    assert lib.fxmig_selftest_timeout(None, 100, None) == fx.FXMIG_EINVAL
    assert lib.fxmig_selftest_timeout(ctypes.c_void_p((1 << 20) + 8), 100, None) == fx.FXMIG_EINVAL
    assert lib.fxmig_selftest_timeout(ok, 0, None) == fx.FXMIG_EINVAL
    assert lib.fxmig_selftest_timeout(ok, (1 << 20) + 1, None) == fx.FXMIG_EINVAL


def _desc3d(fx, **kw):
    v = dict(nx=40, ny=24, nz=12, nt=128, nw=20, i0=3, L=6, nk=64, dx=20.0, dz=10.0, dt=0.004,
             theta_max_deg=65.0, k_max=0.2)
    v.update(kw)
    return fx.Desc3d(**v)


def test_3d_entry_points_reject_bad_arguments(fx):
    # argument checks only: nothing is enqueued on these paths
    lib = fx.lib()
    assert fx.fxmig3d_num_taps(6) == 28 and fx.fxmig3d_num_taps(8) == 45 and fx.fxmig3d_num_taps(0) == 1
    assert lib.fxmig3d_num_taps(9) == fx.FXMIG_EINVAL and lib.fxmig3d_num_taps(-1) == fx.FXMIG_EINVAL
    d = _desc3d(fx)
    nparts = fx.fxmig3d_num_partials(d)
    assert nparts >= 1
    need = fx.fxmig3d_workspace_bytes(d)
    # status head, taps [nk][45 at L = 6 compiled as 6: 28] float4, slowness, norms, second slab
    assert need >= 256 + 64 * 28 * 16 + 12 * 40 * 24 * 4 + 20 * 8 + 20 * 40 * 24 * 8
    for bad in (dict(nx=0), dict(ny=0), dict(L=9), dict(nt=1), dict(i0=0), dict(nw=200), dict(dx=0.0),
                dict(theta_max_deg=95.0)):
        db = _desc3d(fx, **bad)
        assert fx.fxmig3d_workspace_bytes(db) == 0, bad
        assert lib.fxmig3d_num_partials(ctypes.byref(db)) == fx.FXMIG_EINVAL, bad
        assert lib.fxmig3d_design_operators(ctypes.byref(db), ctypes.c_void_p(1 << 20), None, None) == fx.FXMIG_EINVAL
    ok = ctypes.c_void_p(1 << 20)
    mis = ctypes.c_void_p((1 << 20) + 4)
    assert lib.fxmig3d_design_operators(ctypes.byref(d), None, None, None) == fx.FXMIG_EINVAL
    assert lib.fxmig3d_design_operators(ctypes.byref(d), mis, None, None) == fx.FXMIG_EINVAL
    args = dict(slab=ok, vel=ok, table=ok, partials=ok, nparts=nparts, z0=0, z1=d.nz, groups=0, ws=ok)

    def call(**kw):
        a = dict(args)
        a.update(kw)
        return lib.fxmig3d_migrate(ctypes.byref(d), a["slab"], a["vel"], a["table"], a["partials"], a["nparts"],
                                   a["z0"], a["z1"], a["groups"], a["ws"], None)
    assert call(slab=None) == fx.FXMIG_EINVAL
    assert call(vel=None) == fx.FXMIG_EINVAL
    assert call(ws=mis) == fx.FXMIG_EINVAL
    assert call(partials=ctypes.c_void_p((1 << 20) + 8)) == fx.FXMIG_EINVAL
    assert call(z0=5, z1=4) == fx.FXMIG_EINVAL
    assert call(z1=d.nz + 1) == fx.FXMIG_EINVAL
    assert call(groups=-1) == fx.FXMIG_EINVAL
    assert call(nparts=nparts - 1) == fx.FXMIG_ENOSPC
    assert lib.fxmig3d_image(ctypes.byref(d), ok, nparts - 1, ok, None) == fx.FXMIG_ENOSPC
    assert lib.fxmig3d_image(ctypes.byref(d), None, nparts, ok, None) == fx.FXMIG_EINVAL
