"""fxmig_migrate_noalloc: the depth loop for callers that cannot allocate
device memory (their host application or plug-in API hands them buffers but
no allocator, or cudaMalloc is off limits on their real-time path).  It must
give the same wavefield and image as fxmig_migrate_ex in the persistent form,
call after call, although its scratch lives in one fixed device array that
every call reuses.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

from fxhelp import desc_of, layered_inputs, problem, small_layered

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


def _cfn(fx):
    f = fx.lib().fxmig_migrate_noalloc
    f.argtypes = [ctypes.POINTER(fx.Desc)] + [ctypes.c_void_p] * 4 + [ctypes.c_int] * 3 + [ctypes.c_void_p]
    f.restype = ctypes.c_int
    return f


def test_noalloc_matches_workspace_entry_point_twice(fx):
    w = small_layered(nx=520, nz=70, seed=13)
    v, refl, sec = layered_inputs(w)
    pr = problem(w, v, sec)
    d = desc_of(fx, w, pr["k_max"])
    P0 = torch.from_numpy(pr["P0"].astype(np.complex64)).cuda()
    vel = torch.from_numpy(pr["vm"]).cuda()
    table = torch.from_numpy(pr["table"].astype(np.complex64)).cuda()
    launch = fx.Launch(mode=fx.FXMIG_MODE_PERSISTENT)
    nparts = fx.fxmig_num_partials(d, launch)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    # existing entry point with a caller workspace
    slab_ref = P0.clone()
    part_ref = torch.zeros((nparts, d.nz, d.nx), dtype=torch.float32, device="cuda")
    ws = torch.zeros(fx.fxmig_workspace_bytes(d, fx.FXMIG_WS_MIGRATE), dtype=torch.uint8, device="cuda")
    fx.fxmig_migrate_ex(d, launch, slab_ref, vel, table, part_ref, 0, d.nz, ws)
    img_ref = torch.empty((d.nz, d.nx), dtype=torch.float32, device="cuda")
    fx.fxmig_image(d, part_ref, img_ref)

    f = _cfn(fx)
    for _ in range(2):  # two calls in a row share the same fixed scratch
        slab = P0.clone()
        part = torch.full((nparts, d.nz, d.nx), float("nan"), dtype=torch.float32, device="cuda")
        rc = f(ctypes.byref(d), ctypes.c_void_p(slab.data_ptr()), ctypes.c_void_p(vel.data_ptr()),
               ctypes.c_void_p(table.data_ptr()), ctypes.c_void_p(part.data_ptr()), nparts, 0, d.nz, stream)
        assert rc == fx.FXMIG_OK, fx.fxmig_strerror(rc)
        img = torch.empty((d.nz, d.nx), dtype=torch.float32, device="cuda")
        fx.fxmig_image(d, part, img)
        torch.cuda.synchronize()
        # same kernel, same inputs, same arithmetic: bitwise equal
        assert np.array_equal(slab.cpu().numpy(), slab_ref.cpu().numpy())
        assert np.array_equal(img.cpu().numpy(), img_ref.cpu().numpy())
        assert torch.isfinite(img).all()


def test_noalloc_rejects_tables_beyond_its_scratch(fx):
    w = small_layered(nx=64, nz=4, seed=3)
    d = desc_of(fx, w, 0.5)
    d.nk = 1 << 16                        # 65536 entries x 13 taps x 16 B > 8 MiB
    dummy = ctypes.c_void_p(1 << 20)
    rc = _cfn(fx)(ctypes.byref(d), dummy, dummy, dummy, dummy, 1 << 20, 0, 1, None)
    assert rc == fx.FXMIG_ENOSPC
