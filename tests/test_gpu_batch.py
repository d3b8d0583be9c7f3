"""GPU batches of uneven lines in one persistent launch: every line matches
the FP64 oracle and repeats bit for bit; the autotuner leaves the inputs
untouched; the batch replays from a CUDA graph; partial depth ranges."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from fxhelp import TOL_IMAGE, TOL_SLICE, desc_of, layered_inputs, problem, rel_l2

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


def _uneven_lines(n=6, seed0=2000):
    """Small uneven lines: Nx, Nz, band and L drawn like the 64-line batch."""
    out = []
    for i in range(n):
        rng = np.random.default_rng(seed0 + i)
        nx = int(rng.integers(96, 700))
        nz = int(rng.integers(12, 40))
        f_hi = float(rng.integers(30, 61))
        L = int(rng.choice([8, 12, 17]))
        out.append(W.Workload(f"l{i}", nx=nx, dx=12.5, nt=512, dt=0.004, nz=nz, dz=5.0, f_lo=5.0, f_hi=f_hi, L=L,
                              seed=seed0 + i))
    return out


@pytest.fixture(scope="module")
def batch_case(oracle_mod):
    cases = []
    for w in _uneven_lines():
        v, refl, sec = layered_inputs(w)
        pr = problem(w, v, sec)
        table32 = pr["table"].astype(np.complex64)
        P0_32 = pr["P0"].astype(np.complex64)
        P, img = O.migrate(P0_32.astype(np.complex128), pr["vm"], table32.astype(np.complex128), pr["q"])
        cases.append((w, pr, table32, P0_32, P, img))
    return cases


class _Batch:
    """Device buffers of a batch and its fxmig_line array."""

    def __init__(self, fx, cases, plan, z_ranges=None):
        self.fx, self.cases, self.plan = fx, cases, plan
        descs = [desc_of(fx, w, pr["k_max"]) for (w, pr, _, _, _, _) in cases]
        self.nparts = fx.fxmig_batch_num_partials([fx.Line(d=d) for d in descs], plan)
        self.bufs, self.lines = [], []
        for i, ((w, pr, table32, P0_32, _, _), d) in enumerate(zip(cases, descs)):
            b = dict(d=d, slab=_cuda(P0_32, torch.complex64), vel=_cuda(pr["vm"], torch.float32),
                     table=_cuda(table32, torch.complex64),
                     partials=torch.zeros((self.nparts[i], d.nz, d.nx), dtype=torch.float32, device="cuda"),
                     image=torch.empty((d.nz, d.nx), dtype=torch.float32, device="cuda"))
            zb, ze = z_ranges[i] if z_ranges else (0, d.nz)
            self.bufs.append(b)
            self.lines.append(fx.line_of(d, b["slab"], b["vel"], b["table"], b["partials"], zb, ze))
        self.ws = torch.zeros(fx.fxmig_batch_workspace_bytes(self.lines), dtype=torch.uint8, device="cuda")

    def run(self):
        self.fx.fxmig_migrate_batch(self.lines, self.plan, self.ws)
        for b in self.bufs:
            self.fx.fxmig_image(b["d"], b["partials"], b["image"])

    def results(self):
        torch.cuda.synchronize()
        assert self.fx.fxmig_check(self.ws) == self.fx.FXMIG_OK
        return [(b["slab"].cpu().numpy(), b["image"].cpu().numpy()) for b in self.bufs]


# cluster sizes 1 and 2; caps of 1 (every line of a cluster-2 group cut in
# half), 2 (no cut) and 3 (the middle line cut)
@pytest.mark.parametrize("cluster,cap", [(1, 0), (2, 0), (2, 1), (2, 2), (2, 3), (1, 3)])
def test_batch_matches_oracle_and_is_deterministic(fx, batch_case, cluster, cap):
    plan = fx.BatchPlan(cluster=cluster, lines_cap=cap)
    bt = _Batch(fx, batch_case, plan)
    assert all(p >= 1 for p in bt.nparts)
    bt.run()
    got = bt.results()
    for (w, pr, table32, P0_32, P_ref, img_ref), (P, img) in zip(batch_case, got):
        assert rel_l2(P, P_ref) < TOL_SLICE, w.name
        assert rel_l2(img, img_ref) < TOL_IMAGE, w.name
    # the same batch again: bit for bit
    bt2 = _Batch(fx, batch_case, plan)
    bt2.run()
    for (P, img), (P2, img2) in zip(got, bt2.results()):
        assert np.array_equal(P, P2) and np.array_equal(img, img2)


def test_autotune_leaves_inputs_untouched(fx, batch_case):
    bt = _Batch(fx, batch_case, None)
    ws = torch.zeros(fx.fxmig_batch_workspace_bytes(bt.lines, autotune=True), dtype=torch.uint8, device="cuda")
    before = [(b["slab"].clone(), b["partials"].clone()) for b in bt.bufs]
    plan, ms = fx.fxmig_batch_autotune(bt.lines, ws)
    torch.cuda.synchronize()
    assert plan.cluster in (1, 2, 4, 8) and plan.lines_cap >= 0 and ms > 0
    for (s0, p0), b in zip(before, bt.bufs):
        assert torch.equal(s0, b["slab"]) and torch.equal(p0, b["partials"])
    # the tuned plan runs and matches the oracle
    bt2 = _Batch(fx, batch_case, plan)
    bt2.run()
    for (w, _, _, _, P_ref, img_ref), (P, img) in zip(batch_case, bt2.results()):
        assert rel_l2(img, img_ref) < TOL_IMAGE, w.name


def test_batch_replays_from_a_cuda_graph(fx, batch_case):
    plan = fx.BatchPlan(cluster=2)
    eager = _Batch(fx, batch_case, plan)
    eager.run()
    ref = eager.results()
    bt = _Batch(fx, batch_case, plan)
    slab0 = [b["slab"].clone() for b in bt.bufs]
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(stream):
        bt.run()   # warm-up outside capture (sets kernel attributes)
    torch.cuda.current_stream().wait_stream(stream)
    torch.cuda.synchronize()
    for b, s0 in zip(bt.bufs, slab0):
        b["slab"].copy_(s0)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        bt.run()
    for _ in range(2):
        for b, s0 in zip(bt.bufs, slab0):
            b["slab"].copy_(s0)
        g.replay()
        for (P, img), (Pr, ir) in zip(bt.results(), ref):
            assert np.array_equal(P, Pr) and np.array_equal(img, ir)


def test_batch_partial_depth_ranges(fx, batch_case):
    # each line stops half-way; the second batch call continues from there
    plan = fx.BatchPlan(cluster=2)
    halves = [(0, c[0].nz // 2) for c in batch_case]
    rest = [(c[0].nz // 2, c[0].nz) for c in batch_case]
    bt = _Batch(fx, batch_case, plan, halves)
    fx.fxmig_migrate_batch(bt.lines, plan, bt.ws)
    lines2 = [fx.line_of(b["d"], b["slab"], b["vel"], b["table"], b["partials"], zb, ze)
              for b, (zb, ze) in zip(bt.bufs, rest)]
    fx.fxmig_migrate_batch(lines2, plan, bt.ws)
    for b in bt.bufs:
        fx.fxmig_image(b["d"], b["partials"], b["image"])
    full = _Batch(fx, batch_case, plan)
    full.run()
    for (P, img), (Pf, imf) in zip(bt.results(), full.results()):
        assert np.array_equal(P, Pf) and np.array_equal(img, imf)
