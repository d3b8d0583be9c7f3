"""Benchmark: explicit f-x poststack depth migration on GB300.

Metric: extrapolated points x frequencies per second, Nx * Nz * Nw / t, where t
is the CUDA-event time of one depth loop (fxmig_migrate, all depth rows) plus
the imaging reduction (fxmig_image).  Workload: the 2048-trace layered medium
with dipping interfaces and a smoothed lens (Nx=2048, dx=12.5 m, Nt=2000,
dt=2 ms, Nz=800, dz=5 m, 5-60 Hz -> 221 frequencies, 25-tap operators, 1024
table entries); the input section is synthetic (seeded) and stands in for the
SEG/EAGE salt data the paper migrates, which is not available.

One JSON line on stdout (rank 0).  `--impl reference` times the FP64 CPU
oracle instead (the only other place this script runs the oracle is the
`cpu_baseline` leg).  Under torchrun every rank migrates its own, independently
seeded line (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import shutil
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

WORKLOADS = {w.name: w for w in (W.DIFFRACTOR_128, W.LAYERED_LENS_2048, W.LARGE_8192)}
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
NOMINAL_SMS = 152
NOMINAL_SM_MHZ = 2070.0


def ops_per_point(L: int) -> int:
    """Algorithmic FP32 operations per extrapolated point x frequency, each
    occupying one FP32 lane slot (an FMA counts once): L complex pair additions
    (2L), the L+1 complex multiply-adds of Eq. 1 with symmetric taps (4(L+1)):
    6L + 4.  (In flops, FMA = 2: 10L + 6.)"""
    return 6 * L + 4


def env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def __enter__(self):
        exe = shutil.which("nvidia-smi")
        if exe:
            self.proc = subprocess.Popen([exe, f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=5)

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax = float(p[2])
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": smax, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def make_inputs(w: W.Workload, seed: int):
    v, refl = W.layered_lens_model(w, seed=seed)
    sec = W.normal_incidence_section(w, v, refl, seed=seed)
    vm = (0.5 * v).astype(np.float32)            # exploding-reflector migration velocity
    return sec.astype(np.float32), vm


def k_max_of(w: W.Workload, vm_min: float) -> float:
    return 2.0 * math.pi * (w.i0 + w.nw - 1) / (w.nt * w.dt) / vm_min


# sources of the persistent depth-loop kernel (the traffic record is valid
# only for the exact sources it was captured from)
KERNEL_SOURCES = ("paper_1912_05529_gb300/csrc/migrate.cu", "paper_1912_05529_gb300/csrc/depth.cuh",
                  "paper_1912_05529_gb300/csrc/fir.cuh", "paper_1912_05529_gb300/csrc/fxmig_internal.cuh")


def kernel_traffic(workload: str):
    """DRAM bytes per launch of the persistent depth-loop kernel from the ncu
    capture recorded under profiles/, or None if the kernel sources changed
    since that capture (or none exists for this workload)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", f"traffic_k_depth_{workload}.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return rec.get("dram_bytes_per_launch") if rec.get("source_sha256") == h.hexdigest() else None


def load_peaks():
    try:
        with open(PEAKS_PATH) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": NOMINAL_SM_MHZ}, "fallback"


# ------------------------------------------------------------------ oracle legs
def oracle_run(w: W.Workload, sec, vm, threads: int = 0):
    """FP64 oracle migration of the whole workload; returns (seconds of the
    depth loop, final wavefield, image, cores used)."""
    import oracle as O
    om = O.omegas(w.i0, w.nw, w.nt, w.dt)
    kmax = float(om[-1] / float(vm.min()))
    table = O.design_operators(w.nk, kmax, w.dx, w.dz, w.L, w.theta_deg)
    _, dk = O.k_grid(w.nk, kmax)
    P0 = O.band_dft(sec.astype(np.float64), w.i0, w.nw)
    cores = threads or O.max_threads()
    t0 = time.perf_counter()
    P, img = O.migrate(P0, vm, table, O.q_values(om, dk), nthreads=cores)
    return time.perf_counter() - t0, P, img, cores


def oracle_single_thread(w: W.Workload, sec, vm, target_points: float = 3e7):
    """The FP64 oracle's depth loop on one host thread, on a bounded sample of
    the workload: a contiguous block of frequencies (about target_points
    points x frequencies) over the full line and all depth rows.  Returns
    (point*freq/s, sample description)."""
    import oracle as O
    om = O.omegas(w.i0, w.nw, w.nt, w.dt)
    kmax = float(om[-1] / float(vm.min()))
    table = O.design_operators(w.nk, kmax, w.dx, w.dz, w.L, w.theta_deg)
    _, dk = O.k_grid(w.nk, kmax)
    nws = max(1, min(w.nw, int(target_points // (w.nx * w.nz))))
    j0 = (w.nw - nws) // 2
    P0 = O.band_dft(sec.astype(np.float64), w.i0 + j0, nws)
    q = O.q_values(om[j0:j0 + nws], dk)
    t0 = time.perf_counter()
    O.migrate(P0, vm, table, q, nthreads=1)
    secs = time.perf_counter() - t0
    return (w.nx * w.nz * nws / secs,
            f"{nws} of {w.nw} frequencies (bins {w.i0 + j0}..{w.i0 + j0 + nws - 1}), all {w.nx} traces and "
            f"{w.nz} depth rows, one thread, {secs:.2f} s")


def run_reference(args, w):
    """The oracle on the host cores, same metric and workload; each step is a
    bounded sample: a contiguous block of frequencies over the full line and
    all depth rows (the cost per point x frequency does not depend on which
    frequencies are taken)."""
    import oracle as O
    rank, world, _ = env_rank()
    if rank != 0:
        return 0
    sec, vm = make_inputs(w, w.seed)
    om = O.omegas(w.i0, w.nw, w.nt, w.dt)
    kmax = float(om[-1] / float(vm.min()))
    table = O.design_operators(w.nk, kmax, w.dx, w.dz, w.L, w.theta_deg)
    _, dk = O.k_grid(w.nk, kmax)
    nws = min(w.nw, args.ref_freqs)
    j0 = (w.nw - nws) // 2
    P0 = O.band_dft(sec.astype(np.float64), w.i0 + j0, nws)
    q = O.q_values(om[j0:j0 + nws], dk)
    cores = O.max_threads()
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        O.migrate(P0, vm, table, q, nthreads=cores)
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    tot = sum(times)
    pts = w.nx * w.nz * nws
    val = pts * len(times) / tot
    line = {"impl": "reference", "metric": "extrapolated points*freq/s (Nx*Nz*Nw/s)", "value": val,
            "unit": "point*freq/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / len(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded layered+lens model)",
            "config": {"workload": w.name, "nx": w.nx, "nz": w.nz, "nw": w.nw, "L": w.L},
            "cpu_baseline": {"value": val, "unit": "point*freq/s", "cores": cores, "kind": "oracle",
                             "sample": f"{nws} of {w.nw} frequencies (bins {w.i0 + j0}..{w.i0 + j0 + nws - 1}), "
                                       f"all {w.nx} traces and {w.nz} depth rows per step"},
            "e2e": {"value": val, "unit": "point*freq/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def measure_learned(fx, d, b, slab0, steps, flush, train_steps=1000000, n_train=8192, seed=2, lr=(3e-3, 1e-5)):
    """The learned-operator form on the same inputs: train the operator network
    on the GPU (n_train designed operators at k ~ U[0, k_max], seeded), then
    time fxmig_mlp_migrate + fxmig_image like the plain form."""
    import torch
    k = torch.from_numpy(np.random.default_rng(seed).uniform(0.0, d.k_max, n_train)).cuda()
    taps = torch.empty((n_train, d.L + 1), dtype=torch.complex64, device="cuda")
    P = fx.fxmig_mlp_param_count(d.L)
    params = torch.from_numpy(W.mlp_init(seed, n_out=2 * (d.L + 1)).astype(np.float32)).cuda()
    m = torch.zeros(P, device="cuda")
    v = torch.zeros(P, device="cuda")
    ws_t = torch.empty(fx.fxmig_mlp_train_ws_bytes(d.L, n_train), dtype=torch.uint8, device="cuda")
    loss = torch.empty(train_steps, device="cuda")
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record()
    fx.fxmig_design_at(d, k, taps)
    fx.fxmig_mlp_train(d, params, m, v, 0, train_steps, lr[0], lr[1], train_steps, k, taps, ws_t, loss=loss)
    t1.record()
    torch.cuda.synchronize()
    train_ms = t0.elapsed_time(t1)
    nparts = fx.fxmig_mlp_num_partials(d)
    partials = torch.zeros((nparts, d.nz, d.nx), dtype=torch.float32, device="cuda")
    ws = torch.empty(fx.fxmig_workspace_bytes(d, fx.FXMIG_WS_MLP_MIGRATE), dtype=torch.uint8, device="cuda")
    image = torch.empty((d.nz, d.nx), dtype=torch.float32, device="cuda")
    slab = torch.empty_like(slab0)
    stream = torch.cuda.current_stream()
    for _ in range(2):
        slab.copy_(slab0)
        fx.fxmig_mlp_migrate(d, slab, b.vel, params, partials, 0, d.nz, ws)
        fx.fxmig_image(d, partials, image)
    torch.cuda.synchronize()
    if fx.fxmig_check(ws) != fx.FXMIG_OK:
        raise RuntimeError("learned form: device status " + fx.fxmig_strerror(fx.fxmig_check(ws)))
    ms = []
    for _ in range(steps):
        slab.copy_(slab0)
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fx.fxmig_mlp_migrate(d, slab, b.vel, params, partials, 0, d.nz, ws)
        fx.fxmig_image(d, partials, image)
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    l = loss.cpu().numpy()
    return {"ms_per_step": float(np.mean(ms)), "train_ms": train_ms, "train_steps": train_steps,
            "train_samples": n_train, "train_lr": list(lr), "train_loss_first_last": [float(l[0]), float(l[-1])],
            "image": image.cpu().numpy(), "params": params}


PREC_NAMES = ("FP16_SPLIT", "BF16_SPLIT", "FP16", "BF16")


def measure_precision(fx, d, b, slab0, steps, flush, launch, prec):
    """A 16-bit storage form of the persistent depth loop on the same inputs:
    mean CUDA-event time of fxmig_migrate_ex + fxmig_image, and its image."""
    import torch
    lc = fx.Launch(mode=fx.FXMIG_MODE_PERSISTENT, cluster=launch.cluster, groups=launch.groups,
                   warps=launch.warps, precision=prec, ctas_per_sm=launch.ctas_per_sm)
    nparts = fx.fxmig_num_partials(d, lc)
    partials = torch.zeros((nparts, d.nz, d.nx), dtype=torch.float32, device="cuda")
    image = torch.empty((d.nz, d.nx), dtype=torch.float32, device="cuda")
    slab = torch.empty_like(slab0)
    stream = torch.cuda.current_stream()
    for _ in range(2):
        slab.copy_(slab0)
        fx.fxmig_migrate_ex(d, lc, slab, b.vel, b.table, partials, 0, d.nz, b.ws_mig)
        fx.fxmig_image(d, partials, image)
    torch.cuda.synchronize()
    if fx.fxmig_check(b.ws_mig) != fx.FXMIG_OK:
        raise RuntimeError("16-bit form: device status " + fx.fxmig_strerror(fx.fxmig_check(b.ws_mig)))
    ms = []
    for _ in range(steps):
        slab.copy_(slab0)
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fx.fxmig_migrate_ex(d, lc, slab, b.vel, b.table, partials, 0, d.nz, b.ws_mig)
        fx.fxmig_image(d, partials, image)
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    return {"ms_per_step": float(np.mean(ms)), "partials": nparts, "image": image.cpu().numpy()}


def measure_per_depth(fx, d, b, slab0, steps, flush):
    """The per-depth-launch form (one Eq. 1 launch per depth row, the wavefield
    streaming through L2/HBM) on the same inputs: mean CUDA-event time of
    fxmig_migrate_ex + fxmig_image, its image, and the migrate time alone for
    the wavefield-traffic rate (16 bytes per point x frequency)."""
    import torch
    lc = fx.Launch(mode=fx.FXMIG_MODE_PER_DEPTH)
    nparts = fx.fxmig_num_partials(d, lc)
    partials = torch.zeros((nparts, d.nz, d.nx), dtype=torch.float32, device="cuda")
    image = torch.empty((d.nz, d.nx), dtype=torch.float32, device="cuda")
    slab = torch.empty_like(slab0)
    stream = torch.cuda.current_stream()
    for _ in range(2):
        slab.copy_(slab0)
        fx.fxmig_migrate_ex(d, lc, slab, b.vel, b.table, partials, 0, d.nz, b.ws_mig)
        fx.fxmig_image(d, partials, image)
    torch.cuda.synchronize()
    if fx.fxmig_check(b.ws_mig) != fx.FXMIG_OK:
        raise RuntimeError("per-depth form: device status " + fx.fxmig_strerror(fx.fxmig_check(b.ws_mig)))
    ms, mig = [], []
    for _ in range(steps):
        slab.copy_(slab0)
        flush.fill_(1)
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        fx.fxmig_migrate_ex(d, lc, slab, b.vel, b.table, partials, 0, d.nz, b.ws_mig)
        e1.record(stream)
        fx.fxmig_image(d, partials, image)
        e2.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e2))
        mig.append(e0.elapsed_time(e1))
    # the ceiling while the wavefield stays in L2: a device copy of a buffer
    # of the wavefield's size, back and forth (read + write bytes per second)
    nb = d.nw * d.nx * 8
    src = torch.empty(nb, dtype=torch.uint8, device="cuda")
    dst = torch.empty_like(src)
    for _ in range(20):
        dst.copy_(src)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 400
    e0.record(stream)
    for i in range(reps):
        (dst if i & 1 else src).copy_(src if i & 1 else dst)
    e1.record(stream)
    torch.cuda.synchronize()
    l2_gbs = 2.0 * nb * reps / (e0.elapsed_time(e1) * 1e-3) / 1e9
    # the L2 bandwidth itself: 32 MB buffers (both L2-resident), copied back and forth
    big = 32 << 20
    src = torch.empty(big, dtype=torch.uint8, device="cuda")
    dst = torch.empty_like(src)
    for _ in range(10):
        dst.copy_(src)
    reps = 100
    e0.record(stream)
    for i in range(reps):
        (dst if i & 1 else src).copy_(src if i & 1 else dst)
    e1.record(stream)
    torch.cuda.synchronize()
    l2_bw = 2.0 * big * reps / (e0.elapsed_time(e1) * 1e-3) / 1e9
    return {"ms_per_step": float(np.mean(ms)), "migrate_ms": float(np.mean(mig)), "partials": nparts,
            "kernels_per_step": 4 + d.nz, "graph": "the depth launches replayed as one CUDA graph",
            "l2_copy_gbs": l2_gbs, "l2_bandwidth_gbs": l2_bw, "image": image.cpu().numpy()}


# --------------------------------------------------------- the large line
LARGE_WINDOW = (3968, 256)   # traces [x0, x0 + n) of the 8192-trace line for the oracle check


def measure_large(fx, flush, steps: int = 3, oracle_check: bool = True):
    """The 8192-trace line (35-tap operators, 601 frequencies, 2000 depth
    steps): FP32 and every 16-bit storage form of the persistent depth loop
    over the whole line (mean CUDA-event time of fxmig_migrate_ex +
    fxmig_image, L2 flushed), and each form's image on a 256-trace window of
    the line, migrated as its own problem with the oracle's operator table,
    against the FP64 oracle on that window (the bar is image rel-L2 <= 1e-2)."""
    import torch

    import oracle as O
    w = W.LARGE_8192
    sec, vm = make_inputs(w, w.seed)
    k_max = k_max_of(w, float(vm.min()))
    d = fx.Desc(nx=w.nx, nz=w.nz, nt=w.nt, nw=w.nw, i0=w.i0, L=w.L, nk=w.nk, dx=w.dx, dz=w.dz, dt=w.dt,
                theta_max_deg=w.theta_deg, k_max=k_max)
    table = torch.empty((w.nk, w.L + 1), dtype=torch.complex64, device="cuda")
    fx.fxmig_design_operators(d, table)
    slab0 = torch.empty((w.nw, w.nx), dtype=torch.complex64, device="cuda")
    ws_t = torch.empty(fx.fxmig_workspace_bytes(d, fx.FXMIG_WS_T2F), dtype=torch.uint8, device="cuda")
    fx.fxmig_t2f(d, torch.from_numpy(sec).cuda(), slab0, ws_t)
    del ws_t
    vel = torch.from_numpy(vm).cuda()
    slab = torch.empty_like(slab0)
    ws = torch.empty(fx.fxmig_workspace_bytes(d, fx.FXMIG_WS_MIGRATE), dtype=torch.uint8, device="cuda")
    image = torch.empty((w.nz, w.nx), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    names = ("FP32",) + PREC_NAMES
    res = {}
    for name in names:
        lc = fx.Launch(mode=fx.FXMIG_MODE_PERSISTENT, precision=getattr(fx, "FXMIG_PREC_" + name))
        partials = torch.empty((fx.fxmig_num_partials(d, lc), w.nz, w.nx), dtype=torch.float32, device="cuda")
        ms = []
        for it in range(steps + 1):
            slab.copy_(slab0)
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fx.fxmig_migrate_ex(d, lc, slab, vel, table, partials, 0, w.nz, ws)
            fx.fxmig_image(d, partials, image)
            e1.record(stream)
            torch.cuda.synchronize()
            if it > 0:
                ms.append(e0.elapsed_time(e1))
        if fx.fxmig_check(ws) != fx.FXMIG_OK:
            raise RuntimeError(f"large line {name}: device status " + fx.fxmig_strerror(fx.fxmig_check(ws)))
        shape = fx.fxmig_launch_shape(d, lc)
        res[name] = {"ms_per_step": float(np.mean(ms)), "value": w.points / (float(np.mean(ms)) * 1e-3),
                     "launch": {"cluster": shape.cluster, "groups": shape.groups, "waves": shape.waves,
                                "items_per_lane": shape.items_per_lane}}
        del partials
    del slab, slab0, ws, image, vel, table
    torch.cuda.empty_cache()

    plain = res["FP32"]["ms_per_step"]
    if not oracle_check:
        return {"large_8192_" + nm.lower(): {"value": r["value"], "unit": "point*freq/s",
                                             "ms_per_step": r["ms_per_step"],
                                             "speedup_vs_plain": plain / r["ms_per_step"], "launch": r["launch"]}
                for nm, r in res.items()}
    # the window problem: the same line's model and section, 256 traces
    x0, n = LARGE_WINDOW
    om = O.omegas(w.i0, w.nw, w.nt, w.dt)
    tab = O.design_operators(w.nk, k_max, w.dx, w.dz, w.L, w.theta_deg).astype(np.complex64)
    _, dk = O.k_grid(w.nk, k_max)
    P0 = O.band_dft(sec[x0:x0 + n].astype(np.float64), w.i0, w.nw).astype(np.complex64)
    vmw = np.ascontiguousarray(vm[:, x0:x0 + n])
    ts = time.perf_counter()
    _, img_ref = O.migrate(P0.astype(np.complex128), vmw, tab.astype(np.complex128), O.q_values(om, dk))
    oracle_s = time.perf_counter() - ts
    dwin = fx.Desc(nx=n, nz=w.nz, nt=w.nt, nw=w.nw, i0=w.i0, L=w.L, nk=w.nk, dx=w.dx, dz=w.dz, dt=w.dt,
                   theta_max_deg=w.theta_deg, k_max=k_max)
    ws = torch.empty(fx.fxmig_workspace_bytes(dwin, fx.FXMIG_WS_MIGRATE), dtype=torch.uint8, device="cuda")
    velw, tabw = torch.from_numpy(vmw).cuda(), torch.from_numpy(tab).cuda()
    imgw = torch.empty((w.nz, n), dtype=torch.float32, device="cuda")
    bar = 1e-2
    forms = {}
    for name in names:
        lc = fx.Launch(mode=fx.FXMIG_MODE_PERSISTENT, precision=getattr(fx, "FXMIG_PREC_" + name))
        parts = torch.empty((fx.fxmig_num_partials(dwin, lc), w.nz, n), dtype=torch.float32, device="cuda")
        sl = torch.from_numpy(P0).cuda()
        fx.fxmig_migrate_ex(dwin, lc, sl, velw, tabw, parts, 0, w.nz, ws)
        fx.fxmig_image(dwin, parts, imgw)
        torch.cuda.synchronize()
        e = float(np.linalg.norm(imgw.cpu().numpy() - img_ref) / np.linalg.norm(img_ref))
        r = res[name]
        f = {"value": r["value"], "unit": "point*freq/s", "ms_per_step": r["ms_per_step"],
             "speedup_vs_plain": plain / r["ms_per_step"],
             "what": ("FP32 wavefield and taps" if name == "FP32" else
                      "wavefield lines and taps stored in 16 bits" + (" (taps as hi + lo)" if "SPLIT" in name else "")
                      + ", FP32 arithmetic") + "; 8192 traces x 2000 depths x 601 frequencies, L = 17",
             "launch": r["launch"],
             "image_rel_l2_window_vs_fp64_oracle": e,
             "window": f"traces [{x0}, {x0 + n}) as a {n}-trace problem, all 2000 depths and 601 frequencies"}
        if name != "FP32":
            f["bar"] = bar
            f["status"] = "meets bar" if e <= bar else "above bar"
        forms["large_8192_" + name.lower()] = f
    forms["large_8192_fp32"]["oracle_window_seconds"] = oracle_s
    return forms


# ------------------------------------------------ 3-D, 2-D extrapolators
FX3D_CHECK_LINES = (0, 35, 70)   # frequency lines of the band migrated by the oracle (all depths, full grid)


def ops_per_point_3d(L: int, nx_thread: int = 4) -> int:
    """FP32-pipe lane operations per point x frequency of the 3-D step as the
    kernel takes it: the sums of rows y + j and y - j over a thread's window
    (L (nx_thread + 2L) complex additions shared by its nx_thread points),
    then per point and row pair L column-pair additions and L + 1 complex
    multiply-adds (two packed f32x2 operations each)."""
    f2 = L * (nx_thread + 2 * L) / nx_thread + (L + 1) * L + 2 * (L + 1) ** 2
    return int(round(2 * f2))


def measure_fx3d(fx, flush, steps: int = 3, oracle_check: bool = True):
    """3-D migration with 2-D extrapolators on the 128 x 128 x 150 layered +
    lens model (71 frequencies, 13 x 13 stencils): t->f of the flattened
    section, the 2-D operator table and the image on the GPU; the mean
    CUDA-event time of fxmig3d_migrate + fxmig3d_image (L2 flushed); and three
    frequency lines migrated by the GPU and by the FP64 oracle from the same
    inputs (all depths, the whole grid)."""
    import torch

    import oracle as O
    w = W.LAYERED_LENS_3D
    v, refl = W.layered_lens_model_3d(w)
    vm = (0.5 * v).astype(np.float32)
    sec = W.normal_incidence_section_3d(w, v, refl).astype(np.float32)
    om = O.omegas(w.i0, w.nw, w.nt, w.dt)
    k_max = float(om[-1] / float(vm.min()))
    d = fx.Desc3d(nx=w.nx, ny=w.ny, nz=w.nz, nt=w.nt, nw=w.nw, i0=w.i0, L=w.L, nk=w.nk, dx=w.dx, dz=w.dz,
                  dt=w.dt, theta_max_deg=w.theta_deg, k_max=k_max)
    d2 = fx.flat_desc(d)
    npts = w.nx * w.ny
    slab0 = torch.empty((w.nw, npts), dtype=torch.complex64, device="cuda")
    ws_t = torch.empty(fx.fxmig_workspace_bytes(d2, fx.FXMIG_WS_T2F), dtype=torch.uint8, device="cuda")
    fx.fxmig_t2f(d2, torch.from_numpy(sec.reshape(npts, w.nt)).cuda(), slab0, ws_t)
    del ws_t
    table = torch.empty((w.nk, fx.fxmig3d_num_taps(w.L)), dtype=torch.complex64, device="cuda")
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record()
    fx.fxmig3d_design_operators(d, table)
    t1.record()
    torch.cuda.synchronize()
    design_ms = t0.elapsed_time(t1)
    vel = torch.from_numpy(vm).cuda()
    slab = torch.empty_like(slab0)
    partials = torch.empty((fx.fxmig3d_num_partials(d), w.nz, npts), dtype=torch.float32, device="cuda")
    ws = torch.empty(fx.fxmig3d_workspace_bytes(d), dtype=torch.uint8, device="cuda")
    image = torch.empty((w.nz, npts), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    ms = []
    for it in range(steps + 2):
        slab.copy_(slab0)
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fx.fxmig3d_migrate(d, slab, vel, table, partials, 0, w.nz, ws)
        fx.fxmig3d_image(d, partials, image)
        e1.record(stream)
        torch.cuda.synchronize()
        if it >= 2:
            ms.append(e0.elapsed_time(e1))
    if fx.fxmig_check(ws) != fx.FXMIG_OK:
        raise RuntimeError("3-D form: device status " + fx.fxmig_strerror(fx.fxmig_check(ws)))
    t = float(np.mean(ms))
    ops = ops_per_point_3d(w.L)
    peaks, _ = load_peaks()
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    props = torch.cuda.get_device_properties(0)
    fp32_peak = props.multi_processor_count * 128 * sm_mhz * 1e6
    # shared-memory bytes per output: a thread's 2L + 1 row loads of its
    # window (4 + 2L values of 8 bytes) for its 4 points, and the tile store
    smem_bytes = 8 * ((2 * w.L + 1) * (4 + 2 * w.L) / 4.0 + (8 + 2 * w.L) * (128 + 2 * w.L) / 1024.0)
    smem_peak = props.multi_processor_count * 128 * sm_mhz * 1e6   # 128 bytes per cycle and SM
    out = {"value": w.points / (t * 1e-3), "unit": "point*freq/s", "ms_per_step": t,
           "what": "3-D f-x migration with 2-D extrapolators (13 x 13 stencils, 28 unique taps, table lookup per "
                   "point), one launch per depth step, 4 points per thread; 128 x 128 points x 150 depths x 71 "
                   "frequencies",
           "design_ms": design_ms, "ops_per_point": ops,
           "frac_of_fp32_peak": w.points * ops / (t * 1e-3) / fp32_peak,
           "smem_bytes_per_point": smem_bytes,
           "frac_of_smem_bandwidth": w.points * smem_bytes / (t * 1e-3) / smem_peak,
           "bound": "latency of the per-plane tile loads and the tap loads (neither the FP32 pipe nor shared "
                    "memory is saturated; ncu: long-scoreboard stalls first)"}
    del slab, partials, image, ws
    if not oracle_check:
        return out
    # the oracle on three frequency lines (the GPU migrates the same lines as a problem of their own)
    lines = list(FX3D_CHECK_LINES)
    P0 = slab0.cpu().numpy().reshape(w.nw, w.ny, w.nx)[lines]
    tab = table.cpu().numpy()
    _, dk = O.k_grid(w.nk, k_max)
    q = O.q_values(om, dk)[lines]
    import oracle.fx3d as F
    ts = time.perf_counter()
    _, img_ref = F.migrate3d(P0.astype(np.complex128), vm, tab.astype(np.complex128), q)
    oracle_s = time.perf_counter() - ts
    errs = []
    img_sum = np.zeros_like(img_ref)
    for j, line in enumerate(lines):
        dj = fx.Desc3d(nx=w.nx, ny=w.ny, nz=w.nz, nt=w.nt, nw=1, i0=w.i0 + line, L=w.L, nk=w.nk, dx=w.dx,
                       dz=w.dz, dt=w.dt, theta_max_deg=w.theta_deg, k_max=k_max)
        sl = torch.from_numpy(np.ascontiguousarray(P0[j:j + 1])).cuda()
        pj = torch.empty((fx.fxmig3d_num_partials(dj), w.nz, npts), dtype=torch.float32, device="cuda")
        wsj = torch.empty(fx.fxmig3d_workspace_bytes(dj), dtype=torch.uint8, device="cuda")
        ij = torch.empty((w.nz, npts), dtype=torch.float32, device="cuda")
        fx.fxmig3d_migrate(dj, sl, vel, table, pj, 0, w.nz, wsj)
        fx.fxmig3d_image(dj, pj, ij)
        torch.cuda.synchronize()
        img_sum += ij.cpu().numpy().reshape(img_ref.shape)
    err = float(np.linalg.norm(img_sum - img_ref) / np.linalg.norm(img_ref))
    out.update({"image_rel_l2_vs_fp64_oracle": err,
                "check": f"frequency lines {lines} of the band, the whole grid and all depths, each migrated "
                         "by the GPU and by the FP64 oracle (oracle/fx3d.py) with the GPU's table",
                "oracle_seconds": oracle_s})
    return out


# ------------------------------------------------- the learned form's judge
LEARNED_WINDOW = (1024, 256)                           # traces of the 2048-trace line (the lens's left edge)
LEARNED_BLOCKS = ((0, 8), (71, 8), (142, 8), (213, 8))  # frequency blocks (first line, lines) of the band


def phase_errors(h, k, dx, dz, theta_deg, n=256):
    """Per tap set h[i] (designed for wavenumber k[i]): the largest phase error
    |arg(H(kx) / exp(i sqrt(k^2 - kx^2) dz))| over the design passband
    kx <= k sin(theta), H(kx) = h0 + 2 sum_n h_n cos(n kx dx)."""
    kx = np.linspace(0.0, 1.0, n)[None, :] * (k[:, None] * math.sin(math.radians(theta_deg)))
    L = h.shape[1] - 1
    c = np.where(np.arange(L + 1) == 0, 1.0, 2.0)
    H = np.einsum("kn,kmn->km", h, c * np.cos(kx[:, :, None] * dx * np.arange(L + 1)))
    D = np.exp(1j * np.sqrt(np.maximum(k[:, None] ** 2 - kx ** 2, 0.0)) * dz)
    return np.abs(np.angle(H / D)).max(axis=1)


def judge_learned(fx, d, params, w, sec, vm):
    """The learned-operator form against the continuous-velocity FP64 reference
    (operators designed at every point's exact wavenumber, oracle
    migrate_pointwise with the oracle's design), on a 256-trace window of the
    line through the lens edge, all 800 depth steps, 4 blocks of 8
    frequencies spread over the band; the table form on the same window
    against the same reference for comparison; and the phase error of the
    network's tap sets and of the designed ones over the band of k."""
    import torch

    import oracle as O
    x0, n = LEARNED_WINDOW
    om = O.omegas(w.i0, w.nw, w.nt, w.dt)
    J = np.concatenate([np.arange(j0, j0 + nb) for j0, nb in LEARNED_BLOCKS])
    P0 = O.band_dft(sec[x0:x0 + n].astype(np.float64), w.i0, w.nw)[J].astype(np.complex64)
    vmw = np.ascontiguousarray(vm[:, x0:x0 + n])
    # operators designed once per distinct (frequency, slowness) of the window
    su = np.unique(O.slowness(vmw))
    ku = np.unique((om[J][:, None] * su.astype(np.float64)[None, :]).ravel())
    ts = time.perf_counter()
    hu = O.design_at(ku, w.dx, w.dz, w.L, w.theta_deg)
    design_s = time.perf_counter() - ts

    def taps_fn(wp, sp):   # design_taps_fn with the designs computed above
        k = np.asarray(wp, dtype=np.float64) * np.asarray(sp, dtype=np.float32).astype(np.float64)
        return hu[np.searchsorted(ku, k)]
    ts = time.perf_counter()
    _, img_ref = O.migrate_pointwise(P0.astype(np.complex128), vmw, om[J], taps_fn)
    oracle_s = time.perf_counter() - ts
    k_max = d.k_max
    tab = O.design_operators(w.nk, k_max, w.dx, w.dz, w.L, w.theta_deg).astype(np.complex64)
    velw, tabw = torch.from_numpy(vmw).cuda(), torch.from_numpy(tab).cuda()
    img_l = np.zeros((w.nz, n))
    img_t = np.zeros((w.nz, n))
    pos = 0
    for j0, nb in LEARNED_BLOCKS:
        db = fx.Desc(nx=n, nz=w.nz, nt=w.nt, nw=nb, i0=w.i0 + j0, L=w.L, nk=w.nk, dx=w.dx, dz=w.dz, dt=w.dt,
                     theta_max_deg=w.theta_deg, k_max=k_max)
        imgb = torch.empty((w.nz, n), dtype=torch.float32, device="cuda")
        # learned operators
        parts = torch.zeros((fx.fxmig_mlp_num_partials(db), w.nz, n), dtype=torch.float32, device="cuda")
        wsm = torch.empty(fx.fxmig_workspace_bytes(db, fx.FXMIG_WS_MLP_MIGRATE), dtype=torch.uint8, device="cuda")
        sl = torch.from_numpy(np.ascontiguousarray(P0[pos:pos + nb])).cuda()
        fx.fxmig_mlp_migrate(db, sl, velw, params, parts, 0, w.nz, wsm)
        fx.fxmig_image(db, parts, imgb)
        torch.cuda.synchronize()
        if fx.fxmig_check(wsm) != fx.FXMIG_OK:
            raise RuntimeError("learned window: device status " + fx.fxmig_strerror(fx.fxmig_check(wsm)))
        img_l += imgb.cpu().numpy()
        # the operator table
        wst = torch.empty(fx.fxmig_workspace_bytes(db, fx.FXMIG_WS_MIGRATE), dtype=torch.uint8, device="cuda")
        parts = torch.empty((fx.fxmig_num_partials(db), w.nz, n), dtype=torch.float32, device="cuda")
        sl = torch.from_numpy(np.ascontiguousarray(P0[pos:pos + nb])).cuda()
        fx.fxmig_migrate_ex(db, None, sl, velw, tabw, parts, 0, w.nz, wst)
        fx.fxmig_image(db, parts, imgb)
        torch.cuda.synchronize()
        img_t += imgb.cpu().numpy()
        pos += nb
    rel = lambda a: float(np.linalg.norm(a - img_ref) / np.linalg.norm(img_ref))
    # phase error per tap set over k in (0, k_max]
    kk = np.linspace(k_max / 64, k_max, 64)
    tk = torch.empty((kk.size, w.L + 1), dtype=torch.complex64, device="cuda")
    fx.fxmig_mlp_taps(d, params, torch.from_numpy(kk).cuda(), tk)
    torch.cuda.synchronize()
    pe_net = phase_errors(tk.cpu().numpy().astype(np.complex128), kk, w.dx, w.dz, w.theta_deg)
    pe_des = phase_errors(O.design_at(kk, w.dx, w.dz, w.L, w.theta_deg), kk, w.dx, w.dz, w.theta_deg)
    return {"image_rel_l2_vs_continuous_fp64": rel(img_l),
            "table_image_rel_l2_vs_continuous_fp64": rel(img_t),
            "bar": 1e-2, "status": "meets bar" if rel(img_l) <= 1e-2 else "above bar",
            "window": f"traces [{x0}, {x0 + n}) of the line as a {n}-trace problem, all {w.nz} depth steps, "
                      f"frequency lines {', '.join(f'[{a}, {a + b})' for a, b in LEARNED_BLOCKS)} of {w.nw}",
            "reference": "oracle migrate_pointwise with operators designed at every point's exact k = w s "
                         f"({ku.size} designs, {design_s:.1f} s; depth loop {oracle_s:.1f} s)",
            "phase_error_rad": {"k_samples": int(kk.size),
                                "network": {"max": float(pe_net.max()), "mean": float(pe_net.mean())},
                                "designed": {"max": float(pe_des.max()), "mean": float(pe_des.mean())}}}


# ------------------------------------------------------------ batched lines
BATCH_NAME = "batched_64"


def batch_inputs(seed0: int):
    """64 uneven lines (seeded Nx, Nz, band, L), each with its own seeded
    layered velocity model; the wavefield at the surface is a seeded random
    band of complex values (the migration's cost does not depend on them)."""
    out = []
    for w in W.batched_lines(64, seed0=seed0):
        v, _ = W.layered_lens_model(w, lens=False)
        vm = (0.5 * v).astype(np.float32)
        rng = np.random.default_rng(w.seed + 77)
        P0 = (rng.standard_normal((w.nw, w.nx)) + 1j * rng.standard_normal((w.nw, w.nx))).astype(np.complex64)
        out.append((w, vm, P0))
    return out


def batch_setup(fx, rank: int):
    """The 64 uneven lines on the device, the autotuned batch plan and one CUDA
    graph of the whole step (batch depth loop + per-line imaging)."""
    import torch
    inputs = batch_inputs(1000 + 1000 * rank)
    bufs = []
    for w, vm, P0 in inputs:
        d = fx.Desc(nx=w.nx, nz=w.nz, nt=w.nt, nw=w.nw, i0=w.i0, L=w.L, nk=w.nk, dx=w.dx, dz=w.dz, dt=w.dt,
                    theta_max_deg=w.theta_deg, k_max=k_max_of(w, float(vm.min())))
        b = dict(d=d, w=w, slab0=torch.from_numpy(P0).cuda(), vel=torch.from_numpy(vm).cuda(),
                 table=torch.empty((w.nk, w.L + 1), dtype=torch.complex64, device="cuda"),
                 image=torch.empty((w.nz, w.nx), dtype=torch.float32, device="cuda"))
        b["slab"] = b["slab0"].clone()
        fx.fxmig_design_operators(d, b["table"])
        bufs.append(b)

    def lines_for(plan):
        nparts = fx.fxmig_batch_num_partials([fx.Line(d=b["d"]) for b in bufs], plan)
        out = []
        for b, p in zip(bufs, nparts):
            b["partials"] = torch.empty((p, b["d"].nz, b["d"].nx), dtype=torch.float32, device="cuda")
            out.append(fx.line_of(b["d"], b["slab"], b["vel"], b["table"], b["partials"]))
        return out

    # autotune on scratch copies, then the chosen plan
    lines = lines_for(None)
    ws_t = torch.empty(fx.fxmig_batch_workspace_bytes(lines, autotune=True), dtype=torch.uint8, device="cuda")
    plan, tune_ms = fx.fxmig_batch_autotune(lines, ws_t)
    del ws_t
    lines = lines_for(plan)
    ws = torch.empty(fx.fxmig_batch_workspace_bytes(lines), dtype=torch.uint8, device="cuda")

    def step():
        fx.fxmig_migrate_batch(lines, plan, ws)
        for b in bufs:
            fx.fxmig_image(b["d"], b["partials"], b["image"])

    def restore():
        for b in bufs:
            b["slab"].copy_(b["slab0"])

    restore()
    step()   # eager run (kernel attributes), then capture the whole step in one graph
    torch.cuda.synchronize()
    if fx.fxmig_check(ws) != fx.FXMIG_OK:
        raise RuntimeError("batch: device status " + fx.fxmig_strerror(fx.fxmig_check(ws)))
    graph = torch.cuda.CUDAGraph()
    restore()
    with torch.cuda.graph(graph):
        step()
    return dict(inputs=inputs, bufs=bufs, plan=plan, tune_ms=tune_ms, ws=ws, graph=graph, restore=restore,
                points=sum(b["w"].points for b in bufs),
                ops=sum(b["w"].points * ops_per_point(b["w"].L) for b in bufs))


def batch_timed(B, steps: int, flush):
    """CUDA-event times (ms) of `steps` graph replays, L2 flushed before each."""
    import torch
    stream = torch.cuda.current_stream()
    ms = []
    for _ in range(steps):
        B["restore"]()
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        B["graph"].replay()
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    return ms


def batch_compare(fx, B):
    """The comparison forms, once each: a persistent launch per line, and one
    launch per line per depth step (ms for all 64 lines)."""
    import torch
    stream = torch.cuda.current_stream()

    def per_line(launch):
        total = 0.0
        for b in B["bufs"]:
            d = b["d"]
            n = fx.fxmig_num_partials(d, launch)
            parts = torch.empty((n, d.nz, d.nx), dtype=torch.float32, device="cuda")
            wsl = torch.empty(fx.fxmig_workspace_bytes(d, fx.FXMIG_WS_MIGRATE), dtype=torch.uint8, device="cuda")
            b["slab"].copy_(b["slab0"])
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fx.fxmig_migrate_ex(d, launch, b["slab"], b["vel"], b["table"], parts, 0, d.nz, wsl)
            fx.fxmig_image(d, parts, b["image"])
            e1.record(stream)
            torch.cuda.synchronize()
            total += e0.elapsed_time(e1)
        return total
    per_line(None)   # warm-up (kernel attributes, first-touch)
    return per_line(None), per_line(fx.Launch(mode=fx.FXMIG_MODE_PER_DEPTH))


def batch_parity(inputs, img_gpu, n=2):
    """FP64 oracle on the n smallest lines: (seconds of the depth loops, points,
    image rel-L2 per sampled line)."""
    import oracle as O
    O.build()
    small = sorted(range(len(inputs)), key=lambda i: inputs[i][0].points)[:n]
    secs, errs, pts = 0.0, [], 0
    for i in small:
        w, vm, P0 = inputs[i]
        om = O.omegas(w.i0, w.nw, w.nt, w.dt)
        k_max = float(om[-1] / float(vm.min()))
        table = O.design_operators(w.nk, k_max, w.dx, w.dz, w.L, w.theta_deg).astype(np.complex64)
        _, dk = O.k_grid(w.nk, k_max)
        ts = time.perf_counter()
        _, img_ref = O.migrate(P0.astype(np.complex128), vm, table.astype(np.complex128), O.q_values(om, dk))
        secs += time.perf_counter() - ts   # the depth loop only
        pts += w.points
        errs.append(float(np.linalg.norm(img_gpu[i] - img_ref) / np.linalg.norm(img_ref)))
    return secs, pts, errs


def run_batch(args):
    import torch
    import torch.distributed as dist
    rank, world, local = env_rank()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_1912_05529_gb300 import build
    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        dist.barrier()
    import paper_1912_05529_gb300 as fx

    B = batch_setup(fx, rank)
    inputs, bufs, plan, tune_ms, graph = B["inputs"], B["bufs"], B["plan"], B["tune_ms"], B["graph"]
    points, ops = B["points"], B["ops"]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        B["restore"]()
        graph.replay()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    with ClockSampler(local) as clk:
        time.sleep(0.3)
        ms = batch_timed(B, args.steps, flush)
    tot_ms = sum(ms)
    if world > 1:
        t = torch.tensor([tot_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tot_ms = float(t.item())
    value = world * points * args.steps / (tot_ms * 1e-3)
    img_gpu = [b["image"].cpu().numpy() for b in bufs]

    # end to end: wavefields and velocities from pinned host memory, the
    # captured step, images back to pinned host memory
    slab_h = [torch.from_numpy(P0).pin_memory() for _, _, P0 in inputs]
    vel_h = [torch.from_numpy(vm).pin_memory() for _, vm, _ in inputs]
    img_h = [torch.empty((b["d"].nz, b["d"].nx), dtype=torch.float32, pin_memory=True) for b in bufs]
    e2e_ms = []
    for it in range(args.steps + 1):
        flush.fill_(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for b, sh, vh in zip(bufs, slab_h, vel_h):
            b["slab"].copy_(sh, non_blocking=True)
            b["vel"].copy_(vh, non_blocking=True)
        graph.replay()
        for b, ih in zip(bufs, img_h):
            ih.copy_(b["image"], non_blocking=True)
        torch.cuda.synchronize()
        if it > 0:
            e2e_ms.append(1e3 * (time.perf_counter() - t0))
    e2e_val = world * points * len(e2e_ms) / (sum(e2e_ms) * 1e-3)
    h2d = sum(P0.nbytes + vm.nbytes for _, vm, P0 in inputs)
    d2h = sum(b["d"].nz * b["d"].nx * 4 for b in bufs)
    t_persistent, t_per_depth = batch_compare(fx, B)

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0
    peaks, peak_src = load_peaks()
    sm_max = float(peaks.get("sm_max_mhz", NOMINAL_SM_MHZ))
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    peak_tops = sms * 128 * sm_max * 1e6 / 1e12
    mean_ms = tot_ms / args.steps
    achieved = ops / (mean_ms * 1e-3) / 1e12
    line = {
        "metric": "extrapolated points*freq/s (Nx*Nz*Nw/s)", "value": value, "unit": "point*freq/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean_ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (64 seeded layered models, seeded random surface wavefields)",
        "config": {"workload": BATCH_NAME, "lines": len(bufs), "points": points,
                   "nx": [min(b["d"].nx for b in bufs), max(b["d"].nx for b in bufs)],
                   "nz": [min(b["d"].nz for b in bufs), max(b["d"].nz for b in bufs)],
                   "nw": [min(b["d"].nw for b in bufs), max(b["d"].nw for b in bufs)],
                   "L": sorted({b["d"].L for b in bufs}),
                   "plan": {"cluster": plan.cluster, "lines_cap": plan.lines_cap, "autotune_ms": tune_ms},
                   "launch": "one persistent batch kernel + per-line imaging, replayed as one CUDA graph",
                   "l2": "flushed between steps (256 MiB write)",
                   "parallelism": f"{world} independent batches" if world > 1 else "1 batch"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tops, "unit": "TOP/s (FP32 pipe)",
                     "frac": achieved / peak_tops, "traffic": None, "kernel": "k_migrate_batch",
                     "peak_source": f"{sms} SMs x 128 FP32 lanes x {sm_max:.0f} MHz ({peak_src} max clock)",
                     "ops_per_point": "6L+4 per line"},
        "e2e": {"value": e2e_val, "unit": "point*freq/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h),
                "includes": "H2D wavefields+velocities, batch depth loop, imaging, D2H images"},
        "gpu_launches": (3 + len(bufs)) * args.steps,
        "clocks": clk.summary(),
        "compare": {
            "per_line_persistent": {"ms": t_persistent, "value": points / (t_persistent * 1e-3),
                                    "batch_speedup": t_persistent / mean_ms},
            "per_line_per_depth": {"ms": t_per_depth, "value": points / (t_per_depth * 1e-3),
                                   "batch_speedup": t_per_depth / mean_ms,
                                   "launches": sum(b["d"].nz for b in bufs)}},
    }
    if not args.no_cpu_baseline and world == 1:
        import oracle as O
        secs, pts, errs = batch_parity(inputs, img_gpu)
        line["cpu_baseline"] = {"value": pts / secs, "unit": "point*freq/s", "cores": O.max_threads(),
                                "kind": "oracle", "sample": f"the 2 smallest lines ({pts} points x frequencies), "
                                "FP64 depth loop", "seconds": secs}
        line["parity"] = {"image_rel_l2_sampled_lines": errs}
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def measure_batch_form(fx, flush, steps: int = 3, warmup: int = 3, oracle_check: bool = True):
    """The batched_64 workload as a form of the default line: graph replays,
    speedups against per-line persistent and per-depth launches, and the FP64
    oracle on the two smallest lines."""
    import torch
    B = batch_setup(fx, 0)
    for _ in range(warmup):
        B["restore"]()
        B["graph"].replay()
    torch.cuda.synchronize()
    ms = batch_timed(B, steps, flush)
    mean_ms = float(np.mean(ms))
    img_gpu = [b["image"].cpu().numpy() for b in B["bufs"]]
    t_persistent, t_per_depth = batch_compare(fx, B)
    out = {"value": B["points"] / (mean_ms * 1e-3), "unit": "point*freq/s", "ms_per_step": mean_ms,
           "ops_per_s": B["ops"] / (mean_ms * 1e-3),
           "what": "64 uneven lines (Nx {}-{}, Nz {}-{}, {}-{} frequencies, L {}) in one persistent batch "
                   "kernel + per-line imaging, replayed as one CUDA graph".format(
                       min(b["d"].nx for b in B["bufs"]), max(b["d"].nx for b in B["bufs"]),
                       min(b["d"].nz for b in B["bufs"]), max(b["d"].nz for b in B["bufs"]),
                       min(b["d"].nw for b in B["bufs"]), max(b["d"].nw for b in B["bufs"]),
                       "/".join(str(v) for v in sorted({b["d"].L for b in B["bufs"]}))),
           "plan": {"cluster": B["plan"].cluster, "lines_cap": B["plan"].lines_cap, "autotune_ms": B["tune_ms"]},
           "batch_speedup_vs_per_line_persistent": t_persistent / mean_ms,
           "batch_speedup_vs_per_line_per_depth": t_per_depth / mean_ms,
           "per_line_persistent_ms": t_persistent, "per_line_per_depth_ms": t_per_depth}
    if oracle_check:
        secs, pts, errs = batch_parity(B["inputs"], img_gpu)
        out["image_rel_l2_sampled_lines_vs_fp64_oracle"] = errs
    del B
    torch.cuda.empty_cache()
    return out


# ------------------------------------------------------------------ GPU leg
FORM_NAMES = ("learned", "precision", "per_depth", "large", "batch", "fx3d")


def run_native(args, w):
    import torch
    import torch.distributed as dist
    rank, world, local = env_rank()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_1912_05529_gb300 import build
    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        dist.barrier()
    import paper_1912_05529_gb300 as fx

    seed = w.seed + 1000 * rank
    sec, vm = make_inputs(w, seed)
    d = fx.Desc(nx=w.nx, nz=w.nz, nt=w.nt, nw=w.nw, i0=w.i0, L=w.L, nk=w.nk, dx=w.dx, dz=w.dz, dt=w.dt,
                theta_max_deg=w.theta_deg, k_max=k_max_of(w, float(vm.min())))
    launch = fx.Launch(mode=args.mode, cluster=args.cluster, groups=args.groups, warps=args.warps,
                       ctas_per_sm=args.ctas_per_sm)
    b = fx.allocate(d, launch)
    b.section.copy_(torch.from_numpy(sec))
    b.vel.copy_(torch.from_numpy(vm))
    fx.fxmig_design_operators(d, b.table)
    fx.fxmig_t2f(d, b.section, b.slab, b.ws_t2f)
    slab0 = b.slab.clone()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")   # > 129 MB L2
    stream = torch.cuda.current_stream()

    def step():
        fx.fxmig_migrate_ex(d, launch, b.slab, b.vel, b.table, b.partials, 0, d.nz, b.ws_mig)
        fx.fxmig_image(d, b.partials, b.image)

    for _ in range(args.warmup):
        b.slab.copy_(slab0)
        step()
    torch.cuda.synchronize()
    if fx.fxmig_check(b.ws_mig) != fx.FXMIG_OK:
        raise RuntimeError("device status after warm-up: " + fx.fxmig_strerror(fx.fxmig_check(b.ws_mig)))

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        time.sleep(0.3)
        for e0, e1, e2 in ev:
            b.slab.copy_(slab0)
            flush.fill_(1)
            e0.record(stream)
            fx.fxmig_migrate_ex(d, launch, b.slab, b.vel, b.table, b.partials, 0, d.nz, b.ws_mig)
            e1.record(stream)
            fx.fxmig_image(d, b.partials, b.image)
            e2.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    mig_ms = [e0.elapsed_time(e1) for e0, e1, _ in ev]
    step_ms = [e0.elapsed_time(e2) for e0, _, e2 in ev]
    tot_ms = sum(step_ms)
    if world > 1:
        t = torch.tensor([tot_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tot_ms = float(t.item())
    value = world * w.points * args.steps / (tot_ms * 1e-3)

    # end to end through the public call with host buffers (pinned)
    sec_h = torch.from_numpy(sec).pin_memory()
    vm_h = torch.from_numpy(vm).pin_memory()
    img_h = torch.empty((d.nz, d.nx), dtype=torch.float32, pin_memory=True)
    for _ in range(2):
        fx.migrate_section(d, sec_h, vm_h, b, launch, img_h, design=False)
    torch.cuda.synchronize()
    e2e_ms = []
    for _ in range(args.steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fx.migrate_section(d, sec_h, vm_h, b, launch, img_h, design=False)
        torch.cuda.synchronize()
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
    e2e_val = world * w.points * len(e2e_ms) / (sum(e2e_ms) * 1e-3)

    learned, precs, per_depth, large, batched, fx3d = None, {}, None, {}, None, None
    oracle_leg = not args.no_cpu_baseline and world == 1
    forms = set() if args.no_forms else {f.strip() for f in args.forms.split(",") if f.strip()}
    if forms - set(FORM_NAMES):
        raise SystemExit(f"unknown forms: {sorted(forms - set(FORM_NAMES))}")
    if world == 1:
        if "learned" in forms and d.L <= 15:
            learned = measure_learned(fx, d, b, slab0, args.steps, flush, train_steps=args.train_steps,
                                      lr=tuple(args.train_lr))
        if "precision" in forms:
            for name in PREC_NAMES:
                precs[name] = measure_precision(fx, d, b, slab0, args.steps, flush, launch,
                                                getattr(fx, "FXMIG_PREC_" + name))
        if "per_depth" in forms and args.mode != 2:
            per_depth = measure_per_depth(fx, d, b, slab0, min(args.steps, 5), flush)
        if w.name == "layered_lens_2048":
            # the 8192-trace line and the 64 uneven lines, recorded with this line
            if "large" in forms:
                large = measure_large(fx, flush, oracle_check=oracle_leg)
            if "batch" in forms:
                batched = measure_batch_form(fx, flush, oracle_check=oracle_leg)
            if "fx3d" in forms:
                fx3d = measure_fx3d(fx, flush, oracle_check=oracle_leg)

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0

    peaks, peak_src = load_peaks()
    sm_max = float(peaks.get("sm_max_mhz", NOMINAL_SM_MHZ))
    props = torch.cuda.get_device_properties(local)
    sms = props.multi_processor_count
    # FP32 pipe: 128 lanes per SM, one operation per lane per cycle (packed
    # f32x2 instructions take two cycles), at the maximum SM clock
    peak_tops = sms * 128 * sm_max * 1e6 / 1e12
    mig_avg = sum(mig_ms) / len(mig_ms)
    achieved = ops_per_point(w.L) * w.points / (mig_avg * 1e-3) / 1e12
    nparts = b.partials.shape[0]
    line = {
        "metric": "extrapolated points*freq/s (Nx*Nz*Nw/s)", "value": value, "unit": "point*freq/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded layered+lens model, normal-incidence section)",
        "config": {"workload": w.name, "nx": w.nx, "nz": w.nz, "nw": w.nw, "L": w.L, "nk": w.nk,
                   "mode": "persistent" if args.mode != 2 else "per_depth",
                   "l2": "flushed between steps (256 MiB write)", "partials": nparts,
                   "parallelism": f"{world} independent lines" if world > 1 else "1 line"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tops, "unit": "TOP/s (FP32 pipe)",
                     "frac": achieved / peak_tops,
                     "traffic": kernel_traffic(w.name) if args.mode != 2 else None,
                     "kernel": "k_depth" if args.mode != 2 else "k_migrate_step",
                     "peak_source": f"{sms} SMs x 128 FP32 lanes x {sm_max:.0f} MHz ({peak_src} max clock)",
                     "ops_per_point": ops_per_point(w.L), "migrate_ms": mig_avg,
                     "image_ms": float(np.mean([b_ - a_ for a_, b_ in zip(mig_ms, step_ms)]))},
        "e2e": {"value": e2e_val, "unit": "point*freq/s",
                "h2d_bytes_per_step": int(sec.nbytes + vm.nbytes), "d2h_bytes_per_step": int(d.nz * d.nx * 4),
                "includes": "H2D section+velocity, t->f, depth loop, imaging, D2H image (table resident)"},
        # per timed step: table expansion, slowness, line norms (image scale),
        # depth loop, image (persistent); the same with one launch per depth
        # row (per-depth form)
        "gpu_launches": (5 if args.mode != 2 else 4 + d.nz) * args.steps,
        "clocks": clk.summary(),
    }
    img_ref = None
    if not args.no_cpu_baseline and world == 1:
        secs, P_ref, img_ref, cores = oracle_run(w, sec, vm)
        img_gpu = b.image.cpu().numpy()
        # b.slab now holds the wavefield after the last e2e run (same inputs)
        P_gpu = b.slab.cpu().numpy()
        st_val, st_sample = oracle_single_thread(w, sec, vm)
        line["cpu_baseline"] = {"value": w.points / secs, "unit": "point*freq/s", "cores": cores,
                                "kind": "oracle", "sample": "whole workload, FP64 depth loop (design and "
                                "t->f excluded)", "seconds": secs,
                                "single_thread": {"value": st_val, "unit": "point*freq/s", "cores": 1,
                                                  "sample": st_sample}}
        line["parity"] = {"image_rel_l2": float(np.linalg.norm(img_gpu - img_ref) / np.linalg.norm(img_ref)),
                          "final_slice_rel_l2": float(np.linalg.norm(P_gpu - P_ref) / np.linalg.norm(P_ref))}
    rel = lambda a, r: float(np.linalg.norm(a - r) / np.linalg.norm(r))
    img_plain = b.image.cpu().numpy()
    forms = {}
    for name, r in precs.items():
        img_p = r.pop("image")
        val_p = w.points / (r["ms_per_step"] * 1e-3)
        forms[name.lower()] = {
            "value": val_p, "unit": "point*freq/s", "speedup_vs_plain": val_p / value,
            "what": "persistent form, wavefield lines and taps stored in 16 bits "
                    + ("(taps as hi + lo)" if "SPLIT" in name else "") + ", FP32 arithmetic",
            "image_rel_l2_vs_fp64_oracle": rel(img_p, img_ref) if img_ref is not None else None,
            "image_rel_l2_vs_plain_gpu": rel(img_p, img_plain), **r}
        if img_ref is not None:
            forms[name.lower()]["bar"] = 1e-2
            forms[name.lower()]["status"] = "meets bar" if rel(img_p, img_ref) <= 1e-2 else "above bar"
    if per_depth is not None:
        img_d = per_depth.pop("image")
        gbs = 16.0 * w.points / (per_depth["migrate_ms"] * 1e-3) / 1e9
        hbm = float(peaks.get("hbm_gbs", 6800.0))
        l2c = per_depth["l2_copy_gbs"]
        slab_mb = d.nw * d.nx * 8 / 1e6
        forms["per_depth"] = {
            "value": w.points / (per_depth["ms_per_step"] * 1e-3), "unit": "point*freq/s",
            "speedup_vs_plain": w.points / (per_depth["ms_per_step"] * 1e-3) / value,
            "what": "one Eq. 1 launch per depth row (k_migrate_step), wavefield read and written "
                    "through L2/HBM every step; the launches replayed as one CUDA graph",
            "wavefield_gbs": gbs, "ceiling": "l2_copy_gbs", "frac_of_l2_copy": gbs / l2c,
            "frac_of_l2_bandwidth": gbs / per_depth["l2_bandwidth_gbs"],
            "hbm_peak_gbs": hbm, "frac_of_hbm": gbs / hbm,
            "note": f"algorithmic 16 B per point*freq; the {slab_mb:.1f} MB wavefield stays in the "
                    "129 MB L2 between launches: l2_copy_gbs is a device copy of that size (one launch "
                    "per copy, like one launch per depth step), l2_bandwidth_gbs a copy of 32 MB "
                    "buffers that stay in L2 (the L2's own rate); HBM is not the ceiling here",
            "image_rel_l2_vs_fp64_oracle": rel(img_d, img_ref) if img_ref is not None else None,
            "image_rel_l2_vs_plain_gpu": rel(img_d, img_plain), **per_depth}
    forms.update(large)
    if batched is not None:
        forms["batched_64"] = batched
    if fx3d is not None:
        forms["fx3d_layered_lens_128"] = fx3d
    if forms:
        line["forms"] = forms
    if learned is not None:
        img_l = learned.pop("image")
        params_l = learned.pop("params")
        val_l = w.points / (learned["ms_per_step"] * 1e-3)
        line.setdefault("forms", {})
        line["forms"]["learned"] = {
            "value": val_l, "unit": "point*freq/s", "speedup_vs_plain": val_l / value,
            "what": "operators generated by the network (split-BF16 tensor-core MLP) for every distinct "
                    "(frequency, slowness) pair of each row; one Eq. 1 launch per depth row",
            "image_rel_l2_vs_plain_gpu": rel(img_l, img_plain), **learned}
        if oracle_leg:
            line["forms"]["learned"].update(judge_learned(fx, d, params_l, w, sec, vm))
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--workload", default="layered_lens_2048", choices=sorted(WORKLOADS) + [BATCH_NAME])
    ap.add_argument("--mode", type=int, default=0, help="0 auto, 1 persistent, 2 per-depth")
    ap.add_argument("--cluster", type=int, default=0)
    ap.add_argument("--groups", type=int, default=0)
    ap.add_argument("--warps", type=int, default=0)
    ap.add_argument("--ctas-per-sm", type=int, default=0, help="persistent form: 1, 2, or 0 (auto)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the other forms (learned operators, 16-bit "
                    "storage, per-depth launches, the 8192-trace line, the 64-line batch)")
    ap.add_argument("--forms", default=",".join(FORM_NAMES),
                    help="comma-separated subset of the other forms to run: " + ", ".join(FORM_NAMES))
    ap.add_argument("--train-steps", type=int, default=1000000, help="Adam steps of the operator network")
    ap.add_argument("--train-lr", type=float, nargs=2, default=[3e-3, 1e-5], metavar=("MAX", "MIN"),
                    help="cosine learning-rate schedule of the operator network")
    ap.add_argument("--ref-freqs", type=int, default=24, help="frequencies per oracle step (reference arm)")
    args = ap.parse_args(argv)
    if args.workload == BATCH_NAME:
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the reference arm times the oracle on the "
                              "single-line workloads"}), flush=True)
            return 0
        return run_batch(args)
    w = WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, w)
    return run_native(args, w)


if __name__ == "__main__":
    sys.exit(main())
