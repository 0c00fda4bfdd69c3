"""Benchmark of the MPR gap fill on GB300 (one JSON line on stdout, rank 0).

A step is one whole gap fill of a 4096 x 4096 Whittle-Matern grid (nu = 1, correlation
length 32, half of the sites missing as random disks of radius 8-64 plus random sites):
Eq. 1 map and lattice set-up, Eq. 4 sample energy, T-hat from the e(T, L) table, the
Algorithm 2 relaxation with the slope test, M = 100 equilibrium sweeps and the averaging /
back-transform.  The metric is gap-site updates per second (one update = over-relaxation +
Metropolis step of one gap site).

  value : inputs and output already in device memory (torch tensors)
  e2e   : the same call with pinned host buffers, host<->device copies inside the step
The e(T, L) table depends only on the lattice shape and the sampler parameters; it is
built once per shape during warm-up (its build time is reported) and reused by every step.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mpr|reference]
With N > 1 (torchrun) every rank fills its own map (independent seeds): weak scaling,
no collective on the data path; the reported time is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOAD = "mpr-fill-4096x4096-wm-nu1-xi32-p0.5-disks"
METRIC = "MPR site-updates/s"
UNIT = "site-updates/s"
L = 4096
M = 100


def reduce_over_ranks(times_ms, updates, dist=None, device="cpu"):
    """Whole-job numbers of a weak-scaling run: the slowest rank's times (every rank filled
    its own map, so the job ends when the last one does) and the sum of the site updates of
    all ranks.  dist: torch.distributed (initialised) or None for one process."""
    import torch
    t = torch.tensor([float(x) for x in times_ms], dtype=torch.float64, device=device)
    u = torch.tensor([float(x) for x in updates], dtype=torch.float64, device=device)
    if dist:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return t.tolist(), u.tolist()


def make_inputs(seed_offset: int):
    from paper_1811_01604_gb300 import synth
    z = synth.wm_field(L, 1.0, 32.0, seed=3 + seed_offset)
    mask = synth.mask_disks(L, L, 0.5, seed=1_000_003 + seed_offset)
    return z, mask


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            for name, v in zip(names, r[4:8]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


# DRAM bytes per sweep of k_tile_sweep on this grid, per compiled tile configuration and
# phase: dram__bytes_read.sum + dram__bytes_write.sum of one ncu capture of the profile case
# fill4096 (the relaxation launch, 261 sweeps, and the accumulating launch, 100 sweeps),
# divided by the launch's sweeps; valid for the kernel sources with this hash only.
TILE_TRAFFIC_PER_SWEEP = {2: {"relax": (48.008288e9 + 36.125516e9) / 261, "acc": (18.341778e9 + 16.763368e9) / 100}}
TILE_TRAFFIC_SOURCE_HASH = "61db15acd72b83d5"


def tile_kernel_hash():
    """Hash of the sweep kernel's sources with comments and blank lines removed (an edit of
    a comment leaves the captured counters valid; any change of code does not)."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in ("mpr_tile.cu", "mpr_internal.cuh"):
        with open(os.path.join(ROOT, "paper_1811_01604_gb300", "csrc", f), encoding="utf-8") as fh:
            t = fh.read()
        t = re.sub(r"/\*.*?\*/", "", t, flags=re.S)
        t = re.sub(r"//[^\n]*", "", t)
        t = "\n".join(line.rstrip() for line in t.splitlines() if line.strip())
        h.update(t.encode())
    return h.hexdigest()[:16]


# Arithmetic of one gap-site update counted for the ALU roof: about 60 FP32 and 70 integer
# operations (Philox4x32-10, the reflection, the proposal and the Metropolis test), the
# per-update figure of the method's operation count; the unit-vector lattice replaces the
# neighbours' transcendentals by plain arithmetic, so the MUFU roof (about 5 per update) is
# far below both others.
ALU_OPS_PER_UPDATE = 130
LANES_PER_SM = 128                 # 4 schedulers x 32 lanes issue one operation each per clock


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def cpu_baseline(z, mask, T):
    """The FP64 oracle on 512 x 512 crops of the same workload (fixed T-hat, slope-test
    relaxation + M sweeps): once on one core, then one crop per host core on as many
    threads (the C oracle runs outside the GIL)."""
    from concurrent.futures import ThreadPoolExecutor
    import oracle.oracle as orc
    c = 512
    crops = []
    for i in range(max(1, os.cpu_count() or 1)):
        y0, x0 = (i // 8) * c % (z.shape[0] - c + 1), (i % 8) * c % (z.shape[1] - c + 1)
        crops.append((np.ascontiguousarray(z[y0:y0 + c, x0:x0 + c]),
                      np.ascontiguousarray(mask[y0:y0 + c, x0:x0 + c])))
    prm = orc.params(seed=0, M=M)

    def one(zm):
        _, _, out = orc.fill(zm[0], zm[1], prm, T_fixed=T)
        return out.n_gap * (out.eq.sweeps + M)

    t0 = time.perf_counter()
    u1 = one(crops[0])
    t1 = time.perf_counter() - t0
    cores = len(crops)
    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=cores) as ex:
        un = sum(ex.map(one, crops))
    tn = time.perf_counter() - t0
    return {"value": u1 / t1, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"512x512 crop of the step's grid, fixed T-hat, slope-test relaxation + "
                      f"M={M}: {u1} site-updates in {t1:.1f} s on one core",
            "all_cores": {"value": un / tn, "unit": UNIT, "cores": cores,
                          "sample": f"{cores} different 512x512 crops on {cores} threads "
                                    f"(host cores: {os.cpu_count()}): {un} site-updates in {tn:.1f} s"}}


def run_reference(args, rank):
    """--impl reference: the oracle as it stands, each step a 256 x 256 crop fill."""
    if rank != 0:
        return
    import oracle.oracle as orc
    orc.build()
    z, mask = make_inputs(0)
    c = 256
    zc = np.ascontiguousarray(z[:c, :c])
    mc = np.ascontiguousarray(mask[:c, :c])
    prm = orc.params(seed=0, M=M, KT=8, T_W=32, T_H=32, M_T=50)
    _, _, out0 = orc.fill(zc, mc, prm)                      # T-hat of the crop
    T = out0.T_hat
    for _ in range(args.warmup):
        orc.fill(zc, mc, prm, T_fixed=T)
    t0 = time.perf_counter()
    updates = 0
    for _ in range(args.steps):
        _, _, out = orc.fill(zc, mc, prm, T_fixed=T)
        updates += out.n_gap * (out.eq.sweeps + M)
    dt = time.perf_counter() - t0
    v = updates / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample": "256x256 crop",
                                              "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"256x256 crop of the 4096^2 step grid, fixed T-hat "
                                       f"{T:.4f}, slope-test relaxation + M={M} per step"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def trace_summary(it, ctl, relax, n_sms):
    """Where a phase's time goes, from the sweep kernel's timestamps (mpr_debug_trace).
    it: int64 [sweeps][tiles][6] item stamps in ns (taken, copy issued, copy landed, both
    colours updated, written back; block | SM << 32), zero where an item was not run;
    ctl: int64 [k][2] control-step stamps (ticket that completed a sweep, published), zero
    where unused.  Per item medians (us) of the wait for its inputs, the copy, the update
    and the write-back; the fraction of block time spent updating; the time per sweep; for
    a relaxation (relax), the serial gap of the Algorithm 2 control step (last update to
    the ticket, the control step, its publication to the next sweep's first copy landing)
    and how a mid-relaxation sweep's tiles fall on the n_sms SMs."""
    S = it.shape[0]
    ok = it[:, :, 1] > 0
    t = [it[:, :, k][ok] for k in range(5)]
    d = lambda a, b: float(np.median(b - a)) / 1e3
    last = np.where(ok, it[:, :, 3], 0).max(axis=1)
    r = {"sweeps": S, "items": int(ok.sum()),
         "us_wait": d(t[0], t[1]), "us_copy": d(t[1], t[2]), "us_update": d(t[2], t[3]),
         "us_writeback": float(np.median((t[4] - t[3])[t[4] > 0])) / 1e3,
         "us_per_sweep": float(np.median(np.diff(last))) / 1e3}
    nb = int((it[:, :, 5][ok] & 0xFFFFFFFF).max()) + 1
    r["blocks"] = nb
    r["update_share_of_block_time"] = float((t[3] - t[2]).sum() / (nb * (t[3].max() - t[0].min())))
    if relax:
        tix = np.sort(ctl[:, 0][ctl[:, 0] > 0])
        pub = np.sort(ctl[:, 1][ctl[:, 1] > 0])
        n = min(len(pub), S) - 1
        first = np.where(ok, it[:, :, 2], np.iinfo(np.int64).max).min(axis=1)
        r["us_last_update_to_ticket"] = float(np.median(tix[:n] - last[:n])) / 1e3
        r["us_control_step"] = float(np.median(pub[:n] - tix[:n])) / 1e3
        r["us_publish_to_first_copy_landed"] = float(np.median(first[1:n + 1] - pub[:n])) / 1e3
        sm = (it[S // 2, :, 5] >> 32)[ok[S // 2]]
        cnt = np.bincount(sm.astype(np.int64), minlength=n_sms)
        r["mid_sweep_tiles_per_sm"] = {"max": int(cnt.max()), "idle_sms": int((cnt == 0).sum()),
                                       "histogram": np.bincount(cnt).tolist()}
    return r


def trace_phases(z, mask, W, H, T, tile_cfg):
    """trace_summary of the relaxation launch and the M accumulating sweeps of one fill at
    a fixed T (mpr_debug_trace)."""
    import torch
    from paper_1811_01604_gb300 import mpr
    g = mpr.mpr_default_params(seed=1, M=M, tile_cfg=tile_cfg)
    ctx = mpr.mpr_init(z, mask, W, H, g)
    out = {}
    try:
        mpr.mpr_set_T(ctx, T)
        th, tw = {0: (16, 128), 1: (32, 64), 2: (32, 128)}[tile_cfg]
        ntiles = -(-H // th) * -(-W // tw)
        buf = torch.zeros(ntiles * 10002 * 6 + 8192, dtype=torch.int64, device="cuda")
        K = (buf.numel() - 8192) // 6
        for phase in ("relax", "acc"):
            buf.zero_()
            mpr.mpr_debug_trace(buf)
            if phase == "relax":
                S = mpr.mpr_equilibrate(ctx).sweeps
            else:
                S = M
                mpr.mpr_predict(ctx, M, torch.empty_like(z))
            torch.cuda.synchronize()
            mpr.mpr_debug_trace(None)
            it = buf[: ntiles * S * 6].cpu().numpy().astype(np.int64).reshape(S, ntiles, 6)
            ctl = buf[K * 6:].cpu().numpy().astype(np.int64).reshape(-1, 2)
            out[phase] = trace_summary(it, ctl, phase == "relax",
                                       torch.cuda.get_device_properties(0).multi_processor_count)
    finally:
        mpr.mpr_free(ctx)
    return out


def profile_case(name, tile_cfg=0):
    """sweep4096: 4096^2 bench grid, T = 0.05, 24 sweeps at a = 8 (one launch of the
    persistent sweep kernel; a few set-up kernels before it).
    fill4096: the 4096^2 bench grid at its T-hat (set directly: no table build): the
    relaxation (one launch of the sweep kernel) and M = 100 accumulating sweeps (one
    launch), as in a timed step.
    copy4096: a plain device copy of the bytes a ping-pong sweep of the 4096^2 grid moves
    (one unit-vector lattice buffer of 134 MB read, one written), timed with CUDA events:
    the memory floor of a sweep that rewrites its whole lattice.
    net4096: two warm-start forward passes (untrained network) on the 4096^2 bench grid.
    net128: two training steps of the warm-start network on a batch of 32 128^2 grids.
    net1024: two warm-start forward passes (untrained network) on a 1024^2 grid.
    sweep64_4096: the 4096^2 bench grid in FP64 (MPR_PREC_F64, list kernels), T = 0.05,
    3 sweeps at a = 8 (6 half-sweep launches).
    trace4096, trace1024: per-item timestamps of the sweep kernel over one fill
    (trace_phases).
    hostlink: the host<->device bandwidth of the end-to-end line's copies (pinned host
    memory; torch copies, which are cudaMemcpyAsync)."""
    import torch
    from paper_1811_01604_gb300 import mpr
    if name == "copy4096":
        n = 4096 * 4096                             # float2 elements of one lattice buffer (2 planes)
        src = torch.ones(2 * n, dtype=torch.float32, device="cuda")
        dst = torch.empty_like(src)
        ms = []
        for _ in range(23):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            dst.copy_(src)
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        t = statistics.median(ms[3:])
        print(json.dumps({"profile_case": name, "bytes_read": 8 * n, "bytes_written": 8 * n,
                          "median_ms": t, "GB_per_s": 2 * 8 * n / (t * 1e-3) / 1e9}))
        return
    if name == "hostlink":
        # the end-to-end line's copies: 83.9 MB from pinned host memory to the device (the
        # 4096^2 grid's data and mask) and 67.1 MB back (its estimates), timed with CUDA events
        out = {"profile_case": name}
        for what, nbytes in (("h2d", 5 * 4096 * 4096), ("d2h", 4 * 4096 * 4096)):
            h = torch.ones(nbytes, dtype=torch.uint8).pin_memory()
            d = torch.ones(nbytes, dtype=torch.uint8, device="cuda")
            ms = []
            for _ in range(13):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                if what == "h2d":
                    d.copy_(h, non_blocking=True)
                else:
                    h.copy_(d, non_blocking=True)
                e1.record()
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
            t = statistics.median(ms[3:])
            out[what] = {"bytes": nbytes, "median_ms": t, "GB_per_s": nbytes / (t * 1e-3) / 1e9}
        print(json.dumps(out))
        return
    if name == "net128":
        B, S = 32, 128
        g = torch.Generator(device="cuda")
        g.manual_seed(0)
        z = torch.rand((B, S, S), generator=g, device="cuda")
        m = (torch.rand((B, S, S), generator=g, device="cuda") > 0.4).to(torch.uint8)
        phi = 6.283 * torch.rand((B, S, S), generator=g, device="cuda")
        net = mpr.mpr_net_create(0)
        try:
            for _ in range(2):
                mpr.mpr_net_train_step(net, z, m, phi, np.zeros(B), np.ones(B), B, S, S, 1e-3)
            torch.cuda.synchronize()
        finally:
            mpr.mpr_net_free(net)
        print(f"profile case {name}: done")
        return
    if name in ("trace4096", "trace1024"):
        if name == "trace4096":
            z_np, m_np = make_inputs(0)
            T = 9.869677377227477e-4
        else:
            from paper_1811_01604_gb300 import synth
            z_np = synth.wm_field(1024, 0.5, 16.0, seed=1)
            m_np = synth.mask_uniform(1024, 1024, 0.33, seed=1_000_034)
            T = None
        z = torch.from_numpy(np.ascontiguousarray(z_np, np.float32)).cuda()
        mask = torch.from_numpy(np.ascontiguousarray(m_np, np.uint8)).cuda()
        H, W = z.shape
        if T is None:
            ctx = mpr.mpr_init(z, mask, W, H, mpr.mpr_default_params(seed=1, M=M))
            try:
                T, _ = mpr.mpr_estimate_T(ctx)
            finally:
                mpr.mpr_free(ctx)
        print(json.dumps({"profile_case": name, "tile_cfg": tile_cfg, "T": T,
                          **trace_phases(z, mask, W, H, T, tile_cfg)}))
        return
    if name == "net1024":
        from paper_1811_01604_gb300 import synth
        z = synth.wm_field_gpu(1024, 1024, 0.5, 16.0, 1)
        mask = synth.mask_uniform_gpu(1024, 1024, 0.33, 1_000_001)
        H, W = 1024, 1024
    else:
        z_np, m_np = make_inputs(0)
        H, W = z_np.shape
        z = torch.from_numpy(z_np).cuda()
        mask = torch.from_numpy(m_np).cuda()
    extra = dict(precision=mpr.MPR_PREC_F64) if name == "sweep64_4096" else dict(tile_cfg=tile_cfg)
    ctx = mpr.mpr_init(z, mask, W, H, mpr.mpr_default_params(seed=1, **extra))
    try:
        if name in ("net4096", "net1024"):
            net = mpr.mpr_net_create(0)
            try:
                for _ in range(2):
                    mpr.mpr_warmstart_init(ctx, net)
                torch.cuda.synchronize()
            finally:
                mpr.mpr_net_free(net)
            print(f"profile case {name}: done")
            return
        if name == "fill4096":
            mpr.mpr_set_T(ctx, 9.869677377227477e-4)
            eq = mpr.mpr_equilibrate(ctx)
            out = torch.empty_like(z)
            mpr.mpr_predict(ctx, M, out)
            torch.cuda.synchronize()
            print(f"profile case {name}: relaxation {eq.sweeps} sweeps, then {M}")
            return
        mpr.mpr_set_T(ctx, 0.05)
        st = mpr.mpr_sweep(ctx, 3 if name == "sweep64_4096" else 24, 8.0)
        torch.cuda.synchronize()
    finally:
        mpr.mpr_free(ctx)
    print(f"profile case {name}: acceptance {st.acceptance:.3f} e {st.e:.6f}")


def run_batch(args):
    """256 grids (sides log-uniform in [128, 2048], own nu, correlation length, missing
    fraction), M = 32 each: one batched fill per step, against the same grids filled one
    at a time with the same chains and temperatures.  --batch-warm adds the batched fill
    with the learned warm start (network trained first, untimed, as in the warm workloads)."""
    import torch
    from paper_1811_01604_gb300 import mpr, synth
    Mb = 32
    spec = synth.batch_workload(256)
    zs, ms = [], []
    for sp in spec:
        zs.append(synth.wm_field_gpu(sp["L"], sp["L"], sp["nu"], sp["xi"], sp["seed"]))
        ms.append(synth.mask_uniform_gpu(sp["L"], sp["L"], sp["p"], sp["seed"] + 1_000_000))
    outs = [torch.empty_like(z) for z in zs]
    prm = mpr.mpr_default_params(seed=4, M=Mb)
    gaps = [int((m == 0).sum().item()) for m in ms]
    stream = torch.cuda.current_stream()

    net = None
    if args.batch_warm:
        from paper_1811_01604_gb300 import warmstart
        groups = warmstart.training_grids(n64=args.train_n64, n128=args.train_n128, seed=10_000,
                                          n256=args.train_n256)
        sets = [warmstart.equilibrium_states(z, m, states_per_grid=4, spacing=20, seed=20_000)
                for z, m in groups]
        net = warmstart.WarmStartNet(seed=0, stride=args.warm_stride)
        warmstart.train(net, sets, steps=args.train_steps, batch=32, lr=1e-3, seed=0)
        torch.cuda.synchronize()

    # the tile shape is chosen once, by the autotuner in the first (untimed) fill, and
    # passed in the parameters of every later fill, as for the single map
    tuned = {}

    def batched(use_net=False):
        ctx = mpr.mpr_init_batch(zs, ms, prm, stream.cuda_stream)
        try:
            mpr.mpr_estimate_T(ctx)
            if not tuned:
                t0 = time.perf_counter()
                tuned.update(mpr.mpr_autotune(ctx))
                torch.cuda.synchronize()
                tuned["autotune_s"] = time.perf_counter() - t0
                prm.tile_cfg = tuned["tile_cfg"]
            tune = tuned
            if use_net:
                net.warmstart(ctx)
            mpr.mpr_equilibrate(ctx)
            mpr.mpr_predict_batch(ctx, Mb, outs)
            info = mpr.mpr_batch_info_all(ctx)
        finally:
            mpr.mpr_free(ctx)
        return info, tune

    t0 = time.perf_counter()
    info, tune = batched()                       # builds and caches the e(T, L) tables
    torch.cuda.synchronize()
    t_first = time.perf_counter() - t0
    for _ in range(max(0, args.warmup - 1)):
        batched()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        info, tune = batched()
    e1.record(stream)
    torch.cuda.synchronize()
    batch_ms = e0.elapsed_time(e1) / args.steps
    updates = sum(P * (inf["sweeps"] + Mb) for P, inf in zip(gaps, info))

    def maes():
        return [float((o - z)[m == 0].abs().mean()) for o, z, m in zip(outs, zs, ms)]

    mae_plain = maes()
    warm = None
    if net is not None:
        batched(True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            info_w, _ = batched(True)
        e1.record(stream)
        torch.cuda.synchronize()
        warm_ms = e0.elapsed_time(e1) / args.steps
        mae_w = maes()
        warm = {"ms": warm_ms, "speedup_vs_batched_plain": batch_ms / warm_ms,
                "relax_sweeps_max": max(i["sweeps"] for i in info_w),
                "relax_sweeps_mean": float(np.mean([i["sweeps"] for i in info_w])),
                "mae_mean": float(np.mean(mae_w)), "mae_mean_plain": float(np.mean(mae_plain)),
                "mae_ratio_max": float(max(a / b for a, b in zip(mae_w, mae_plain))),
                "net_stride": args.warm_stride}

    def sequential():
        for g, (z, m) in enumerate(zip(zs, ms)):
            H, W = z.shape
            ctx = mpr.mpr_init(z, m, W, H, mpr.mpr_default_params(seed=4, M=Mb, chain=g,
                                                                  tile_cfg=prm.tile_cfg),
                               stream.cuda_stream)
            try:
                mpr.mpr_set_T(ctx, info[g]["T"])
                mpr.mpr_equilibrate(ctx)
                mpr.mpr_predict(ctx, Mb, outs[g])
            finally:
                mpr.mpr_free(ctx)

    sequential()
    torch.cuda.synchronize()
    e0.record(stream)
    sequential()
    e1.record(stream)
    torch.cuda.synchronize()
    seq_ms = e0.elapsed_time(e1)
    line = {"metric": METRIC, "value": updates / (batch_ms * 1e-3), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": batch_ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "mpr-batch-256-grids-L128-2048", "grids": len(zs),
                       "sites": int(sum(z.numel() for z in zs)), "gap_sites": int(sum(gaps)),
                       "M": Mb, "relax_sweeps_max": max(i["sweeps"] for i in info),
                       "relax_sweeps_mean": float(np.mean([i["sweeps"] for i in info])),
                       "autotune": tune, "first_fill_s_incl_tables": t_first,
                       "note": "temperatures of the sequential runs are the batch's"},
            "sequential": {"ms": seq_ms, "value": updates / (seq_ms * 1e-3),
                           "speedup_batched": seq_ms / batch_ms}}
    if warm:
        line["batched_warm_start"] = warm
    print(json.dumps(line), flush=True)


def net_flops_per_site():
    """Useful multiply-adds x 2 of one forward pass per full-resolution site (the first
    convolution counted with its 3 used input channels)."""
    lev = [0, 0, 1, 1, 2, 2, 3, 3, 2, 2, 1, 1, 0, 0]
    cin = [3, 32, 32, 64, 64, 128, 128, 256, 384, 128, 192, 64, 96, 32]
    cout = [32, 32, 64, 64, 128, 128, 256, 256, 128, 128, 64, 64, 32, 32]
    return sum(2 * 9 * a * b / 4 ** l for a, b, l in zip(cin, cout, lev)) + 2 * 32 * 2


def run_warm(args):
    """Learned warm start against the plain random start on the same maps: a step fills one
    map twice (plain, then warm-started), each timed with CUDA events; the network is
    trained first (untimed) on equilibrium states of 64^2 grids and 128^2 crops of 1024^2
    fields made by the library's own MCMC."""
    import torch
    from paper_1811_01604_gb300 import mpr, synth, warmstart
    Lw = 1024 if args.workload == "warm1024" else 4096
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    groups = warmstart.training_grids(n64=args.train_n64, n128=args.train_n128, seed=10_000,
                                      n256=args.train_n256)
    sets = [warmstart.equilibrium_states(z, m, states_per_grid=4, spacing=20, seed=20_000) for z, m in groups]
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    net = warmstart.WarmStartNet(seed=0, stride=args.warm_stride)
    t0 = time.perf_counter()
    losses = warmstart.train(net, sets, steps=args.train_steps, batch=32, lr=1e-3, seed=0)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    if Lw == 1024:
        z = synth.wm_field_gpu(1024, 1024, 0.5, 16.0, 1)
        mask = synth.mask_uniform_gpu(1024, 1024, 0.33, 1_000_001)
        wl = "mpr-warmstart-1024x1024-wm-nu0.5-xi16-p0.33"
    else:
        z_np, m_np = make_inputs(0)
        z, mask = torch.from_numpy(z_np).cuda(), torch.from_numpy(m_np).cuda()
        wl = "mpr-warmstart-4096x4096-wm-nu1-xi32-p0.5-disks"
    H, W = z.shape
    gap = mask == 0
    P = int(gap.sum().item())
    out = torch.empty_like(z)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    prm = mpr.mpr_default_params(seed=1, M=M)

    def fill(use_net):
        ctx = mpr.mpr_init(z, mask, W, H, prm, stream.cuda_stream)
        try:
            mpr.mpr_estimate_T(ctx)
            if use_net:
                net.warmstart(ctx)
            st = mpr.mpr_equilibrate(ctx)
            mpr.mpr_predict(ctx, M, out)
        finally:
            mpr.mpr_free(ctx)
        return st.sweeps

    def timed(use_net, n):
        ms, sw = [], []
        for _ in range(n):
            flush.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sw.append(fill(use_net))
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        mae = float((out - z)[gap].abs().mean())
        return ms, sw, mae

    for _ in range(args.warmup):
        fill(False)
        fill(True)
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    l0 = mpr.mpr_kernel_launches()
    ms_w, sw_w, mae_w = timed(True, args.steps)
    launches = mpr.mpr_kernel_launches() - l0
    ms_p, sw_p, mae_p = timed(False, args.steps)
    # inference alone: the warm start of a fresh context, timed on the context's stream
    ctx = mpr.mpr_init(z, mask, W, H, prm, stream.cuda_stream)
    try:
        inf = []
        for _ in range(3):
            flush.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            net.warmstart(ctx)
            e1.record(stream)
            torch.cuda.synchronize()
            inf.append(e0.elapsed_time(e1))
    finally:
        mpr.mpr_free(ctx)
    clk = clocks.stop()
    inf_ms = statistics.median(inf)
    S = args.warm_stride
    Hp, Wp = ((H + S - 1) // S + 7) // 8 * 8, ((W + S - 1) // S + 7) // 8 * 8      # network frame
    flops = net_flops_per_site() * Hp * Wp
    peaks, src = measured_peaks()
    peak = float(peaks.get("bf16_tflops", 1900.0))
    ach = flops / (inf_ms * 1e-3) / 1e12
    n_states = sum(s.n for s in sets)
    line = {"metric": "s per map (warm start)", "value": statistics.mean(ms_w) * 1e-3, "unit": "s/map",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": statistics.mean(ms_w), "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 lattice, bf16 network", "data": "synthetic",
            "config": {"workload": wl, "W": W, "H": H, "gap_sites": P, "M": M,
                       "net_stride": S, "net_frame": [Hp, Wp],
                       "l2": "512 MB buffer written between steps (L2 flush)",
                       "train": {"states": n_states, "steps": args.train_steps, "batch": "32 x 128^2 sites",
                                 "groups": [list(st.z.shape) for st in sets],
                                 "data_s": t_data, "train_s": t_train,
                                 "loss_first20": float(np.mean(losses[:20])),
                                 "loss_last20": float(np.mean(losses[-20:]))}},
            "warm": {"s_per_map": statistics.mean(ms_w) * 1e-3, "relax_sweeps": sw_w, "mae": mae_w,
                     "inference_ms": inf_ms},
            "plain": {"s_per_map": statistics.mean(ms_p) * 1e-3, "relax_sweeps": sw_p, "mae": mae_p},
            "speedup_vs_plain": statistics.mean(ms_p) / statistics.mean(ms_w),
            "gpu_launches": int(launches),
            "roofline": {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                         "frac": ach / peak, "traffic": None,
                         "kernel": "warm-start forward (14 x k_conv3x3 + 9 small kernels)",
                         "flops_per_launch": flops, "ms_per_launch": inf_ms,
                         "peak_source": f"{src} bf16_tflops"},
            "clocks": clk}
    net.close()
    print(json.dumps(line), flush=True)


def run_chains(args):
    """Independent chains against the paper's single chain at equal total sweeps: per seed,
    one 1024^2 map (nu 0.5, correlation length 16, 33 % gaps) is relaxed once; from that
    state mpr_predict_chains runs K chains x 100/K averaged sweeps for K in 1, 4, 10, 25
    (K = 1 is the single-chain estimator), and K = 4, 10 after 25 burn-in sweeps per chain.
    Reports MAE / RMSE against the hidden field, the estimator's Monte Carlo error (RMS
    distance at the gaps to the posterior mean, estimated by 32 chains x (200 burn-in + 200
    averaged) sweeps from the same state) and the time of each prediction (CUDA events)."""
    import torch
    from paper_1811_01604_gb300 import mpr, synth
    stream = torch.cuda.current_stream()
    variants = ((1, 0), (4, 0), (10, 0), (25, 0), (4, 25), (10, 25))        # (K, burn-in)
    total = 100
    res = {v: {"mae": [], "rmse": [], "noise": [], "ms": []} for v in variants}
    seeds = tuple(range(1, 1 + max(1, args.steps)))
    for seed in seeds:
        z = synth.wm_field_gpu(1024, 1024, 0.5, 16.0, 100 + seed)
        mask = synth.mask_uniform_gpu(1024, 1024, 0.33, 1_000_100 + seed)
        gap = mask == 0
        ctx = mpr.mpr_init(z, mask, 1024, 1024, mpr.mpr_default_params(seed=seed, M=total),
                           stream.cuda_stream)
        try:
            mpr.mpr_estimate_T(ctx)
            mpr.mpr_equilibrate(ctx)
            # the posterior mean at the gaps, nearly free of the shared start: 32 chains that
            # first run 200 unaveraged sweeps, then average 200 each
            ref = torch.empty_like(z)
            mpr.mpr_predict_chains(ctx, 32, 200, ref, burn_in=200)
            out = torch.empty_like(z)
            for v in variants:
                K, burn = v
                for _ in range(2 if seed == seeds[0] else 1):       # first seed: one untimed warm-up
                    torch.cuda.synchronize()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    mpr.mpr_predict_chains(ctx, K, total // K, out, burn_in=burn)
                    e1.record(stream)
                    torch.cuda.synchronize()
                res[v]["ms"].append(e0.elapsed_time(e1))
                err = (out - z)[gap].double()
                res[v]["mae"].append(float(err.abs().mean()))
                res[v]["rmse"].append(float(err.pow(2).mean().sqrt()))
                res[v]["noise"].append(float((out - ref)[gap].double().pow(2).mean().sqrt()))
        finally:
            mpr.mpr_free(ctx)
    rows = {"K%d_burn%d" % v: {k: float(np.mean(x)) for k, x in res[v].items()} for v in variants}
    line = {"metric": "estimator MC noise at equal averaged sweeps (independent chains)",
            "value": rows["K10_burn25"]["noise"],
            "unit": "z units (RMS)", "n_gpus": 1, "steps": len(seeds), "warmup": 1,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "mpr-chains-1024x1024-wm-nu0.5-xi16-p0.33", "total_sweeps": total,
                       "seeds": list(seeds), "reference": "posterior mean: 32 chains x (200 burn-in + 200 averaged) sweeps"},
            "by_chains_and_burn_in": rows}
    print(json.dumps(line), flush=True)


def run_or_modes(args):
    """Eq. 6 readings on whole fills: 1024^2 maps (nu 0.5, correlation length 16, 33 % gaps),
    filled with the energy-conserving reflection (the library's reading), the formula as
    printed (the q = 1 reflection) and no over-relaxation, at each grid's own T-hat; MAE /
    RMSE against the hidden field, T-hat, relaxation sweeps, time per map and the part of it
    spent up to T-hat (the e(T, L) table relaxes with the same reflection), over seeds."""
    import torch
    from paper_1811_01604_gb300 import mpr, synth
    stream = torch.cuda.current_stream()
    modes = (("conserving", mpr.MPR_OR_CONSERVING), ("literal", mpr.MPR_OR_LITERAL),
             ("none", mpr.MPR_OR_NONE))
    rows = {name: {"mae": [], "rmse": [], "T": [], "sweeps": [], "ms": [], "ms_T": []} for name, _ in modes}
    seeds = tuple(range(1, 1 + max(1, args.steps)))
    for seed in seeds:
        z = synth.wm_field_gpu(1024, 1024, 0.5, 16.0, 300 + seed)
        mask = synth.mask_uniform_gpu(1024, 1024, 0.33, 1_000_300 + seed)
        gap = mask == 0
        out = torch.empty_like(z)
        for name, mode in modes:
            for _ in range(2 if seed == seeds[0] else 1):           # first seed: one untimed warm-up
                torch.cuda.synchronize()
                e0, eT, e1 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
                e0.record(stream)
                ctx = mpr.mpr_init(z, mask, 1024, 1024, mpr.mpr_default_params(seed=seed, or_mode=mode),
                                   stream.cuda_stream)
                try:
                    T_hat, _ = mpr.mpr_estimate_T(ctx)
                    eT.record(stream)
                    st = mpr.mpr_equilibrate(ctx)
                    mpr.mpr_predict(ctx, M, out)
                finally:
                    mpr.mpr_free(ctx)
                e1.record(stream)
                torch.cuda.synchronize()
            err = (out - z)[gap].double()
            r = rows[name]
            r["mae"].append(float(err.abs().mean()))
            r["rmse"].append(float(err.pow(2).mean().sqrt()))
            r["T"].append(T_hat)
            r["sweeps"].append(st.sweeps)
            r["ms"].append(e0.elapsed_time(e1))
            r["ms_T"].append(e0.elapsed_time(eT))
    summary = {name: {k: float(np.mean(v)) for k, v in r.items()} for name, r in rows.items()}
    line = {"metric": "MAE of the fill by Eq. 6 reading", "value": summary["literal"]["mae"],
            "unit": "z units", "n_gpus": 1, "steps": len(seeds), "warmup": 1, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "mpr-or-modes-1024x1024-wm-nu0.5-xi16-p0.33", "M": M, "seeds": list(seeds)},
            "by_mode": summary}
    print(json.dumps(line), flush=True)


def run_config2(args):
    """The 1024^2 workloads: Whittle-Matern fields (nu = 0.5 and 2.5, correlation length 16,
    Gaussian and pointwise lognormal), 33 % and 66 % of the sites removed at random; each
    filled by the whole method (T-hat from the e(T, L) table, relaxation with the slope
    test, M = 100) -- one JSON line per grid with MAE, RMSE and correlation against the
    hidden field at the gap sites, and site-updates/s and ms per map (CUDA events, device-
    resident inputs, L2 flushed before each fill, the table built in the warm-up)."""
    import torch
    from paper_1811_01604_gb300 import mpr, synth
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    Lc = 1024
    tile_cfg = None                    # chosen once by the autotuner, untimed, on the first grid
    for nu in (0.5, 2.5):
        for kind in ("gauss", "lognormal"):
            for p in (0.33, 0.66):
                seed = 1 if nu == 0.5 else 2
                z_np = synth.wm_field(Lc, nu, 16.0, seed=seed)
                if kind == "lognormal":
                    z_np = synth.lognormal(z_np).astype(np.float32)
                m_np = synth.mask_uniform(Lc, Lc, p, seed=1_000_000 + seed + int(100 * p))
                z = torch.from_numpy(np.ascontiguousarray(z_np, np.float32)).cuda()
                mask = torch.from_numpy(np.ascontiguousarray(m_np, np.uint8)).cuda()
                gap = mask == 0
                P = int(gap.sum().item())
                out = torch.empty_like(z)
                if tile_cfg is None:
                    ctx = mpr.mpr_init(z, mask, Lc, Lc, mpr.mpr_default_params(seed=1, M=M), stream.cuda_stream)
                    try:
                        mpr.mpr_estimate_T(ctx)
                        tile_cfg = mpr.mpr_autotune(ctx)["tile_cfg"]
                    finally:
                        mpr.mpr_free(ctx)
                prm = mpr.mpr_default_params(seed=1, M=M, tile_cfg=tile_cfg)

                def fill():
                    ctx = mpr.mpr_init(z, mask, Lc, Lc, prm, stream.cuda_stream)
                    try:
                        T, _ = mpr.mpr_estimate_T(ctx)
                        st = mpr.mpr_equilibrate(ctx)
                        mpr.mpr_predict(ctx, M, out)
                    finally:
                        mpr.mpr_free(ctx)
                    return T, st.sweeps

                for _ in range(max(1, args.warmup)):
                    fill()
                ms, sw = [], []
                for _ in range(args.steps):
                    flush.zero_()
                    torch.cuda.synchronize()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    T, n = fill()
                    e1.record(stream)
                    torch.cuda.synchronize()
                    ms.append(e0.elapsed_time(e1))
                    sw.append(n)
                zt, zh = z[gap].double(), out[gap].double()
                err = zh - zt
                corr = float(torch.corrcoef(torch.stack([zh, zt]))[0, 1])
                updates = sum(P * (n + M) for n in sw)
                line = {"metric": METRIC, "value": updates / (sum(ms) * 1e-3), "unit": UNIT, "n_gpus": 1,
                        "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.mean(ms),
                        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                        "data": "synthetic",
                        "config": {"workload": f"mpr-fill-1024x1024-wm-nu{nu}-xi16-{kind}-p{p}", "M": M,
                                   "tile_cfg": tile_cfg,
                                   "gap_sites": P, "T_hat": T, "relax_sweeps": sw,
                                   "l2": "512 MB buffer written between fills (L2 flush)"},
                        "mae": float(err.abs().mean()), "rmse": float(err.pow(2).mean().sqrt()),
                        "corr": corr}
                print(json.dumps(line), flush=True)


def run_dpsp(args):
    """Single versus double precision (Sect. 4, the DP/SP time ratio against the grid side
    for p = 33 % and 66 %): Whittle-Matern fields nu = 0.5, kappa = 0.2 (correlation length
    5), gaps removed uniformly at random, L = 32 .. 4096.  Per grid: the whole fill (e(T, L)
    table built afresh, T-hat, relaxation, M = 100 averaged sweeps) in FP32 (the tile
    kernel) and in FP64 (MPR_PREC_F64, the list kernels), the time of one equilibrium sweep
    of each (FP32 also on the list kernels, the like-for-like ratio), and the MAE of each."""
    import torch
    from paper_1811_01604_gb300 import mpr, synth
    stream = torch.cuda.current_stream()
    sides = (32, 64, 128, 256, 512, 1024, 2048, 4096)
    variants = (("sp", dict()), ("dp", dict(precision=mpr.MPR_PREC_F64)))

    def fill(z, mask, L, seed, extra):
        out = torch.empty_like(z)
        prm = mpr.mpr_default_params(seed=seed, **extra)
        torch.cuda.synchronize()
        e0, eT, e1 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        ctx = mpr.mpr_init(z, mask, L, L, prm, stream.cuda_stream)
        try:
            T_hat, _ = mpr.mpr_estimate_T(ctx)
            eT.record(stream)
            st = mpr.mpr_equilibrate(ctx)
            mpr.mpr_predict(ctx, M, out)
            e1.record(stream)
            torch.cuda.synchronize()
        finally:
            mpr.mpr_free(ctx)
        # one sweep at a = 1, 10 timed after 3, on fresh contexts at T-hat (both FP32 kernels)
        sweep_ms = {}
        kernels = (("list", mpr.MPR_EXEC_LIST),) if extra else (("tile", mpr.MPR_EXEC_TILE),
                                                                ("list", mpr.MPR_EXEC_LIST))
        for name, ex in kernels:
            c2 = mpr.mpr_init(z, mask, L, L, mpr.mpr_default_params(seed=seed, exec_mode=ex, **extra),
                              stream.cuda_stream)
            try:
                mpr.mpr_set_T(c2, T_hat)
                mpr.mpr_time_sweeps(c2, 3, 1.0)
                sweep_ms[name] = mpr.mpr_time_sweeps(c2, 10, 1.0)
            finally:
                mpr.mpr_free(c2)
        gap = mask == 0
        mae = float((out - z)[gap].double().abs().mean())
        return dict(T=T_hat, sweeps=st.sweeps, ms=e0.elapsed_time(e1), ms_T=e0.elapsed_time(eT),
                    sweep_ms=sweep_ms, mae=mae)

    for _, extra in variants:                                    # untimed warm-up
        zw = synth.wm_field_gpu(64, 64, 0.5, 5.0, 1)
        fill(zw, synth.mask_uniform_gpu(64, 64, 0.33, 2), 64, 999, extra)
    rows = []
    for L in sides:
        for p in (0.33, 0.66):
            z = synth.wm_field_gpu(L, L, 0.5, 5.0, 700 + L)
            mask = synth.mask_uniform_gpu(L, L, p, 800 + L + int(100 * p))
            r = {"L": L, "p": p}
            for name, extra in variants:
                r[name] = fill(z, mask, L, 31 + L + int(1000 * p), extra)   # own seed: no cached table
            r["ratio_fill"] = r["dp"]["ms"] / r["sp"]["ms"]
            r["ratio_sweep_list"] = r["dp"]["sweep_ms"]["list"] / r["sp"]["sweep_ms"]["list"]
            r["ratio_sweep_tile"] = r["dp"]["sweep_ms"]["list"] / r["sp"]["sweep_ms"]["tile"]
            rows.append(r)
            print(json.dumps(r), file=sys.stderr, flush=True)
    big = [r for r in rows if r["L"] >= 1024]
    line = {"metric": "DP/SP time ratio of a whole fill, L >= 1024",
            "value": float(np.mean([r["ratio_fill"] for r in big])), "unit": "ratio",
            "n_gpus": 1, "steps": 1, "warmup": 1, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32/f64", "data": "synthetic",
            "config": {"workload": "mpr-dpsp-wm-nu0.5-xi5-p0.33,0.66-L32..4096", "M": M},
            "rows": rows}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mpr", choices=["mpr", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-case", default=None,
                    choices=["sweep4096", "fill4096", "copy4096", "net4096", "net1024", "net128",
                             "sweep64_4096", "trace4096", "trace1024", "hostlink"],
                    help="run a small fixed sweep workload for ncu instead of the benchmark")
    ap.add_argument("--workload", default="fill4096", choices=["fill4096", "config1024", "batch256", "warm1024",
                                                                "warm4096", "chains1024", "ormodes1024", "dpsp"],
                    help="fill4096: one 4096^2 map per step (default); config1024: the eight 1024^2 "
                         "grids (nu 0.5 / 2.5, Gaussian / lognormal, 33 / 66 %% gaps), one line each; "
                         "batch256: 256 grids of "
                         "sides 128-2048 filled in one batch, against the same grids one at a time; "
                         "warm1024 / warm4096: learned warm start against the plain random start; "
                         "chains1024: independent chains against one chain at equal sweeps; "
                         "ormodes1024: fills with the Eq. 6 readings (conserving, printed, none); "
                         "dpsp: FP32 against FP64 fills, L = 32 .. 4096")
    ap.add_argument("--tile-cfg", type=int, default=0, help="profile cases: compiled tile configuration")
    ap.add_argument("--train-steps", type=int, default=2000, help="warm start: Adam steps")
    ap.add_argument("--warm-stride", type=int, default=4, choices=[1, 2, 4, 8],
                    help="warm start: sites per network pixel along each axis")
    ap.add_argument("--batch-warm", action="store_true",
                    help="batch256: also time the batched fill with the learned warm start")
    ap.add_argument("--train-n64", type=int, default=1024, help="warm start: 64^2 training grids")
    ap.add_argument("--train-n128", type=int, default=4096, help="warm start: 128^2 training crops")
    ap.add_argument("--train-n256", type=int, default=1024,
                    help="warm start: 256^2 training crops with the 4096^2 workload's disk gaps")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if args.profile_case:
        profile_case(args.profile_case, args.tile_cfg)
        return
    if args.workload == "batch256":
        run_batch(args)
        return
    if args.workload in ("warm1024", "warm4096"):
        run_warm(args)
        return
    if args.workload == "chains1024":
        run_chains(args)
        return
    if args.workload == "ormodes1024":
        run_or_modes(args)
        return
    if args.workload == "dpsp":
        run_dpsp(args)
        return
    if args.workload == "config1024":
        run_config2(args)
        return

    import torch
    from paper_1811_01604_gb300 import mpr

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)

    z_np, m_np = make_inputs(rank)
    H, W = z_np.shape
    z = torch.from_numpy(z_np).to(dev)
    mask = torch.from_numpy(m_np).to(dev)
    zhat = torch.empty_like(z)
    z_h = torch.from_numpy(z_np).pin_memory()
    m_h = torch.from_numpy(m_np).pin_memory()
    zhat_h = torch.empty_like(z_h).pin_memory()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # 512 MB > L2
    prm = mpr.mpr_default_params(seed=1 + rank, M=M)
    stream = torch.cuda.current_stream(dev)

    N = H * W
    P = int(m_np.size - m_np.sum())                     # gap sites (host work, outside every timed region)

    def one_fill(zi, mi, out, p=prm):
        ctx = mpr.mpr_init(zi, mi, W, H, p, stream.cuda_stream)
        try:
            T, _ = mpr.mpr_estimate_T(ctx)
            st = mpr.mpr_equilibrate(ctx)
            mpr.mpr_predict(ctx, M, out)
        finally:
            mpr.mpr_free(ctx)
        return P * (st.sweeps + M), st, T

    # warm-up (the first one loads the library's kernels and builds and caches the e(T, L)
    # table of this shape); the library's autotuner then picks the tile configuration for
    # this grid shape, used by every later fill
    one_fill(z, mask, zhat)
    torch.cuda.synchronize()
    ctx = mpr.mpr_init(z, mask, W, H, prm, stream.cuda_stream)
    try:
        mpr.mpr_estimate_T(ctx)
        tune = mpr.mpr_autotune(ctx)
    finally:
        mpr.mpr_free(ctx)
    prm.tile_cfg = tune["tile_cfg"]
    for _ in range(max(0, args.warmup - 1)):
        one_fill(z, mask, zhat)

    # a first map of a new shape pays for its e(T, L) table: a fill with a seed whose table
    # is not cached yet (the table depends on the seed), timed alone
    cold_prm = mpr.mpr_default_params(seed=1_000_001 + rank, M=M, tile_cfg=prm.tile_cfg)
    flush.zero_()
    torch.cuda.synchronize()
    c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    c0.record(stream)
    one_fill(z, mask, zhat, cold_prm)
    c1.record(stream)
    torch.cuda.synchronize()
    cold_ms = c0.elapsed_time(c1)

    def timed(zi, mi, out):
        total_ms, updates, launches, sweeps = 0.0, 0, 0, []
        for _ in range(args.steps):
            flush.zero_()                                  # L2 flush between steps
            torch.cuda.synchronize()
            if dist:
                dist.barrier()
            l0 = mpr.mpr_kernel_launches()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            u, st, T = one_fill(zi, mi, out)
            e1.record(stream)
            torch.cuda.synchronize()
            launches += mpr.mpr_kernel_launches() - l0
            total_ms += e0.elapsed_time(e1)
            updates += u
            sweeps.append(st.sweeps)
        return total_ms, updates, launches, sweeps, T

    clocks = ClockSampler(local)
    clocks.start()
    torch.cuda.profiler.start()        # an ncu run with --profile-from-start off sees these steps
    mpr.mpr_sweep_timing_start()       # CUDA events around every sweep-kernel launch of the steps
    dev_ms, dev_updates, launches, sweeps, T = timed(z, mask, zhat)
    swt = mpr.mpr_sweep_timing_read(stop=True)
    torch.cuda.profiler.stop()
    one_fill(z_h, m_h, zhat_h)         # untimed: the first fill from these host buffers
    torch.cuda.synchronize()
    e2e_ms, e2e_updates, _, _, _ = timed(z_h, m_h, zhat_h)
    clk = clocks.stop()

    # the same sweeps with the fast transcendentals (__sincosf, ex2.approx), for reference
    ctx = mpr.mpr_init(z, mask, W, H, mpr.mpr_default_params(seed=1 + rank, M=M, trig_mode=mpr.MPR_TRIG_FAST,
                                                             tile_cfg=prm.tile_cfg), stream.cuda_stream)
    try:
        mpr.mpr_set_T(ctx, T)
        mpr.mpr_sweep(ctx, 20, 1.0)
        sweep_ms_fast = mpr.mpr_time_sweeps(ctx, 100, 1.0)
    finally:
        mpr.mpr_free(ctx)
    # roofline of the dominant kernel (the persistent sweep kernel: one launch per phase of
    # a fill), from the CUDA-event durations of its launches in the timed steps.  Algorithmic
    # bytes of one sweep: every site's angle read once (4 B) plus the gap sites' angles
    # read and written (8 B) plus the mask bits (N / 4 B); the unit-vector lattice's own
    # bytes are 8 B per site read and 10 B per gap site (vector written, list entry read).
    peaks, peak_src = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    k_ms = swt["ms"]
    k_launches = max(1, swt["launches"])
    bytes_alg = 4.25 * swt["site_sweeps"] + 8.0 * swt["gap_updates"]
    bytes_uv = 8.0 * swt["site_sweeps"] + 10.0 * swt["gap_updates"]
    achieved = bytes_alg / (k_ms * 1e-3) / 1e9 if k_ms > 0 else 0.0
    sweeps_total = swt["site_sweeps"] / N
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_mhz = clk.get("sm_mhz") or float(peaks.get("sm_max_mhz", 2070.0))
    alu_peak = sms * LANES_PER_SM * sm_mhz * 1e6                 # lane operations / s
    alu_achieved = ALU_OPS_PER_UPDATE * swt["gap_updates"] / (k_ms * 1e-3) if k_ms > 0 else 0.0
    binding = "alu" if ALU_OPS_PER_UPDATE * swt["gap_updates"] / alu_peak > bytes_alg / (hbm * 1e9) else "hbm"
    tr = TILE_TRAFFIC_PER_SWEEP.get(tune["tile_cfg"]) if tile_kernel_hash() == TILE_TRAFFIC_SOURCE_HASH else None
    # per launch of the timed steps: each step is one relaxation launch and one of M sweeps
    traffic_launch = ((sum(sweeps) * tr["relax"] + args.steps * M * tr["acc"]) / k_launches) if tr else None

    (dev_ms, e2e_ms), (dev_updates, e2e_updates) = reduce_over_ranks(
        [dev_ms, e2e_ms], [dev_updates, e2e_updates], dist, dev)

    if rank == 0:
        line = {
            "metric": METRIC, "value": dev_updates / (dev_ms * 1e-3), "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dev_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "W": W, "H": H, "gap_sites": P, "M": M,
                       "relax_sweeps": sweeps, "T_hat": T,
                       "s_per_map": dev_ms * 1e-3 / args.steps,
                       "cold_s_per_map": cold_ms * 1e-3,
                       "T_table": "cached per lattice shape and sampler parameters; every timed step "
                                  "reuses it, cold_s_per_map includes building it",
                       "tile_cfg": tune["tile_cfg"], "autotune_ms_per_sweep": tune["ms_per_sweep"],
                       "trig": "accurate (Taylor sincos, expf); fast-trig sweep in roofline.ms_per_sweep_fast",
                       "l2": "512 MB buffer written between steps (L2 flush)",
                       "parallelism": f"replicas{world}"},
            "e2e": {"value": e2e_updates / (e2e_ms * 1e-3), "unit": UNIT,
                    "h2d_bytes_per_step": N * 5, "d2h_bytes_per_step": N * 4},
            "gpu_launches": int(launches),
            # the binding roof of the algorithmic counts (the larger of the two times, the
            # fraction of the roofline model: max(bytes / BW, ops / ALU peak) / time)
            "roofline": {"bound": binding,
                         "achieved": alu_achieved * 1e-12 if binding == "alu" else achieved,
                         "peak": alu_peak * 1e-12 if binding == "alu" else hbm,
                         "unit": "Top/s" if binding == "alu" else "GB/s",
                         "frac": alu_achieved / alu_peak if binding == "alu" else achieved / hbm,
                         "traffic": traffic_launch,
                         "hbm": {"achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm},
                         "kernel": "k_tile_sweep", "tile_cfg": tune["tile_cfg"],
                         "launches": swt["launches"], "ms_per_launch": k_ms / k_launches,
                         "bytes_per_launch": bytes_alg / k_launches,
                         "bytes_model": "(4 + 8p) N + N/4 per sweep",
                         "sweeps_per_launch": sweeps_total / k_launches,
                         "ms_per_sweep": k_ms / sweeps_total if sweeps_total else None,
                         "ms_per_sweep_fast": sweep_ms_fast,
                         "peak_source": f"{peak_src} hbm_gbs",
                         "frac_unit_vector_bytes": bytes_uv / (k_ms * 1e-3) / 1e9 / hbm if k_ms > 0 else None,
                         "traffic_per_sweep": ({"relax": tr["relax"], "acc": tr["acc"]} if tr else None),
                         "alu": {"ops_per_update": ALU_OPS_PER_UPDATE, "sms": sms,
                                 "lanes_per_sm": LANES_PER_SM, "sm_mhz": sm_mhz,
                                 "peak_ops": alu_peak, "achieved_ops": alu_achieved},
                         "frac_alu": alu_achieved / alu_peak,
                         "binding": binding},
            "clocks": clk,
        }
        if not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline(z_np, m_np, T)
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
