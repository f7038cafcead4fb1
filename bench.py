#!/usr/bin/env python3
"""Throughput of the Radon forward projection + exact adjoint on one GB300 (or N, one rank each).

Workload (default): fan beam, 16 x 512^2 seeded ellipse phantoms, 720 views over [0, 2 pi),
source 1000 px, detector 500 px, 1024 bins x 1.5 px.  One step = the forward projection of the
whole image batch and the adjoint of a whole sinogram batch (independent inputs), i.e. every
kernel of the hot path once.  Metric: bilinear samples per second, 2 B S / (t_fwd + t_adj), with
S the per-image sample count the geometry enumerates in FP64; images/s = B / (t_fwd + t_adj).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle on the host
cores on a bounded sample of the same workload.
"""

from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from synth import WORKLOADS, workload_geometry_args, workload_images  # noqa: E402

DEFAULT_WORKLOAD = "fan_b16_n512_v720_d1024"
L2_BYTES = 126 * 1024 * 1024
METRIC = "Radon fwd+adjoint bilinear samples/s and images/s at 512^2; chosen vs plain FP32"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 50 ms around the timed region; each sample
    carries its host arrival time, and the summary covers the samples inside the region marked by
    ``region(t0, t1)`` (all samples if none fell inside)."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    PERIOD_MS = 50

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self._t = None
        self._region = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", str(self.PERIOD_MS)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self._t = threading.Thread(target=self._read, daemon=True)
        self._t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.monotonic(), line.strip()))

    def region(self, t0: float, t1: float):
        """Host monotonic times bracketing the timed region."""
        self._region = (t0, t1)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self._t is not None:
            self._t.join(timeout=2)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        parsed = []
        for t, ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                parsed.append((t, float(parts[1]), float(parts[2]),
                               {n for n, v in zip(names, parts[5:9]) if v.lower() == "active"}))
            except ValueError:
                continue
        if not parsed:
            return None
        inside = parsed
        if self._region is not None:
            # a line arrives up to one period after the GPU state it reports
            t0, t1 = self._region
            inside = [p for p in parsed if t0 <= p[0] <= t1 + self.PERIOD_MS / 1000.0] or parsed
        reasons = set().union(*(p[3] for p in inside))
        return {"sm_mhz": statistics.median(p[1] for p in inside), "sm_max_mhz": max(p[2] for p in parsed),
                "samples": len(inside), "samples_total": len(parsed), "period_ms": self.PERIOD_MS,
                "reasons": sorted(reasons)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


ADJ_OPS_PER_SAMPLE = 18
ADJ_PRODUCTS_PER_SAMPLE = 2.5


def max_over_ranks(values, device=None):
    """Element-wise maximum of ``values`` over the ranks of the default process group (if any)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor(values, dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def whole_job_value(units_per_rank_step, world, ms_per_step):
    """Units all ranks processed per second: every rank runs its own replica of the step (weak
    scaling), and the step time is the slowest rank's."""
    return units_per_rank_step * world / (ms_per_step * 1e-3)


def workload_config(workload, storage, algo, geom):
    """The ``config`` object of the GPU arm's JSON line: the workload and its library geometry."""
    w = WORKLOADS[workload]
    return {"workload": workload, "geometry": geom.kind, "batch": w.batch, "n": geom.n, "views": geom.n_angles,
            "det_count": geom.det_count, "det_spacing": geom.det_spacing, "source_distance": geom.source_distance,
            "det_distance": geom.det_distance, "storage": storage, "algo": algo,
            "samples_per_image": geom.sample_count,
            "parallelism": "replica per GPU (batch sharding, no exchange)"}


def oracle_workload_config(workload, storage, algo):
    """The same ``config`` object built from the oracle's geometry alone (the reference arm never
    loads the library): defaults resolved and samples counted by ``oracle``."""
    import oracle as O
    w = WORKLOADS[workload]
    og = O.Geometry.from_args(workload_geometry_args(w))
    return {"workload": workload, "geometry": og.kind, "batch": w.batch, "n": og.n, "views": og.n_angles,
            "det_count": int(og.det_count), "det_spacing": float(og.det_spacing),
            "source_distance": float(og.source_distance), "det_distance": float(og.det_distance),
            "storage": storage, "algo": algo, "samples_per_image": O.sample_count(og),
            "parallelism": "replica per GPU (batch sharding, no exchange)"}


def roofline(samples, ms, sm_count, per_sm, clk_mhz, basis, traffic):
    """Achieved vs peak bilinear samples/s of one kernel (``alu``: an on-chip pipe bounds it)."""
    peak = sm_count * per_sm * clk_mhz * 1e6 / 1e9
    achieved = samples / (ms * 1e-3) / 1e9
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Gsamples/s", "frac": achieved / peak,
            "traffic": traffic, "peak_basis": basis + " (sm_max_mhz of MEASURED_PEAKS.json)"}


# ----------------------------------------------------------------------------- GPU arm

def _try_adjoint_table(geom, L):
    """Builds the geometry's adjoint weight table (once per geometry, outside any timed region);
    returns (bytes, seconds, overflow fraction) or None where the library refuses it."""
    t0 = time.perf_counter()
    try:
        geom.build_adjoint_table()
    except L.RadonError:
        return None
    return geom.adjoint_table_bytes(), time.perf_counter() - t0, geom.adjoint_table_overflow()


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2009_14788_gb300 import (Geometry, _lib as L, backward_raw, forward_images_per_cta, forward_raw,
                                        launch_config)
    from paper_2009_14788_gb300.build import build

    world, rank, local = _dist()
    if WORKLOADS[args.workload].kind not in ("parallel", "fan"):
        raise SystemExit("the timed step takes a parallel or fan workload; %s is measured in the secondary "
                         "section of the default run" % args.workload)
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build()
    w = WORKLOADS[args.workload]
    gargs = workload_geometry_args(w)
    kind = gargs.pop("kind")
    geom = Geometry(kind, **gargs)
    B = w.batch
    S = geom.sample_count
    dtypes = {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}
    dt = dtypes[args.storage]
    chosen = launch_config(args.algo)
    plain = launch_config("plain")
    # the exact adjoint's weight table: built once per geometry, before anything is timed (a GB300
    # memory-for-compute trade: the packed adjoint then reads its bilinear weights, same bits)
    table = None if args.no_adjoint_table else _try_adjoint_table(geom, L)

    x64 = workload_images(w)
    bytes_per_set = (B * geom.n * geom.n + B * geom.n_angles * geom.det_count) * 2 * torch.empty((), dtype=dt).element_size()
    n_sets = max(2, int(np.ceil(2.5 * L2_BYTES / bytes_per_set)))
    xs = [torch.from_numpy(x64).to(device="cuda", dtype=dt) for _ in range(n_sets)]
    y0 = forward_raw(geom, xs[0].float()).to(dt)
    ys = [y0.clone() for _ in range(n_sets)]
    outs_y = [torch.empty_like(y0) for _ in range(n_sets)]
    outs_x = [torch.empty_like(xs[0]) for _ in range(n_sets)]
    stream = torch.cuda.current_stream()

    def step(i, cfg, sets, ev=None):
        xset, yset, oy, ox = sets
        j = i % len(xset)
        if ev is not None:
            ev[0].record(stream)
        forward_raw(geom, xset[j], cfg, out=oy[j])
        if ev is not None:
            ev[1].record(stream)
        backward_raw(geom, yset[j], cfg, out=ox[j])
        if ev is not None:
            ev[2].record(stream)

    def timed(cfg, steps, warmup, sets, launches=None):
        for i in range(warmup):
            step(i, cfg, sets)
        torch.cuda.synchronize()
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        n0 = L.radon_kernel_launch_count()
        t0.record(stream)
        for i in range(steps):
            step(i, cfg, sets, evs[i])
        t1.record(stream)
        if launches is not None:
            launches["count"] = int(L.radon_kernel_launch_count() - n0)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        total = t0.elapsed_time(t1)
        fwd = [e[0].elapsed_time(e[1]) for e in evs]
        adj = [e[1].elapsed_time(e[2]) for e in evs]
        return total, fwd, adj

    # supplementary: the plain FP32 form on the same workload (outside the headline timed region);
    # FP32 sets rotate over more than 2x L2 as well
    n32 = max(2, int(np.ceil(2.5 * L2_BYTES / ((B * geom.n * geom.n + B * geom.n_angles * geom.det_count) * 8))))
    x32 = xs[0].float()
    y32 = ys[0].float()
    sets32 = ([x32.clone() for _ in range(n32)], [y32.clone() for _ in range(n32)],
              [torch.empty_like(y32) for _ in range(n32)], [torch.empty_like(x32) for _ in range(n32)])
    p_steps = max(2, min(5, args.steps))
    p_total, p_fwd, p_adj = timed(plain, p_steps, 1, sets32)
    plain_ms = p_total / p_steps
    # supplementary: the same tuned kernels with FP32 storage (Section 3.3 compares 16-bit with FP32
    # storage in one design)
    t_steps = max(3, min(20, args.steps))
    t_total, t_fwd, t_adj = timed(chosen, t_steps, 3, sets32)
    tuned32_ms = t_total / t_steps
    del sets32, x32, y32
    torch.cuda.empty_cache()
    # supplementary: the FP16 forward with FP16 weights in mixed-precision FMAs (opt-in), timed alone,
    # and its departure from the FP32-weight forward on the same input
    f16w = None
    if args.storage == "f16":
        cfg_w2 = launch_config(args.algo, weights=2)
        for i in range(3):
            forward_raw(geom, xs[i % n_sets], cfg_w2, out=outs_y[i % n_sets])
        torch.cuda.synchronize()
        wev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(t_steps)]
        for i in range(t_steps):
            wev[i][0].record(stream)
            forward_raw(geom, xs[i % n_sets], cfg_w2, out=outs_y[i % n_sets])
            wev[i][1].record(stream)
        torch.cuda.synchronize()
        w2_ms = statistics.mean(e[0].elapsed_time(e[1]) for e in wev)
        y_w2 = forward_raw(geom, xs[0], cfg_w2).double()
        y_w0 = forward_raw(geom, xs[0], chosen).double()
        f16w = {"fwd_ms": w2_ms, "samples_per_s": B * S / (w2_ms * 1e-3),
                "max_abs_diff_rel_to_max": float((y_w2 - y_w0).abs().max() / y_w0.abs().max()),
                "rel_l2_vs_fp32_weights": float(torch.linalg.vector_norm(y_w2 - y_w0) / torch.linalg.vector_norm(y_w0)),
                "weights": "FP16 (each weight rounded once, relative error <= 2^-12), exact FP16 x FP16 products "
                           "accumulated in FP32 (fma.rn.f32.f16)"}
        del y_w2, y_w0

    # supplementary: the adjoint with its weights computed on the fly (the table freed for the
    # measurement and rebuilt before the headline), the same bits
    no_table = None
    if table is not None:
        geom.free_adjoint_table()
        for i in range(3):
            backward_raw(geom, ys[i % n_sets], chosen, out=outs_x[i % n_sets])
        torch.cuda.synchronize()
        aev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(t_steps)]
        for i in range(t_steps):
            aev[i][0].record(stream)
            backward_raw(geom, ys[i % n_sets], chosen, out=outs_x[i % n_sets])
            aev[i][1].record(stream)
        torch.cuda.synchronize()
        nt_ms = statistics.mean(e[0].elapsed_time(e[1]) for e in aev)
        ref_x = backward_raw(geom, ys[0], chosen)
        table = _try_adjoint_table(geom, L)
        same = table is not None and bool(torch.equal(backward_raw(geom, ys[0], chosen), ref_x))
        no_table = {"adj_ms": nt_ms, "samples_per_s": B * S / (nt_ms * 1e-3), "same_bits_as_table": same}
        del ref_x

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    launches = {}
    th0 = time.monotonic()
    total_ms, fwd_ms, adj_ms = timed(chosen, args.steps, args.warmup, (xs, ys, outs_y, outs_x), launches)
    clocks.region(th0, time.monotonic())
    time.sleep(0.2)
    clk = clocks.stop()

    # end to end through the public API with pinned host buffers: every step uploads its inputs and
    # downloads both results inside the timed region.  Three streams pipeline the steps the way a
    # streaming user would (step i+1 uploads while step i computes and step i-1 downloads); two
    # device buffer sets with events order each buffer's reuse.
    hx = [torch.from_numpy(x64).to(dtype=dt).pin_memory() for _ in range(2)]
    hy = [ys[0].cpu().pin_memory() for _ in range(2)]
    hox = [torch.empty(outs_x[0].shape, dtype=dt).pin_memory() for _ in range(2)]
    hoy = [torch.empty(outs_y[0].shape, dtype=dt).pin_memory() for _ in range(2)]
    dx = [torch.empty_like(xs[0]) for _ in range(2)]
    dy = [torch.empty_like(ys[0]) for _ in range(2)]
    dox = [torch.empty_like(outs_x[0]) for _ in range(2)]
    doy = [torch.empty_like(outs_y[0]) for _ in range(2)]
    up, down = torch.cuda.Stream(), torch.cuda.Stream()
    e_steps = max(3, min(args.steps, 10))
    uploaded = [torch.cuda.Event() for _ in range(2)]
    computed = [torch.cuda.Event() for _ in range(2)]
    downloaded = [torch.cuda.Event() for _ in range(2)]
    for ev in computed + downloaded:
        ev.record(stream)
    for i in range(args.warmup + e_steps):
        if i == args.warmup:
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            up.wait_event(e0)
        j = i % 2
        with torch.cuda.stream(up):
            up.wait_event(computed[j])         # step i-2 has finished reading dx[j], dy[j]
            dx[j].copy_(hx[j], non_blocking=True)
            dy[j].copy_(hy[j], non_blocking=True)
            uploaded[j].record(up)
        stream.wait_event(uploaded[j])
        stream.wait_event(downloaded[j])       # step i-2's results have left dox[j], doy[j]
        forward_raw(geom, dx[j], chosen, out=doy[j])
        backward_raw(geom, dy[j], chosen, out=dox[j])
        computed[j].record(stream)
        with torch.cuda.stream(down):
            down.wait_event(computed[j])
            hoy[j].copy_(doy[j], non_blocking=True)
            hox[j].copy_(dox[j], non_blocking=True)
            downloaded[j].record(down)
    for ev in downloaded:
        stream.wait_event(ev)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / e_steps
    h2d = hx[0].numel() * hx[0].element_size() + hy[0].numel() * hy[0].element_size()
    d2h = hox[0].numel() * hox[0].element_size() + hoy[0].numel() * hoy[0].element_size()
    assert torch.equal(hoy[(args.warmup + e_steps - 1) % 2], outs_y[0].cpu()), "e2e forward result differs"
    assert torch.equal(hox[(args.warmup + e_steps - 1) % 2], outs_x[0].cpu()), "e2e adjoint result differs"
    del dx, dy, dox, doy

    # max over ranks
    total_ms, e2e_ms = max_over_ranks([total_ms, e2e_ms], device="cuda")
    ms_per_step = total_ms / args.steps
    samples_per_step = 2 * B * S
    value = whole_job_value(samples_per_step, world, ms_per_step)

    mean_fwd = statistics.mean(fwd_ms)
    mean_adj = statistics.mean(adj_ms)
    dom = "forward" if mean_fwd >= mean_adj else "backward"
    peaks = _peaks()
    sm_count = torch.cuda.get_device_properties(local).multi_processor_count
    clk_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    bytes_per_texel = torch.empty((), dtype=dt).element_size()
    traffic_tab = {}
    tfile = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tfile):
        try:
            with open(tfile) as f:
                traffic_tab = json.load(f).get(args.workload, {}).get(args.storage, {})
        except (OSError, ValueError):
            traffic_tab = {}
    # the gather-ceiling probe over as many texel groups per sample as the chosen forward's CTAs take
    probe = ctypes.c_double(0.0)
    dt_code = {"f32": L.RADON_F32, "f16": L.RADON_F16, "bf16": L.RADON_BF16}[args.storage]
    bg = 4 if args.storage == "f32" else 8
    fwd_groups = max(1, forward_images_per_cta(geom, dt, B, chosen) // bg)
    L.check(L.radon_probe_gather_ceiling_groups(dt_code, 0, fwd_groups, ctypes.byref(probe)),
            "radon_probe_gather_ceiling_groups")
    rooflines = {
        # forward: 4 texels per sample through the shared-memory / L1 load pipe, 128 B/clk/SM
        "forward": roofline(B * S, mean_fwd, sm_count, 128.0 / (4.0 * bytes_per_texel), clk_mhz,
                            "%d SMs x %.0f samples/clk/SM (128 B/clk/SM load pipe / 4 texels x %d B) x %.0f MHz"
                            % (sm_count, 128.0 / (4.0 * bytes_per_texel), bytes_per_texel, clk_mhz),
                            traffic_tab.get("forward")),
        # adjoint: FP32 issue, 128 lanes/clk/SM over ~18 FP32 operations per sample (4 weight pairs)
        "backward": roofline(B * S, mean_adj, sm_count, 128.0 / ADJ_OPS_PER_SAMPLE, clk_mhz,
                             "%d SMs x %.2f samples/clk/SM (128 FP32 lanes/clk/SM / %d ops per sample) x %.0f MHz"
                             % (sm_count, 128.0 / ADJ_OPS_PER_SAMPLE, ADJ_OPS_PER_SAMPLE, clk_mhz),
                             traffic_tab.get("backward_table" if table is not None else "backward")),
    }

    # the same adjoint against a products-only floor: one FP32 FMA per image, pixel and candidate ray
    # that carries weight (~2.6 such rays per pixel and view, ~1.04 samples per pixel and view on the
    # headline geometry: ~2.5 FMAs per image-sample), the weights shared by a group's images counted
    # as free -- the ceiling a perfect use of the weight sharing would approach
    floor = sm_count * (128.0 / ADJ_PRODUCTS_PER_SAMPLE) * clk_mhz * 1e6 / 1e9
    rooflines["backward"]["products_floor"] = floor
    rooflines["backward"]["frac_of_products_floor"] = rooflines["backward"]["achieved"] / floor
    rooflines["backward"]["products_floor_basis"] = (
        "%d SMs x %.1f samples/clk/SM (128 FP32 FMA lanes/clk/SM / %.1f products per image-sample) x %.0f MHz"
        % (sm_count, 128.0 / ADJ_PRODUCTS_PER_SAMPLE, ADJ_PRODUCTS_PER_SAMPLE, clk_mhz))
    if table is not None:
        # with the weight table the adjoint no longer evaluates weights: its floor is the products (the
        # per-sample weight-evaluation basis above stays as the table-free adjoint's), and it streams
        # the table from HBM once per launch
        weight_basis = dict(rooflines["backward"])
        rooflines["backward"] = roofline(
            B * S, mean_adj, sm_count, 128.0 / ADJ_PRODUCTS_PER_SAMPLE, clk_mhz,
            "%d SMs x %.1f samples/clk/SM (128 FP32 FMA lanes/clk/SM / %.1f products per image-sample) x %.0f MHz"
            % (sm_count, 128.0 / ADJ_PRODUCTS_PER_SAMPLE, ADJ_PRODUCTS_PER_SAMPLE, clk_mhz),
            traffic_tab.get("backward_table"))
        hbm = float(peaks.get("hbm_gbs", 6764.0))
        rooflines["backward"]["table_hbm"] = {"achieved": table[0] / (mean_adj * 1e-3) / 1e9, "peak": hbm,
                                              "unit": "GB/s", "frac": table[0] / (mean_adj * 1e-3) / 1e9 / hbm,
                                              "bytes": table[0], "peak_basis": "hbm_gbs of MEASURED_PEAKS.json"}
        rooflines["backward"]["frac_of_weight_evaluation_basis"] = weight_basis["frac"]
    rooflines["forward"]["probe_ceiling"] = probe.value / 1e9
    rooflines["forward"]["frac_of_probe"] = rooflines["forward"]["achieved"] / (probe.value / 1e9)
    rooflines["forward"]["images_per_cta"] = fwd_groups * bg
    if f16w is not None:
        probe2 = ctypes.c_double(0.0)
        w2_groups = max(1, forward_images_per_cta(geom, dt, B, launch_config(args.algo, weights=2)) // 8)
        L.check(L.radon_probe_gather_ceiling_groups(L.RADON_F16, 2, w2_groups, ctypes.byref(probe2)),
                "radon_probe_gather_ceiling_groups")
        f16w["roofline"] = roofline(B * S, f16w["fwd_ms"], sm_count, 128.0 / (4.0 * bytes_per_texel), clk_mhz,
                                    rooflines["forward"]["peak_basis"].split(" (")[0], None)
        f16w["roofline"]["probe_ceiling"] = probe2.value / 1e9
        f16w["roofline"]["frac_of_probe"] = f16w["samples_per_s"] / probe2.value
    tuned32 = {"ms_per_step": tuned32_ms, "samples_per_s": samples_per_step / (tuned32_ms * 1e-3),
               "images_per_s": B / (tuned32_ms * 1e-3), "fwd_ms": statistics.mean(t_fwd),
               "adj_ms": statistics.mean(t_adj),
               "roofline_forward": roofline(B * S, statistics.mean(t_fwd), sm_count, 128.0 / 16.0, clk_mhz,
                                            "%d SMs x 8 samples/clk/SM (128 B/clk/SM load pipe / 4 texels x 4 B) x %.0f MHz"
                                            % (sm_count, clk_mhz), None),
               "roofline_backward": roofline(B * S, statistics.mean(t_adj), sm_count, 128.0 / ADJ_OPS_PER_SAMPLE,
                                             clk_mhz, rooflines["backward"]["peak_basis"].split(" (")[0], None)}
    secondary = None
    if rank == 0 and world == 1 and not args.no_secondary:
        secondary = run_secondary(args)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_sample(w, args.cpu_seconds)

    if rank == 0:
        line = {
            "metric": METRIC,
            "value": value,
            "unit": "samples/s",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": ms_per_step,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32",
            "data": "synthetic",
            "config": dict(workload_config(args.workload, args.storage, args.algo, geom),
                           arithmetic="FP32 (FP32 bilinear weights, FP32 accumulation; storage %s)" % args.storage,
                           adjoint_weights=("precomputed once per geometry (%.2f GB table in HBM, built outside the "
                                            "timed region; same bits as computing them)" % (table[0] / 1e9)
                                            if table is not None else "computed on the fly"),
                           l2="rotating %d input/output sets, %.0f MB total (> 2x L2)" % (
                               n_sets, n_sets * bytes_per_set / 2**20)),
            "images_per_s": B * world / (ms_per_step * 1e-3),
            "fwd_ms": mean_fwd,
            "adj_ms": mean_adj,
            "plain_f32": {"ms_per_step": plain_ms, "samples_per_s": samples_per_step / (plain_ms * 1e-3),
                          "fwd_ms": statistics.mean(p_fwd), "adj_ms": statistics.mean(p_adj)},
            "speedup_vs_plain_f32": plain_ms / ms_per_step,
            "tuned_f32": tuned32,
            "speedup_16bit_storage_vs_tuned_f32": tuned32_ms / ms_per_step,
            "fp16_weights_forward": f16w,
            "adjoint_weight_table": (None if table is None else
                                     {"bytes": table[0], "build_s": table[1], "overflow_fraction": table[2],
                                      "table_read_gbs": table[0] / (mean_adj * 1e-3) / 1e9,
                                      "frac_of_hbm": table[0] / (mean_adj * 1e-3) / 1e9 / float(peaks.get("hbm_gbs", 6764.0)),
                                      "adjoint_without_table": no_table}),
            "roofline": dict(rooflines[dom], kernel=dom),
            "roofline_forward": rooflines["forward"],
            "roofline_backward": rooflines["backward"],
            "e2e": {"value": whole_job_value(samples_per_step, world, e2e_ms), "unit": "samples/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms},
            "gpu_launches": launches["count"],
            "clocks": clk,
            "cpu_baseline": cpu,
        }
        if secondary is not None:
            line["secondary"] = secondary
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def _flush_l2(buf):
    buf.zero_()   # a write larger than L2 between timed iterations (outside the timed brackets)


def run_secondary(args):
    """The two secondary points, each over a few L2-flushed iterations on the same GPU.

    * Landweber (8 x 512^2 parallel, 60 views in [0, pi), 725 detectors, bf16 storage): the step
      size by 20 power iterations, 10 Landweber iterations forward, and the reverse pass to the
      gradients w.r.t. y and alpha (per-iteration checkpoints: 3 projections per iteration); the
      iterations again with the geometry's adjoint weight table.
    * The paper's batch benchmark shape (32 x 512^2 parallel, 512 views in [0, pi), 512
      detectors): forward + adjoint, chosen 16-bit form against the plain FP32 form, without and
      with the geometry's adjoint weight table.
    * The uneven batch (64 images, 16 each of 128^2 .. 1024^2, each with its own parallel geometry,
      fp16): one forward plan and one adjoint plan (autotuned at creation) replayed as one CUDA
      graph, against one library call per image and direction.
    * Filtered backprojection at the paper's FBP setting (512^2, 512 views, 725 detectors, Ram-Lak),
      and CGNE (20 iterations) at the same setting; the batched ones also with the geometry's adjoint
      weight table.
    * The pixel-driven interpolating backprojector against the exact adjoint on the headline workload.
    """
    import torch

    from paper_2009_14788_gb300 import Geometry, Landweber, _lib as L, backward_raw, forward_raw, launch_config
    from synth import power_start, uniform_angles, workload_noise

    flush = torch.empty(2 * L2_BYTES, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def time_it(fn, reps, warm=2):
        for _ in range(warm):
            fn()
        ts = []
        for _ in range(reps):
            _flush_l2(flush)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    out = {}
    # Landweber
    w = WORKLOADS["landweber_b8_n512_v60_d725"]
    ga = workload_geometry_args(w)
    kind = ga.pop("kind")
    g = Geometry(kind, **ga)
    S = g.sample_count
    K = w.extra["iterations"]
    P = w.extra["power_iterations"]
    x_true = workload_images(w)
    sino_shape = (w.batch, g.n_angles, g.det_count)
    xt = torch.from_numpy(x_true).to("cuda", torch.float32)
    y32 = forward_raw(g, xt) + torch.from_numpy(workload_noise(w, sino_shape)).to("cuda", torch.float32)
    y = y32.to(torch.bfloat16)
    lw = Landweber(g)
    v0 = torch.from_numpy(power_start(g.n, 2000 * w.number)).to("cuda", torch.float32)
    ms_power = time_it(lambda: lw.power(P, v0=v0), 3)
    alpha, lam = lw.power(P, v0=v0)
    x0 = torch.zeros((w.batch, g.n, g.n), dtype=torch.bfloat16, device="cuda")
    yg = y.clone().requires_grad_(True)
    ag = alpha.clone().requires_grad_(True)
    ms_fwd = time_it(lambda: lw.run(x0, yg, ag, K), 3)

    def fwd_bwd():
        xk = lw.run(x0, yg, ag, K)
        loss = ((xk.float() - xt) ** 2).sum()
        loss.backward()
    ms_fb = time_it(fwd_bwd, 3)
    # the same with the geometry's adjoint weight table (its 8-image groups read the weights)
    tab = _try_adjoint_table(g, L)
    ms_fwd_t = time_it(lambda: lw.run(x0, yg, ag, K), 3) if tab is not None else None
    ms_fb_t = time_it(fwd_bwd, 3) if tab is not None else None
    if tab is not None:
        g.free_adjoint_table()
    proj_fwd = 2 * K * w.batch * S
    proj_bwd = 3 * K * w.batch * S
    out["landweber"] = {
        "workload": w.name, "storage": "bf16", "iterations": K, "power_iterations": P,
        "lambda": float(lam.item()), "alpha": float(alpha.item()),
        "ms_power_iteration": ms_power, "ms_forward": ms_fwd, "ms_forward_backward": ms_fb,
        "samples_per_s_forward": proj_fwd / (ms_fwd * 1e-3),
        "samples_per_s_forward_backward": (proj_fwd + proj_bwd) / (ms_fb * 1e-3),
        "samples_per_s_power_iteration": 2 * P * S / (ms_power * 1e-3),
        "with_adjoint_table": (None if tab is None else
                               {"bytes": tab[0], "ms_forward": ms_fwd_t, "ms_forward_backward": ms_fb_t,
                                "samples_per_s_forward_backward": (proj_fwd + proj_bwd) / (ms_fb_t * 1e-3)}),
        "l2": "flushed (2x L2 write) before each timed iteration",
    }
    del g, xt, y32, y, yg, ag, x0
    # paper-shaped batch point
    g = Geometry("parallel", 512, uniform_angles(512, np.pi), det_count=512, det_spacing=1.0)
    S = g.sample_count
    B = 32
    from synth import ellipse_phantom
    xs = np.stack([ellipse_phantom(512, 10, 9000 + b) for b in range(B)])
    res = {"workload": "parallel_b32_n512_v512_d512", "samples_per_image": S,
           "l2": "flushed (2x L2 write) before each timed step"}
    for label, dt, cfg in (("chosen_f16", torch.float16, launch_config("auto")),
                           ("tuned_f32", torch.float32, launch_config("auto")),
                           ("plain_f32", torch.float32, launch_config("plain"))):
        x = torch.from_numpy(xs).to("cuda", dt)
        yb = forward_raw(g, x, cfg)
        oy, ox = torch.empty_like(yb), torch.empty_like(x)

        def fa():
            forward_raw(g, x, cfg, out=oy)
            backward_raw(g, yb, cfg, out=ox)
        ms = time_it(fa, 3 if label == "plain_f32" else 5, warm=1)
        res[label] = {"ms_per_step": ms, "samples_per_s": 2 * B * S / (ms * 1e-3), "images_per_s": B / (ms * 1e-3)}
        del x, yb, oy, ox
    res["speedup_chosen_vs_plain_f32"] = res["plain_f32"]["ms_per_step"] / res["chosen_f16"]["ms_per_step"]
    res["speedup_chosen_vs_tuned_f32"] = res["tuned_f32"]["ms_per_step"] / res["chosen_f16"]["ms_per_step"]
    # the same two tuned forms with the geometry's adjoint weight table (16-image groups reading it)
    tab = _try_adjoint_table(g, L)
    if tab is not None:
        res["adjoint_table_bytes"] = tab[0]
        for label, dt in (("chosen_f16_table", torch.float16), ("tuned_f32_table", torch.float32)):
            cfg = launch_config("auto")
            x = torch.from_numpy(xs).to("cuda", dt)
            yb = forward_raw(g, x, cfg)
            oy, ox = torch.empty_like(yb), torch.empty_like(x)

            def fa():
                forward_raw(g, x, cfg, out=oy)
                backward_raw(g, yb, cfg, out=ox)
            ms = time_it(fa, 5, warm=1)
            res[label] = {"ms_per_step": ms, "samples_per_s": 2 * B * S / (ms * 1e-3), "images_per_s": B / (ms * 1e-3)}
            del x, yb, oy, ox
        g.free_adjoint_table()
        res["speedup_chosen_table_vs_plain_f32"] = (res["plain_f32"]["ms_per_step"] /
                                                    res["chosen_f16_table"]["ms_per_step"])
    out["paper_batch"] = res
    del xs
    # the uneven batch: 64 images of 128^2..1024^2, each with its own geometry, in one persistent
    # launch per direction, both captured in one CUDA graph; against one library call per image
    from paper_2009_14788_gb300 import BatchPlan
    from synth import uneven_items
    w = WORKLOADS["uneven_b64_n128-1024"]
    items = uneven_items(w)
    geoms = []
    for k in range(len(items)):
        a = workload_geometry_args(w, k)
        kind = a.pop("kind")
        geoms.append(Geometry(kind, **a))
    S_tot = sum(g.sample_count for g in geoms)
    imgs = workload_images(w)
    xs16 = [torch.from_numpy(x[None]).to("cuda", torch.float16) for x in imgs]
    ys16 = [forward_raw(g, x.float()).to(torch.float16) for g, x in zip(geoms, xs16)]
    oy = [torch.empty_like(y) for y in ys16]
    ox = [torch.empty_like(x) for x in xs16]
    t0 = time.perf_counter()
    pf = BatchPlan(list(zip(geoms, xs16, oy)), "forward")
    pa = BatchPlan(list(zip(geoms, ys16, ox)), "adjoint")
    t_plan = time.perf_counter() - t0
    cs = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(cs):
        pf.launch()
        pa.launch()
        torch.cuda.synchronize()
        with torch.cuda.graph(graph, stream=cs):
            pf.launch()
            pa.launch()
    ms_graph = time_it(graph.replay, 5)
    ms_fwd = time_it(pf.launch, 5)
    ms_adj = time_it(pa.launch, 5)
    # the library defaults without the autotuner (forward: 8 views x 1 lane per ray block; adjoint:
    # chunks of 32 views where they fit), on the same buffers
    df = BatchPlan(list(zip(geoms, xs16, oy)), "forward", autotune=False)
    da = BatchPlan(list(zip(geoms, ys16, ox)), "adjoint", autotune=False)
    ms_fwd_default = time_it(df.launch, 5)
    ms_adj_default = time_it(da.launch, 5)
    df.close()
    da.close()
    # the staged forward alone (image slabs copied into shared memory by bulk copies), its own shapes
    # tuned: the alternative the autotuner weighs against the L1 gather at every image size
    sf = BatchPlan(list(zip(geoms, xs16, oy)), "forward", forward_kernel="staged")
    ms_fwd_staged = time_it(sf.launch, 5)
    cfg_staged = sorted({(items[k]["n"],) + sf.item_shape(k) + (sf.item_rows(k),) for k in range(len(items))})
    sf.close()

    def per_item():
        for g, x, y, a_, b_ in zip(geoms, xs16, ys16, oy, ox):
            forward_raw(g, x, out=a_)
            backward_raw(g, y, out=b_)
    ms_loop = time_it(per_item, 3, warm=1)
    cfg_f = sorted({(items[k]["n"],) + pf.item_shape(k) + (pf.item_rows(k),) for k in range(len(items))})
    cfg_a = sorted({(items[k]["n"], pa.item_config(k)) for k in range(len(items))})
    out["uneven"] = {
        "workload": w.name, "storage": "f16", "images": len(items), "samples_per_pass": S_tot,
        "ms_graph_fwd_adj": ms_graph, "ms_plan_fwd": ms_fwd, "ms_plan_adj": ms_adj,
        "samples_per_s": 2 * S_tot / (ms_graph * 1e-3), "images_per_s": len(items) / (ms_graph * 1e-3),
        "per_image_calls_ms": ms_loop, "speedup_vs_per_image_calls": ms_loop / ms_graph,
        "plan_create_s": t_plan,
        "autotuned_forward_n_views_lanes_rows": cfg_f,
        "forward_kernel_note": "rows 0: the L1 gather; rows > 0: the staged kernel with that many texel rows per slab",
        "staged_forward_ms_plan_fwd": ms_fwd_staged, "staged_forward_n_views_lanes_rows": cfg_staged,
        "autotuned_adjoint_n_views": cfg_a,
        "default_shapes_ms_plan_fwd": ms_fwd_default, "default_shapes_ms_plan_adj": ms_adj_default,
        "autotuned_speedup_vs_default_shapes": (ms_fwd_default + ms_adj_default) / (ms_fwd + ms_adj),
        "work_items": [pf.info["work_items"], pa.info["work_items"]],
        "ctas": [pf.info["ctas"], pa.info["ctas"]],
        "l2": "flushed (2x L2 write) before each timed launch",
    }
    pf.close()
    pa.close()
    # filtered backprojection at the paper's setting (Section 3.1.3): 512^2, 512 views in [0, pi),
    # ceil(512 sqrt 2) = 725 detectors, Ram-Lak; batch 1 (latency) and 16 (throughput), FP32
    from paper_2009_14788_gb300 import filter_sinogram
    D = int(np.ceil(512 * np.sqrt(2.0)))
    g = Geometry("parallel", 512, uniform_angles(512, np.pi), det_count=D, det_spacing=1.0)
    res = {"workload": "parallel_n512_v512_d725_ramlak", "storage": "f32",
           "l2": "flushed (2x L2 write) before each timed call"}
    for B, table in ((1, False), (16, False), (16, True)):
        if table and _try_adjoint_table(g, L) is None:
            continue
        x = torch.from_numpy(np.stack([ellipse_phantom(512, 10, 4242 + b) for b in range(B)])).to("cuda", torch.float32)
        y = forward_raw(g, x)
        q = torch.empty_like(y)
        rec = torch.empty_like(x)
        ms_f = time_it(lambda: filter_sinogram(g, y, "ram-lak", out=q), 5)

        def fbp():
            filter_sinogram(g, y, "ram-lak", out=q)
            backward_raw(g, q, out=rec)
        ms_fbp = time_it(fbp, 5)
        res["batch%d%s" % (B, "_table" if table else "")] = {"ms_filter": ms_f, "ms_fbp": ms_fbp,
                                                            "images_per_s": B / (ms_fbp * 1e-3)}
        del x, y, q, rec
    g.free_adjoint_table()
    out["fbp"] = res
    # CGNE at the same setting (Section 4.2 runs 500 iterations): 20 iterations, batch 1 and 8
    from paper_2009_14788_gb300 import cgne
    res = {"workload": "parallel_n512_v512_d725", "storage": "f32", "iterations": 20,
           "l2": "flushed (2x L2 write) before each timed call"}
    for B, table in ((1, False), (8, False), (8, True)):
        if table and _try_adjoint_table(g, L) is None:
            continue
        x = torch.from_numpy(np.stack([ellipse_phantom(512, 10, 4242 + b) for b in range(B)])).to("cuda", torch.float32)
        y = forward_raw(g, x)
        x0 = torch.zeros_like(x)
        ms = time_it(lambda: cgne(g, x0, y, 20), 3, warm=1)
        res["batch%d%s" % (B, "_table" if table else "")] = {
            "ms": ms, "ms_per_iteration": ms / 20, "samples_per_s": 2 * 20 * B * g.sample_count / (ms * 1e-3)}
        del x, y, x0
    g.free_adjoint_table()
    out["cgne"] = res
    # the pixel-driven interpolating backprojector against the exact adjoint, headline workload
    from paper_2009_14788_gb300 import backproject_interpolating
    w = WORKLOADS[DEFAULT_WORKLOAD]
    ga = workload_geometry_args(w)
    kind = ga.pop("kind")
    g = Geometry(kind, **ga)
    x = torch.from_numpy(workload_images(w)).to("cuda", torch.float16)
    y = forward_raw(g, x)
    ox = torch.empty_like(x)
    ms_i = time_it(lambda: backproject_interpolating(g, y, out=ox), 5)
    ms_a = time_it(lambda: backward_raw(g, y, out=ox), 5)
    ms_t = time_it(lambda: backward_raw(g, y, out=ox), 5) if _try_adjoint_table(g, L) is not None else None
    g.free_adjoint_table()
    out["interpolating_backprojection"] = {"workload": w.name, "storage": "f16", "ms": ms_i,
                                           "exact_adjoint_ms": ms_a, "speedup_vs_exact_adjoint": ms_a / ms_i,
                                           "exact_adjoint_with_table_ms": ms_t}
    del x, y, ox
    del flush
    torch.cuda.empty_cache()
    return out


def run_profile(args):
    """Only the chosen form's kernels: warmup + steps launches of forward and adjoint, no timing."""
    import torch

    from paper_2009_14788_gb300 import Geometry, _lib as L, backward_raw, forward_raw, launch_config
    from paper_2009_14788_gb300.build import build

    build()
    w = WORKLOADS[args.workload]
    dt = {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}[args.storage]
    if w.kind == "uneven":
        # the uneven batch: one forward plan and one adjoint plan (default tile shapes, no autotuning)
        from paper_2009_14788_gb300 import BatchPlan
        from synth import uneven_items
        geoms = []
        for k in range(len(uneven_items(w))):
            a = workload_geometry_args(w, k)
            kd = a.pop("kind")
            geoms.append(Geometry(kd, **a))
        xs = [torch.from_numpy(x[None]).to("cuda", dt) for x in workload_images(w)]
        ys = [torch.zeros((1,) + g.sino_shape, dtype=dt, device="cuda") for g in geoms]
        ox = [torch.empty_like(x) for x in xs]
        pf = BatchPlan(list(zip(geoms, xs, ys)), "forward", autotune=False)
        pa = BatchPlan(list(zip(geoms, ys, ox)), "adjoint", autotune=False)
        for _ in range(1 + args.warmup + args.steps):
            pf.launch()
            pa.launch()
        torch.cuda.synchronize()
        print("profile run: %s %s, %d launches of each plan" % (args.workload, args.storage,
                                                                1 + args.warmup + args.steps))
        return
    gargs = workload_geometry_args(w)
    kind = gargs.pop("kind")
    geom = Geometry(kind, **gargs)
    if not args.no_adjoint_table:
        _try_adjoint_table(geom, L)
    cfg = launch_config(args.algo)
    x = torch.from_numpy(workload_images(w)).to(device="cuda", dtype=dt)
    y = forward_raw(geom, x, cfg)
    for _ in range(args.warmup + args.steps):
        forward_raw(geom, x, cfg, out=y)
        backward_raw(geom, y, cfg, out=x)
    torch.cuda.synchronize()
    print("profile run: %s %s %s, %d launches of each operator" % (args.workload, args.storage, args.algo,
                                                                  1 + args.warmup + args.steps))


# ----------------------------------------------------------------------------- CPU oracle

def _oracle_sample_geometry(w, stride):
    import oracle as O
    gargs = workload_geometry_args(w)
    gargs["angles"] = gargs["angles"][::stride]
    return O.Geometry.from_args(gargs)


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the platform string)."""
    import platform
    import subprocess
    try:
        r = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10)
        for line in r.stdout.splitlines():
            if line.split(":")[0].strip() == "Model name":
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


def cpu_oracle_sample(w, seconds):
    """The FP64 oracle as it stands on the host cores: fwd + adjoint of the whole image batch on every
    ``stride``-th view, with the stride picked so the run takes roughly ``seconds``."""
    import oracle as O
    x = workload_images(w)
    stride = 64
    result = None
    while True:
        g = _oracle_sample_geometry(w, stride)
        S = O.sample_count(g)
        y = O.forward(g, x)            # warm (builds / loads the library)
        t0 = time.perf_counter()
        y = O.forward(g, x)
        O.adjoint(g, y)
        dt = time.perf_counter() - t0
        result = {"value": 2 * x.shape[0] * S / dt, "unit": "samples/s", "cores": O.num_threads(), "cpu": cpu_model(),
                  "kind": "oracle",
                  "sample": "fwd + adjoint of all %d images on every %d-th view (%d of %d views), %.1f s" % (
                      x.shape[0], stride, g.n_angles, w.n_views, dt),
                  "seconds": dt}
        if dt * 3 > seconds or stride == 1:
            break
        stride = max(1, stride // 4)
    one = cpu_oracle_one_core(w.name)
    if one is not None:
        result["one_core"] = one
    return result


ONE_CORE_STRIDE = 64


def cpu_oracle_one_core(workload: str):
    """The same oracle on one host core (OpenMP limited to one thread in a child interpreter), on every
    64th view of the workload: samples/s, or None if the child fails."""
    import subprocess
    code = (
        "import json, sys, time\n"
        "sys.path.insert(0, %r)\n"
        "import oracle as O\n"
        "from bench import _oracle_sample_geometry\n"
        "from synth import WORKLOADS, workload_images\n"
        "w = WORKLOADS[%r]\n"
        "x = workload_images(w)\n"
        "g = _oracle_sample_geometry(w, %d)\n"
        "O.forward(g, x[:1])\n"
        "t0 = time.perf_counter(); y = O.forward(g, x); O.adjoint(g, y); dt = time.perf_counter() - t0\n"
        "print(json.dumps({'samples': 2 * x.shape[0] * O.sample_count(g), 'seconds': dt, 'views': g.n_angles,\n"
        "                  'threads': O.num_threads(), 'images': int(x.shape[0])}))\n"
    ) % (os.path.dirname(os.path.abspath(__file__)), workload, ONE_CORE_STRIDE)
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=600)
        d = json.loads(r.stdout.strip().splitlines()[-1])
    except (OSError, subprocess.SubprocessError, ValueError, IndexError):
        return None
    return {"value": d["samples"] / d["seconds"], "unit": "samples/s", "cores": d["threads"],
            "sample": "fwd + adjoint of all %d images on every %d-th view (%d views), %.1f s" % (
                d["images"], ONE_CORE_STRIDE, d["views"], d["seconds"])}


def run_reference(args):
    world, rank, local = _dist()
    if rank != 0:
        return
    import oracle as O
    w = WORKLOADS[args.workload]
    x = workload_images(w)
    stride = args.reference_stride
    g = _oracle_sample_geometry(w, stride)
    S = O.sample_count(g)
    y = O.forward(g, x)
    for _ in range(args.warmup):
        O.forward(g, x)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        yy = O.forward(g, x)
        O.adjoint(g, yy)
        times.append(time.perf_counter() - t0)
    _ = y
    ms = 1e3 * statistics.mean(times)
    value = 2 * x.shape[0] * S / (ms * 1e-3)
    line = {"metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": dict(oracle_workload_config(args.workload, args.storage, args.algo),
                           sample="every %d-th view" % stride),
            "cpu_baseline": {"value": value, "unit": "samples/s", "cores": O.num_threads(), "cpu": cpu_model(),
                             "kind": "oracle",
                             "sample": "fwd + adjoint of all %d images on every %d-th view (%d of %d views) per step"
                                       % (x.shape[0], stride, g.n_angles, w.n_views)},
            "e2e": {"value": value, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS),
                    help="timed runs take the parallel / fan workloads; --profile takes any")
    ap.add_argument("--storage", choices=["f32", "f16", "bf16"], default="f16")
    ap.add_argument("--algo", choices=["auto", "plain", "tiled"], default="auto")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the Landweber and paper-shaped secondary measurements")
    ap.add_argument("--reference-stride", type=int, default=16)
    ap.add_argument("--no-adjoint-table", action="store_true",
                    help="leave the geometry without its adjoint weight table (weights computed on the fly)")
    ap.add_argument("--profile", action="store_true",
                    help="run --warmup + --steps fwd/adjoint launches of the chosen form only (for ncu)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.profile:
        run_profile(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
