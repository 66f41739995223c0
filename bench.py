"""Benchmark of the SG-Splatting rasterizer on one node.

Headline (printed as ONE JSON line by rank 0): forward+backward views/s of the batched
path -- 3 M clustered Gaussians (SH degree 1 + 4 SG lobes), 16 cameras of mixed
resolution {640x360, 1280x720, 1600x900, 1920x1080} rendered, L1-compared with seeded
U(0,1) targets and differentiated in one batched pass per step.  Beside it: the same
views as 16 sequential plain (one view per launch) passes, render FPS of the 1 M-Gaussian
1280x720 scene with SH-1 + 3 SG lobes and with SH degree 3 (48 coefficients), per-kernel
times from CUDA events inside the timed region, the roofline of the dominant kernel, an
end-to-end number through host buffers, and the CPU oracle timed on a bounded sample.

Usage: python bench.py [--gpus N --steps K --warmup W] [--impl reference]
Under torchrun each rank renders its own batch against a replica of the Gaussians (weak
scaling) and every step ends with one all-reduce of the gradient planes (view-sharded
training's exchange); times are the max over ranks.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2501_00342_b300 import inputs as I  # noqa: E402

METRIC = "fwd+bwd views/sec (batched launch, 16 mixed-resolution views)"
UNIT = "views/s"
WORKLOAD = ("3M clustered Gaussians, SH-1 + 4 SG lobes (free axes), 16 orbit views at mixed "
            "{640x360,1280x720,1600x900,1920x1080}, L1 vs U(0,1) targets, forward + backward")


# DRAM bytes per unit of work of the profiled kernels (profiles/dram_traffic.json), valid
# while the kernel's source file keeps the hash recorded there
def _traffic_rates():
    import hashlib
    rates = {}
    try:
        with open(os.path.join(ROOT, "profiles", "dram_traffic.json")) as f:
            table = json.load(f)["kernels"]
    except (OSError, ValueError, KeyError):
        return rates
    for kernel, e in table.items():
        path = os.path.join(ROOT, "paper_2501_00342_b300", "csrc", e["source"])
        try:
            now = hashlib.sha1(open(path, "rb").read()).hexdigest()[:12]
        except OSError:
            continue
        if now == e["sha1"]:
            rates[kernel] = (e["unit"], float(e["bytes_per_unit"]))
    return rates


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), float(p.get("sm_max_mhz", 2032.0)), "measured"
    except Exception:
        return 6400.0, 2032.0, "fallback"


# ------------------------------------------------------------------------------ clocks
class ClockSampler:
    """Samples SM clock and throttle reasons with nvidia-smi while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index, self.rows, self.proc = index, [], None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[k] for r in self.rows for k in range(4)
                          if len(r) > 3 + k and r[3 + k].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "samples": len(self.rows), "reasons": reasons}


def measure_alu_peak(index: int, reps: int = 10, iters: int = 1 << 19):
    """FP32 throughput of this GPU, measured: the library's probe kernel (8 independent
    multiply-add chains per thread over a multiple of the SM count) timed with CUDA events,
    as scalar fma.rn.f32 and as packed fma.rn.f32x2, with the SM clock sampled meanwhile.
    Returns Tops/s (a multiply-add counted as one operation, like the kernels' counts)."""
    import torch
    from paper_2501_00342_b300 import binding as B
    stream = torch.cuda.current_stream()
    out = torch.empty(B.alu_probe_size(), dtype=torch.float32, device="cuda")
    res = {}
    for label, packed in (("ffma", False), ("ffma2", True)):
        B.alu_probe(packed, 1024, out.data_ptr(), stream.cuda_stream)  # warm-up
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(index) as clk:
            a.record(stream)
            ops = 0.0
            for _ in range(reps):
                ops += B.alu_probe(packed, iters, out.data_ptr(), stream.cuda_stream)
            b.record(stream)
            torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        res[label] = {"tops": round(ops / (ms / 1e3) / 1e12, 3), "ms": round(ms, 2), "clocks": clk.summary()}
    return res


def copy_bandwidth(nbytes: int = 1 << 30, reps: int = 5):
    """Pinned host <-> device copy rates (GB/s): host-to-device alone, device-to-host alone,
    and both at once on two streams, as the end-to-end leg overlaps them (CUDA events, best
    of `reps`)."""
    import torch
    h_src, h_dst = (torch.empty(nbytes, dtype=torch.uint8).pin_memory() for _ in range(2))
    d_dst, d_src = (torch.empty(nbytes, dtype=torch.uint8, device="cuda") for _ in range(2))
    up, down = torch.cuda.Stream(), torch.cuda.Stream()
    main = torch.cuda.current_stream()
    out = {}
    for name, h2d, d2h in (("h2d", True, False), ("d2h", False, True), ("both", True, True)):
        best = None
        for _ in range(reps):
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(main)
            for st, on, dst, src in ((up, h2d, d_dst, h_src), (down, d2h, h_dst, d_src)):
                if on:
                    st.wait_event(a)
                    with torch.cuda.stream(st):
                        dst.copy_(src, non_blocking=True)
                    main.wait_stream(st)
            b.record(main)
            torch.cuda.synchronize()
            ms = a.elapsed_time(b)
            best = ms if best is None else min(best, ms)
        out[name] = round((int(h2d) + int(d2h)) * nbytes / (best / 1e3) / 1e9, 1)
    del h_src, h_dst, d_dst, d_src
    return out


# ------------------------------------------------------------------------------ GPU arm
def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_max(x: float, world: int, device) -> float:
    """Max of a per-rank number over all ranks (the host-side timing collective)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, views_per_rank: int, ms_max: float) -> float:
    """Whole-job views/s: every rank renders its own batch; the slowest rank sets the time."""
    return world * views_per_rank / (ms_max / 1e3)


def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_2501_00342_b300 import binding as B
    from paper_2501_00342_b300.render import GaussianModel, Rasterizer, RenderSettings, l1_loss
    from paper_2501_00342_b300.train import GradientBucket

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    def max_over_ranks(x: float) -> float:
        return reduce_max(x, world, "cuda")

    stream = torch.cuda.current_stream()
    settings = RenderSettings(tile_w=args.tile[0], tile_h=args.tile[1], batch_depth=args.batch_depth,
                              digit_bits=args.digit_bits, fwd_pixels=args.fwd_pixels, bwd_pixels=args.bwd_pixels)
    from paper_2501_00342_b300.autotune import autotune
    if args.workload == "single":  # small profiling case: 1 M Gaussians, one 1280x720 view
        scene, cams = I.workload(1, sh_degree=1, num_lobes=4)
        cams = cams[:1]
    elif args.workload == "medium":  # profiling case: the 3 M scene, two 1920x1080 views
        scene, cams = I.workload(3)
        cams = [c for c in cams if c.width == 1920][:2]
    else:
        scene, cams = I.workload(3)
    n, nv = scene.n, len(cams)
    model = GaussianModel.from_scene(scene)
    targets = I.target_images(cams, config=3)
    target = torch.from_numpy(np.concatenate([t.reshape(-1) for t in targets])).cuda()
    tune_log = []
    if args.autotune:
        settings = autotune(model, cams, base=settings, steps=2, log=tune_log)
    rast = Rasterizer(model, cams, settings)
    img = torch.empty(3 * rast.num_pixels, device="cuda")
    rast.forward(model, out_rgb=img, sync=True)  # sizes the instance capacity
    M = rast.num_instances
    rast = Rasterizer(model, cams, settings, capacity=int(M * 1.02) + 4096)
    # Under torchrun every rank renders its own batch of views against a replica of the
    # Gaussians (the same 16 cameras on every rank in this synthetic workload) and the step
    # ends with the one exchange of view-sharded training: an all-reduce (sum) of all the
    # gradient planes, held in one flat buffer.  The L1 of each rank is normalised by the
    # pixel values of all ranks, so the summed gradient is that of the job's mean L1.
    norm = world * img.numel() if world > 1 else None

    def make_grads():
        if world == 1:
            return model.empty_grads(), None
        bucket = GradientBucket(model)
        return bucket.planes, bucket

    grads, bucket = make_grads()

    def exchange(bk):
        if bk is not None:
            bk.allreduce()

    def step(sync=False):
        rast.forward(model, out_rgb=img, sync=sync)
        loss, dimg = l1_loss(img, target, norm=norm)
        rast.backward(model, dimg, grads=grads)
        return loss

    step(sync=True)
    assert rast.num_instances == M and rast.device_status() == 0
    names = B.EVENTS

    def probe_events():
        evs = [torch.cuda.Event(enable_timing=True) for _ in names]
        for e in evs:  # creates the driver events before they are handed to the library
            e.record(stream)
        return evs, C_void_p_array(len(names))(*[e.cuda_event for e in evs])

    # eager run of the same step (also the fallback source of the per-kernel times)
    eager_evs, handles = probe_events()
    B.set_events(rast.plan, handles)
    for _ in range(args.warmup):
        step()
        exchange(bucket)
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        step()
        exchange(bucket)
    t1.record(stream)
    torch.cuda.synchronize()
    eager_ms = t0.elapsed_time(t1) / args.steps

    # the headline: one batched step captured as a CUDA graph (probe events become graph
    # nodes), replayed K times
    graph_evs, handles = probe_events()
    B.set_events(rast.plan, handles)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph(keep_graph=True)
    with torch.cuda.graph(graph):
        graph_loss = step()
    B.set_events(rast.plan, None)
    kernel_nodes = _graph_kernel_nodes(graph.raw_cuda_graph())
    graph.instantiate()
    for _ in range(args.warmup):
        graph.replay()
        exchange(bucket)
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t0.record(stream)
        for _ in range(args.steps):
            graph.replay()
            exchange(bucket)
        t1.record(stream)
        torch.cuda.synchronize()
    barrier()
    ms = max_over_ranks(t0.elapsed_time(t1) / args.steps)
    value = job_rate(world, nv, ms)
    try:  # the probe events of the last replay of the timed loop
        graph_evs[0].elapsed_time(graph_evs[1])
        ev_sets, stage_source = [graph_evs], "CUDA events inside the graph, last timed replay"
    except RuntimeError:
        ev_sets, stage_source = [eager_evs], "CUDA events of the last eager step"

    def span(a, b):
        ia, ib = names.index(a), names.index(b)
        return float(np.mean([ev[ia].elapsed_time(ev[ib]) for ev in ev_sets]))

    P = rast.plan.sort_passes
    stages = {
        "preprocess": span("PRE_BEGIN", "PRE_END"),
        "scan": span("BIN_BEGIN", "SCAN_END"),
        "duplicate": span("SCAN_END", "DUP_END"),
        "sort_histogram": span("DUP_END", "HIST_END"),
        "sort_onesweep_all_passes": span("HIST_END", "SORT_END"),
        "ranges": span("SORT_END", "RANGES_END"),
        "blend": span("BLEND_BEGIN", "BLEND_END"),
        "loss": span("BLEND_END", "BWD_BEGIN"),
        "backward_tile_order": span("BWD_BEGIN", "BWD_ZERO_END"),
        "backward_blend": span("BWD_ZERO_END", "BWD_BLEND_END"),
        "backward_preprocess": span("BWD_BLEND_END", "BWD_PRE_END"),
    }

    # algorithmic work of each kernel
    tiles = rast.region("TILES", torch.int32)[:n * nv]
    visible = int((tiles != 0).sum().item())
    # one more forward with the per-pixel pair counters on (the timed kernels skip them)
    rast.plan.settings.count_pairs = 1
    rast.forward(model, out_rgb=img, sync=False)
    rast.plan.settings.count_pairs = 0
    torch.cuda.synchronize()
    counts = rast.region("PIX_COUNT", torch.int32)[:2 * rast.num_pixels].view(-1, 2).to(torch.int64)
    e_eval, e_contrib = int(counts[:, 0].sum().item()), int(counts[:, 1].sum().item())
    p_bytes = 4 * scene.floats_per_gaussian()
    hbm, sm_max, peak_kind = _peaks()
    # FP32 peak measured on this GPU (scalar and packed multiply-adds); when the probe ran at
    # a lower SM clock than the timed step, it is scaled up to the step's clock, so that the
    # blend kernels' fractions are not inflated by a slower probe
    alu = measure_alu_peak(local)
    step_mhz = clk.summary().get("sm_mhz") or sm_max
    best = max(("ffma", "ffma2"), key=lambda k: alu[k]["tops"])
    probe_mhz = alu[best]["clocks"].get("sm_mhz") or step_mhz
    alu_peak = alu[best]["tops"] * max(1.0, step_mhz / probe_mhz)
    alu["peak_tops"] = round(alu_peak, 3)
    alu["peak_from"] = f"{best} at {probe_mhz:.0f} MHz, scaled to the timed step's {step_mhz:.0f} MHz" \
        if step_mhz > probe_mhz else f"{best} at {probe_mhz:.0f} MHz"
    alu["sm_count"] = torch.cuda.get_device_properties(local).multi_processor_count
    fwd_name = "blend_pair_kernel" if settings.fwd_pixels in (0, 2) else "blend_kernel"
    bwd_name = "blend_pair_backward_kernel" if settings.bwd_pixels in (0, 2) else "blend_backward_kernel"
    # algorithmic bytes of each HBM-bound kernel: everything this design's kernel must read
    # and write ("work"), and, for the preprocess kernels, a narrower count too: the
    # parameters plus a minimal 44-byte record per (view, Gaussian) and, backward, 36 bytes
    # of 2D gradients per visible record ("narrow_work")
    R = n * nv
    kernels = {
        # parameters once; per visible record its 48-byte record and the row table's first
        # 32-byte sector; per record its rectangle, tile count, flags and record-sort pair
        "preprocess_kernel": dict(ms=stages["preprocess"], launches=1, bound="hbm",
                                  work=n * p_bytes + visible * (48 + 32) + R * (8 + 4 + 4 + 8),
                                  narrow_work=n * p_bytes + R * 44),
        # the instances written (u32 tile id + u32 record id); per visible record its row
        # table sector, sorted position and scan offset read
        "duplicate_kernel": dict(ms=stages["duplicate"], launches=1, bound="hbm", work=8 * M + visible * (32 + 8)),
        "onesweep_kernel": dict(ms=stages["sort_onesweep_all_passes"] / max(P, 1), launches=P, bound="hbm",
                                work=16 * M),  # u32 tile id + u32 record id, read and written
        # two pixels per thread run the packed-pair kernels
        fwd_name: dict(ms=stages["blend"], launches=1, bound="alu", work=8 * e_eval + 11 * e_contrib),
        bwd_name: dict(ms=stages["backward_blend"], launches=1, bound="alu", work=8 * e_eval + 40 * e_contrib),
        # parameters read and their gradients written; per record its flags; per visible
        # record its 36-byte 2D gradient read and cleared
        "preprocess_backward_kernel": dict(ms=stages["backward_preprocess"], launches=1, bound="hbm",
                                           work=2 * n * p_bytes + R * 4 + visible * 72,
                                           narrow_work=2 * n * p_bytes + visible * 36),
    }
    dom_name = max(kernels, key=lambda k: kernels[k]["ms"] * kernels[k]["launches"])
    units = {"pixel": rast.num_pixels, "instance": M, "record": R}
    rates = _traffic_rates()

    def traffic(name):
        if name not in rates or rates[name][0] not in units:
            return None
        return int(rates[name][1] * units[rates[name][0]])

    roofs = {}
    for name, k in kernels.items():
        if k["work"] is None:
            continue
        if k["bound"] == "hbm":
            achieved = k["work"] / (k["ms"] / 1e3) / 1e9
            roofs[name] = {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                           "frac": round(achieved / hbm, 4), "traffic": traffic(name),
                           "algorithmic_bytes_per_launch": int(k["work"]), "ms_per_launch": round(k["ms"], 4)}
            if "narrow_work" in k:
                roofs[name]["narrow_bytes_per_launch"] = int(k["narrow_work"])
                roofs[name]["frac_narrow_count"] = round(k["narrow_work"] / (k["ms"] / 1e3) / 1e9 / hbm, 4)
        else:
            achieved = k["work"] / (k["ms"] / 1e3) / 1e12
            roofs[name] = {"bound": "alu", "achieved": round(achieved, 3), "peak": round(alu_peak, 2),
                           "unit": "Tops/s (FP32 ops)", "frac": round(achieved / alu_peak, 4), "traffic": traffic(name),
                           "algorithmic_ops_per_launch": int(k["work"]), "ms_per_launch": round(k["ms"], 4)}
    dominant = dict(roofs.get(dom_name, {}))
    dominant["kernel"] = dom_name
    dominant["peak_source"] = (f"hbm: {peak_kind} (MEASURED_PEAKS.json hbm_gbs); alu: measured FP32 multiply-add "
                               f"throughput of this GPU ({alu['peak_from']})")
    dominant["traffic_source"] = ("ncu DRAM bytes per unit on a smaller case, scaled by this workload's units "
                                  "(profiles/dram_traffic.json)")

    out = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded; stands in for Mip-NeRF360/T&T/DB)",
        "config": {"workload": {"batched": WORKLOAD,
                                "single": "profiling case: 1M clustered Gaussians, SH-1 + 4 SG, one 1280x720 view",
                                "medium": "profiling case: 3M clustered Gaussians, SH-1 + 4 SG, two 1920x1080 views",
                                }[args.workload],
                   "gaussians": n, "views": nv,
                   "resolutions": [[c.width, c.height] for c in cams], "pixels": int(rast.num_pixels),
                   "instances": M, "sort_passes": P, "key_bits": int(rast.plan.key_bits),
                   "tile": [settings.tile_w, settings.tile_h], "batch_depth": settings.batch_depth,
                   "digit_bits": settings.digit_bits, "fwd_pixels": settings.fwd_pixels,
                   "bwd_pixels": settings.bwd_pixels,
                   "l2": f"inputs larger than L2: {n * p_bytes / 1e6:.0f} MB parameters, "
                         f"{rast.nbytes / 1e9:.2f} GB workspace",
                   "parallelism": (f"view-sharded x{world}: each rank renders its own 16-view batch, one "
                                   f"all-reduce of the gradient planes per step") if world > 1
                                  else "one GPU, one 16-view batch per step"},
        "stages_ms": {k: round(v, 4) for k, v in stages.items()},
        "blend_evaluations": e_eval, "blend_contributions": e_contrib, "visible_records": visible,
        "roofline": dominant, "roofline_all": roofs,
        "gpu_launches": None if kernel_nodes is None else kernel_nodes * args.steps,
        "kernels_per_step": kernel_nodes, "cuda_graph": True, "eager_ms_per_step": round(eager_ms, 4),
        "stage_timing": stage_source,
        "autotune": {"chosen": {k: v for k, v in dataclasses.asdict(settings).items() if k != "bg"},
                     "trials": [dict({k: v for k, v in t["settings"].items() if k != "bg"}, ms=round(t["ms"], 3))
                                for t in tune_log]},
        "clocks": clk.summary(),
        "alu_peak": alu,
    }

    # ---- the same views as 16 plain launches (one view each)
    if args.extras:
        plain = []
        for c in cams:
            r1 = Rasterizer(model, [c], settings)
            r1.forward(model, sync=True)
            r1 = Rasterizer(model, [c], settings, capacity=int(r1.num_instances * 1.02) + 4096)
            i1 = torch.empty(3 * r1.num_pixels, device="cuda")
            plain.append([r1, i1, None, model.empty_grads()])
        offs = rast.pixel_base
        for v, pl in enumerate(plain):  # view v's slice of the packed targets
            pl[2] = target[3 * offs[v]:3 * offs[v + 1]]

        def plain_step():
            for r1, i1, tv, g1 in plain:
                r1.forward(model, out_rgb=i1, sync=False)
                _, d1 = l1_loss(i1, tv)
                r1.backward(model, d1, grads=g1)

        for _ in range(max(1, args.warmup)):
            plain_step()
        torch.cuda.synchronize()
        barrier()
        a, b2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(args.steps):
            plain_step()
        b2.record(stream)
        torch.cuda.synchronize()
        pms_eager = max_over_ranks(a.elapsed_time(b2) / args.steps)
        # like for like with the headline: the 16 one-view steps captured as one CUDA graph
        plain_graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(plain_graph):
            plain_step()
        for _ in range(max(1, args.warmup)):
            plain_graph.replay()
        torch.cuda.synchronize()
        barrier()
        a.record(stream)
        for _ in range(args.steps):
            plain_graph.replay()
        b2.record(stream)
        torch.cuda.synchronize()
        pms = max_over_ranks(a.elapsed_time(b2) / args.steps)
        out["plain"] = {"ms_per_16_views": round(pms, 4), "views_per_s": round(job_rate(world, nv, pms), 3),
                        "batched_over_plain": round(pms / ms, 4), "timing": "CUDA graph replays, as the headline",
                        "eager_ms_per_16_views": round(pms_eager, 4)}
        del plain, plain_graph

        # ---- render FPS, 1 M Gaussians at 1280x720: SG colour vs SH degree 3
        fps = {}
        for label, L, K, adaptive, mode in (("sh1_sg3", 1, 3, None, I.AXIS_FREE), ("sh3", 3, 0, None, I.AXIS_FREE),
                                            ("adaptive_sh012_sg3", 2, 3, (0.5, 0.9), I.AXIS_FREE),
                                            ("dc_sg3_frame", 0, 3, None, I.AXIS_ORTHO_FRAME)):
            sc1, cams1 = I.workload(1, sh_degree=L, num_lobes=K, axis_mode=mode)
            if adaptive:
                # degree 0 for the smaller half of the records, 1 up to the 90th percentile
                # of the pixel radius, 2 above (the paper: most Gaussians are small)
                probe = Rasterizer(GaussianModel.from_scene(sc1), cams1[:1], settings)
                probe.forward(GaussianModel.from_scene(sc1), sync=True)
                rad = probe.region("REC1", torch.float32)[:4 * sc1.n].view(-1, 4)[:, 3]
                rad = rad[probe.region("TILES", torch.int32)[:sc1.n] != 0]
                adaptive = tuple(float(torch.quantile(rad, q).ceil()) for q in adaptive)
                sc1.sh_adaptive, sc1.sh_radius = 1, adaptive
                del probe
            m1 = GaussianModel.from_scene(sc1)
            rs = []
            for c in cams1:
                r1 = Rasterizer(m1, [c], settings)
                r1.forward(m1, sync=True)
                r1 = Rasterizer(m1, [c], settings, capacity=int(r1.num_instances * 1.02) + 4096)
                rs.append((r1, torch.empty(3 * r1.num_pixels, device="cuda")))
            for r1, o1 in rs:
                r1.forward(m1, out_rgb=o1, sync=False)
            torch.cuda.synchronize()
            a.record(stream)
            reps = max(2, args.steps)
            for _ in range(reps):
                for r1, o1 in rs:
                    r1.forward(m1, out_rgb=o1, sync=False)
            b2.record(stream)
            torch.cuda.synchronize()
            fms = max_over_ranks(a.elapsed_time(b2) / (reps * len(rs)))
            # the same 32 views in one batched forward launch
            rb_ = Rasterizer(m1, cams1, settings)
            ob = torch.empty(3 * rb_.num_pixels, device="cuda")
            rb_.forward(m1, out_rgb=ob, sync=True)
            rb_ = Rasterizer(m1, cams1, settings, capacity=int(rb_.num_instances * 1.02) + 4096)
            ob = torch.empty(3 * rb_.num_pixels, device="cuda")
            for _ in range(2):
                rb_.forward(m1, out_rgb=ob, sync=False)
            torch.cuda.synchronize()
            a.record(stream)
            for _ in range(reps):
                rb_.forward(m1, out_rgb=ob, sync=False)
            b2.record(stream)
            torch.cuda.synchronize()
            bms = max_over_ranks(a.elapsed_time(b2) / reps)
            fps[label] = {"ms_per_frame": round(fms, 4), "fps": round(1e3 / fms, 1),
                          "batched_32_views_ms": round(bms, 4), "batched_fps": round(len(cams1) * 1e3 / bms, 1),
                          "floats_per_gaussian": sc1.floats_per_gaussian(),
                          "model_mb": round(sc1.n * 4 * sc1.floats_per_gaussian() / 1e6, 1)}
            del rb_, ob
            if adaptive:  # share of the visible records that summed bands up to 0, 1, 2
                rad = torch.cat([r1.region("REC1", torch.float32)[:4 * sc1.n].view(-1, 4)[:, 3][
                    r1.region("TILES", torch.int32)[:sc1.n] != 0] for r1, _ in rs])
                deg = torch.where(rad < adaptive[0], 0, torch.where(rad < adaptive[1], 1, 2))
                fps[label]["thresholds_px"] = list(adaptive)
                fps[label]["records_per_degree"] = [round(float((deg == d).float().mean()), 4) for d in range(3)]
            del rs, m1
        fps["sg_over_sh3_speedup"] = round(fps["sh3"]["ms_per_frame"] / fps["sh1_sg3"]["ms_per_frame"], 4)
        fps["adaptive_over_sh3_speedup"] = round(fps["sh3"]["ms_per_frame"] / fps["adaptive_sh012_sg3"]["ms_per_frame"], 4)
        fps["frame_over_sh3_speedup"] = round(fps["sh3"]["ms_per_frame"] / fps["dc_sg3_frame"]["ms_per_frame"], 4)
        fps["workload"] = ("1M clustered Gaussians, 32 orbit views at 1280x720, forward only: one view per launch "
                           "(fps) and all 32 in one batched launch (batched_fps)")
        out["render_fps"] = fps

        # ---- training iterations (render, L1, backward, fused Adam) on 2.5M Gaussians, one
        # 1264x832 view, U(0,1) target; the lobes train from iteration 0 here (past sg_start)
        from paper_2501_00342_b300.train import TrainConfig, Trainer
        sc2, cams2 = I.workload(2)
        m2 = GaussianModel.from_scene(sc2)
        t2 = torch.from_numpy(I.target_images(cams2, config=2)[0].reshape(-1)).cuda()
        trainer = Trainer(m2, cams2, t2, settings, TrainConfig(sg_start=0, extent=4.0))
        trainer.step(sync=True)
        for _ in range(args.warmup):
            trainer.step()
        iters = max(5, args.steps)
        ad0, ad1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for k in range(iters):
            trainer.rast.forward(m2, out_rgb=trainer.img, sync=False)
            _, d2 = l1_loss(trainer.img, t2)
            trainer.rast.backward(m2, d2, grads=trainer.grads)
            if k == iters - 1:
                ad0.record(stream)
            B.adam_step(m2.struct(), *trainer._structs, trainer.adam_config(trainer.iteration), stream.cuda_stream)
            if k == iters - 1:
                ad1.record(stream)
            trainer.iteration += 1
        b2.record(stream)
        torch.cuda.synchronize()
        tms = a.elapsed_time(b2) / iters
        adam_ms = ad0.elapsed_time(ad1)
        entries = sc2.n * sc2.floats_per_gaussian()
        adam_bytes = entries * 28 + sc2.n * 4 * 4  # raw, grad, m, v in; raw, m, v out; act of scale and opacity
        out["train_2.5M_1264x832"] = {
            "workload": "2.5M clustered Gaussians, SH-1 + 4 SG, one 1264x832 view, L1 vs U(0,1) target",
            "ms_per_iteration": round(tms, 4), "iterations_per_s": round(1e3 / tms, 1),
            "adam_ms": round(adam_ms, 4), "adam_entries": int(entries),
            "adam_roofline": {"bound": "hbm", "achieved": round(adam_bytes / (adam_ms / 1e3) / 1e9, 1), "peak": hbm,
                              "unit": "GB/s", "frac": round(adam_bytes / (adam_ms / 1e3) / 1e9 / hbm, 4),
                              "algorithmic_bytes": int(adam_bytes)}}
        del trainer, m2, t2, sc2

        # ---- 8M Gaussians, 8 views at 3840x2160: one batched fwd+bwd step, peak device memory
        sc4, cams4 = I.workload(4)
        m4 = GaussianModel.from_scene(sc4)
        r4 = Rasterizer(m4, cams4, settings)
        i4 = torch.empty(3 * r4.num_pixels, device="cuda")
        r4.forward(m4, out_rgb=i4, sync=True)  # sizes the instance capacity
        M4 = r4.num_instances
        del r4
        torch.cuda.synchronize()
        base = torch.cuda.memory_allocated()  # parameters and image of this workload included below
        base -= sum(t.numel() * 4 for t in m4.planes.values() if t is not None) + i4.numel() * 4
        torch.cuda.reset_peak_memory_stats()
        r4 = Rasterizer(m4, cams4, settings, capacity=int(M4 * 1.02) + 4096)
        t4 = torch.from_numpy(np.concatenate([t.reshape(-1) for t in I.target_images(cams4, config=4)])).cuda()
        g4 = m4.empty_grads()

        def step4():
            r4.forward(m4, out_rgb=i4, sync=False)
            _, d4 = l1_loss(i4, t4)
            r4.backward(m4, d4, grads=g4)

        step4()
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(max(2, args.steps // 2)):
            step4()
        b2.record(stream)
        torch.cuda.synchronize()
        ms4 = a.elapsed_time(b2) / max(2, args.steps // 2)
        out["workload_8M_4k"] = {
            "workload": "8M clustered Gaussians, SH-1 + 4 SG, 8 orbit views at 3840x2160, fwd+bwd batched",
            "ms_per_step": round(ms4, 3), "views_per_s": round(8 / (ms4 / 1e3), 2), "instances": int(M4),
            "status": r4.device_status(),
            "peak_device_bytes": int(torch.cuda.max_memory_allocated() - base),
            "workspace_bytes": int(r4.nbytes), "parameter_bytes": int(sum(
                t.numel() * 4 for t in m4.planes.values() if t is not None))}
        del r4, m4, i4, t4, g4, sc4
        torch.cuda.empty_cache()

    # ---- end to end: host (pinned) parameters and targets in, loss and every parameter
    # gradient plane out, every step.  The inputs are double-buffered: while step k runs on
    # the compute stream, the copies of step k + 1's inputs run on a copy stream into the
    # other buffer.  Each buffer's step is captured as two graphs, the forward and then the
    # loss with the backward, so that a step's forward waits only for its parameters and its
    # targets arrive during the forward.  Each buffer has its own gradient planes, read back
    # into pinned host memory on a second copy stream (the other direction of the link)
    # while the next step runs; a buffer's planes are rewritten only after that read-back.
    # Every step's copies are in the timed region, and the timed region ends after the last
    # step's gradients have reached the host.
    host_planes = {p: (None if t is None else t.cpu().pin_memory()) for p, t in model.planes.items()}
    host_target = target.cpu().pin_memory()
    h2d = sum(t.numel() * 4 for t in host_planes.values() if t is not None) + host_target.numel() * 4
    loss_host = [torch.empty(1).pin_memory(), torch.empty(1).pin_memory()]
    model_b = model.with_planes(**{p: t.clone() for p, t in model.planes.items() if t is not None})
    target_b = target.clone()
    second = make_grads()
    grad_sets, buckets = [grads, second[0]], [bucket, second[1]]
    host_grads = [{p: (None if t is None else torch.empty(t.shape, dtype=t.dtype).pin_memory())
                   for p, t in g.items()} for g in grad_sets]
    d2h = sum(t.numel() * 4 for t in grads.values() if t is not None) + 4

    def capture_split(m, t, g):
        torch.cuda.synchronize()
        gf, gb = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
        with torch.cuda.graph(gf):
            rast.forward(m, out_rgb=img, sync=False)
        with torch.cuda.graph(gb):
            loss, dimg = l1_loss(img, t, norm=norm)
            rast.backward(m, dimg, grads=g)
        return gf, gb, loss

    bufs = [(model, target), (model_b, target_b)]
    splits = [capture_split(m, t, g) for (m, t), g in zip(bufs, grad_sets)]
    copy_stream, d2h_stream = torch.cuda.Stream(), torch.cuda.Stream()
    params_in = [torch.cuda.Event(), torch.cuda.Event()]
    target_in = [torch.cuda.Event(), torch.cuda.Event()]
    consumed = [torch.cuda.Event(), torch.cuda.Event()]
    grads_ready = [torch.cuda.Event(), torch.cuda.Event()]
    grads_read = [torch.cuda.Event(), torch.cuda.Event()]

    def upload(k):  # inputs of step k into buffer k % 2, on the copy stream
        m, t = bufs[k % 2]
        with torch.cuda.stream(copy_stream):
            if k >= 2:
                copy_stream.wait_event(consumed[k % 2])  # step k - 2 is done with the buffer
            for p, h in host_planes.items():
                if h is not None:
                    m.planes[p].copy_(h, non_blocking=True)
            params_in[k % 2].record(copy_stream)
            t.copy_(host_target, non_blocking=True)
            target_in[k % 2].record(copy_stream)

    def download(k):  # gradients and loss of step k to the host, on the second copy stream
        b = k % 2
        with torch.cuda.stream(d2h_stream):
            d2h_stream.wait_event(grads_ready[b])
            for p, t in grad_sets[b].items():
                if t is not None:
                    host_grads[b][p].copy_(t, non_blocking=True)
            loss_host[b].copy_(splits[b][2], non_blocking=True)
            grads_read[b].record(d2h_stream)

    def e2e_run(steps):
        upload(0)
        for k in range(steps):
            b = k % 2
            gf, gb, _ = splits[b]
            stream.wait_event(params_in[b])
            gf.replay()
            stream.wait_event(target_in[b])
            if k >= 2:
                stream.wait_event(grads_read[b])  # step k - 2's gradients have left this buffer
            gb.replay()
            exchange(buckets[b])
            consumed[b].record(stream)
            grads_ready[b].record(stream)
            download(k)
            if k + 1 < steps:
                upload(k + 1)
        stream.wait_stream(d2h_stream)

    e2e_run(2)
    torch.cuda.synchronize()
    barrier()
    a, b2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    copy_stream.wait_event(a)
    e2e_run(args.steps)
    b2.record(stream)
    torch.cuda.synchronize()
    ems = max_over_ranks(a.elapsed_time(b2) / args.steps)
    link = copy_bandwidth()
    out["e2e_parameter_roundtrip"] = {
        "value": round(job_rate(world, nv, ems), 3), "unit": UNIT, "ms_per_step": round(ems, 4),
        "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "link_gbps": link,
        "overlap": "step k+1's uploads (parameters, targets) on one copy stream and step k's "
                   "read-back (all gradient planes, loss) on another during the compute; "
                   "double-buffered inputs and gradients"}
    del splits, bufs, model_b, target_b, grad_sets, host_grads

    # ---- end to end as a training iteration, through the trainer a user calls: the step's
    # input (the 16 target images) comes from pinned host memory each step and its result
    # (the loss) goes back to pinned host memory each step; the Gaussians and the Adam
    # state stay on the device, as they do in training, and every step ends with the fused
    # Adam update (work the headline step does not include).  The targets are
    # double-buffered: step k + 1's copy runs on a copy stream while step k computes.
    from paper_2501_00342_b300.train import ShardedTrainer, TrainConfig, Trainer
    model_t = model.with_planes(**{p: t.clone() for p, t in model.planes.items() if t is not None})
    tbufs = [torch.empty_like(target), torch.empty_like(target)]
    for t in tbufs:
        t.copy_(host_target)
    if world > 1:
        trainer = ShardedTrainer(model_t, cams, tbufs[0], world * img.numel(), settings, TrainConfig(sg_start=0))
    else:
        trainer = Trainer(model_t, cams, tbufs[0], settings, TrainConfig(sg_start=0))
    # room for the instance count to drift while Adam moves the Gaussians
    trainer.rast = Rasterizer(model_t, cams, settings, capacity=int(M * 1.3) + 4096)
    t_in = [torch.cuda.Event(), torch.cuda.Event()]
    t_used = [torch.cuda.Event(), torch.cuda.Event()]
    loss_pin = [torch.empty(1).pin_memory() for _ in range(2)]

    def train_run(steps):
        def upload_target(k):
            with torch.cuda.stream(copy_stream):
                if k >= 2:
                    copy_stream.wait_event(t_used[k % 2])  # step k - 2 is done with the buffer
                tbufs[k % 2].copy_(host_target, non_blocking=True)
                t_in[k % 2].record(copy_stream)

        upload_target(0)
        for k in range(steps):
            if k + 1 < steps:
                upload_target(k + 1)
            stream.wait_event(t_in[k % 2])
            trainer.target = tbufs[k % 2]
            loss = trainer.step()
            t_used[k % 2].record(stream)
            loss_pin[k % 2].copy_(loss.view(1), non_blocking=True)

    trainer.step(sync=True)
    train_run(args.warmup)
    torch.cuda.synchronize()
    barrier()
    a.record(stream)
    copy_stream.wait_event(a)
    train_run(args.steps)
    b2.record(stream)
    torch.cuda.synchronize()
    tms = max_over_ranks(a.elapsed_time(b2) / args.steps)
    out["e2e"] = {"value": round(job_rate(world, nv, tms), 3), "unit": UNIT, "ms_per_step": round(tms, 4),
                  "h2d_bytes_per_step": int(host_target.numel() * 4), "d2h_bytes_per_step": 4,
                  "link_gbps": link,
                  "what": "training iteration through Trainer.step (ShardedTrainer under torchrun): forward, "
                          "L1, backward, fused Adam; the targets in and the loss out every step, the "
                          "Gaussians and the optimiser state resident on the device",
                  "overlap": "step k+1's targets on a copy stream during step k; double-buffered",
                  "parameter_roundtrip_views_per_s": out["e2e_parameter_roundtrip"]["value"],
                  "loss_finite": bool(np.isfinite(float(loss_pin[(args.steps - 1) % 2][0]))),
                  "status": trainer.rast.device_status()}
    del trainer, model_t, tbufs

    # ---- CPU oracle on a bounded sample (rank 0, N = 1 only); same sample checks parity
    if rank == 0 and world == 1 and args.cpu_baseline:
        out["cpu_baseline"], out["oracle_parity"] = cpu_baseline(scene, cams, img, rast, args)
    if world > 1:
        dist.destroy_process_group()
    return out if rank == 0 else None


def _graph_kernel_nodes(raw_graph):
    """Kernel nodes of a captured CUDA graph (every kernel the step launches)."""
    try:
        from cuda.bindings import runtime as rt
        g = rt.cudaGraph_t(init_value=raw_graph)
        err, _, count = rt.cudaGraphGetNodes(g, 0)
        err, nodes, count = rt.cudaGraphGetNodes(g, count)
        kinds = [rt.cudaGraphNodeGetType(nd)[1] for nd in nodes[:count]]
        return sum(1 for k in kinds if k == rt.cudaGraphNodeType.cudaGraphNodeTypeKernel)
    except Exception:
        return None


def C_void_p_array(k):
    import ctypes
    return ctypes.c_void_p * k


def _oracle_sample(scene, cams, patches=1, views=(0, 1)):
    rows = []
    for v in views:
        p = I.sample_pixels([cams[v]], patches_per_view=patches, patch=16, stream=v)
        p[:, 0] = v
        rows.append(p)
    return np.concatenate(rows)


def cpu_baseline(scene, cams, img, rast, args):
    """The oracle as it stands, timed on this host's cores on a bounded sample of the
    workload (forward + adjoint of sampled pixels, brute force over all Gaussians)."""
    import oracle as O
    threads = O.default_threads()
    pix = _oracle_sample(scene, cams)
    t = time.time()
    ref = O.render_pixels(scene, cams, pix, threads=threads)
    w = np.random.default_rng(0).normal(size=(len(pix), 3))
    O.adjoint_pixels(scene, cams, pix, w, threads=threads)
    secs = time.time() - t
    avg_pix = sum(c.width * c.height for c in cams) / len(cams)
    views_per_s = len(pix) / secs / avg_pix
    base = {"value": views_per_s, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{len(pix)} pixels (one 16x16 patch in each of views 0 and 1), FP64 forward + "
                      f"adjoint, brute force over all {scene.n} Gaussians; {secs:.1f} s; views/s "
                      f"extrapolated by the mean pixels per view ({avg_pix:.0f})"}
    # parity of the timed GPU image on the same pixels
    got = np.empty((len(pix), 3))
    flat = img.cpu().numpy()
    for j, (v, x, y) in enumerate(pix):
        c = cams[v]
        b = rast.plan.pixel_base[v]
        hw = c.width * c.height
        for ch in range(3):
            got[j, ch] = flat[3 * b + ch * hw + y * c.width + x]
    ok = ref["margin"][:, 0] >= 1e-5
    err = float(np.abs(got - ref["rgb"]).max(1)[ok].max()) if ok.any() else None
    parity = {"pixels": int(len(pix)), "ambiguous": int((~ok).sum()), "max_abs_err": err, "tolerance": 1e-4,
              "pass": bool(err is not None and err <= 1e-4)}
    return base, parity


# ------------------------------------------------------------------------------ reference arm
def run_reference(args):
    """The oracle as the reference implementation, on the host cores: each step is a
    bounded sample of the same workload (one 16x16 patch, forward + adjoint)."""
    world, rank, _ = _dist()
    if rank != 0:
        return None
    import oracle as O
    threads = O.default_threads()
    scene, cams = I.workload(3)
    avg_pix = sum(c.width * c.height for c in cams) / len(cams)

    def one(k):
        pix = I.sample_pixels([cams[k % len(cams)]], patches_per_view=1, patch=16, stream=100 + k)
        pix[:, 0] = k % len(cams)
        t = time.time()
        O.render_pixels(scene, cams, pix, threads=threads)
        O.adjoint_pixels(scene, cams, pix, np.ones((len(pix), 3)), threads=threads)
        return len(pix), time.time() - t

    for k in range(args.warmup):
        one(k)
    tot_pix = tot_s = 0.0
    for k in range(args.steps):
        p, s = one(args.warmup + k)
        tot_pix += p
        tot_s += s
    v = tot_pix / tot_s / avg_pix
    sample = (f"per step one 16x16 patch of one view, FP64 forward + adjoint, brute force over all "
              f"{scene.n} Gaussians; views/s extrapolated by mean pixels per view ({avg_pix:.0f})")
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=("ours", "reference"))
    ap.add_argument("--tile", type=int, nargs=2, default=(32, 32))
    ap.add_argument("--batch-depth", type=int, default=1024)
    ap.add_argument("--digit-bits", type=int, default=9)
    ap.add_argument("--fwd-pixels", type=int, default=0, help="pixels per thread, forward blend (0: library's)")
    ap.add_argument("--bwd-pixels", type=int, default=0, help="pixels per thread, backward blend (0: library's)")
    ap.add_argument("--workload", default="batched", choices=("batched", "single", "medium"),
                    help="single: 1M Gaussians, one 1280x720 view; medium: the 3M scene, two "
                         "1920x1080 views (smaller cases for profilers)")
    ap.add_argument("--no-extras", dest="extras", action="store_false")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    out = run_reference(args) if args.impl == "reference" else run_gpu(args)
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
