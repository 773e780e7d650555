"""Benchmark of the resampling hot path on one B300 (or N independent replicas).

Workload (one "step"): a 4096x4096x3 FP32 image of 64 random plane waves plus
N(0, 0.05^2) noise, clipped to [0, 1] (synthetic; seeded), resampled with
Lanczos-3 and the mirror boundary by scale 1.37 (-> 5612x5612x3) and by scale
0.3 with antialiasing (-> 1229x1229x3, ~20 taps per axis).  Each step runs the
whole path on the GPU: the FP64 weight-table and band kernels of both plans and
the two resample kernels, each scale on its own stream (the scales are
independent, so their kernels overlap), replayed as one CUDA graph (the
step's launches captured once; replaying them removes the host launch gaps
between the short table kernels).  Inputs stay resident in HBM; the input (201 MB) is larger
than L2 (126 MB), so no explicit flush is needed between steps.  The
dominant kernel is also timed alone (K launches between CUDA events on its
stream) for the roofline.

Printed line (rank 0): output Mpixel/s over the K timed steps, the roofline of
the dominant kernel (the x1.37 resample), an end-to-end figure through the C
ABI with host buffers (H2D of the input and D2H of both outputs inside the
timed region), SM clocks sampled during the timed region, the FP64 CPU
oracle timed on the host cores on a bounded sample of the same workload, and
side figures: the C1 FP64 call latency, the C4 batch, the C5 serving trace,
16-bit storage, and the paper's clustering.

``--impl reference`` times that oracle alone (the project has no other
reference implementation: the paper ships no code).  Under torchrun each rank
runs an independent replica (no collective on the data path); rank 0 prints.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "output Mpixel/s, 4096x4096x3 FP32 Lanczos-3 mirror, x1.37 + x0.3 (antialiased)"
UNIT = "Mpixel/s"
SCALES = [1.37, 0.3]
N_IN = 4096
C = 3


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-sample-s", type=float, default=12.0,
                    help="target seconds of oracle work for the cpu_baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="keep the model-chosen kernel configuration")
    ap.add_argument("--batch-n", type=int, default=512, help="images in the batched section")
    ap.add_argument("--serve-seconds", type=float, default=60.0, help="length of the serving trace")
    ap.add_argument("--serve-plain-seconds", type=float, default=5.0,
                    help="arrivals of the trace replayed through the plain FP32 path")
    ap.add_argument("--serve-plain-cap", type=float, default=60.0,
                    help="wall seconds after which the plain FP32 replay stops")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving section")
    ap.add_argument("--serve-only", action="store_true", help="run only the serving section")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched section")
    ap.add_argument("--no-tc", action="store_true", help="skip the 16-bit tensor-core section")
    ap.add_argument("--no-cluster", action="store_true", help="skip the clustering section")
    ap.add_argument("--no-c1", action="store_true", help="skip the C1 FP64 latency section")
    ap.add_argument("--cluster-frames", type=int, default=592, help="204x204 ToF frames per clustering run")
    ap.add_argument("--cluster-only", action="store_true", help="run only the clustering section")
    ap.add_argument("--tc-only", action="store_true",
                    help="run only the 16-bit tensor-core section (profiling); prints its object")
    ap.add_argument("--batch-only", action="store_true",
                    help="run only the batched section (profiling); prints its object")
    ap.add_argument("--tune-cache", default=None,
                    help="JSON-lines autotuner cache (a hit skips the tuning launches)")
    ap.add_argument("--size", type=int, default=4096,
                    help="input side (profiling runs only; the benchmark workload is 4096)")
    ap.add_argument("--scales", type=str, default="1.37,0.3",
                    help="comma-separated scales (profiling runs only)")
    ap.add_argument("--case", action="store_true",
                    help="profiling: run one plan (--size, first of --scales, --case-*) --case-launches times "
                         "and print its configuration; no timing, no JSON line")
    ap.add_argument("--case-dtype", default="f32", choices=["f32", "f16", "bf16"])
    ap.add_argument("--case-channels", type=int, default=3)
    ap.add_argument("--case-kernel", default="lanczos")
    ap.add_argument("--case-param", type=float, default=3.0)
    ap.add_argument("--case-boundary", default="mirror")
    ap.add_argument("--case-flags", default="", help="comma-separated RS_* plan flag names without the prefix")
    ap.add_argument("--case-form", default="",
                    help="streaming form kind,h_warps,v_warps,staged_blocks,strip_width,row_ranges "
                         "(rs_plan_set_stream_form; zeros: defaults)")
    ap.add_argument("--case-launches", type=int, default=4)
    a = ap.parse_args()
    global N_IN, SCALES
    N_IN = a.size
    SCALES = [float(v) for v in a.scales.split(",")]
    return a


def dist_info():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(ms, device):
    """The timed region of the slowest rank (the bench reports whole-job
    throughput over it): a MAX all-reduce of each rank's milliseconds, then a
    barrier.  Needs an initialised process group (NCCL on the GPUs; the CPU
    tests use gloo)."""
    import torch

    t = torch.tensor([float(ms)], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    torch.distributed.barrier()
    return float(t.item())


def out_sizes(reference: bool = False):
    """Output sides of the workload's scales: the library's rule (our arm; host
    only) or the oracle's own (the reference arm runs the oracle alone)."""
    if reference:
        import oracle

        return [oracle.out_size(N_IN, s) for s in SCALES]
    import paper_1110_5450_b300 as rs

    return [rs.rs_desc_out_size(rs.make_desc(N_IN, N_IN, C, 0, 0, s, s, kernel="lanczos", param=3.0,
                                             boundary="mirror"))[0] for s in SCALES]


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


# the device code of the dominant kernel (the pipelined streaming kernel,
# FP32): a change to it voids a recorded traffic figure, and so does another
# configuration (the recorded form is compared as well)
TRAFFIC_SOURCES = ("rs_xstream.cuh", "rs_xstream_f32.cu", "rs_stream.cuh", "rs_fused.cuh")


def kernel_source_hash(files=TRAFFIC_SOURCES):
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1110_5450_b300", "csrc")
    for f in sorted(files):
        h.update(f.encode())
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(form=None):
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summary, only if it was taken on the current kernel sources and, when
    `form` (the streaming form tuple in use) is given, on that form."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        if d.get("source_hash") != kernel_source_hash():
            return None
        if form is not None and list(d.get("form", [])) != list(form):
            return None
        return float(d["dram_bytes_per_launch"])
    except Exception:
        return None


def stream_form(rs, plan):
    """(kind, h_warps, v_warps, staged_blocks, strip_width, row_ranges) of a
    streaming plan, else None."""
    if plan.path not in ("stream", "tcstream"):
        return None
    f = rs.rs_plan_get_stream_form(plan.handle)
    return [f.kind, f.h_warps, f.v_warps, f.staged_blocks, f.strip_width, f.row_ranges]


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 100 ms while running
    (the bench runs it over a 0.4 s burst of the timed step's own replays and
    the timed region)."""

    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 6:
                self.samples.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "", 1).isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "", 1).isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in self.samples for k in range(4) if s[2 + k] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def cpu_baseline(img, budget_s: float, outs):
    """The FP64 oracle on the host cores, on a band of output rows of both
    scales sized to about ``budget_s`` seconds; returns (Mpixel/s, cores, text)."""
    import oracle

    import numpy as np

    o = oracle.default()
    img = np.ascontiguousarray(img, dtype=np.float64)  # exact upcast, once, outside the timing
    # grow a central band of output rows per scale until it has taken its
    # share of the budget (per-call set-up makes tiny samples unrepresentative)
    total_px = sum(n * n for n in outs)
    full_s, dt, rows = 0.0, 0.0, []
    for n in outs:
        share = budget_s * (n * n) / total_px
        k = 16
        while True:
            k = min(k, n)
            y0 = (n - k) // 2
            t0 = time.perf_counter()
            o.resample(img, n, n, "lanczos", "mirror", param=3.0, rows=(y0, y0 + k))
            t = time.perf_counter() - t0
            if t >= 0.5 * share or k == n:
                break
            k = int(k * min(8.0, max(2.0, share / max(t, 1e-3))))
        rows.append(k)
        dt += t
        full_s += t * (n / k)  # seconds for all n rows at the sampled rate
    if all(k == n for k, n in zip(rows, outs)):
        # the whole workload fits the budget: repeat it to fill the budget
        passes = 1
        while dt < budget_s:
            t0 = time.perf_counter()
            for n in outs:
                o.resample(img, n, n, "lanczos", "mirror", param=3.0)
            t = time.perf_counter() - t0
            dt += t
            passes += 1
        value = passes * total_px / dt / 1e6
        sample = "the whole workload (both outputs), %d passes (%.1f s)" % (passes, dt)
        return value, o.default_threads(), sample
    value = total_px / full_s / 1e6
    sample = "central bands of %s output rows of the x1.37 and x0.3 outputs (%.1f s)" % (
        "+".join(str(k) for k in rows), dt)
    return value, o.default_threads(), sample


def sample_rows(n: int, k: int = 6, seed: int = 17):
    """Rows checked against the oracle: both edges, the middle, k random."""
    import numpy as np

    g = np.random.default_rng(seed)
    return sorted(r for r in set([0, 1, n // 2, n - 2, n - 1]) | set(int(v) for v in g.integers(0, n, k))
                  if 0 <= r < n)


def accuracy_item(group, dtype, path, make_input, oh, ow, kernel, param, boundary, rows, gpu, tol):
    """One result to check against the oracle: the device output on `rows`
    (None: every row) and how to rebuild its exact (quantised) input."""
    return {"group": group, "dtype": dtype, "path": path, "input": make_input, "oh": oh, "ow": ow,
            "kernel": kernel, "param": param, "boundary": boundary, "rows": rows, "gpu": gpu, "tol": tol}


def oracle_accuracy(items):
    """Part of the CPU-baseline leg: the FP64 oracle on the sampled rows of
    every collected result, fed the same quantised input; per result group the
    largest absolute error and the RMS error."""
    import numpy as np

    import oracle

    groups = {}
    for it in items:
        exact = it["input"]()
        if it["rows"] is None:
            want = oracle.resample(exact, it["oh"], it["ow"], it["kernel"], it["boundary"], param=it["param"])
        else:
            want = np.concatenate([oracle.resample(exact, it["oh"], it["ow"], it["kernel"], it["boundary"],
                                                   param=it["param"], rows=(r, r + 1)) for r in it["rows"]])
        d = np.abs(np.asarray(it["gpu"], dtype=np.float64).reshape(want.shape) - want)
        g = groups.setdefault(it["group"], {"result": it["group"], "dtype": it["dtype"], "path": it["path"],
                                            "max_abs": 0.0, "sq": 0.0, "n": 0, "rows": 0, "tol": it["tol"]})
        g["max_abs"] = max(g["max_abs"], float(d.max()))
        g["sq"] += float((d * d).sum())
        g["n"] += d.size
        g["rows"] += want.shape[0]
        if it["path"] != g["path"]:
            g["path"] = "mixed"
    out = []
    for g in groups.values():
        out.append({"result": g["result"], "dtype": g["dtype"], "path": g["path"], "max_abs": g["max_abs"],
                    "rms": math.sqrt(g["sq"] / max(1, g["n"])), "rows_checked": g["rows"], "tol": g["tol"],
                    "within_tol": g["max_abs"] <= g["tol"]})
    return out


def run_case(args):
    """--case: one plan, a few launches, for profilers (no timing)."""
    import torch

    import paper_1110_5450_b300 as rs
    import synth

    dt = {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}[args.case_dtype]
    flags = 0
    for name in filter(None, args.case_flags.split(",")):
        flags |= getattr(rs, "RS_" + name.strip().upper())
    img = synth.sinusoids(N_IN, N_IN, args.case_channels, seed=synth.SEED_C2)
    x = torch.from_numpy(img).to(dt).cuda()
    p = rs.Plan(N_IN, N_IN, args.case_channels, scale=SCALES[0], kernel=args.case_kernel, param=args.case_param,
                boundary=args.case_boundary, dtype=dt, flags=flags)
    y = torch.empty(p.out_shape, dtype=dt, device="cuda")
    if args.tune_cache:
        p.autotune(x, y, cache_path=args.tune_cache)
    if args.case_form:
        kind, hw, vw, ns, sw, nr = [int(v) for v in args.case_form.split(",")]
        rs.rs_plan_set_stream_form(p.handle, kind, hw, ns, sw, 0, torch.cuda.current_stream().cuda_stream,
                                   vw, nr)
        p.info = rs.rs_plan_get_info(p.handle)
    for _ in range(args.case_launches):
        p(x, out=y)
    torch.cuda.synchronize()
    p.check()
    i = p.info
    print("path", p.path, "tile", [i.tile_h, i.tile_w], "group", i.group_h, "band", [i.span_h, i.span_w],
          "stages", i.stages, "warps_pass1", i.warps_pass1, "smem", i.smem_bytes, "ctas_per_sm", i.ctas_per_sm,
          "form", stream_form(rs, p))
    p.close()


def batched_section(args, dev, stream, acc=None):
    """Uneven batch (512 single-channel FP16 images, sides U{64..2048}, scale
    logU[1/4, 4], kernel U{tent, Keys -1/2, Lanczos-3}, mirror) in one
    persistent launch replayed as a CUDA graph, against the plain per-image
    FP32 path on the same images."""
    import numpy as np
    import torch

    import paper_1110_5450_b300 as rs
    import synth

    specs = synth.batch_specs(args.batch_n)
    tdt = torch.float16
    ins16, ins32, pitches = [], [], []
    for sp in specs:
        img = synth.sinusoids(sp.in_h, sp.in_w, 1, seed=sp.seed)
        t16 = torch.from_numpy(img).to(tdt)
        pitch = (sp.in_w + 7) // 8 * 8          # 16-byte row pitch (TMA eligible)
        b16 = torch.zeros((sp.in_h, pitch), dtype=tdt, device=dev)
        b16[:, :sp.in_w] = t16[:, :, 0].to(dev)
        ins16.append(b16)
        ins32.append(torch.from_numpy(img).to(dev))
        pitches.append(pitch)
    bspecs = [dict(in_h=sp.in_h, in_w=sp.in_w, scale=sp.scale, kernel=sp.kernel, param=sp.param,
                   boundary="mirror") for sp in specs]
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        batch = rs.Batch(bspecs, channels=1, dtype=tdt, in_pitches=pitches, stream=stream)
    create_s = time.perf_counter() - t0
    outs16 = []
    for d in batch.descs:
        oh, ow = rs.rs_desc_out_size(d)
        outs16.append(torch.empty((oh, ow, 1), dtype=tdt, device=dev))
    t0 = time.perf_counter()
    if not args.no_tune:
        batch.autotune(ins16, outs16, stream=stream, cache_path=args.tune_cache)
    tune_s = time.perf_counter() - t0
    info = batch.info
    for _ in range(3):
        batch(ins16, outs16, stream=stream)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    reps = 10
    a.record(stream)
    for _ in range(reps):
        batch(ins16, outs16, stream=stream)
    b.record(stream)
    torch.cuda.synchronize()
    ms_batch = a.elapsed_time(b) / reps
    # plain per-image FP32 path: one plan and one launch per image
    plans, outs32 = [], []
    with torch.cuda.stream(stream):
        for sp in specs:
            pl = rs.Plan(sp.in_h, sp.in_w, 1, scale=sp.scale, kernel=sp.kernel, param=sp.param,
                         boundary="mirror", dtype=torch.float32, stream=stream)
            plans.append(pl)
            outs32.append(torch.empty(pl.out_shape, dtype=torch.float32, device=dev))
    torch.cuda.synchronize()

    def plain():
        for pl, x, y in zip(plans, ins32, outs32):
            pl(x, out=y, stream=stream)

    plain()
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(3):
        plain()
    b.record(stream)
    torch.cuda.synchronize()
    ms_plain = a.elapsed_time(b) / 3
    # FP16 batch against the per-image FP32 path; every 64th image's sampled
    # rows go to the oracle leg
    diff = max(float((o16.float() - o32).abs().max()) for o16, o32 in zip(outs16, outs32))
    if acc is not None:
        for k in range(0, len(specs), 64):
            sp, y = specs[k], outs16[k]
            rows = sample_rows(y.shape[0], 2, seed=k)
            acc.append(accuracy_item(
                "C4 batch of %d FP16 images (every 64th)" % len(specs), "f16", "batch",
                (lambda sp=sp: torch.from_numpy(synth.sinusoids(sp.in_h, sp.in_w, 1, seed=sp.seed))
                 .to(tdt).to(torch.float64).numpy()),
                y.shape[0], y.shape[1], sp.kernel, sp.param, "mirror", rows,
                y[rows].double().cpu().numpy(), 2e-3))
    for pl in plans:
        pl.close()
    batch.close()
    peak, _ = measured_peaks()
    mpx = info.out_pixels / 1e6
    alg = info.in_bytes + info.out_bytes
    return {"workload": "%d single-channel FP16 images, sides U{64..2048}, scale logU[1/4,4], "
                        "kernel U{tent, Keys -1/2, Lanczos-3}, mirror; one persistent launch (CUDA graph)"
                        % len(specs),
            "value": mpx / (ms_batch / 1e3), "unit": UNIT, "ms_per_batch": ms_batch,
            "hbm_frac": alg / (ms_batch / 1e3) / 1e9 / peak, "algorithmic_bytes": alg,
            "plain_fp32_per_image": {"value": mpx / (ms_plain / 1e3), "unit": UNIT, "ms": ms_plain,
                                     "launches": len(specs)},
            "speedup_vs_plain_fp32": ms_plain / ms_batch,
            "max_abs_diff_fp16_vs_fp32_path": diff, "create_s": round(create_s, 2), "autotune_s": round(tune_s, 2),
            "config": {"streamed_images": info.n_streamed, "group": info.group, "warps_pass1": info.warps_pass1, "stages": info.stages,
                       "use_tma": info.use_tma, "smem": info.smem_bytes, "ctas_per_sm": info.ctas_per_sm,
                       "tiles": info.total_tiles}}


def tc_section(args, dev, stream, acc=None):
    """Precision form: the 4096x4096x3 sinusoid image stored in BF16 and FP16
    (FP32 accumulation), Lanczos-3 mirror, x1.37, x0.3 and x0.125.  Per dtype
    and scale: the autotuned plan ("auto": the fastest of the kernels below),
    then each kernel forced where it applies -- the tensor-core streaming
    downscale (stream form 3: the horizontal pass as a tcgen05 GEMM), the
    fused tiles with the tcgen05 vertical pass, the SIMT tile kernel and the
    SIMT row-streaming kernels (untuned form); kernel time (CUDA events per
    launch, L2 flushed before each: the 16-bit input, 101 MB, would fit the
    126 MB L2), HBM fraction, and the largest difference from the FP32 path
    on the same input (the autotuned results' errors against the FP64
    oracle: the line's accuracy_vs_fp64_oracle)."""
    import torch

    import paper_1110_5450_b300 as rs
    import synth

    img = synth.sinusoids(4096, 4096, 3, seed=synth.SEED_C2)
    x32 = torch.from_numpy(img).to(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    peak, _ = measured_peaks()
    res = {"workload": "4096x4096x3 sinusoids+noise, Lanczos-3 mirror, BF16/FP16 storage, FP32 accumulation",
           "l2": "256 MB buffer written before each timed launch", "runs": []}
    # (label, plan flags, stream form forced after creation or None, autotune)
    variants = (("auto", 0, None, True), ("tcstream", 0, 3, False), ("tcgen05", rs.RS_FORCE_TC, None, True),
                ("tile", rs.RS_FORCE_SIMT | rs.RS_NO_STREAM, None, True), ("stream", rs.RS_FORCE_STREAM, -1, False))
    s = stream.cuda_stream
    for tdt, name in ((torch.bfloat16, "bf16"), (torch.float16, "f16")):
        x = x32.to(tdt)
        for sc in (1.37, 0.3, 0.125):
            with torch.cuda.stream(stream):
                p32 = rs.Plan(4096, 4096, 3, scale=sc, kernel="lanczos", param=3.0, boundary="mirror",
                              dtype=torch.float32, stream=stream)
                y32 = p32(x32, stream=stream)
            for label, flags, form, tune in variants:
                try:
                    with torch.cuda.stream(stream):
                        p = rs.Plan(4096, 4096, 3, scale=sc, kernel="lanczos", param=3.0, boundary="mirror",
                                    dtype=tdt, flags=flags, stream=stream)
                    if form == 3:
                        rs.rs_plan_set_stream_form(p.handle, 3, 0, 0, 0, 0, s)
                        p.info = rs.rs_plan_get_info(p.handle)
                    elif form == -1 and p.path == "tcstream":
                        # the SIMT streaming kernels: the band kernel's untuned form
                        rs.rs_plan_set_stream_form(p.handle, 1, 0, 0, 0, 0, s)
                        p.info = rs.rs_plan_get_info(p.handle)
                except (RuntimeError, rs.RSError) as e:
                    if "unsupported" not in str(e):
                        raise
                    continue  # this kernel does not apply to this scale
                with torch.cuda.stream(stream):
                    y = torch.empty(p.out_shape, dtype=tdt, device=dev)
                    if tune and not args.no_tune:
                        p.autotune(x, out=y, stream=stream, cache_path=args.tune_cache)
                    for _ in range(3):
                        p(x, out=y, stream=stream)
                torch.cuda.synchronize()
                reps = 10
                ev = []
                with torch.cuda.stream(stream):
                    for _ in range(reps):
                        flush.fill_(1)
                        a = torch.cuda.Event(enable_timing=True)
                        b = torch.cuda.Event(enable_timing=True)
                        a.record(stream)
                        p(x, out=y, stream=stream)
                        b.record(stream)
                        ev.append((a, b))
                torch.cuda.synchronize()
                p.check()
                us = sum(a.elapsed_time(b) for a, b in ev) / reps * 1e3
                alg = x.numel() * 2 + y.numel() * 2
                info = p.info
                if acc is not None and label == "auto":
                    rows = sample_rows(y.shape[0])
                    acc.append(accuracy_item(
                        "C3 4096x4096x3 x%g %s" % (sc, name.upper()), name, rs.PATHS[info.path],
                        (lambda tdt=tdt: torch.from_numpy(img).to(tdt).to(torch.float64).numpy()),
                        y.shape[0], y.shape[1], "lanczos", 3.0, "mirror", rows, y[rows].double().cpu().numpy(),
                        1e-2 if name == "bf16" else 2e-3))
                run = {
                    "dtype": name, "scale": sc, "variant": label, "path": rs.PATHS[info.path], "us": us,
                    "GBps": alg / (us / 1e6) / 1e9, "hbm_frac": alg / (us / 1e6) / 1e9 / peak,
                    "out_mpx_s": y.shape[0] * y.shape[1] / us,
                    "max_abs_diff_vs_fp32_path": float((y.float() - y32).abs().max()),
                    "tile": [info.tile_h, info.tile_w], "group": info.group_h, "band": info.span_h,
                    "smem": info.smem_bytes, "ctas_per_sm": info.ctas_per_sm}
                if info.path in (3, 5):
                    run["form"] = stream_form(rs, p)
                res["runs"].append(run)
                p.close()
            p32.close()
    return res


def c1_section(dev, stream, acc=None):
    """C1: 256x256x1 FP64 U[0,1) -> 512x512, Keys a = -1/2, clamp, FP64
    accumulation.  2.6 MB move in 0.4 us at full HBM bandwidth, so there is
    no meaningful roofline: after autotuning, the device time of one call
    (weight tables, bands if any, and resample; CUDA events over 200 calls on
    the stream) and the host round trip of one call (call plus synchronize;
    p50 / p99 of 200)."""
    import torch

    import paper_1110_5450_b300 as rs
    import synth

    img = torch.from_numpy(synth.uniform(256, 256, 1, seed=synth.SEED_C1)).to(dev)
    with torch.cuda.stream(stream):
        p = rs.Plan(256, 256, 1, 512, 512, kernel="cubic", param=-0.5, boundary="clamp",
                    dtype=torch.float64, stream=stream)
        y = torch.empty(p.out_shape, dtype=torch.float64, device=dev)
    # measured choice of kernel (tile, two-pass) for this small problem
    p.autotune(img, out=y, stream=stream)

    def call():
        p.recompute(stream)
        p(img, out=y, stream=stream)

    for _ in range(20):
        call()
    torch.cuda.synchronize()
    a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(200):
        call()
    b_.record(stream)
    torch.cuda.synchronize()
    dev_us = a.elapsed_time(b_) / 200 * 1e3
    rt = []
    for _ in range(200):
        t0 = time.perf_counter()
        call()
        stream.synchronize()
        rt.append((time.perf_counter() - t0) * 1e6)
    p.check()
    info = p.info
    if acc is not None:
        host = img.cpu().numpy()
        acc.append(accuracy_item("C1 256x256x1 FP64 x2 Keys (whole output)", "f64", rs.PATHS[info.path],
                                 lambda: host, 512, 512, "cubic", -0.5, "clamp", None,
                                 y.cpu().numpy(), 1e-12))
    p.close()
    rt.sort()
    return {"workload": "C1 256x256x1 FP64 U[0,1) -> 512x512, Keys -1/2, clamp",
            "path": rs.PATHS[info.path], "device_us_per_call": dev_us,
            "roundtrip_us_p50": rt[len(rt) // 2], "roundtrip_us_p99": rt[int(0.99 * len(rt))],
            "launches_per_call": 3, "autotuned": True}


def cluster_section(args, dev, stream):
    """The paper's own data-parallel path: parallel merging clustering of
    synthetic 204 x 204 ToF frames (depth, distance, intensity), Table 1
    thresholds and weights, one thread block per frame, all frames in one
    launch.  Frames per second over the batch and the merge rounds it took;
    the paper's Table 2 gives 44 ms per frame for its three clustering steps
    on a GeForce GTX 480 (context, not a target)."""
    import numpy as np
    import torch

    import paper_1110_5450_b300 as rs
    import synth

    n = args.cluster_frames
    Z, D, I = synth.tof_frames(min(n, 16))
    reps = (n + Z.shape[0] - 1) // Z.shape[0]
    z, d, inten = (torch.from_numpy(np.ascontiguousarray(np.concatenate([a] * reps)[:n])).to(dev) for a in (Z, D, I))
    c = rs.Cluster(n, 204, 204)
    with torch.cuda.stream(stream):
        labels, rounds = c(z, d, inten, stream=stream)   # warm-up
        stream.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        labels, rounds = c(z, d, inten, stream=stream)
        b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    r = rounds.cpu().numpy()
    regions = [int(np.unique(labels[k].cpu().numpy()).size) for k in range(min(n, 4))]
    c.close()
    return {"workload": "%d synthetic 204x204 ToF frames (piecewise-planar scenes), t_z 0.04 m, t_phi 0.009 rad, "
                        "alpha_z 8/pi, alpha_phi 4/3; one block per frame, one launch" % n,
            "frames_per_s": n / (ms / 1e3), "ms_per_batch": ms, "ms_per_frame_latency": ms,
            "rounds_mean": float(r.mean()), "rounds_max": int(r.max()), "final_regions_first_frames": regions,
            "paper_context": "Table 2: 44 ms per frame (Find Mergepartner 29 + Merge 5 + Update 10) on a GTX 480"}


def serving_section(args, dev):
    """Open-loop serving trace: Poisson arrivals at 2000 req/s, square BF16
    images (side logU[32, 4096], 1 or 3 channels, scale logU[1/8, 8], kernel
    U{Keys -1/2, Lanczos-3}, mirror), continuous batching under a 40 GB budget.
    Inputs are crops of two resident 4096x4096 base images; outputs are
    allocated by the server and released as soon as each request completes.
    Latency = completion (host callback) - arrival time in the trace.

    The comparator replays the first --serve-plain-seconds of the SAME trace
    open loop through the plain FP32 path: one worker takes the requests in
    arrival order, each one (plan creation + resample + synchronise + destroy)
    starting at its arrival or when the previous one ends, whichever is later;
    its latency is completion - arrival too.  The replay stops after
    --serve-plain-cap seconds; requests not finished by then are counted with
    the latency they had reached (a lower bound) and reported as unfinished.
    The server's latencies over the same prefix of arrivals are reported
    beside it."""
    import numpy as np
    import torch

    import paper_1110_5450_b300 as rs
    import synth

    trace = synth.serving_trace(duration_s=args.serve_seconds)
    bases, bases32 = {}, {}
    for C in (1, 3):
        img = synth.sinusoids(4096, 4096, C, seed=synth.SEED_C5 + C)
        bases[C] = torch.from_numpy(img).to(torch.bfloat16).to(dev).reshape(4096, 4096 * C)
        bases32[C] = torch.from_numpy(img).to(dev).reshape(4096, 4096 * C)
    descs = []
    for r in trace:
        sp = r.spec
        descs.append(rs.make_desc(sp.in_h, sp.in_w, sp.channels, scale_h=sp.scale, scale_w=sp.scale,
                                  kernel=sp.kernel, param=sp.param, boundary="mirror", dtype=torch.bfloat16,
                                  in_row_stride=4096 * sp.channels))
    srv = rs.rs_server_create(40 << 30, max_inflight=4, max_batch=256)
    torch.cuda.synchronize()
    outstanding = {}
    lat = np.full(len(trace), np.nan)
    out_px, batch_sizes = 0, []
    t0_ns = time.monotonic_ns()       # the server stamps with the same (steady) clock
    i = 0
    n = len(trace)
    lag = []
    while i < n or outstanding:
        now = (time.monotonic_ns() - t0_ns) * 1e-9
        # submit everything whose arrival time has come
        first = i
        while i < n and trace[i].arrival_s <= now:
            i += 1
        if i > first:
            reqs = [rs.rs_request(descs[k], bases[trace[k].spec.channels].data_ptr(), None) for k in range(first, i)]
            tk = rs.rs_batch_submit(srv, reqs)
            for k in range(first, i):
                outstanding[tk + (k - first)] = k
                lag.append(now - trace[k].arrival_s)
        # collect completions
        done = []
        for tk in list(outstanding.keys())[:512]:
            st = rs.rs_batch_poll(srv, tk)
            if st.status == rs.RS_ERR_BUSY:
                continue
            k = outstanding[tk]
            if st.status == rs.RS_OK:
                lat[k] = (st.t_done_ns - t0_ns) / 1e6 - trace[k].arrival_s * 1e3
                out_px += st.out_h * st.out_w
                batch_sizes.append(st.batch_size)
            rs.rs_server_release(srv, tk)
            done.append(tk)
        for tk in done:
            del outstanding[tk]
        if not done and i < n:
            time.sleep(0.0002)
    wall = (time.monotonic_ns() - t0_ns) * 1e-9
    stats = rs.rs_server_get_stats(srv)
    rs.rs_server_drain(srv)
    rs.rs_server_destroy(srv)
    ok = ~np.isnan(lat)

    # the plain FP32 path, open loop on the first seconds of the same trace
    m = sum(1 for r in trace if r.arrival_s < args.serve_plain_seconds)
    dd = []
    for r in trace[:m]:
        sp = r.spec
        d = rs.make_desc(sp.in_h, sp.in_w, sp.channels, scale_h=sp.scale, scale_w=sp.scale, kernel=sp.kernel,
                         param=sp.param, boundary="mirror", dtype=torch.float32, in_row_stride=4096 * sp.channels)
        oh, ow = rs.rs_desc_out_size(d)
        dd.append((d, oh * ow * sp.channels))
    y = torch.empty(max([e for _, e in dd] + [1]), dtype=torch.float32, device=dev)   # reused output
    torch.cuda.synchronize()
    plat, px32 = np.zeros(m), 0
    t1_ns = time.monotonic_ns()
    cap_ns = int(args.serve_plain_cap * 1e9)
    served = 0
    for k in range(m):
        arr = t1_ns + int(trace[k].arrival_s * 1e9)
        while time.monotonic_ns() < arr:
            pass
        h = rs.rs_plan_create(dd[k][0], 0)
        rs.rs_resample(h, bases32[trace[k].spec.channels].data_ptr(), y.data_ptr(), 0)
        torch.cuda.synchronize()
        rs.rs_destroy(h)
        t = time.monotonic_ns()
        plat[k] = (t - arr) / 1e6
        px32 += dd[k][1] // trace[k].spec.channels
        served = k + 1
        if t - t1_ns > cap_ns:
            break
    stop_ns = time.monotonic_ns()
    for k in range(served, m):          # still waiting when the replay stopped: a lower bound
        plat[k] = max(0.0, (stop_ns - t1_ns) / 1e6 - trace[k].arrival_s * 1e3)
    plain_wall = (stop_ns - t1_ns) * 1e-9
    del y
    pre = ok[:m]
    return {"workload": "Poisson %d req/s for %.0f s, square BF16, side logU[32,4096], C in {1,3}, "
                        "scale logU[1/8,8], kernel U{Keys -1/2, Lanczos-3}, mirror; 40 GB budget"
                        % (2000, args.serve_seconds),
            "requests": int(ok.sum()), "rejected": int(stats.rejected), "launches": int(stats.launches),
            "streamed_launches": int(stats.streamed),
            "value": out_px / wall / 1e6, "unit": UNIT, "wall_s": wall,
            "p50_ms": float(np.percentile(lat[ok], 50)), "p99_ms": float(np.percentile(lat[ok], 99)),
            "latency": "completion (host callback) - arrival in the trace",
            "mean_batch": float(np.mean(batch_sizes)) if batch_sizes else 0.0,
            "max_bytes_in_use": int(stats.max_bytes_in_use),
            "submit_lag_p99_ms": float(np.percentile(lag, 99) * 1e3) if lag else 0.0,
            "same_prefix": {"arrivals_s": args.serve_plain_seconds, "requests": m,
                            "server_p50_ms": float(np.percentile(lat[:m][pre], 50)) if pre.any() else None,
                            "server_p99_ms": float(np.percentile(lat[:m][pre], 99)) if pre.any() else None,
                            "plain_fp32_open_loop": {
                                "served": served, "unfinished": m - served,
                                "p50_ms": float(np.percentile(plat, 50)) if m else None,
                                "p99_ms": float(np.percentile(plat, 99)) if m else None,
                                "value": px32 / plain_wall / 1e6, "unit": UNIT, "wall_s": plain_wall,
                                "how": "one worker, arrival order, rs_plan_create + rs_resample + sync + "
                                       "rs_destroy per request, FP32, one reused output buffer; "
                                       "latency = completion - arrival (unfinished: lower bound at the cap)"}}}


def run_reference(args, rank, world):
    """--impl reference: the FP64 oracle on the host cores (rank 0 only)."""
    if rank != 0:
        return
    import synth

    img = synth.sinusoids(N_IN, N_IN, C, seed=synth.SEED_C2)
    per_step = max(2.0, 60.0 / max(1, args.steps + args.warmup))
    outs = out_sizes(reference=True)
    for _ in range(args.warmup):
        cpu_baseline(img, min(per_step, 2.0), outs)
    vals, cores, sample = [], 0, ""
    t0 = time.perf_counter()
    for _ in range(args.steps):
        v, cores, sample = cpu_baseline(img, per_step, outs)
        vals.append(v)
    wall = time.perf_counter() - t0
    value = statistics.median(vals)
    mpx_step = sum(n * n for n in outs) / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": mpx_step / value * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": "C2 4096x4096x3 x1.37+x0.3 Lanczos-3 mirror"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample + "; per step, %d steps in %.1f s" % (args.steps, wall)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_info()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.case:
        run_case(args)
        return

    import torch

    import paper_1110_5450_b300 as rs
    import synth

    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.Stream()
    outs = out_sizes()
    if args.batch_only:
        print(json.dumps(batched_section(args, dev, stream)), flush=True)
        return
    if args.serve_only:
        print(json.dumps(serving_section(args, dev)), flush=True)
        return
    if args.tc_only:
        print(json.dumps(tc_section(args, dev, stream)), flush=True)
        return
    if args.cluster_only:
        print(json.dumps(cluster_section(args, dev, stream)), flush=True)
        return

    img = synth.sinusoids(N_IN, N_IN, C, seed=synth.SEED_C2 + rank)
    x = torch.from_numpy(img).to(dev)
    with torch.cuda.stream(stream):
        plans = [rs.Plan(N_IN, N_IN, C, scale=s, kernel="lanczos", param=3.0, boundary="mirror",
                         dtype=torch.float32, stream=stream) for s in SCALES]
        ys = [torch.empty(p.out_shape, dtype=torch.float32, device=dev) for p in plans]
    torch.cuda.synchronize()
    # measured autotuning of each plan on its own buffers (outside the timed region)
    t_tune = time.perf_counter()
    if not args.no_tune:
        for p, y in zip(plans, ys):
            p.autotune(x, out=y, stream=stream, cache_path=args.tune_cache)
    torch.cuda.synchronize()
    t_tune = time.perf_counter() - t_tune
    # our kernels per step and plan: the weight tables, the band tables (one
    # launch for both bands of a band-streaming or tile plan; none for the
    # pipelined kernel, which builds its bands on chip) and the resample
    launches_per_step = sum(2 if (stream_form(rs, p) or [0])[0] == 2 else 3 for p in plans)

    side = torch.cuda.Stream()

    def step():
        # the plans are independent: each plan's tables and resample on its
        # own stream, so the short table kernels overlap and the second
        # resample's CTAs fill the SMs the first one leaves idle (measured
        # 0.258 against 0.266 ms per step with the resamples in sequence)
        side.wait_stream(stream)
        for p, y in zip(plans[1:], ys[1:]):
            p.recompute(side)
            p(x, out=y, stream=side)
        plans[0].recompute(stream)
        plans[0](x, out=ys[0], stream=stream)
        stream.wait_stream(side)

    for _ in range(2):
        step()
    torch.cuda.synchronize()
    # The step as one CUDA graph: its launches are short (the weight and band
    # kernels take microseconds), so replaying them from a graph removes the
    # host launch gaps between them.  The graph holds exactly the eager step.
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        step()
    with torch.cuda.stream(stream):
        for _ in range(max(3, args.warmup)):
            graph.replay()
    torch.cuda.synchronize()

    # each scale's resample alone, K launches captured in a CUDA graph: the
    # kernel timings below replay it between CUDA events, so that no host gap
    # (the clock sampler's process competes for the host) opens between the
    # launches and inflates their average
    kgraphs = []
    for i in (0, 1):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            for _ in range(args.steps):
                plans[i](x, out=ys[i], stream=stream)
        kgraphs.append(g)
    with torch.cuda.stream(stream):
        for g in kgraphs:
            g.replay()
    torch.cuda.synchronize()

    sampler = ClockSampler(dev.index or 0)
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler.start()
    # keep the GPU under this step's load (untimed replays of the same graph)
    # for 0.4 s, so that the sampler's 100 ms samples see the clocks the
    # workload runs at; the timed steps follow without a gap
    t_load = time.perf_counter()
    with torch.cuda.stream(stream):
        while time.perf_counter() - t_load < 0.4:
            for _ in range(40):
                graph.replay()
            stream.synchronize()
    with torch.cuda.stream(stream):
        t_start.record(stream)
        for _ in range(args.steps):
            graph.replay()
        t_end.record(stream)
    torch.cuda.synchronize()
    # the dominant kernel (the x1.37 resample) on its stream, K launches
    # between CUDA events, right after the timed steps and on the same buffers
    ka = torch.cuda.Event(enable_timing=True)
    kb = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        ka.record(stream)
        kgraphs[0].replay()
        kb.record(stream)
    # and the x0.3 resample, the same way (its own roofline figure)
    kc = torch.cuda.Event(enable_timing=True)
    kd = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        kc.record(stream)
        kgraphs[1].replay()
        kd.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = t_start.elapsed_time(t_end)
    kms = [ka.elapsed_time(kb) / args.steps]
    if world > 1:
        ms = max_over_ranks(ms, dev)

    mpx_step = sum(n * n for n in outs) / 1e6
    value = world * args.steps * mpx_step / (ms / 1e3)

    # roofline of the dominant kernel: the x1.37 resample
    in_bytes = N_IN * N_IN * C * 4
    out_bytes = outs[0] * outs[0] * C * 4
    alg = in_bytes + out_bytes
    k_avg_s = statistics.mean(kms) / 1e3
    peak, peak_kind = measured_peaks()
    achieved = alg / k_avg_s / 1e9
    k2_s = kc.elapsed_time(kd) / args.steps / 1e3
    alg2 = in_bytes + outs[1] * outs[1] * C * 4

    # end to end through the C ABI with host buffers: every step copies its
    # input from pinned host memory, recomputes the tables, resamples both
    # scales and copies both outputs back.  Steps are double-buffered over
    # three streams (host->device copy, compute, device->host copy) so that
    # step k+1's input upload and step k's download use the two copy
    # directions at once; the timed region spans all steps, first upload to
    # last download.
    e2e = None
    if not args.no_e2e:
        h_in = torch.from_numpy(img).pin_memory()
        h_outs = [[torch.empty(p.out_shape, dtype=torch.float32).pin_memory() for p in plans] for _ in range(2)]
        d_ins = [torch.empty_like(x) for _ in range(2)]
        d_outs = [ys, [torch.empty_like(y) for y in ys]]
        s_up, s_down = torch.cuda.Stream(), torch.cuda.Stream()
        ev = {k: [torch.cuda.Event() for _ in range(2)] for k in ("up", "comp", "down")}
        used = [False, False]

        def e2e_step(k):
            b = k % 2
            with torch.cuda.stream(s_up):
                if used[b]:
                    s_up.wait_event(ev["comp"][b])  # buffer b's previous input is consumed
                d_ins[b].copy_(h_in, non_blocking=True)
                ev["up"][b].record(s_up)
            stream.wait_event(ev["up"][b])
            if used[b]:
                stream.wait_event(ev["down"][b])  # buffer b's previous outputs are downloaded
            with torch.cuda.stream(stream):
                for p, y in zip(plans, d_outs[b]):
                    p.recompute(stream)
                    rs.rs_resample(p.handle, d_ins[b].data_ptr(), y.data_ptr(), stream.cuda_stream)
                ev["comp"][b].record(stream)
            with torch.cuda.stream(s_down):
                s_down.wait_event(ev["comp"][b])
                for y, h in zip(d_outs[b], h_outs[b]):
                    h.copy_(y, non_blocking=True)
                ev["down"][b].record(s_down)
            used[b] = True

        for k in range(2):
            e2e_step(k)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b_ = torch.cuda.Event(enable_timing=True)
        n_e2e = max(3, min(args.steps, 10))
        a.record(s_up)
        for k in range(n_e2e):
            e2e_step(k)
        stream.wait_stream(s_down)
        b_.record(stream)
        torch.cuda.synchronize()
        e_ms = a.elapsed_time(b_) / n_e2e
        e2e = {"value": mpx_step / (e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": in_bytes,
               "d2h_bytes_per_step": sum(n * n * C * 4 for n in outs), "ms_per_step": e_ms,
               "pipelining": "double-buffered steps over upload / compute / download streams"}

    for p in plans:
        p.check()
    # the timed step's outputs on sampled rows, for the oracle leg
    acc = [] if rank == 0 and not args.no_cpu_baseline else None
    if acc is not None:
        import numpy as np

        img64 = img.astype(np.float64)
        for sc, p, y in zip(SCALES, plans, ys):
            rows = sample_rows(y.shape[0])
            acc.append(accuracy_item("C2 %dx%dx%d x%g FP32 (timed step)" % (N_IN, N_IN, C, sc), "f32",
                                     rs.PATHS[p.info.path], lambda: img64, y.shape[0], y.shape[1], "lanczos",
                                     3.0, "mirror", rows, y[rows].double().cpu().numpy(), 2e-6))

    batched = None
    if not args.no_batch:
        batched = batched_section(args, dev, stream, acc)
    clustering = None
    if not args.no_cluster and rank == 0:
        clustering = cluster_section(args, dev, stream)
    c1 = c1_section(dev, stream, acc) if rank == 0 and not args.no_c1 else None
    tc16 = None
    if not args.no_tc and rank == 0:
        tc16 = tc_section(args, dev, stream, acc)
    serving = None
    if not args.no_serve and rank == 0:
        serving = serving_section(args, dev)

    # the CPU-baseline leg: the FP64 oracle timed on the host cores, and the
    # error of every collected result against it
    cpu = None
    accuracy = None
    if rank == 0 and not args.no_cpu_baseline:
        v, cores, sample = cpu_baseline(img, args.cpu_sample_s, outs)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}
        accuracy = oracle_accuracy(acc)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "C2 4096x4096x3 FP32 sinusoids+noise, Lanczos-3 mirror, x1.37 and x0.3",
                       "outputs": ["%dx%dx%d" % (n, n, C) for n in outs],
                       "step": "weight-table + band kernels + resample, both scales (one stream per scale), replayed as one CUDA graph",
                       "autotune_s": round(t_tune, 3),
                       "l2": "input 201 MB > 126 MB L2, no flush",
                       "parallelism": "replicas" if world > 1 else "single",
                       "plans": {str(sc): {"path": rs.PATHS[pl.info.path], "tile": [pl.info.tile_h, pl.info.tile_w],
                                           "group": pl.info.group_h, "band": pl.info.span_h,
                                           "warps_pass1": pl.info.warps_pass1, "stages": pl.info.stages,
                                           "smem": pl.info.smem_bytes, "ctas_per_sm": pl.info.ctas_per_sm}
                                 for sc, pl in zip(SCALES, plans)}},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": recorded_traffic(stream_form(rs, plans[0])),
                         "form": stream_form(rs, plans[0]),
                         "kernel": "resample x1.37 (%s kernel)" % rs.PATHS[plans[0].info.path], "algorithmic_bytes": alg,
                         "avg_kernel_ms": k_avg_s * 1e3, "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)"},
            "roofline_x0.3": {"bound": "hbm", "achieved": alg2 / k2_s / 1e9, "peak": peak, "unit": "GB/s",
                              "frac": alg2 / k2_s / 1e9 / peak, "algorithmic_bytes": alg2,
                              "avg_kernel_ms": k2_s * 1e3, "form": stream_form(rs, plans[1]),
                              "kernel": "resample x0.3 (%s kernel)" % rs.PATHS[plans[1].info.path]},
            "e2e": e2e,
            "gpu_launches": launches_per_step * args.steps,
            "clocks": clocks,
            "cpu_baseline": cpu,
            "accuracy_vs_fp64_oracle": accuracy,
            "batched": batched,
            "clustering": clustering,
            "c1_latency": c1,
            "precision_16bit": tc16,
            "serving": serving,
        }
        print(json.dumps(line), flush=True)
    for p in plans:
        p.close()
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
