"""Run one resampling configuration a few times, for profilers.

    python -m paper_1110_5450_b300.profile_case --size 4096 --channels 3 \
        --dtype bf16 --scale 0.125 --flags FORCE_TC --launches 4

Builds the synthetic sinusoid image of the given size, creates the plan
(optionally autotuned against a cache file), runs the resample `--launches`
times on one stream and checks the plan's device error word.  It prints the
plan's kernel path and configuration, nothing else, so that a profiler's
launch counting (`-s`, `-c`) is predictable: the plan's table kernels first,
then the resample launches.
"""
from __future__ import annotations

import argparse
import os
import sys


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--size", type=int, default=4096)
    ap.add_argument("--channels", type=int, default=3)
    ap.add_argument("--dtype", default="f32", choices=["f32", "f16", "bf16"])
    ap.add_argument("--scale", type=float, default=1.37)
    ap.add_argument("--kernel", default="lanczos")
    ap.add_argument("--param", type=float, default=3.0)
    ap.add_argument("--boundary", default="mirror")
    ap.add_argument("--flags", default="", help="comma-separated RS_* flag names without the prefix")
    ap.add_argument("--launches", type=int, default=4)
    ap.add_argument("--tune-cache", default=None, help="autotune against this cache file first")
    a = ap.parse_args(argv)

    import torch

    here = os.path.dirname(os.path.abspath(__file__))
    sys.path.insert(0, os.path.dirname(here))
    import paper_1110_5450_b300 as rs
    import synth

    dt = {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}[a.dtype]
    flags = 0
    for name in filter(None, a.flags.split(",")):
        flags |= getattr(rs, "RS_" + name.strip().upper())
    img = synth.sinusoids(a.size, a.size, a.channels, seed=synth.SEED_C2)
    x = torch.from_numpy(img).to(dt).cuda()
    p = rs.Plan(a.size, a.size, a.channels, scale=a.scale, kernel=a.kernel, param=a.param,
                boundary=a.boundary, dtype=dt, flags=flags)
    y = torch.empty(p.out_shape, dtype=dt, device="cuda")
    if a.tune_cache:
        p.autotune(x, y, cache_path=a.tune_cache)
    for _ in range(a.launches):
        p(x, out=y)
    torch.cuda.synchronize()
    p.check()
    i = p.info
    print("path", p.path, "tile", [i.tile_h, i.tile_w], "group", i.group_h, "band", [i.span_h, i.span_w],
          "stages", i.stages, "smem", i.smem_bytes, "ctas_per_sm", i.ctas_per_sm)
    p.close()


if __name__ == "__main__":
    main()
