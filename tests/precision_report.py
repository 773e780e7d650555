"""Error of the CUDA path against the FP64 oracle per storage type (needs a GPU).

    python tests/precision_report.py [--rows 16]

Prints a markdown table: for every configuration, the largest absolute error
and the RMS error of the device result against the oracle fed the same
quantised input (full outputs for the small images, sampled rows of the
4096x4096x3 ones, every 64th image of the uneven FP16 batch).
"""
from __future__ import annotations

import argparse
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

import oracle  # noqa: E402
import synth  # noqa: E402
from gpu_helpers import quantise, torch_dtype  # noqa: E402


def _rows(n, k, seed=7):
    g = np.random.default_rng(seed)
    return sorted(set([0, n // 2, n - 1]) | set(int(r) for r in g.integers(0, n, k)))


def _stats(got, want):
    d = np.abs(got - want)
    return float(d.max()), float(np.sqrt(np.mean(d * d)))


def full_image(rs, label, img, dt, oh, ow, kernel, boundary, param, flags=0):
    import torch

    t, exact = quantise(img, dt)
    H, W, C = img.shape
    p = rs.Plan(H, W, C, oh, ow, kernel=kernel, param=param, boundary=boundary, dtype=torch_dtype(dt),
                flags=flags)
    y = p(t.cuda())
    torch.cuda.synchronize()
    p.check()
    path = p.path
    p.close()
    want = oracle.resample(exact, oh, ow, kernel, boundary, param=param)
    return (label, dt, path) + _stats(y.double().cpu().numpy(), want)


def sampled(rs, label, img, dt, scale, flags, nrows):
    import torch

    t, exact = quantise(img, dt)
    H, W, C = img.shape
    p = rs.Plan(H, W, C, scale=scale, kernel="lanczos", param=3.0, boundary="mirror", dtype=torch_dtype(dt),
                flags=flags)
    y = p(t.cuda())
    torch.cuda.synchronize()
    p.check()
    path, oh, ow = p.path, p.info.out_h, p.info.out_w
    p.close()
    got = y.double().cpu().numpy()
    mx, sq, n = 0.0, 0.0, 0
    for r in _rows(oh, nrows):
        want = oracle.resample(exact, oh, ow, "lanczos", "mirror", param=3.0, rows=(r, r + 1))[0]
        d = np.abs(got[r] - want)
        mx = max(mx, float(d.max()))
        sq += float((d * d).sum())
        n += d.size
    return (label, dt, path, mx, float(np.sqrt(sq / n)))


def batch_rows(rs, n_images):
    import torch

    specs = synth.batch_specs(n_images)
    ins, exact, pitches = [], [], []
    for sp in specs:
        img = synth.sinusoids(sp.in_h, sp.in_w, 1, seed=sp.seed)
        t16 = torch.from_numpy(img).to(torch.float16)
        pitch = (sp.in_w + 7) // 8 * 8
        buf = torch.zeros((sp.in_h, pitch), dtype=torch.float16, device="cuda")
        buf[:, :sp.in_w] = t16[:, :, 0].cuda()
        ins.append(buf)
        pitches.append(pitch)
        exact.append(t16.double().numpy())
    b = rs.Batch([dict(in_h=sp.in_h, in_w=sp.in_w, scale=sp.scale, kernel=sp.kernel, param=sp.param,
                       boundary="mirror") for sp in specs], channels=1, dtype=torch.float16, in_pitches=pitches)
    outs = [torch.empty((rs.out_size(sp.in_h, sp.scale), rs.out_size(sp.in_w, sp.scale), 1),
                        dtype=torch.float16, device="cuda") for sp in specs]
    b(ins, outs)
    torch.cuda.synchronize()
    b.close()
    mx, rms = 0.0, []
    for i in range(0, len(specs), 64):
        sp = specs[i]
        got = outs[i].double().cpu().numpy()
        want = oracle.resample(exact[i], got.shape[0], got.shape[1], sp.kernel, "mirror", param=sp.param)
        m, r = _stats(got, want)
        mx = max(mx, m)
        rms.append(r)
    return ("%d uneven images, every 64th" % n_images, "f16", "batch", mx, float(np.mean(rms)))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--rows", type=int, default=16, help="sampled output rows per 4096x4096 case")
    ap.add_argument("--batch-n", type=int, default=512)
    a = ap.parse_args()
    import paper_1110_5450_b300 as rs

    rows = []
    c1 = synth.uniform(256, 256, 1, seed=synth.SEED_C1)
    rows.append(full_image(rs, "256x256 x2 Keys clamp (fused)", c1, "f64", 512, 512, "cubic", "clamp", -0.5))
    rows.append(full_image(rs, "256x256 x2 Keys clamp (two-pass)", c1, "f64", 512, 512, "cubic", "clamp", -0.5,
                           rs.RS_TWO_PASS))
    rows.append(full_image(rs, "256x256 x2 Keys clamp", c1, "f32", 512, 512, "cubic", "clamp", -0.5))
    big = synth.sinusoids(4096, 4096, 3, seed=synth.SEED_C2)
    tile = rs.RS_FORCE_SIMT | rs.RS_NO_STREAM
    for s in (1.37, 0.3):
        rows.append(sampled(rs, "4096x4096x3 x%g Lanczos-3" % s, big, "f32", s, 0, a.rows))
        rows.append(sampled(rs, "4096x4096x3 x%g Lanczos-3" % s, big, "f32", s, tile, a.rows))
    for dt in ("bf16", "f16"):
        for s in (1.37, 0.3, 0.125):
            # the default kernel, then the other kernels that apply
            rows.append(sampled(rs, "4096x4096x3 x%g Lanczos-3" % s, big, dt, s, 0, a.rows))
            rows.append(sampled(rs, "4096x4096x3 x%g Lanczos-3" % s, big, dt, s, tile, a.rows))
            if s == 0.3:
                rows.append(sampled(rs, "4096x4096x3 x%g Lanczos-3" % s, big, dt, s, rs.RS_FORCE_STREAM, a.rows))
    rows.append(batch_rows(rs, a.batch_n))
    print("| configuration | storage | path | max abs error | RMS error |")
    print("|---|---|---|---|---|")
    for label, dt, path, mx, rms in rows:
        print("| %s | %s | %s | %.3g | %.3g |" % (label, dt, path, mx, rms))


if __name__ == "__main__":
    main()
