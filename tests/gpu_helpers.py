"""Shared helpers of the GPU parity tests: run the CUDA path through the C
ABI binding and quantise inputs exactly the way the device sees them."""
from __future__ import annotations

import numpy as np

TOL = {"f64": 1e-12, "f32": 2e-6, "f16": 2e-3, "bf16": 1e-2}


def torch_dtype(name):
    import torch

    return {"f64": torch.float64, "f32": torch.float32, "f16": torch.float16,
            "bf16": torch.bfloat16}[name]


def quantise(img: np.ndarray, dt: str):
    """(torch CPU tensor in dtype, exact float64 numpy copy of it)."""
    import torch

    t = torch.from_numpy(np.ascontiguousarray(img)).to(torch_dtype(dt))
    return t, t.to(torch.float64).numpy()


def run_gpu(t_in, out_h, out_w, kernel, boundary, param=None, flags=0, scale=None):
    """Resample a CPU tensor (H, W, C) on cuda:0; returns (float64 numpy, plan info)."""
    import torch

    import paper_1110_5450_b300 as rs

    H, W, C = t_in.shape
    x = t_in.to("cuda").contiguous()
    if scale is not None:
        p = rs.Plan(H, W, C, scale=scale, kernel=kernel, param=param, boundary=boundary,
                    dtype=x.dtype, flags=flags)
    else:
        p = rs.Plan(H, W, C, out_h, out_w, kernel=kernel, param=param, boundary=boundary,
                    dtype=x.dtype, flags=flags)
    y = p(x)
    torch.cuda.synchronize()
    p.check()
    info = p.info
    res = y.to(torch.float64).cpu().numpy()
    p.close()
    return res, info
