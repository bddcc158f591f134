"""Helpers for the GPU tests: run the CUDA path through the C ABI."""
import numpy as np

torch = None


def _torch():
    global torch
    if torch is None:
        import torch as t
        torch = t
    return torch


def run_gpu(tiling, src, u, tgt=None, levels=0, p=0, eps=1e-6, prec="mixed", f32=False,
            domain=None, keep=False, leaf_size=None):
    """Build + evaluate through the C ABI on cuda:0; returns (phi, plan)."""
    from paper_1204_3105_gb300 import fmm2d

    t = _torch()
    dev = t.device("cuda:0")
    flags = {"fp64": fmm2d.PREC_FP64, "mixed": fmm2d.PREC_MIXED, "tc": fmm2d.PREC_MIXED_TC,
             "hybrid": fmm2d.PREC_HYBRID, "split": fmm2d.PREC_SPLIT}[prec]
    dt = np.float32 if f32 else np.float64
    if f32:
        flags |= fmm2d.IN_F32
    if leaf_size is not None:      # adaptive tree
        flags |= fmm2d.ADAPTIVE
    plan = fmm2d.Plan(tiling, levels=levels, p=p, eps=eps, flags=flags)
    if leaf_size is not None:
        plan.set_leaf_size(leaf_size)
    if domain is not None:
        plan.set_domain(*domain)
    s_d = t.from_numpy(np.ascontiguousarray(src, dt)).to(dev)
    same = tgt is None
    t_d = s_d if same else t.from_numpy(np.ascontiguousarray(tgt, dt)).to(dev)
    n_src = len(src)
    n_tgt = n_src if same else len(tgt)
    u_d = t.from_numpy(np.ascontiguousarray(u, dt)).to(dev)
    out = t.full((max(1, n_tgt),), float("nan"), dtype=t.float64, device=dev)
    plan.build(s_d, n_src, t_d, n_tgt)
    plan.evaluate(u_d, out)
    t.cuda.synchronize()
    phi = out.cpu().numpy()[:n_tgt]
    if keep:
        return phi, plan
    plan.close()
    return phi, None
