"""Helpers shared by the GPU tests (not collected as tests)."""

import numpy as np

from oracle import dwf as orc
from paper_2602_14454_gb300 import inputs


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def maxrel(a, b):
    """max |a - b| over max |b| (element-wise bound)."""
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


# error bounds written out per precision (FP64 and FP32 from the target, FP16
# from the storage format: 11-bit significands of input, links and output,
# each relative to the per-site maximum, summed over 8 hops and Ls slices)
TOL = {"f64": 1e-12, "f32": 1e-5, "f16": 3e-3}


def make_pair(dims, Ls, M0, mf, b, c, form, alpha, eps=0.5, seed=1, bc=(1, 1, 1, -1), U=None):
    import torch
    from paper_2602_14454_gb300 import dwf
    if U is None:
        U = inputs.random_links(dims, eps, seed)
    op = dwf.Operator(dims, Ls, M0, mf, b, c, form=form, alpha=alpha, bc=bc)
    op.set_gauge(torch.from_numpy(U).cuda())
    ref = orc.DWF(U, dims, Ls, M0, mf, b, c, form=form, alpha=alpha, bc=bc)
    return op, ref


def to_gpu(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def to_np(t):
    return t.cpu().numpy()
