"""Helpers shared by the GPU tests: column-major device buffers and a handle wrapper."""
import numpy as np

import paper_1602_01768_gb300._binding as B


def to_dev(A, dtype):
    """Column-major copy of a 2-D numpy array in a CUDA tensor (ld = rows)."""
    import torch

    A = np.asarray(A)
    t = torch.from_numpy(np.ascontiguousarray(A.T)).to(dtype=dtype, device="cuda")
    return t


def empty_dev(rows, cols, dtype):
    import torch

    return torch.zeros(cols, rows, dtype=dtype, device="cuda")


def from_dev(t):
    """numpy float64 matrix from a column-major CUDA tensor made by to_dev/empty_dev."""
    import torch

    torch.cuda.synchronize()
    return t.detach().double().cpu().numpy().T.copy()


def torch_dtype(prec):
    import torch

    return torch.float64 if prec == B.RB_FP64 else torch.float32


def stream_ptr():
    import torch

    return torch.cuda.current_stream().cuda_stream


def export(h, n, prec, what):
    out = empty_dev(n, n, torch_dtype(prec))
    B.rbfgs_export(h, what, out.data_ptr(), n)
    return from_dev(out)


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
