"""torch.autograd.Function for K unrolled HSDE-ADMM iterations.

Forward runs the iterations inside libhsde (hsde_unrolled_forward) for data
(C on the pattern, b) given as tensors; backward calls the library's reverse
sweep (hsde_unrolled_backward: Daleckii-Krein adjoint of the clique
projections, adjoint affine solve with the cached factor, checkpointing).
This module only moves values between tensors and the C-ABI.

The handle must run the literal iteration on the data as given: create it
with ``**LITERAL`` (alpha = 1, no data scaling), because the scaling factors
depend on c and b and the library differentiates the unscaled steps.
"""
from __future__ import annotations

import numpy as np
import torch

from . import hsde

# options of a handle that can be differentiated (the library refuses others)
LITERAL = dict(alpha=1.0, scaling=0)


def pattern_weights(handle) -> np.ndarray:
    """1 for diagonal pattern entries, 2 off the diagonal (full-vec inner products)."""
    st = handle.hsde_get_structure(0)
    col = np.repeat(np.arange(st["pat_colptr"].shape[0] - 1), np.diff(st["pat_colptr"]))
    return np.where(st["pat_row"] == col, 1.0, 2.0)


def pattern_values(handle, rows, cols, vals) -> np.ndarray:
    """Scatter a lower-triangle COO matrix onto the handle's pattern order."""
    st = handle.hsde_get_structure(0)
    n = st["pat_colptr"].shape[0] - 1
    col = np.repeat(np.arange(n), np.diff(st["pat_colptr"]))
    key_pat = col.astype(np.int64) * n + st["pat_row"]
    key = np.asarray(cols, np.int64) * n + np.asarray(rows, np.int64)
    pos = np.searchsorted(key_pat, key)
    if np.any(pos >= key_pat.shape[0]) or np.any(key_pat[np.minimum(pos, key_pat.shape[0] - 1)] != key):
        raise ValueError("entry outside the pattern")
    out = np.zeros(key_pat.shape[0])
    out[pos] = vals
    return out


class UnrolledHSDE(torch.autograd.Function):
    """(c, b) -> (x_K, y_K, tau_K, kappa_K) after K iterations from the standard start."""

    @staticmethod
    def forward(ctx, c, b, handle, K: int, ckpt: int):
        handle.hsde_set_data(0, c.detach().to("cpu", torch.float64).numpy(),
                             b.detach().to("cpu", torch.float64).numpy())
        x, y, tau, kappa = handle.hsde_unrolled_forward(K, ckpt)
        ctx.handle = handle
        ctx.meta = (c.device, c.dtype, b.device, b.dtype)
        f = lambda a, d, t: torch.as_tensor(np.asarray(a), dtype=t, device=d)
        return f(x, c.device, c.dtype), f(y, b.device, b.dtype), f(tau, c.device, c.dtype), f(kappa, c.device, c.dtype)

    @staticmethod
    def backward(ctx, gx, gy, gtau, gkappa):
        cdev, cdt, bdev, bdt = ctx.meta
        sz = ctx.handle.sizes[0]
        np_ = lambda t, n: (t.detach().to("cpu", torch.float64).numpy() if t is not None else np.zeros(n))
        gC, gb = ctx.handle.hsde_unrolled_backward(np_(gx, sz.N), np_(gy, sz.m),
                                                   float(gtau) if gtau is not None else 0.0,
                                                   float(gkappa) if gkappa is not None else 0.0)
        return (torch.as_tensor(gC, dtype=cdt, device=cdev), torch.as_tensor(gb, dtype=bdt, device=bdev),
                None, None, None)


def unrolled_objective(c, b, handle, K: int, ckpt: int = 20, weights=None):
    """f(C, b) = c^T x_K / (tau_K + kappa_K) (full-vec inner product), differentiable in c and b."""
    if weights is None:
        weights = torch.as_tensor(pattern_weights(handle), dtype=c.dtype, device=c.device)
    x, y, tau, kappa = UnrolledHSDE.apply(c, b, handle, K, ckpt)
    return (weights * c * x).sum() / (tau + kappa)
