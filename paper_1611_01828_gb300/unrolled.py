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


def _f64(t):
    return t.detach().to(torch.float64).contiguous()


class UnrolledHSDE(torch.autograd.Function):
    """(c, b) -> (x_K, y_K, tau_K, kappa_K) after K iterations from the standard start.

    CUDA tensors on the handle's GPU go to the library as device addresses
    (no host copy of C, b, the outputs or the upstream gradients); CPU
    tensors go as host arrays."""

    @staticmethod
    def forward(ctx, c, b, handle, K: int, ckpt: int):
        sz = handle.sizes[0]
        ctx.handle = handle
        ctx.meta = (c.device, c.dtype, b.device, b.dtype)
        if c.is_cuda:
            c64, b64 = _f64(c), _f64(b.to(c.device))
            x = torch.empty(sz.N, dtype=torch.float64, device=c.device)
            y = torch.empty(sz.m, dtype=torch.float64, device=c.device)
            torch.cuda.current_stream(c.device).synchronize()
            handle.hsde_set_data(0, c64.data_ptr(), b64.data_ptr())
            _, _, tau, kappa = handle.hsde_unrolled_forward(K, ckpt, x=x.data_ptr(), y=y.data_ptr())
        else:
            handle.hsde_set_data(0, _f64(c).numpy(), _f64(b).numpy())
            xh, yh, tau, kappa = handle.hsde_unrolled_forward(K, ckpt)
            x, y = torch.from_numpy(xh), torch.from_numpy(yh)
        sc = lambda v: torch.tensor(v, dtype=c.dtype, device=c.device)
        return x.to(c.dtype), y.to(device=b.device, dtype=b.dtype), sc(tau), sc(kappa)

    @staticmethod
    def backward(ctx, gx, gy, gtau, gkappa):
        cdev, cdt, bdev, bdt = ctx.meta
        sz = ctx.handle.sizes[0]
        taubar = float(gtau) if gtau is not None else 0.0
        kappabar = float(gkappa) if gkappa is not None else 0.0
        if cdev.type == "cuda":
            xb = _f64(gx) if gx is not None else None
            yb = _f64(gy.to(cdev)) if gy is not None else None
            gC = torch.empty(sz.N, dtype=torch.float64, device=cdev)
            gb = torch.empty(sz.m, dtype=torch.float64, device=cdev)
            torch.cuda.current_stream(cdev).synchronize()
            ctx.handle.hsde_unrolled_backward(xb.data_ptr() if xb is not None else None,
                                              yb.data_ptr() if yb is not None else None,
                                              taubar, kappabar, gC=gC.data_ptr(), gb=gb.data_ptr())
        else:
            xb = _f64(gx).numpy() if gx is not None else None
            yb = _f64(gy).numpy() if gy is not None else None
            gCh, gbh = ctx.handle.hsde_unrolled_backward(xb, yb, taubar, kappabar)
            gC, gb = torch.from_numpy(gCh), torch.from_numpy(gbh)
        return gC.to(cdt), gb.to(device=bdev, dtype=bdt), None, None, None


def unrolled_objective(c, b, handle, K: int, ckpt: int = 20, weights=None):
    """f(C, b) = c^T x_K / (tau_K + kappa_K) (full-vec inner product), differentiable in c and b."""
    if weights is None:
        weights = torch.as_tensor(pattern_weights(handle), dtype=c.dtype, device=c.device)
    x, y, tau, kappa = UnrolledHSDE.apply(c, b, handle, K, ckpt)
    return (weights * c * x).sum() / (tau + kappa)
