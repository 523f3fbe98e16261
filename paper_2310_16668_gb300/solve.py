"""Iterative solves with the skeletonized apply as the matrix-vector product.

The apply costs one pass of Algorithm 2 per product while the plan (tree and
interpolative decompositions) is built once, so an iterative method on
(sigma I + A~) x = b amortises the build over all its iterations and over all
right-hand sides. ``gmres`` runs restarted GMRES on every column of b at once:
each Krylov step is one batched apply of all columns, and the Arnoldi
orthogonalisation (modified Gram-Schmidt, one small least-squares problem per
column) runs on the GPU with torch. No step of the solver leaves the device
except the per-column residual norms read back once per restart cycle.
"""
from __future__ import annotations

import torch

from .api import SkelFMM


def _apply_cols(fmm: SkelFMM, sigma: float, x: torch.Tensor, precision: str, transpose: bool) -> torch.Tensor:
    """(sigma I + A~) x for x of shape (n, m), column by column in one apply."""
    y = fmm.apply_transpose(x, precision) if transpose else fmm.apply(x, precision)
    return y + sigma * x if sigma != 0.0 else y


def gmres(fmm: SkelFMM, b: torch.Tensor, sigma: float = 0.0, precision: str = "fp64", restart: int = 30,
          max_restarts: int = 20, rtol: float = 1e-10, transpose: bool = False, x0: torch.Tensor | None = None):
    """Solve (sigma I + A~) x = b (or its transpose) for every column of b.

    b: CUDA tensor (n,) or (n, m) in the apply's dtype (float64 / complex128
    for precision "fp64"). Returns (x, info) where info holds the relative
    residual of each column and the number of applies performed.
    """
    squeeze = b.dim() == 1
    B = b.reshape(b.shape[0], 1) if squeeze else b
    n, m = B.shape
    dt = B.dtype
    X = torch.zeros_like(B) if x0 is None else (x0.reshape(n, -1).clone())
    bnorm = torch.linalg.vector_norm(B, dim=0).real.clamp_min(torch.finfo(B.real.dtype).tiny)
    applies = 0
    rel = None
    for _ in range(max_restarts):
        R = B - _apply_cols(fmm, sigma, X, precision, transpose)
        applies += 1
        beta = torch.linalg.vector_norm(R, dim=0).real
        rel = beta / bnorm
        if bool((rel <= rtol).all()):
            break
        V = torch.zeros((restart + 1, n, m), dtype=dt, device=B.device)
        H = torch.zeros((m, restart + 1, restart), dtype=dt, device=B.device)
        V[0] = R / beta.clamp_min(torch.finfo(beta.dtype).tiny).to(dt)
        k_used = 0
        for j in range(restart):
            w = _apply_cols(fmm, sigma, V[j], precision, transpose)
            applies += 1
            for i in range(j + 1):                        # modified Gram-Schmidt, all columns at once
                h = torch.sum(V[i].conj() * w, dim=0)
                H[:, i, j] = h
                w = w - V[i] * h
            hn = torch.linalg.vector_norm(w, dim=0).real
            H[:, j + 1, j] = hn.to(dt)
            V[j + 1] = w / hn.clamp_min(torch.finfo(hn.dtype).tiny).to(dt)
            k_used = j + 1
        # per column: min || beta e1 - H y ||, then X += V y
        e1 = torch.zeros((m, k_used + 1, 1), dtype=dt, device=B.device)
        e1[:, 0, 0] = beta.to(dt)
        y = torch.linalg.lstsq(H[:, :k_used + 1, :k_used], e1).solution[:, :, 0]     # (m, k)
        X = X + torch.einsum("kim,mk->im", V[:k_used], y)
    R = B - _apply_cols(fmm, sigma, X, precision, transpose)
    applies += 1
    rel = torch.linalg.vector_norm(R, dim=0).real / bnorm
    info = {"relres": rel.detach().cpu().numpy(), "applies": applies}
    return (X.reshape(n) if squeeze else X), info
