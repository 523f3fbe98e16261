"""The batched GMRES of paper_2310_16668_gb300.solve, on the CPU with a dense
stand-in for the skeletonized apply (same call signature): it must solve
(sigma I + A) x = b for every column, for real and complex systems, and for
the transposed operator."""
import numpy as np
import pytest
import torch

from paper_2310_16668_gb300.solve import gmres


class DenseOperator:
    def __init__(self, A):
        self.A = A

    def apply(self, x, precision="fp64"):
        return self.A @ x

    def apply_transpose(self, x, precision="fp64"):
        return self.A.T @ x


@pytest.mark.parametrize("dtype", [torch.float64, torch.complex128])
@pytest.mark.parametrize("transpose", [False, True])
def test_gmres_dense_standin(dtype, transpose):
    g = torch.Generator().manual_seed(3)
    n, m = 120, 3
    A = torch.randn(n, n, generator=g, dtype=torch.float64) / np.sqrt(n)
    if dtype == torch.complex128:
        A = A + 1j * torch.randn(n, n, generator=g, dtype=torch.float64) / np.sqrt(n)
    b = torch.randn(n, m, generator=g, dtype=torch.float64).to(dtype)
    sigma = 3.0
    x, info = gmres(DenseOperator(A), b, sigma=sigma, restart=25, max_restarts=30, rtol=1e-12, transpose=transpose)
    M = (A.T if transpose else A) + sigma * torch.eye(n, dtype=dtype)
    ref = torch.linalg.solve(M, b)
    assert info["relres"].max() < 1e-11
    assert torch.linalg.vector_norm(x - ref) / torch.linalg.vector_norm(ref) < 1e-10


def test_gmres_single_column_and_restarts():
    g = torch.Generator().manual_seed(5)
    n = 80
    A = torch.randn(n, n, generator=g, dtype=torch.float64) / np.sqrt(n)
    b = torch.randn(n, generator=g, dtype=torch.float64)
    x, info = gmres(DenseOperator(A), b, sigma=2.0, restart=5, max_restarts=60, rtol=1e-12)
    assert x.shape == (n,)
    assert info["relres"].max() < 1e-11
    assert info["applies"] > 10                      # several restart cycles were needed
