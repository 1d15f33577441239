"""The GPU path runs ADMM of Sec. III-D in an algebraically equivalent form with the
shifted multiplier U = Y - theta*A_k(L)V (derived from the Z-, L- and Y-updates using
V V^T = I and A_k^* A_k = k I):

    s_i   = max(0, 1 - 1/||U_i||)                     (Z-update, shrink factor)
    L'    = P_Omega^perp(L + A_k^*(U D V^T)/(k theta)) + P_Omega(M),  D = diag(1 - s)
    U'    = U D - A_k((theta + theta') L' - theta L) V

This test runs that form in FP64 and checks it reproduces the paper-order oracle
iterate, so the rewrite the kernels rely on is pinned to the paper's algorithm.
"""
import numpy as np
import pytest

from oracle import icnnm_oracle as O
from paper_2604_17001_gb300 import synth


def shifted_dual_solve(M, mask, V, kdims, iters, lam=np.inf, rho=1.1, theta_max=1e10):
    T, H, W = M.shape
    k = V.shape[0]
    msk = mask.astype(bool)
    L = np.where(msk, M, 0.0).astype(np.float64)
    theta = O.theta0_default(M, mask, V, kdims)
    U = -theta * O.conv_matrix_times(L, V, kdims)
    for _ in range(iters):
        n = np.linalg.norm(U, axis=0)
        s = np.where(n > 1, 1 - 1 / np.where(n > 0, n, 1), 0.0)
        D = 1 - s
        Delta = O.adjoint_of_product(U * D[None, :], V, (T, H, W), kdims)
        if np.isinf(lam):
            Ln = np.where(msk, M, L + Delta / (k * theta))
        else:
            Ln = (Delta / k + theta * L + lam * np.where(msk, M, 0)) / (lam * msk + theta)
        thn = min(rho * theta, theta_max)
        U = U * D[None, :] - O.conv_matrix_times((theta + thn) * Ln - theta * L, V, kdims)
        L, theta = Ln, thn
    return L


@pytest.mark.parametrize("lam", [np.inf, 1000.0])
def test_shifted_dual_form_equals_paper_order(lam):
    w = synth.workload(1, dims=(10, 12, 6), n_ref=3)
    kd = (3, 3, 2)
    V, _ = O.learn_V(w["refs"], kd)
    Lo, _ = O.icnnm_solve(w["M"], w["mask"], V, kd, lam=lam, max_iters=60)
    Ls = shifted_dual_solve(w["M"].astype(np.float64), w["mask"], V, kd, 60, lam=lam)
    assert np.linalg.norm(Ls - Lo) / np.linalg.norm(Lo) < 1e-10
