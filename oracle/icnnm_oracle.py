"""FP64 CPU oracle for ICNNM (Inductive Convolution Nuclear Norm Minimization).

TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the benchmark's
CPU-baseline leg may import this module. The product path (the CUDA library and
its Python binding) never imports, calls or links anything under ``oracle/``; the
two share no code. Inputs come from the seeded generators, never from the GPU.

Everything is plain numpy in float64, written from the paper's definitions and
algorithm, in the paper's order and notation. Library primitives used as steps:
``numpy`` matmul, ``numpy.linalg.eigh`` / ``svd`` and ``np.bincount`` (the
transpose of a gather). There is no fusion or reordering beyond what the
definitions state; the only structure added is splitting the rows of the
convolution matrix into chunks, to bound memory.

Conventions (a reading; the paper's vec() is MATLAB's):
  * a tensor of dims (H, W, T) is a numpy array of shape (T, H, W); the voxel index
    is i = (t*H + h)*W + w; 2-D images use T = 1 and a kernel with k3 = 1;
  * kernel dims (k1, k2, k3) run along (h, w, t); tap index s = (st*k1 + sh)*k2 + sw;
  * V (the paper's K) is a k x k array whose column i is vec(kappa_i), indexed by tap.

Parity pins (tests/test_oracle_pins.py) cover every function below; the full
multi-iteration ADMM iterate has no printed worked example in the paper, so its
value is pinned only through its steps and the properties the paper states.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "conv_index", "conv_matrix", "conv_matrix_times", "adjoint", "adjoint_of_product",
    "P_Omega", "column_norms", "norm_21", "gram", "learn_V", "canonical_signs",
    "prox_21", "icnnm_init", "icnnm_iteration", "icnnm_solve", "cnnm_solve",
    "relative_eigvals", "spectral_correlation", "relative_rank", "active_coherence",
    "theta0_default", "primal_residual",
]

CHUNK_ROWS = 8192
_IDX_CACHE: dict = {}
_IDX_CACHE_MAX_BYTES = 4 << 30


def _chunk_index(dims_thw, kdims, r0, r1):
    """conv_index for rows [r0, r1), memoised (int32) so that repeated products with
    the same tensor shape do not recompute the index arithmetic."""
    key = (tuple(dims_thw), tuple(kdims), r0, r1)
    idx = _IDX_CACHE.get(key)
    if idx is None:
        idx = conv_index(dims_thw, kdims, np.arange(r0, r1))
        if idx.size * 4 + sum(v.nbytes for v in _IDX_CACHE.values()) <= _IDX_CACHE_MAX_BYTES:
            idx = idx.astype(np.int32)
            _IDX_CACHE[key] = idx
    return idx


# ----------------------------------------------------------------------------------
# Sec. II-B: circular convolution and the convolution matrix A_k
# ----------------------------------------------------------------------------------
def _shape3(a: np.ndarray) -> tuple[int, int, int]:
    if a.ndim == 2:
        return 1, a.shape[0], a.shape[1]
    T, H, W = a.shape
    return T, H, W


def conv_index(dims_thw: tuple[int, int, int], kdims: tuple[int, int, int],
               rows: np.ndarray | None = None) -> np.ndarray:
    """Index array of A_k: idx[r, s] = linear index of the voxel (i - s) mod dims.

    Sec. II-B, the entry formula of L * X: [L * X]_i = sum_s [L]_{i-s} [X]_s, where an
    index i_j - s_j below range wraps by +m_j (circular convolution). With Eq. (ak),
    vec(L * X) = A_k(L) vec(X), row i of A_k(L) holds [L]_{i-s} for every tap s.
    Indices are 0-based here (the paper is 1-based; the two differ by a cyclic shift
    of the rows of A_k, which changes neither A_k^T A_k nor any column norm).
    """
    T, H, W = dims_thw
    k1, k2, k3 = kdims
    m = T * H * W
    if rows is None:
        rows = np.arange(m)
    rows = np.asarray(rows, dtype=np.int64)
    t = rows // (H * W)
    h = (rows // W) % H
    w = rows % W
    st, sh, sw = np.meshgrid(np.arange(k3), np.arange(k1), np.arange(k2), indexing="ij")
    st, sh, sw = st.ravel(), sh.ravel(), sw.ravel()          # tap s = (st*k1 + sh)*k2 + sw
    tt = (t[:, None] - st[None, :]) % T
    hh = (h[:, None] - sh[None, :]) % H
    ww = (w[:, None] - sw[None, :]) % W
    return (tt * H + hh) * W + ww


def conv_matrix(L: np.ndarray, kdims, rows=None) -> np.ndarray:
    """A_k(L) (or the given rows of it), m x k, Eq. (ak)."""
    T, H, W = _shape3(L)
    idx = conv_index((T, H, W), kdims, rows)
    return np.asarray(L, dtype=np.float64).ravel()[idx]


def conv_matrix_times(L: np.ndarray, V: np.ndarray, kdims) -> np.ndarray:
    """A_k(L) @ V (m x k'), forming the rows of A_k(L) chunk by chunk."""
    T, H, W = _shape3(L)
    m = T * H * W
    V = np.asarray(V, dtype=np.float64)
    out = np.empty((m, V.shape[1]), dtype=np.float64)
    Lf = np.asarray(L, dtype=np.float64).ravel()
    for r0 in range(0, m, CHUNK_ROWS):
        r1 = min(m, r0 + CHUNK_ROWS)
        out[r0:r1] = Lf[_chunk_index((T, H, W), kdims, r0, r1)] @ V
    return out


def adjoint(G: np.ndarray, dims_thw, kdims) -> np.ndarray:
    """Hermitian adjoint A_k^*: R^{m x k} -> tensors (Sec. III-D names it).

    A_k^* is the transpose of the linear map L -> A_k(L). Since entry (i, s) of
    A_k(L) is [L]_{idx[i, s]}, the transpose adds G[i, s] into voxel idx[i, s]:
    [A_k^*(G)]_j = sum_s G[(j + s) mod m, s].
    """
    T, H, W = dims_thw
    m = T * H * W
    out = np.zeros(m, dtype=np.float64)
    G = np.asarray(G, dtype=np.float64)
    for r0 in range(0, m, CHUNK_ROWS):
        rows = np.arange(r0, min(m, r0 + CHUNK_ROWS))
        idx = conv_index(dims_thw, kdims, rows)
        out += np.bincount(idx.ravel(), weights=G[rows].ravel(), minlength=m)
    return out.reshape(T, H, W)


def adjoint_of_product(Wm: np.ndarray, V: np.ndarray, dims_thw, kdims) -> np.ndarray:
    """A_k^*(Wm V^T), the adjoint applied to an m x k matrix times V^T (Sec. III-D,
    L-update numerator)."""
    T, H, W = dims_thw
    m = T * H * W
    out = np.zeros(m, dtype=np.float64)
    Vt = np.asarray(V, dtype=np.float64).T
    for r0 in range(0, m, CHUNK_ROWS):
        r1 = min(m, r0 + CHUNK_ROWS)
        idx = _chunk_index(dims_thw, kdims, r0, r1)
        out += np.bincount(idx.ravel(), weights=(Wm[r0:r1] @ Vt).ravel(), minlength=m)
    return out.reshape(T, H, W)


# ----------------------------------------------------------------------------------
# Sec. II-A notation: projection onto Omega and matrix norms
# ----------------------------------------------------------------------------------
def P_Omega(L: np.ndarray, mask: np.ndarray) -> np.ndarray:
    """[P_Omega(L)]_i = [L]_i if i in Omega else 0 (Sec. II-A)."""
    return np.where(np.asarray(mask).astype(bool), L, 0.0)


def column_norms(Mat: np.ndarray) -> np.ndarray:
    """l2 norm of each column."""
    return np.sqrt(np.sum(np.asarray(Mat, dtype=np.float64) ** 2, axis=0))


def norm_21(Mat: np.ndarray) -> float:
    """||M||_{2,1}: sum of the l2 norms of the columns (Sec. II-A)."""
    return float(np.sum(column_norms(Mat)))


# ----------------------------------------------------------------------------------
# Sec. III-C: learning the convolution eigenvectors from reference tensors
# ----------------------------------------------------------------------------------
def gram(refs, kdims) -> np.ndarray:
    """A^T A for A = [A_k(L_1); ...; A_k(L_b)] (Eq. (A)), accumulated as
    sum_j A_k(L_j)^T A_k(L_j) over row chunks. Reference tensors may differ in dims
    as long as every dim is at least the kernel's."""
    k = int(np.prod(kdims))
    Gm = np.zeros((k, k), dtype=np.float64)
    for Lj in refs:
        T, H, W = _shape3(Lj)
        m = T * H * W
        Lf = np.asarray(Lj, dtype=np.float64).ravel()
        for r0 in range(0, m, CHUNK_ROWS):
            A = Lf[_chunk_index((T, H, W), kdims, r0, min(m, r0 + CHUNK_ROWS))]
            Gm += A.T @ A
    return Gm


def canonical_signs(V: np.ndarray) -> np.ndarray:
    """Sign convention (a reading; the paper fixes none): in each column the entry of
    largest magnitude is made positive (ties: the lowest index)."""
    V = np.array(V, dtype=np.float64, copy=True)
    for i in range(V.shape[1]):
        j = int(np.argmax(np.abs(V[:, i])))
        if V[j, i] < 0:
            V[:, i] = -V[:, i]
    return V


def learn_V(refs, kdims):
    """Convolution eigenvectors of a tensor ensemble (Sec. III-C, Definition 3, Eq. (A)).

    The eigenvectors of the ensemble are the right singular vectors of A, i.e. the
    eigenvectors of A^T A, ordered by decreasing eigenvalue sigma_i (which is the
    maximised value sum_j ||L_j * X||_F^2 of the definition). Returns (V, sigma).
    """
    Gm = gram(refs, kdims)
    evals, evecs = np.linalg.eigh(Gm)
    order = np.argsort(-evals, kind="stable")
    return canonical_signs(evecs[:, order]), evals[order]


# ----------------------------------------------------------------------------------
# Sec. III-A definitions: relative convolution eigenvalues, rank, alpha_K
# ----------------------------------------------------------------------------------
def relative_eigvals(L0, V, kdims) -> np.ndarray:
    """sigma_i^K(L0) = ||L0 * kappa_i||_F = ||A_k(L0) v_i||_2 (Definition 2)."""
    return column_norms(conv_matrix_times(L0, V, kdims))


def relative_rank(L0, V, kdims, tol=1e-9) -> int:
    """r_K(L0) = ||A_k(L0) K||_{2,0}, number of nonzero columns (Eq. (rkL0))."""
    s = relative_eigvals(L0, V, kdims)
    return int(np.sum(s > tol * max(1.0, s.max())))


def spectral_correlation(L0, V, kdims, tol=1e-9) -> float:
    """alpha_K(L0) = ||A_k(L0) K D|| with D = diag(1/sigma_i^K) on the column support
    and 0 elsewhere (Eq. (alphaK))."""
    Q = conv_matrix_times(L0, V, kdims)
    s = column_norms(Q)
    sup = s > tol * max(1.0, s.max())
    d = np.where(sup, 1.0 / np.where(sup, s, 1.0), 0.0)
    return float(np.linalg.norm(Q * d[None, :], 2))


def active_coherence(L0, V, kdims, tol=1e-9) -> float:
    """mu_K^I = mu_1(K_I), the first coherence (Eq. (coherence)) of the active submatrix
    K_I, the columns of K on the column support I of A_k(L0)K (Sec. III-A). K_I has
    orthonormal columns, so its skinny SVD has left factor K_I itself and
    mu_1(K_I) = (k / r) max_s ||[K_I]_{s,:}||^2. Zero when I is empty."""
    s = relative_eigvals(L0, V, kdims)
    sup = s > tol * max(1.0, s.max())
    r = int(sup.sum())
    if r == 0:
        return 0.0
    U, sv, _ = np.linalg.svd(V[:, sup], full_matrices=False)
    Ur = U[:, sv > 1e-12]
    return float(V.shape[0] / Ur.shape[1] * np.max(np.sum(Ur * Ur, axis=1)))


# ----------------------------------------------------------------------------------
# Sec. III-D: ADMM for  min ||A_k(L)K||_{2,1} + (lambda k / 2)||P_Omega(L - M)||_F^2
# ----------------------------------------------------------------------------------
def prox_21(R: np.ndarray, tau: float) -> np.ndarray:
    """argmin_Z tau*||Z||_{2,1} + 1/2 ||Z - R||_F^2, column-wise shrinkage
    Z_i = max(0, 1 - tau/||R_i||) R_i (Z-update of Sec. III-D; the closed form the
    paper cites). A zero column stays zero."""
    n = column_norms(R)
    scale = np.where(n > tau, 1.0 - tau / np.where(n > 0, n, 1.0), 0.0)
    return R * scale[None, :]


def primal_residual(Z, Q, L, k) -> float:
    """Stopping quantity (a reading; the paper states no stopping rule): the primal
    residual of the split Z = A_k(L)K, ||Z - A_k(L)K||_F, relative to
    ||A_k(L)K||_F = sqrt(k)||L||_F (A_k^*A_k = kI and K orthogonal), with Q = A_k(L)K
    of the current L."""
    return float(np.linalg.norm(Z - Q) / (np.sqrt(k) * max(np.linalg.norm(L), 1e-300)))


def theta0_default(M, mask, V, kdims) -> float:
    """Initial penalty (a reading; the paper is silent): 1/||A_k(P_Omega M) V||_{2,inf}."""
    Q0 = conv_matrix_times(P_Omega(M, mask), V, kdims)
    return 1.0 / float(column_norms(Q0).max())


def icnnm_init(M, mask, V, kdims, theta0=None):
    """Initial state (a reading): L0 = P_Omega(M), Y0 = 0, theta0 as above."""
    L = P_Omega(np.asarray(M, dtype=np.float64), mask)
    T, H, W = _shape3(L)
    k = int(np.prod(kdims))
    Y = np.zeros((T * H * W, V.shape[1]), dtype=np.float64)
    th = theta0_default(M, mask, V, kdims) if theta0 is None or theta0 <= 0 else float(theta0)
    return L, Y, th


def icnnm_iteration(L, Y, theta, M, mask, V, kdims, lam=np.inf, Q=None):
    """One ADMM iteration in the paper's order (Sec. III-D): Z, then L, then Y.

    Z = prox_{(1/theta)||.||_{2,1}}(A_k(L)K - Y/theta)
    L = (A_k^*((Y + theta Z) K^T)/k + lambda P_Omega(M)) / (lambda Theta_Omega + theta)
    Y = Y + theta (Z - A_k(L) K)          (the multiplier step of ADMM; the sign
                                           follows the Lagrangian's <Z - A_k(L)K, Y>)
    With lambda = inf the L-update reads P_Omega^perp(A_k^*(.)/(k theta)) + P_Omega(M),
    i.e. the observed entries are restored exactly (the constraint of Eq.
    (InductiveCNNM)). Returns (L_new, Y_new, Z, Q_new) with Q_new = A_k(L_new)K.
    """
    T, H, W = _shape3(L)
    dims = (T, H, W)
    k = int(np.prod(kdims))
    msk = np.asarray(mask).astype(bool).reshape(T, H, W)
    Mf = np.asarray(M, dtype=np.float64).reshape(T, H, W)
    if Q is None:
        Q = conv_matrix_times(L, V, kdims)
    Z = prox_21(Q - Y / theta, 1.0 / theta)
    num = adjoint_of_product(Y + theta * Z, V, dims, kdims) / k
    if np.isinf(lam):
        Lnew = np.where(msk, Mf, num / theta)
    else:
        Lnew = (num + lam * np.where(msk, Mf, 0.0)) / (lam * msk + theta)
    Qnew = conv_matrix_times(Lnew, V, kdims)
    Ynew = Y + theta * (Z - Qnew)
    return Lnew, Ynew, Z, Qnew


def icnnm_solve(M, mask, V, kdims, lam=np.inf, theta0=None, rho=1.1, theta_max=1e10,
                max_iters=100, tol=0.0, check_every=1, return_history=False, record_every=0):
    """ICNNM by ADMM (Sec. III-D) from the initial state of ``icnnm_init``.

    After each iteration theta <- min(rho*theta, theta_max) (a reading of "updated
    according to the instructions of ADMM"). If tol > 0, every ``check_every``
    iterations the run stops once ||Z - A_k(L)K||_F / (sqrt(k)||L||_F) <= tol.
    Returns (L, stats) with stats = dict(iters, residual, objective, theta); with
    ``record_every`` > 0, stats["checkpoints"] maps every iteration count that is a
    multiple of it to (L, residual) after that iteration (bookkeeping only).
    """
    V = np.asarray(V, dtype=np.float64)
    k = int(np.prod(kdims))
    L, Y, theta = icnnm_init(M, mask, V, kdims, theta0)
    Q = conv_matrix_times(L, V, kdims)
    hist = []
    ckpt = {}
    it = 0
    resid = float("nan")
    for it in range(1, max_iters + 1):
        L, Y, Z, Q = icnnm_iteration(L, Y, theta, M, mask, V, kdims, lam, Q)
        theta = min(rho * theta, theta_max)
        if return_history:
            hist.append(dict(objective=norm_21(Q), L=L.copy()))
        if record_every and it % record_every == 0:
            ckpt[it] = (L.copy(), primal_residual(Z, Q, L, k))
        if tol > 0 and it % check_every == 0:
            resid = primal_residual(Z, Q, L, k)
            if resid <= tol:
                break
    if not (tol > 0 and it % check_every == 0):
        resid = primal_residual(Z, Q, L, k)
    stats = dict(iters=it, residual=resid, objective=norm_21(Q), theta=theta)
    if return_history:
        stats["history"] = hist
    if record_every:
        stats["checkpoints"] = ckpt
    return L, stats


# ----------------------------------------------------------------------------------
# Eq. (cnnm): CNNM by the same ADMM with singular-value thresholding (tiny inputs)
# ----------------------------------------------------------------------------------
def cnnm_solve(M, mask, kdims, rho=1.1, theta_max=1e10, max_iters=300, theta0=None):
    """min ||A_k(L)||_* s.t. P_Omega(L) = P_Omega(M) (Eq. (cnnm)), solved by the same
    augmented-Lagrangian scheme: Z = SVT_{1/theta}(A_k(L) - Y/theta),
    L = P_Omega^perp(A_k^*(Y + theta Z)/(k theta)) + P_Omega(M),
    Y = Y + theta (Z - A_k(L)). For tiny inputs only (dense SVD each step)."""
    T, H, W = _shape3(np.asarray(M))
    M = np.asarray(M, dtype=np.float64).reshape(T, H, W)
    msk = np.asarray(mask).astype(bool).reshape(T, H, W)
    dims = (T, H, W)
    k = int(np.prod(kdims))
    L = np.where(msk, M, 0.0)
    A = conv_matrix(L, kdims)
    Y = np.zeros_like(A)
    theta = 1.0 / np.linalg.norm(A, 2) if theta0 is None else theta0
    for _ in range(max_iters):
        U, s, Vt = np.linalg.svd(A - Y / theta, full_matrices=False)
        Z = (U * np.maximum(s - 1.0 / theta, 0.0)) @ Vt
        L = np.where(msk, M, adjoint(Y + theta * Z, dims, kdims) / (k * theta))
        A = conv_matrix(L, kdims)
        Y = Y + theta * (Z - A)
        theta = min(rho * theta, theta_max)
    return L
