"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these re-types an oracle formula: each checks the oracle against an
independent route (a brute-force loop over the definition, an FFT, a closed form,
an optimality condition, a property the paper states).
"""
import itertools
import json
import os

import numpy as np
import pytest

from oracle import icnnm_oracle as O
from paper_2604_17001_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
RNG = np.random.default_rng(1234)


def brute_conv(L, X):
    """[L * X]_i = sum_s [L]_{i-s}[X]_s with circular indices (Sec. II-B), by loops."""
    T, H, W = L.shape
    k3, k1, k2 = X.shape
    out = np.zeros_like(L, dtype=np.float64)
    for t, h, w in itertools.product(range(T), range(H), range(W)):
        acc = 0.0
        for st, sh, sw in itertools.product(range(k3), range(k1), range(k2)):
            acc += L[(t - st) % T, (h - sh) % H, (w - sw) % W] * X[st, sh, sw]
        out[t, h, w] = acc
    return out


def fft_conv(L, X):
    """Circular convolution by the convolution theorem (independent route)."""
    T, H, W = L.shape
    Xp = np.zeros((T, H, W))
    Xp[: X.shape[0], : X.shape[1], : X.shape[2]] = X
    return np.real(np.fft.ifftn(np.fft.fftn(L) * np.fft.fftn(Xp)))


SHAPES = [((3, 4, 5), (2, 3, 2)), ((7, 6, 1), (3, 2, 1)), ((4, 3, 4), (3, 3, 4)), ((2, 5, 4), (1, 1, 1))]


@pytest.mark.parametrize("dims,kdims", SHAPES)
def test_conv_matrix_matches_definition_exactly(dims, kdims):
    # dims = (H, W, T), kdims = (k1, k2, k3); integers => the sums are exact
    H, W, T = dims
    k1, k2, k3 = kdims
    L = RNG.integers(-5, 6, size=(T, H, W)).astype(np.float64)
    X = RNG.integers(-3, 4, size=(k3, k1, k2)).astype(np.float64)
    got = O.conv_matrix(L, kdims) @ X.ravel()          # Eq. (ak): A_k(L) vec(X)
    assert np.array_equal(got, brute_conv(L, X).ravel())


@pytest.mark.parametrize("dims,kdims", SHAPES + [((8, 9, 6), (5, 4, 3))])
def test_conv_matrix_matches_fft(dims, kdims):
    H, W, T = dims
    k1, k2, k3 = kdims
    L = RNG.standard_normal((T, H, W))
    X = RNG.standard_normal((k3, k1, k2))
    got = O.conv_matrix(L, kdims) @ X.ravel()
    np.testing.assert_allclose(got, fft_conv(L, X).ravel(), rtol=0, atol=1e-11)


@pytest.mark.parametrize("dims,kdims", SHAPES + [((8, 9, 6), (5, 4, 3))])
def test_adjoint_identity_and_AstarA(dims, kdims):
    H, W, T = dims
    k = int(np.prod(kdims))
    X = RNG.standard_normal((T, H, W))
    G = RNG.standard_normal((H * W * T, k))
    lhs = np.sum(O.conv_matrix(X, kdims) * G)          # <A_k(X), G>
    rhs = np.sum(X * O.adjoint(G, (T, H, W), kdims))   # <X, A_k^*(G)>
    assert abs(lhs - rhs) <= 1e-11 * max(1.0, abs(lhs))
    Xi = RNG.integers(-4, 5, size=(T, H, W)).astype(np.float64)
    assert np.array_equal(O.adjoint(O.conv_matrix(Xi, kdims), (T, H, W), kdims), k * Xi)


def test_adjoint_of_product_matches_adjoint():
    dims, kdims = (5, 6, 4), (3, 2, 2)
    H, W, T = dims
    k = 12
    Wm = RNG.standard_normal((H * W * T, k))
    V = np.linalg.qr(RNG.standard_normal((k, k)))[0]
    np.testing.assert_allclose(O.adjoint_of_product(Wm, V, (T, H, W), kdims),
                               O.adjoint(Wm @ V.T, (T, H, W), kdims), atol=1e-12)


@pytest.mark.parametrize("frac", [0.1, 0.37, 0.9])
def test_convolution_sampling_set_column_counts(frac):
    # Sec. II-B: every column of Theta_{Omega_A} = A_k(Theta_Omega) has exactly |Omega| ones
    H, W, T = 7, 6, 5
    mask = synth.mask_uniform(H, W, T, frac, seed=3).astype(np.float64)
    A = O.conv_matrix(mask, (3, 4, 2))
    assert np.all(A.sum(axis=0) == mask.sum())
    assert set(np.unique(A)) <= {0.0, 1.0}


def test_closed_forms():
    cases = json.load(open(os.path.join(GOLDEN, "closed_forms.json")))["cases"]
    for c in cases:
        H, W, T = c["dims_HWT"]
        kd = tuple(c["kdims"])
        if c["name"] == "constant tensor":
            L = np.full((T, H, W), c["c"])
        elif c["name"].startswith("cosine"):
            L = np.cos(2 * np.pi * c["f"] * np.arange(W) / W).reshape(1, 1, W)
        else:
            L = np.zeros((T, H, W))
            L[0, 0, 0] = 1.0
        A = O.conv_matrix(L, kd)
        s = np.linalg.svd(A, compute_uv=False)
        assert int(np.sum(s > 1e-9)) == c["rank"], c["name"]
        assert abs(s.sum() - c["nuclear_norm"]) < 1e-9, c["name"]
        if "singular_values" in c:
            np.testing.assert_allclose(s[:2], c["singular_values"], atol=1e-10)
        if c["name"] == "unit impulse":
            np.testing.assert_allclose(A.T @ A, np.eye(A.shape[1]), atol=0)


def test_nuclear_norm_rewrite_eq_cnnorm():
    # Eq. (cnnorm): ||A_k(L)||_* = sum_i ||L * kappa_i(L)||_F with L's own eigenvectors;
    # for any other orthonormal V the sum is >= (concavity of sqrt / Ky Fan).
    w = synth.workload(1, dims=(8, 8, 4), n_ref=0)
    L = w["L0"].astype(np.float64)
    kd = (3, 3, 2)
    A = O.conv_matrix(L, kd)
    _, s, Vt = np.linalg.svd(A, full_matrices=False)
    lhs = s.sum()
    rhs = sum(np.linalg.norm(fft_conv(L, Vt[i].reshape(2, 3, 3))) for i in range(len(s)))
    assert abs(lhs - rhs) <= 1e-10 * lhs
    assert abs(O.norm_21(O.conv_matrix_times(L, Vt.T, kd)) - lhs) <= 1e-10 * lhs
    for _ in range(5):
        Vr = np.linalg.qr(RNG.standard_normal((18, 18)))[0]
        assert O.norm_21(O.conv_matrix_times(L, Vr, kd)) >= lhs * (1 - 1e-12)


def autocorr_gram(refs, kdims):
    """A^T A through circular autocorrelations by FFT: entry (u, s) equals
    sum_j sum_i L_j[i-u] L_j[i-s] = sum_j R_j[u - s], R_j[d] = sum_i L_j[i] L_j[i+d]."""
    k1, k2, k3 = kdims
    taps = [(st, sh, sw) for st in range(k3) for sh in range(k1) for sw in range(k2)]
    G = np.zeros((len(taps), len(taps)))
    for L in refs:
        F = np.fft.fftn(L)
        R = np.real(np.fft.ifftn(np.conj(F) * F))     # R[d] = sum_i L[i] L[i+d]
        T, H, W = L.shape
        for a, (ut, uh, uw) in enumerate(taps):
            for b, (st, sh, sw) in enumerate(taps):
                G[a, b] += R[(ut - st) % T, (uh - sh) % H, (uw - sw) % W]
    return G


def test_gram_matches_autocorrelation_route():
    refs = [synth.video(9, 7, 5, seed=s).astype(np.float64) for s in (1, 2, 3)]
    kd = (3, 2, 2)
    np.testing.assert_allclose(O.gram(refs, kd), autocorr_gram(refs, kd), rtol=1e-12, atol=1e-10)


def test_learn_V_properties():
    # Sec. III-C Definition 3: sigma_1 = max_{||X||=1} sum_j ||L_j * X||_F^2, attained by kappa_1
    refs = [synth.video(10, 9, 6, seed=s).astype(np.float64) for s in (11, 12, 13, 14)]
    kd = (3, 3, 2)
    k = 18
    V, sig = O.learn_V(refs, kd)
    np.testing.assert_allclose(V.T @ V, np.eye(k), atol=1e-12)
    assert np.all(np.diff(sig) <= 1e-9 * sig[0])                  # decreasing
    assert np.all(sig >= -1e-9 * sig[0])                          # A^T A is PSD
    # trace(A^T A) = ||A||_F^2 = k * sum_j ||L_j||_F^2 (every voxel appears in k taps)
    assert abs(sig.sum() - k * sum(np.sum(L ** 2) for L in refs)) <= 1e-10 * sig.sum()

    def energy(x):
        X = x.reshape(2, 3, 3)
        return sum(np.sum(fft_conv(L, X) ** 2) for L in refs)

    for i in range(k):
        assert abs(energy(V[:, i]) - sig[i]) <= 1e-9 * sig[0]      # Rayleigh quotient
    for _ in range(50):
        x = RNG.standard_normal(k)
        x /= np.linalg.norm(x)
        assert energy(x) <= sig[0] * (1 + 1e-12)
    # sign convention: largest-magnitude entry of each column is positive
    for i in range(k):
        assert V[np.argmax(np.abs(V[:, i])), i] > 0


def test_prox_21_optimality():
    # Z-update closed form: for tau*||.||_{2,1} + 1/2||Z - R||^2 the optimum shrinks each
    # column; checked by subgradient optimality and against direct numerical minimisation
    from scipy.optimize import minimize
    R = RNG.standard_normal((6, 4))
    R[:, 2] *= 0.05                                  # a column that must vanish
    tau = 0.7
    Z = O.prox_21(R, tau)
    for i in range(4):
        n = np.linalg.norm(Z[:, i])
        if n > 0:
            np.testing.assert_allclose(Z[:, i] - R[:, i] + tau * Z[:, i] / n, 0, atol=1e-12)
        else:
            assert np.linalg.norm(R[:, i]) <= tau
    f = lambda z: tau * np.sum(np.linalg.norm(z.reshape(6, 4), axis=0)) + 0.5 * np.sum((z.reshape(6, 4) - R) ** 2)
    best = minimize(f, R.ravel(), method="Powell", options=dict(xtol=1e-10, ftol=1e-14, maxiter=200000))
    assert f(Z.ravel()) <= best.fun + 1e-9


def _tiny_problem(seed=5, dims=(6, 7, 4), kd=(3, 3, 2), frac=0.6):
    H, W, T = dims
    L0 = synth.video(H, W, T, seed=seed).astype(np.float64)
    mask = synth.mask_uniform(H, W, T, frac, seed=seed + 1)
    M = np.where(mask.astype(bool), L0, 0.0)
    k = int(np.prod(kd))
    V = np.linalg.qr(RNG.standard_normal((k, k)))[0]
    return L0, M, mask, V, kd


@pytest.mark.parametrize("lam", [np.inf, 3.0])
def test_L_update_minimises_augmented_lagrangian(lam):
    # Sec. III-D: the L-update is the exact minimiser of the augmented Lagrangian in L.
    L0, M, mask, V, kd = _tiny_problem()
    T, H, W = L0.shape
    k = V.shape[0]
    msk = mask.astype(bool)
    L = np.where(msk, M, 0.2 * RNG.standard_normal(L0.shape))
    Y = RNG.standard_normal((L.size, k))
    theta = 0.8
    Q = O.conv_matrix_times(L, V, kd)
    Z = O.prox_21(Q - Y / theta, 1 / theta)
    Lnew, Ynew, _, Qnew = O.icnnm_iteration(L, Y, theta, M, mask, V, kd, lam)

    def lag(Lx):
        AK = O.conv_matrix_times(Lx, V, kd)
        pen = 0.0 if np.isinf(lam) else lam * k / 2 * np.sum(np.where(msk, Lx - M, 0) ** 2)
        return pen + np.sum((Z - AK) * Y) + theta / 2 * np.sum((Z - AK) ** 2)

    eps = 1e-5
    free = np.flatnonzero(~msk.ravel()) if np.isinf(lam) else np.arange(L.size)
    for j in RNG.choice(free, 12, replace=False):
        e = np.zeros(L.size)
        e[j] = eps
        e = e.reshape(L.shape)
        g = (lag(Lnew + e) - lag(Lnew - e)) / (2 * eps)
        assert abs(g) < 1e-6 * max(1.0, np.abs(Y).sum() / L.size), (j, g)
    if np.isinf(lam):
        assert np.array_equal(Lnew[msk], M[msk])          # constraint restored exactly


@pytest.mark.parametrize("lam", [np.inf, 3.0])
def test_multiplier_update_dual_feasibility(lam):
    # With the multiplier step Y <- Y + theta(Z - A_k(L)K) after the L-update, the
    # L-subproblem's optimality reads A_k^*(Y_new K^T) = lam*k*P_Omega(L_new - M),
    # i.e. it vanishes off Omega; a wrong sign or order of the Y-step breaks this.
    L0, M, mask, V, kd = _tiny_problem(seed=9)
    T, H, W = L0.shape
    msk = mask.astype(bool)
    L = np.where(msk, M, 0.0)
    Y = RNG.standard_normal((L.size, V.shape[0]))
    Lnew, Ynew, _, _ = O.icnnm_iteration(L, Y, 1.3, M, mask, V, kd, lam)
    g = O.adjoint_of_product(Ynew, V, (T, H, W), kd)
    np.testing.assert_allclose(g[~msk], 0, atol=1e-10)
    if not np.isinf(lam):
        np.testing.assert_allclose(g[msk], lam * V.shape[0] * (Lnew - M)[msk], atol=1e-9)


def test_alpha_K_ground_truth_scheme_and_bounds():
    # Sec. III-A: alpha_K(L0) = 1 when K holds L0's own convolution eigenvectors (the
    # G.T. row of Table I), and 1 <= alpha_K <= sqrt(r_K) in general.
    L0 = synth.video(10, 8, 4, seed=21).astype(np.float64)
    kd = (3, 3, 2)
    V, _ = O.learn_V([L0], kd)
    assert abs(O.spectral_correlation(L0, V, kd) - 1.0) < 1e-9
    for _ in range(3):
        Vr = np.linalg.qr(RNG.standard_normal((18, 18)))[0]
        a = O.spectral_correlation(L0, Vr, kd)
        assert 1 - 1e-12 <= a <= np.sqrt(O.relative_rank(L0, Vr, kd)) + 1e-12


def test_exact_recovery_low_rank_target_theorem1():
    # Theorem 1: a convolutionally low-rank L0 (a single whole-period plane wave, rank 2),
    # with K = L0's own eigenvectors and a high sampling rate, is recovered.
    H, W, T = 12, 12, 1
    hh, ww = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    L0 = (0.5 + 0.4 * np.cos(2 * np.pi * (hh + 2 * ww) / 12.0)).reshape(1, H, W)
    kd = (4, 4, 1)
    V, _ = O.learn_V([L0], kd)
    mask = synth.mask_uniform(H, W, T, 0.85, seed=77)
    M = np.where(mask.astype(bool), L0, 0.0)
    L, st = O.icnnm_solve(M, mask, V, kd, max_iters=400)
    assert np.linalg.norm(L - L0) / np.linalg.norm(L0) < 1e-4, st
    assert O.spectral_correlation(L0, V, kd) == pytest.approx(1.0, abs=1e-9)


def test_solution_objective_not_above_target_and_observed_exact():
    # L0 is feasible for Eq. (InductiveCNNM), so the minimiser's objective is <= L0's.
    w = synth.workload(1, dims=(12, 12, 6), n_ref=4)
    kd = (3, 3, 2)
    V, _ = O.learn_V(w["refs"], kd)
    L, st = O.icnnm_solve(w["M"], w["mask"], V, kd, max_iters=150)
    msk = w["mask"].astype(bool)
    assert np.array_equal(L[msk], w["M"].astype(np.float64)[msk])
    obj0 = O.norm_21(O.conv_matrix_times(w["L0"].astype(np.float64), V, kd))
    assert st["objective"] <= obj0 * (1 + 1e-4)


def test_icnnm_with_cnnm_eigvectors_reaches_cnnm_value():
    # Eq. (cnnorm) with V = the right singular vectors of A_k(L*) (L* from CNNM): the
    # ICNNM objective at L* equals CNNM's optimal value, so ICNNM's minimum is <= it.
    H, W, T = 7, 7, 1
    L0 = synth.video(H, W, T, seed=31).astype(np.float64)
    mask = synth.mask_uniform(H, W, T, 0.7, seed=32)
    M = np.where(mask.astype(bool), L0, 0.0)
    kd = (3, 3, 1)
    Lc = O.cnnm_solve(M, mask, kd, max_iters=250)
    A = O.conv_matrix(Lc, kd)
    _, s, Vt = np.linalg.svd(A)
    cnnm_val = s.sum()
    assert O.norm_21(A @ Vt.T) == pytest.approx(cnnm_val, rel=1e-10)
    Li, st = O.icnnm_solve(M, mask, Vt.T, kd, max_iters=250)
    assert st["objective"] <= cnnm_val * (1 + 1e-5)
    assert np.array_equal(Lc[mask.astype(bool)], M[mask.astype(bool)])


def test_cnnm_feasible_objective_and_low_rank_recovery():
    # Eq. (cnnm): L0 is feasible, so the minimiser's ||A_k(L)||_* is at most L0's; the
    # observed entries are kept; a convolutionally low-rank target (a whole-period plane
    # wave: convolution rank 3) is recovered from most of its entries (the exact-recovery
    # property CNNM is built on, Sec. I).
    nuc = lambda X, kd: np.linalg.svd(O.conv_matrix(X, kd), compute_uv=False).sum()
    L0 = synth.video(8, 8, 3, seed=41).astype(np.float64)
    mask = synth.mask_uniform(8, 8, 3, 0.6, seed=42)
    M = np.where(mask.astype(bool), L0, 0.0)
    kd = (3, 3, 2)
    L = O.cnnm_solve(M, mask, kd, max_iters=300)
    assert np.array_equal(L[mask.astype(bool)], M[mask.astype(bool)])
    assert nuc(L, kd) <= nuc(L0, kd) * (1 + 1e-4)
    hh, ww = np.meshgrid(np.arange(12), np.arange(12), indexing="ij")
    P = (0.5 + 0.4 * np.cos(2 * np.pi * (hh + 2 * ww) / 12.0)).reshape(1, 12, 12)
    pm = synth.mask_uniform(12, 12, 1, 0.85, seed=77)
    Lp = O.cnnm_solve(np.where(pm.astype(bool), P, 0.0), pm, (4, 4, 1), max_iters=400)
    assert np.linalg.norm(Lp - P) / np.linalg.norm(P) < 1e-4


# -------------------------------------------------------------------------------
# Planted mistakes: a plausible bug in the oracle must make a pin above fail.
# -------------------------------------------------------------------------------
def test_planted_adjoint_shift_sign_is_caught(monkeypatch):
    orig = O.conv_index

    def wrong_index(dims, kdims, rows=None):   # (i + s) instead of (i - s)
        T, H, W = dims
        idx = orig(dims, kdims, rows)
        t, h, w = idx // (H * W), (idx // W) % H, idx % W
        r = np.arange(T * H * W) if rows is None else np.asarray(rows)
        rt, rh, rw = r // (H * W), (r // W) % H, r % W
        return (((2 * rt[:, None] - t) % T) * H + (2 * rh[:, None] - h) % H) * W + (2 * rw[:, None] - w) % W

    monkeypatch.setattr(O, "conv_index", wrong_index)
    with pytest.raises(AssertionError):
        test_conv_matrix_matches_definition_exactly((3, 4, 5), (2, 3, 2))


def test_planted_swapped_kernel_axes_is_caught(monkeypatch):
    orig = O.conv_index
    monkeypatch.setattr(O, "conv_index", lambda d, kd, rows=None: orig(d, (kd[1], kd[0], kd[2]), rows))
    with pytest.raises(AssertionError):
        test_conv_matrix_matches_fft((7, 6, 1), (3, 2, 1))


def test_planted_threshold_mistake_is_caught(monkeypatch):
    orig = O.prox_21
    monkeypatch.setattr(O, "prox_21", lambda R, tau: orig(R, 1.0 / tau))
    with pytest.raises(AssertionError):
        test_prox_21_optimality()


def test_planted_multiplier_sign_is_caught(monkeypatch):
    orig = O.icnnm_iteration

    def wrong(L, Y, theta, M, mask, V, kdims, lam=np.inf, Q=None):
        Ln, Yn, Z, Qn = orig(L, Y, theta, M, mask, V, kdims, lam, Q)
        return Ln, 2 * Y - Yn, Z, Qn                      # Y - theta(Z - A_k(L)K)

    monkeypatch.setattr(O, "icnnm_iteration", wrong)
    with pytest.raises(AssertionError):
        test_multiplier_update_dual_feasibility(np.inf)


def test_active_coherence_bounds_and_special_cases():
    # Eq. (coherence): 1 <= mu_1(B) <= p for a p x r matrix B; for K_I (k x r, orthonormal
    # columns) the row norms sum to r and none exceeds 1, so 1 <= mu_K^I <= k / r.
    L0 = synth.video(10, 8, 4, seed=23).astype(np.float64)
    kd = (3, 3, 2)
    k = 18
    # full support and an orthogonal K: every row of K has unit norm, so mu = 1
    Vr = np.linalg.qr(RNG.standard_normal((k, k)))[0]
    assert O.relative_rank(L0, Vr, kd) == k
    assert O.active_coherence(L0, Vr, kd) == pytest.approx(1.0, abs=1e-12)
    # a rank-2 plane wave with its own eigenvectors: I = the two leading columns
    hh, ww = np.meshgrid(np.arange(12), np.arange(12), indexing="ij")
    P = (0.5 + 0.4 * np.cos(2 * np.pi * (hh + 2 * ww) / 12.0)).reshape(1, 12, 12)
    kd2 = (4, 4, 1)
    V, _ = O.learn_V([P], kd2)
    s = O.relative_eigvals(P, V, kd2)
    r = O.relative_rank(P, V, kd2)
    assert r == 3 and np.all(s[3:] < 1e-9 * s[0])            # constant term + the cos pair
    # K_I spans the row space of A_k(P), so K_I K_I^T is the projector pinv(A) A and the
    # squared row norms of K_I are its diagonal
    A = O.conv_matrix(P, kd2)
    proj = np.linalg.pinv(A, rcond=1e-10) @ A
    mu = O.active_coherence(P, V, kd2)
    assert mu == pytest.approx(16 / 3 * np.max(np.diag(proj)), rel=1e-9)
    assert 1 - 1e-12 <= mu <= 16 / 3 + 1e-12
    # K = I (unit taps) keeps full support on a generic tensor, so mu = 1 again
    assert O.active_coherence(L0, np.eye(k), kd) == pytest.approx(1.0, abs=1e-12)


# -------------------------------------------------------------------------------
# theta0 and the stopping rule (readings of the silent Sec. III-D): hand-derived values
# on the rank-2 cosine, and the residual through the multiplier history.
# -------------------------------------------------------------------------------
def _cosine_case():
    c = json.load(open(os.path.join(GOLDEN, "closed_forms.json")))["theta0"]
    H, W, T = c["dims_HWT"]
    L = np.cos(2 * np.pi * c["f"] * np.arange(W) / W).reshape(T, H, W)
    return c, L, tuple(c["kdims"])


def test_theta0_default_hand_values():
    c, L, kd = _cosine_case()
    k = int(np.prod(kd))
    full = np.ones(L.shape, dtype=np.uint8)
    assert O.theta0_default(L, full, np.eye(k), kd) == pytest.approx(c["full_mask_identity_V"]["theta0"], rel=1e-12)
    V, _ = O.learn_V([L], kd)
    assert O.theta0_default(L, full, V, kd) == pytest.approx(c["full_mask_own_V"]["theta0"], rel=1e-12)
    even = np.zeros(L.shape, dtype=np.uint8)
    even[..., 0::2] = 1
    # M carries the full cosine: theta0 must see only its observed entries
    assert O.theta0_default(L, even, np.eye(k), kd) == pytest.approx(c["even_w_observed_identity_V"]["theta0"],
                                                                     rel=1e-12)


def test_residual_closed_form_full_mask():
    c, L, kd = _cosine_case()
    r = c["residual_full_mask_identity_V"]
    k = int(np.prod(kd))
    full = np.ones(L.shape, dtype=np.uint8)
    _, s1 = O.icnnm_solve(L, full, np.eye(k), kd, max_iters=1)
    assert s1["residual"] == pytest.approx(r["residual_iter1"], rel=1e-12)
    _, s2 = O.icnnm_solve(L, full, np.eye(k), kd, max_iters=2)
    assert abs(s2["residual"] - r["residual_iter2"]) <= 1e-14
    # the stopping rule: the first check at or below tol ends the run
    _, s = O.icnnm_solve(L, full, np.eye(k), kd, max_iters=50, tol=0.5, check_every=1)
    assert s["iters"] == 2


def test_residual_equals_multiplier_step():
    # Independent route: the multiplier step Y' = Y + theta(Z - A_k(L')K) gives
    # Z - A_k(L')K = (Y' - Y)/theta, so the residual after iteration t is
    # ||Y_t - Y_{t-1}||_F / (theta_{t-1} sqrt(k) ||L_t||_F); the run stops at the first
    # multiple of check_every where that is <= tol.
    L0 = synth.video(10, 8, 4, seed=91).astype(np.float64)
    mask = synth.mask_uniform(10, 8, 4, 0.45, seed=92)
    M = np.where(mask.astype(bool), L0, 0.0)
    kd = (3, 3, 2)
    k = 18
    V, _ = O.learn_V([synth.video(10, 8, 4, seed=93)], kd)
    L, Y, th = O.icnnm_init(M, mask, V, kd)
    Q = None
    res = []
    for _ in range(40):
        Ln, Yn, Z, Q = O.icnnm_iteration(L, Y, th, M, mask, V, kd, np.inf, Q)
        res.append(np.linalg.norm(Yn - Y) / (th * np.sqrt(k) * np.linalg.norm(Ln)))
        L, Y, th = Ln, Yn, 1.1 * th
    for n in (1, 7, 40):
        _, s = O.icnnm_solve(M, mask, V, kd, max_iters=n)
        assert s["residual"] == pytest.approx(res[n - 1], rel=1e-9)
    srt = np.sort(res[5:30])
    tol, every = float(0.5 * (srt[12] + srt[13])), 3      # between two residuals: no ties
    want = next(t for t in range(every, 41, every) if res[t - 1] <= tol)
    _, s = O.icnnm_solve(M, mask, V, kd, max_iters=40, tol=tol, check_every=every)
    assert s["iters"] == want and s["residual"] == pytest.approx(res[want - 1], rel=1e-9)


def test_planted_theta0_row_norms_is_caught(monkeypatch):
    def rows(M, mask, V, kdims):   # ||.||_{2,inf} taken over rows instead of columns
        Q0 = O.conv_matrix_times(O.P_Omega(M, mask), V, kdims)
        return 1.0 / float(O.column_norms(Q0.T).max())

    monkeypatch.setattr(O, "theta0_default", rows)
    with pytest.raises(AssertionError):
        test_theta0_default_hand_values()


def test_planted_theta0_without_projection_is_caught(monkeypatch):
    def no_proj(M, mask, V, kdims):   # P_Omega forgotten
        return 1.0 / float(O.column_norms(O.conv_matrix_times(M, V, kdims)).max())

    monkeypatch.setattr(O, "theta0_default", no_proj)
    with pytest.raises(AssertionError):
        test_theta0_default_hand_values()


@pytest.mark.parametrize("mistake", ["no_sqrt_k", "norm_of_Z", "squared"])
def test_planted_residual_mistakes_are_caught(monkeypatch, mistake):
    orig = O.primal_residual
    wrong = {
        "no_sqrt_k": lambda Z, Q, L, k: orig(Z, Q, L, 1),
        "norm_of_Z": lambda Z, Q, L, k: orig(Z, 0 * Q, L, k),
        "squared": lambda Z, Q, L, k: orig(Z, Q, L, k) ** 2,
    }[mistake]
    monkeypatch.setattr(O, "primal_residual", wrong)
    with pytest.raises(AssertionError):
        test_residual_closed_form_full_mask()
        test_residual_equals_multiplier_step()
