"""The frequency-domain form of the iteration (the algebra the FFT path runs), written in
numpy FP64 with numpy's FFT, against the paper-order FP64 oracle (Sec. III-D).

The convolution of Sec. II-B is circular, so with kappa_c the kernel of eigenvector c and
^ the 3-D DFT, A_k(X)v_c has the DFT X^ kappa_c^, A_k^*(U D V^T) has the DFT
sum_c D_c U_c^ conj(kappa_c^), and column norms follow from Parseval. Every U_c^ stays a
multiple of kappa_c^, so the iteration can carry y_c = U_c^ conj(kappa_c^) and
q_c = |kappa_c^|^2 only: Delta^ = sum_c D_c y_c, y_c' = D_c y_c - q_c X^,
||U_c'||^2 = (1/m) sum |y_c'|^2 / q_c. These tests check that this recurrence, on real
half spectra with the interior w-frequencies counted twice, reproduces the oracle's
iterate, residual, objective and theta (FP64, 1e-10)."""
import numpy as np
import pytest

from oracle import icnnm_oracle as O
from paper_2604_17001_gb300 import synth


def spectral_solve(M, mask, V, kdims, iters, lam=np.inf, rho=1.1, theta_max=1e10):
    T, H, W = M.shape
    k1, k2, k3 = kdims
    k, m = k1 * k2 * k3, T * H * W
    Wh = W // 2 + 1
    ow = np.arange(Wh)
    wgt = np.where((ow == 0) | (2 * ow == W), 1.0, 2.0)
    rf = np.fft.rfftn
    irf = lambda x: np.fft.irfftn(x, s=(T, H, W), axes=(0, 1, 2))
    q = []
    for c in range(k):
        kap = np.zeros((T, H, W))
        for s in range(k):
            sw, sh, st = s % k2, (s // k2) % k1, s // (k1 * k2)
            kap[st, sh, sw] = V[s, c]
        q.append(np.abs(rf(kap)) ** 2)
    q = np.array(q)
    safe_q = np.where(q > 0, q, 1.0)

    def norm2_over_q(num):            # (1/m) sum |.|^2 / q per column, 0 where q = 0
        return (wgt * np.where(q > 0, num / safe_q, 0.0)).sum(axis=(1, 2, 3)) / m

    msk = mask.astype(bool)
    Mf = M.astype(np.float64)
    L = np.where(msk, Mf, 0.0)
    th = 1.0 / np.sqrt(((wgt * q * np.abs(rf(L)) ** 2).sum(axis=(1, 2, 3)) / m).max())
    y = -q * rf(th * L)[None]

    def shrink(y):
        n = np.sqrt(norm2_over_q(np.abs(y) ** 2))
        s = np.where(n > 1, 1 - 1 / np.maximum(n, 1e-300), 0.0)
        return s, 1 - s

    s, D = shrink(y)
    resid = None
    for it in range(1, iters + 1):
        thn = min(rho * th, theta_max)
        Dl = irf((D[:, None, None, None] * y).sum(0))
        if np.isinf(lam):
            Ln = np.where(msk, Mf, L + Dl / (k * th))
        else:
            lt = np.where(msk, lam, 0.0)
            Ln = (Dl / k + th * L + lt * np.where(msk, Mf, 0.0)) / (lt + th)
        X = (th + thn) * Ln - th * L
        if it == iters:
            r = (s / th)[:, None, None, None] * y + q * rf(Ln)[None]
            resid = np.sqrt(norm2_over_q(np.abs(r) ** 2).sum()) / (np.sqrt(k) * np.linalg.norm(Ln))
        L, th = Ln, thn
        if it == iters:
            break
        y = D[:, None, None, None] * y - q * rf(X)[None]
        s, D = shrink(y)
    obj = np.sqrt((wgt * q * np.abs(rf(L)) ** 2).sum(axis=(1, 2, 3)) / m).sum()
    return L, dict(residual=resid, objective=obj, theta=th)


CASES = [
    ((8, 16, 4), (3, 3, 2), 0.6, np.inf, 25),     # H, W, T; kernel; observed; lambda; iterations
    ((8, 16, 4), (3, 3, 2), 0.6, 1000.0, 25),     # the penalised form
    ((4, 2, 4), (3, 2, 2), 0.5, np.inf, 15),      # W = 2: only the DC and Nyquist w-frequencies
    ((6, 10, 1), (3, 4, 1), 0.5, np.inf, 20),     # an image, dims not powers of two, even kernel
    ((5, 7, 3), (5, 7, 3), 0.7, np.inf, 10),      # the kernel as large as the tensor (odd W)
]


@pytest.mark.parametrize("dims,kdims,frac,lam,iters", CASES)
def test_spectral_recurrence_matches_oracle(dims, kdims, frac, lam, iters):
    H, W, T = dims
    L0 = synth.video(H, W, T, seed=31)
    mask = synth.mask_uniform(H, W, T, frac, seed=32)
    M = np.where(mask.astype(bool), L0, 0.0)
    V, _ = O.learn_V([synth.video(H, W, T, seed=40 + j) for j in range(3)], kdims)
    Lo, so = O.icnnm_solve(M, mask, V, kdims, lam=lam, max_iters=iters)
    L, st = spectral_solve(M.reshape(T, H, W), mask.reshape(T, H, W), V, kdims, iters, lam=lam)
    assert np.abs(L - Lo.reshape(T, H, W)).max() <= 1e-10 * max(1.0, np.abs(Lo).max())
    assert st["residual"] == pytest.approx(so["residual"], rel=1e-8, abs=1e-14)
    assert st["objective"] == pytest.approx(so["objective"], rel=1e-10)
    assert st["theta"] == pytest.approx(so["theta"], rel=1e-12)


def test_parseval_half_spectrum_weights():
    # sum_w x^2 = (1/W) sum over the W/2 + 1 kept frequencies, the interior ones twice
    rng = np.random.default_rng(5)
    for W in (2, 4, 6, 16, 15):
        x = rng.standard_normal((3, 5, W))
        Wh = W // 2 + 1
        ow = np.arange(Wh)
        wgt = np.where((ow == 0) | (2 * ow == W), 1.0, 2.0)
        lhs = (x ** 2).sum()
        rhs = (wgt * np.abs(np.fft.rfftn(x)) ** 2).sum() / x.size
        assert rhs == pytest.approx(lhs, rel=1e-12)


def test_planted_missing_parseval_weight_is_caught(monkeypatch):
    # counting every kept w-frequency once (a plausible mistake) breaks the agreement
    import numpy as _np
    orig = _np.where

    def one_weight(cond, a, b):
        if isinstance(a, float) and a == 1.0 and isinstance(b, float) and b == 2.0:
            return orig(cond, 1.0, 1.0)
        return orig(cond, a, b)
    monkeypatch.setattr(_np, "where", one_weight)
    with pytest.raises(AssertionError):
        test_spectral_recurrence_matches_oracle((8, 16, 4), (3, 3, 2), 0.6, np.inf, 25)
