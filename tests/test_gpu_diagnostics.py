"""GPU parity of icnnm_spectral_diagnostics (Sec. III-A, Definition 2, Eqs. (rkL0) and
(alphaK); the coherence of Eq. (coherence)) with the FP64 oracle on the same tensor and
V: the relative convolution eigenvalues sigma_i, r_K, alpha_K and mu_K.

The GPU forms G = A_k(L0)^T A_k(L0) (FP64 autocorrelations), sigma_i^2 = v_i^T G v_i and
alpha_K^2 = lambda_max(D V^T G V D); the oracle takes column norms and the operator
norm of the explicit A_k(L0) V D. Squaring makes a sigma that is zero in exact
arithmetic come out near sqrt(k eps) sigma_max on the GPU, so the sigma bar is
1e-7 sigma_max absolute; alpha_K agrees to 1e-7 relative while every sigma in the
support is well above the rank threshold; r_K is compared only where no sigma lies
within 10x the sigma bar of the threshold, so that both sides decide alike."""
import numpy as np
import pytest

from oracle import icnnm_oracle as O
from paper_2604_17001_gb300 import icnnm, synth
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu

RNG = np.random.default_rng(20260417)


@pytest.fixture(scope="module")
def ctx():
    need_gpu()
    c = icnnm.Context(0)
    yield c
    c.close()


def plane_wave(H, W, a, b):
    hh, ww = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    return (0.5 + 0.4 * np.cos(2 * np.pi * (a * hh / H + b * ww / W))).reshape(1, H, W).astype(np.float32)


def compare(ctx, L0, V, kd, tol=1e-6):
    g = ctx.icnnm_spectral_diagnostics(L0, V, kd, rank_tol=tol)
    L = L0.astype(np.float64)
    so = O.relative_eigvals(L, V, kd)
    smax = so.max()
    assert np.max(np.abs(g["sigma"] - so)) <= 1e-7 * smax
    thr = tol * max(1.0, smax)
    # both sides decide alike when no sigma lies within 10x the sigma bar of the threshold
    assert not np.any(np.abs(so - thr) <= 10 * 1e-7 * smax), "a sigma too close to the rank threshold"
    assert g["r_K"] == O.relative_rank(L, V, kd, tol)
    ao = O.spectral_correlation(L, V, kd, tol)
    assert abs(g["alpha_K"] - ao) <= 1e-7 * ao
    assert g["mu_K"] == pytest.approx(O.active_coherence(L, V, kd, tol), rel=1e-9)
    return g, ao


def test_video_learned_V(ctx):
    kd = (5, 5, 3)
    L0 = synth.video(24, 20, 6, seed=5)
    V, _ = O.learn_V([synth.video(24, 20, 6, seed=s) for s in (6, 7, 8)], kd)
    g, _ = compare(ctx, L0, V, kd)
    assert g["r_K"] == 75 and 1.0 < g["alpha_K"] <= np.sqrt(75)


def test_random_orthogonal_K_raises_alpha(ctx):
    # Table I's "randomly generated" scheme: a random orthogonal K correlates worse with
    # the target than one learned from similar tensors (alpha_K further above 1).
    kd = (5, 5, 3)
    L0 = synth.video(24, 20, 6, seed=5)
    V, _ = O.learn_V([synth.video(24, 20, 6, seed=s) for s in (6, 7, 8)], kd)
    Vr = np.linalg.qr(RNG.standard_normal((75, 75)))[0]
    a_learned = compare(ctx, L0, V, kd)[1]
    a_random = compare(ctx, L0, Vr, kd)[1]
    assert a_random > a_learned


def test_ground_truth_K_rank_deficient(ctx):
    # Table I's G.T. scheme on a convolution-rank-3 image (a whole-period plane wave plus
    # a constant): r_K = 3 and alpha_K = 1 (Sec. III-A).
    kd = (6, 5, 1)
    P = plane_wave(48, 40, 3, 2)
    V, _ = O.learn_V([P], kd)
    # the null directions come out near 1e-6 sigma_max (the FP32 rounding of P), so the
    # rank threshold sits well above them
    g, _ = compare(ctx, P, V, kd, tol=1e-5)
    assert g["r_K"] == 3
    assert g["alpha_K"] == pytest.approx(1.0, abs=1e-9)


def test_image_workload_size(ctx):
    # the image-completion shape: 200x200, 13x13 kernel, V from the 7 reference images
    w = synth.workload(6)
    V, _ = O.learn_V(w["refs"], w["kdims"])
    g, _ = compare(ctx, w["L0"], V, w["kdims"])
    assert g["r_K"] == 169


def test_zero_tensor_and_invalid(ctx):
    kd = (3, 3, 2)
    V = np.linalg.qr(RNG.standard_normal((18, 18)))[0]
    g = ctx.icnnm_spectral_diagnostics(np.zeros((4, 8, 8), np.float32), V, kd)
    assert g["r_K"] == 0 and g["alpha_K"] == 0.0 and g["mu_K"] == 0.0 and not g["sigma"].any()
    L = synth.video(8, 8, 4, seed=3)
    with pytest.raises(icnnm.ICNNMError):
        ctx.icnnm_spectral_diagnostics(L, V, kd, rank_tol=0.0)
    bad = L.copy()
    bad[1, 2, 3] = np.nan
    with pytest.raises(icnnm.ICNNMError):
        ctx.icnnm_spectral_diagnostics(bad, V, kd)
    with pytest.raises(icnnm.ICNNMError):
        ctx.icnnm_spectral_diagnostics(L, V * 1.01, kd)
