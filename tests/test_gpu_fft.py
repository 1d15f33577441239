"""GPU parity of the frequency-domain solve (icnnm_solve_fft, through the C ABI) against
the FP64 oracle on the same seeded inputs. The frequency-domain path computes the same
ADMM iteration as the oracle (Sec. III-D) with FP32 complex spectra, so it is held to the
FP32 bar of the implicit-GEMM path: relative L2 error <= 1e-5, observed entries bit-exact
(lambda = inf), the same theta and iteration count. At full size it is compared with the
stored FP64 oracle runs of the prediction (128x128x32, k = 405, 500 iterations) and the
interpolation (256x256x64, k = 245, 100 iterations) workloads, whose dims are powers of
two."""
import os

import numpy as np
import pytest

from oracle import icnnm_oracle as O
from paper_2604_17001_gb300 import icnnm, synth
from tests.gpu_util import need_gpu, rel

pytestmark = pytest.mark.gpu

TOL = 1e-5
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def ctx():
    need_gpu()
    c = icnnm.Context(0)
    yield c
    c.close()


def case(dims, kdims, frac=None, last=None, seed=11, nref=3):
    H, W, T = dims
    L0 = synth.video(H, W, T, seed=seed)
    if last is not None:
        mask = synth.mask_last_frames(H, W, T, last)
    else:
        mask = synth.mask_uniform(H, W, T, frac, seed=seed + 1)
    M = np.where(mask.astype(bool), L0, 0).astype(np.float32)
    refs = [synth.video(H, W, T, seed=seed + 10 + j) for j in range(nref)]
    V, _ = O.learn_V(refs, kdims)
    return M, mask, V


CASES = [
    # (dims H,W,T), kernel, mask, iterations
    ((32, 32, 8), (5, 5, 3), dict(frac=0.5), 100),      # the completion workload's shape
    ((16, 8, 4), (3, 4, 2), dict(frac=0.6), 40),        # kernel dims not powers of two
    ((16, 16, 8), (9, 9, 5), dict(last=2), 40),         # k = 405, prediction mask
    ((64, 32, 1), (5, 5, 1), dict(frac=0.5), 60),       # 2-D image (T = 1)
    ((8, 2, 4), (3, 2, 2), dict(frac=0.5), 30),         # W = 2: only DC and Nyquist along w
    ((16, 16, 4), (1, 1, 1), dict(frac=0.5), 20),       # k = 1: V = [1], A_k(L) = vec(L)
    ((4, 4, 4), (4, 4, 4), dict(frac=0.7), 30),         # kernel = the whole tensor
]


@pytest.mark.parametrize("dims,kdims,mk,iters", CASES)
def test_fft_matches_oracle(ctx, dims, kdims, mk, iters):
    M, mask, V = case(dims, kdims, **mk)
    Lo, so = O.icnnm_solve(M, mask, V, kdims, max_iters=iters)
    L, st = ctx.icnnm_solve_fft(M, mask, V, kdims, max_iters=iters)
    e = rel(L, Lo)
    assert e <= TOL, (dims, kdims, e)
    msk = mask.astype(bool)
    assert np.array_equal(L[msk], M[msk])
    assert st["iters"] == iters
    assert st["theta"] == pytest.approx(so["theta"], rel=1e-6)
    assert st["objective"] == pytest.approx(so["objective"], rel=1e-4)


def test_fft_penalised_lambda_1000(ctx):
    M, mask, V = case((32, 16, 8), (5, 5, 3), frac=0.5)
    Lo, _ = O.icnnm_solve(M, mask, V, (5, 5, 3), lam=1000.0, max_iters=60)
    L, _ = ctx.icnnm_solve_fft(M, mask, V, (5, 5, 3), lam=1000.0, max_iters=60)
    assert rel(L, Lo) <= TOL


def test_fft_tolerance_stopping(ctx):
    M, mask, V = case((32, 32, 8), (5, 5, 3), frac=0.5)
    Lo, so = O.icnnm_solve(M, mask, V, (5, 5, 3), max_iters=300, tol=1e-4, check_every=10)
    L, st = ctx.icnnm_solve_fft(M, mask, V, (5, 5, 3), max_iters=300, tol=1e-4, check_every=10)
    assert st["iters"] == so["iters"] < 300
    assert rel(L, Lo) <= TOL
    assert st["residual"] == pytest.approx(so["residual"], rel=2e-2)


def test_fft_agrees_with_implicit_gemm_fp32(ctx):
    M, mask, V = case((32, 64, 8), (7, 7, 3), frac=0.4)
    L1, s1 = ctx.icnnm_solve(M, mask, V, (7, 7, 3), max_iters=50, prec="fp32")
    L2, s2 = ctx.icnnm_solve_fft(M, mask, V, (7, 7, 3), max_iters=50)
    assert rel(L2, L1) <= 2 * TOL
    assert s2["theta"] == pytest.approx(s1["theta"], rel=1e-6)


def test_fft_rejects_what_it_cannot_take(ctx):
    M, mask, V = case((24, 16, 4), (3, 3, 2), frac=0.5)
    with pytest.raises(icnnm.ICNNMError) as ei:
        ctx.icnnm_solve_fft(M, mask, V, (3, 3, 2))
    assert ei.value.status == icnnm.EUNSUPPORTED
    M1 = np.ones((1, 16), dtype=np.float32)                    # H = T = 1: a single row
    with pytest.raises(icnnm.ICNNMError) as ei:
        ctx.icnnm_solve_fft(M1, np.ones((1, 16), dtype=np.uint8), np.eye(3), (1, 3))
    assert ei.value.status == icnnm.EUNSUPPORTED
    M, mask, V = case((16, 16, 4), (3, 3, 2), frac=0.5)
    with pytest.raises(icnnm.ICNNMError) as ei:
        ctx.icnnm_solve_fft(M, np.zeros_like(mask), V, (3, 3, 2))
    assert ei.value.status == icnnm.EINVAL
    with pytest.raises(icnnm.ICNNMError) as ei:
        ctx.icnnm_solve_fft(M, mask, V * 1.01, (3, 3, 2))
    assert ei.value.status == icnnm.EINVAL


def test_fft_prediction_full_size(ctx):
    path = os.path.join(GOLDEN, "prediction_128x128x32_k9x9x5.npz")
    if not os.path.exists(path):
        pytest.skip("stored oracle run not present")
    g = np.load(path)
    w = synth.workload(2, n_ref=0)
    iters = int(g["iters"])
    L, st = ctx.icnnm_solve_fft(w["M"], w["mask"], g["V"], w["kdims"], max_iters=iters)
    msk = w["mask"].astype(bool)
    assert np.array_equal(L[msk], w["M"][msk])
    Lo = L.astype(np.float64).copy()
    Lo[g["frames"]] = g["L_missing"]
    e = float(np.linalg.norm(L - Lo) / np.linalg.norm(Lo))
    assert e <= TOL, e
    assert st["objective"] == pytest.approx(float(g["objective"]), rel=1e-4)
    assert st["theta"] == pytest.approx(float(g["theta"]), rel=1e-12)
    assert st["iters"] == iters


def test_fft_interpolation_full_size(ctx):
    path = os.path.join(GOLDEN, "interpolation_256x256x64_k7x7x5.npz")
    if not os.path.exists(path):
        pytest.skip("stored oracle run not present")
    g = np.load(path)
    w = synth.workload(3, n_ref=0)
    iters = int(g["iters"])
    L, st = ctx.icnnm_solve_fft(w["M"], w["mask"], g["V"], w["kdims"], max_iters=iters)
    msk = w["mask"].astype(bool)
    assert np.array_equal(L[msk], w["M"][msk])
    got = L.reshape(-1)[g["sample_idx"]].astype(np.float64)
    ref = g["L_sample"]
    assert float(np.linalg.norm(got - ref) / np.linalg.norm(ref)) <= TOL
    assert float(np.linalg.norm(L.astype(np.float64))) == pytest.approx(float(g["L_norm"]), rel=TOL)
    assert st["objective"] == pytest.approx(float(g["objective"]), rel=1e-4)
    assert st["iters"] == iters
