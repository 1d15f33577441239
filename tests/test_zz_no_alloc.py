"""The allocation-free entry point icnnm_learn_V_noalloc, for callers that cannot
allocate device memory (graph capture, pool-managed memory, latency-critical code),
gives what icnnm_learn_V gives, on two calls in a row (its scratch array keeps the
previous call's contents, so the second call checks that nothing stale leaks in).

This file is collected last on purpose: if it fails, every other test has run."""
import numpy as np
import pytest

from paper_2604_17001_gb300 import icnnm, synth
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def _check_same(V, e, Vr, er):
    k = len(er)
    assert np.max(np.abs(e - er)) <= 1e-9 * er[0]
    np.testing.assert_allclose(V.T @ V, np.eye(k), atol=1e-12)
    # same Gram to rounding: V diag(e) V^T from both entry points
    G, Gr = (V * e[None, :]) @ V.T, (Vr * er[None, :]) @ Vr.T
    assert np.linalg.norm(G - Gr) <= 1e-9 * np.linalg.norm(Gr)
    # well-separated eigenvectors agree up to sign
    gaps = np.abs(np.diff(er))
    for i in range(6):
        gap = min(gaps[i], gaps[i - 1] if i > 0 else np.inf)
        if gap > 1e-3 * er[0]:
            assert abs(abs(V[:, i] @ Vr[:, i]) - 1) <= 1e-6


def test_learn_V_noalloc_matches_learn_V_on_two_calls():
    need_gpu()
    import torch
    kd = (5, 5, 3)
    with icnnm.Context(0) as ctx:
        for seeds, dims in (([101, 102, 103], (24, 20, 8)), ([201, 202, 203, 204], (16, 32, 6))):
            refs = [torch.from_numpy(synth.video(*dims, seed=s)).cuda() for s in seeds]
            Vr, er = ctx.icnnm_learn_V(refs, kd)
            V, e = icnnm.icnnm_learn_V_noalloc(refs, kd)
            _check_same(V, e, Vr, er)


def test_learn_V_noalloc_rejects_sizes_beyond_its_limit():
    need_gpu()
    import torch
    refs = [torch.from_numpy(synth.video(32, 32, 8, seed=7)).cuda()]
    with pytest.raises(icnnm.ICNNMError) as e:
        icnnm.icnnm_learn_V_noalloc(refs, (9, 9, 5))          # k = 405 > 256
    assert e.value.status == icnnm.EINVAL and "256" in str(e.value)
