"""The allocation-free entry point icnnm_learn_V_noalloc, for callers that cannot
allocate device memory themselves (a framework that hands out device memory only from
its own pool, latency-critical code that must not trigger the synchronisation of a
cudaMalloc), gives what icnnm_learn_V gives, on two calls in a row (its scratch array
keeps the previous call's contents, so the second call checks that nothing stale leaks
in), with host or device outputs, on the default stream or the caller's, and without
allocating device memory.

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


def test_learn_V_noalloc_device_outputs_on_a_stream_allocate_nothing():
    # V_out and eig_out in device memory (the eigensolver writes straight into them), on
    # a caller's stream; the device memory in use is the same before and after the calls
    need_gpu()
    import torch
    kd = (3, 5, 2)
    k = 30
    refs = [torch.from_numpy(synth.video(20, 24, 6, seed=s)).cuda() for s in (301, 302, 303)]
    with icnnm.Context(0) as ctx:
        Vr, er = ctx.icnnm_learn_V(refs, kd)
    s = torch.cuda.Stream()
    Vd = torch.zeros((k, k), dtype=torch.float64, device="cuda")
    ed = torch.zeros(k, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    icnnm.icnnm_learn_V_noalloc(refs, kd, V_out=Vd, eig_out=ed, stream=s.cuda_stream)   # warm-up
    torch.cuda.synchronize()
    used0 = torch.cuda.memory_allocated()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        Vd.zero_()
        ed.zero_()
        torch.cuda.synchronize()
        icnnm.icnnm_learn_V_noalloc(refs, kd, V_out=Vd, eig_out=ed, stream=s.cuda_stream)
        torch.cuda.synchronize()
        # V_out is column-major: row i of the (k, k) buffer is eigenvector i
        _check_same(Vd.cpu().numpy().T, ed.cpu().numpy(), Vr, er)
        Vh, _ = icnnm.icnnm_learn_V_noalloc(refs, kd, eig_out=None, stream=s.cuda_stream)
        _check_same(Vh, ed.cpu().numpy(), Vr, er)
    free1, _ = torch.cuda.mem_get_info()
    assert torch.cuda.memory_allocated() == used0
    assert free1 == free0


def test_learn_V_noalloc_rejects_sizes_beyond_its_limit():
    need_gpu()
    import torch
    refs = [torch.from_numpy(synth.video(32, 32, 8, seed=7)).cuda()]
    with pytest.raises(icnnm.ICNNMError) as e:
        icnnm.icnnm_learn_V_noalloc(refs, (9, 9, 5))          # k = 405 > 256
    assert e.value.status == icnnm.EINVAL and "256" in str(e.value)
