"""Served BF16 against the FP64 oracle on serving-shaped jobs: kernel 7x7x3 (k = 147),
the four mask families of the serving stream (30-70% uniform, last frames missing, every
other frame missing, 16x16 block holes), run to a relative residual of 1e-3 checked every
10 iterations. Every job is submitted to the continuous-batching server at once (so they
step together), and each result is compared with the oracle run for the same iteration
count (the iterate is unique for a given count; the stopping check may land a check
apart on the two sides). Bar: relative L2 <= 1e-3; observed entries bit-exact.

Also long fixed-count runs (300 iterations, no tolerance, so no finish phase) on sparsely
observed jobs, where BF16 rounding has the most iterations to accumulate, in BF16 and in
BF16X3."""
import numpy as np
import pytest

from oracle import icnnm_oracle as O
from paper_2604_17001_gb300 import icnnm, synth
from tests.gpu_util import need_gpu, rel

pytestmark = pytest.mark.gpu

KD = (7, 7, 3)


@pytest.fixture(scope="module")
def setup():
    need_gpu()
    refs = [synth.video(32, 32, 8, synth.seed_for(5, j)) for j in range(1, 5)]
    V, _ = O.learn_V(refs, KD)
    c = icnnm.Context(0)
    yield c, V
    c.close()


def test_served_bf16_tolerance_stopped_matches_oracle(setup):
    ctx, V = setup
    jobs = synth.batch_jobs(8, cfg=5, hw_range=(32, 64), t_range=(8, 16))
    assert len({j["family"][:4] for j in jobs}) >= 3
    kw = dict(max_iters=1000, tol=1e-3, check_every=10)
    ids = [ctx.icnnm_submit(j["M"], j["mask"], V, KD, prec="bf16", **kw) for j in jobs]
    for j, jid in zip(jobs, ids):
        L = np.zeros_like(j["M"])
        r, st = ctx.icnnm_wait(jid, L_out=L, timeout_ms=300000)
        assert r == icnnm.OK and st["residual"] <= 1e-3 and st["iters"] < 1000
        msk = j["mask"].astype(bool)
        assert np.array_equal(L[msk], j["M"][msk])
        Lo, _ = O.icnnm_solve(j["M"], j["mask"], V, KD, max_iters=st["iters"])
        assert rel(L, Lo) <= 1e-3, (j["dims"], j["family"], st["iters"], rel(L, Lo))


# Plain BF16 rounds the forward pass's operands (X and V) to BF16 every iteration; over a
# long fixed run on a sparsely observed job this drifts to about 1e-3 from FP64 (measured
# 1.12e-3 here at 30% observed). BF16X3 splits those operands into hi + lo pairs and keeps
# U as a pair, which takes the drift to about 1e-6.
LONG_BAR = {"bf16": 2e-3, "bf16x3": 1e-5}


@pytest.mark.parametrize("prec", ["bf16", "bf16x3"])
@pytest.mark.parametrize("frac,seed", [(0.3, 71), (0.5, 72)])
def test_long_fixed_run_matches_oracle(setup, frac, seed, prec):
    ctx, V = setup
    H, W, T = 40, 32, 10
    L0 = synth.video(H, W, T, seed=seed)
    mask = synth.mask_uniform(H, W, T, frac, seed=seed + 1)
    M = np.where(mask.astype(bool), L0, 0).astype(np.float32)
    L, st = ctx.icnnm_solve(M, mask, V, KD, max_iters=300, prec=prec)
    Lo, _ = O.icnnm_solve(M, mask, V, KD, max_iters=300)
    assert rel(L, Lo) <= LONG_BAR[prec], (prec, rel(L, Lo))
    assert np.array_equal(L[mask.astype(bool)], M[mask.astype(bool)])
