"""Full-size batching: the 64-tensor workload (H, W in 32..192 step 16, T in 8..48, kernel
7x7x3, mixed masks, 100 iterations) stepped as one batch on the BF16 path. Checked: the
observed entries of every job bit-exact; the three smallest jobs against the FP64 oracle
(<= 1e-3) and against solving them alone (the same within the BF16 tolerance)."""
import numpy as np
import pytest

from oracle import icnnm_oracle as O
from paper_2604_17001_gb300 import icnnm, synth
from tests.gpu_util import need_gpu, rel

pytestmark = pytest.mark.gpu


def test_batch64_full_size():
    need_gpu()
    kd = synth.WORKLOADS[4]["kdims"]
    its = synth.WORKLOADS[4]["iters"]
    jobs = synth.batch_jobs(synth.WORKLOADS[4]["n_jobs"], cfg=4)
    refs = [synth.video(64, 64, 16, synth.seed_for(4, j)) for j in range(1, 9)]
    V, _ = O.learn_V(refs, kd)
    ctx = icnnm.Context(0)
    try:
        outs, _ = ctx.icnnm_solve_batch([j["M"] for j in jobs], [j["mask"] for j in jobs], V, kd, max_iters=its,
                                        prec="bf16")
        for j, L in zip(jobs, outs):
            msk = j["mask"].astype(bool)
            assert np.array_equal(L[msk], j["M"][msk])
        small = sorted(range(len(jobs)), key=lambda i: int(np.prod(jobs[i]["dims"])))[:3]
        for i in small:
            Lo, _ = O.icnnm_solve(jobs[i]["M"], jobs[i]["mask"], V, kd, max_iters=its)
            assert rel(outs[i], Lo) <= 1e-3, (i, jobs[i]["dims"])
            Ls, _ = ctx.icnnm_solve(jobs[i]["M"], jobs[i]["mask"], V, kd, max_iters=its, prec="bf16")
            assert rel(outs[i], Ls) <= 1e-3
    finally:
        ctx.close()
