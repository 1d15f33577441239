"""Full-size parity: the image-completion workload (200x200 image, kernel 13x13, 4x4-pixel
blocks missing at 50%, 500 ADMM iterations, V learned from 7 reference images) through
the C ABI against the stored FP64 oracle run of the same inputs
(tests/golden/image_200x200_k13x13.npz, written by make_image_reference.py, which
calls only the oracle). Bars: relative L2 error of the completed image <= 1e-3 (BF16
path) and <= 1e-5 (FP32 path); observed pixels bit-exact. Also: a batch of images of
this family solved together equals each image solved alone (to the BF16 bar)."""
import os

import numpy as np
import pytest

from paper_2604_17001_gb300 import icnnm, synth
from tests.gpu_util import need_gpu, rel

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "image_200x200_k13x13.npz")
TOL = {"fp32": 1e-5, "bf16": 1e-3}


@pytest.fixture(scope="module")
def setup():
    need_gpu()
    if not os.path.exists(GOLDEN):
        pytest.skip("stored oracle run not present")
    g = np.load(GOLDEN)
    w = synth.workload(6, n_ref=0)
    c = icnnm.Context(0)
    yield c, g, w
    c.close()


@pytest.mark.parametrize("prec", ["bf16", "fp32"])
def test_image_full_size(setup, prec):
    ctx, g, w = setup
    iters = int(g["iters"])
    L, st = ctx.icnnm_solve(w["M"], w["mask"], g["V"], w["kdims"], max_iters=iters, prec=prec)
    msk = w["mask"].astype(bool)
    assert np.array_equal(L[msk], w["M"][msk])
    e = rel(L, g["L"])
    assert e <= TOL[prec], (prec, e)
    assert abs(st["objective"] - float(g["objective"])) <= 10 * TOL[prec] * float(g["objective"])
    assert st["theta"] == pytest.approx(float(g["theta"]), rel=1e-12)
    assert st["iters"] == iters


def test_image_batch_equals_single(setup):
    ctx, g, w = setup
    jobs = synth.image_jobs(6)
    its = 200
    outs, _ = ctx.icnnm_solve_batch([j["M"] for j in jobs], [j["mask"] for j in jobs], g["V"], w["kdims"],
                                    max_iters=its, prec="bf16")
    for j, L in zip(jobs, outs):
        Ls, _ = ctx.icnnm_solve(j["M"], j["mask"], g["V"], w["kdims"], max_iters=its, prec="bf16")
        msk = j["mask"].astype(bool)
        assert np.array_equal(L[msk], j["M"][msk])
        assert rel(L, Ls) <= TOL["bf16"]
