"""Full-size parity: the video-prediction workload (128x128x32, kernel 9x9x5, frames
24..31 missing, 500 ADMM iterations, V learned from 64 reference tensors) through the
C ABI against the stored FP64 oracle run of the same inputs
(tests/golden/prediction_128x128x32_k9x9x5.npz, written by make_prediction_reference.py,
which calls only the oracle). Bars: relative L2 error of the completed tensor <= 1e-3
(BF16 path) and <= 1e-5 (FP32 path); observed frames bit-exact."""
import os

import numpy as np
import pytest

from paper_2604_17001_gb300 import icnnm, synth
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "prediction_128x128x32_k9x9x5.npz")
TOL = {"fp32": 1e-5, "bf16": 1e-3}


@pytest.fixture(scope="module")
def setup():
    need_gpu()
    if not os.path.exists(GOLDEN):
        pytest.skip("stored oracle run not present")
    g = np.load(GOLDEN)
    w = synth.workload(2, n_ref=0)
    c = icnnm.Context(0)
    yield c, g, w
    c.close()


@pytest.mark.parametrize("prec", ["bf16", "fp32"])
def test_prediction_full_size(setup, prec):
    ctx, g, w = setup
    iters = int(g["iters"])
    L, st = ctx.icnnm_solve(w["M"], w["mask"], g["V"], w["kdims"], max_iters=iters, prec=prec)
    frames = g["frames"]
    msk = w["mask"].astype(bool)
    assert np.array_equal(L[msk], w["M"][msk])
    assert not msk[frames].any() and msk[np.setdiff1d(np.arange(L.shape[0]), frames)].all()
    Lo = L.astype(np.float64).copy()
    Lo[frames] = g["L_missing"]
    e = float(np.linalg.norm(L - Lo) / np.linalg.norm(Lo))
    assert e <= TOL[prec], (prec, e)
    assert abs(st["objective"] - float(g["objective"])) <= 10 * TOL[prec] * float(g["objective"])
    assert st["theta"] == pytest.approx(float(g["theta"]), rel=1e-12)
    assert st["iters"] == iters
