"""learn_V at the kernel sizes of the benchmarks (Sec. III-C, Eq. A) against the stored
FP64 oracle runs: k = 405 (9x9x5, 64 reference tensors of 128x128x32, the video-
prediction workload) and k = 245 (7x7x5, 16 reference tensors of 256x256x64, the
interpolation workload). The stored files (tests/golden/*.npz, written by scripts that
call only the oracle) hold the oracle's eigenvalues sigma and eigenvectors V.

Compared: the eigenvalues (FP32 products summed in FP64 on the GPU: to 2e-6 of the
largest), the Gram they reconstruct (V diag(sigma) V^T, to 2e-6), orthonormality of V
(FP64 Jacobi), and the leading eigenvectors whose eigenvalue is well separated from its
neighbours (equal up to the canonical sign, which both sides fix the same way)."""
import os

import numpy as np
import pytest

from paper_2604_17001_gb300 import icnnm, synth
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("cfg,fname", [(2, "prediction_128x128x32_k9x9x5.npz"),
                                       (3, "interpolation_256x256x64_k7x7x5.npz")])
def test_learn_V_full_size_matches_stored_oracle(cfg, fname):
    need_gpu()
    import torch
    g = np.load(os.path.join(GOLDEN, fname))
    Vo, so = g["V"], g["sigma"]
    k = len(so)
    spec = synth.WORKLOADS[cfg]
    H, W, T = spec["dims"]
    with icnnm.Context(0) as ctx:
        refs = [torch.from_numpy(synth.video(H, W, T, synth.seed_for(cfg, j))).cuda()
                for j in range(1, spec["n_ref"] + 1)]
        V, e = ctx.icnnm_learn_V(refs, spec["kdims"])
    assert np.max(np.abs(e - so)) <= 2e-6 * so[0]
    np.testing.assert_allclose(V.T @ V, np.eye(k), atol=1e-11)
    G, Go = (V * e[None, :]) @ V.T, (Vo * so[None, :]) @ Vo.T
    assert np.linalg.norm(G - Go) <= 2e-6 * np.linalg.norm(Go)
    # eigenvectors: by Davis-Kahan, an eigenvector whose eigenvalue is `gap` away from the
    # others moves by at most sin(angle) <= ||dG|| / gap; with ||dG|| <= 2e-6 sigma_0 (the
    # eigenvalue bar above) and a factor 10 of margin, check every leading vector whose
    # bound is below 0.5, up to sign: the Gram is a multilevel Toeplitz matrix, so many
    # eigenvectors are antisymmetric under reversing the taps, their largest entries come
    # in pairs of equal magnitude and opposite sign, and the sign rule (largest entry
    # positive, ties to the lowest index) is then decided by rounding on either side
    gaps = np.abs(np.diff(so))
    checked = 0
    for i in range(16):
        gap = min(gaps[i], gaps[i - 1] if i > 0 else np.inf)
        bound = 2e-5 * so[0] / gap
        if bound < 0.5:
            c = abs(float(V[:, i] @ Vo[:, i]))
            assert np.sqrt(max(0.0, 1 - c * c)) <= bound, (i, c, bound)
            checked += 1
    assert checked >= 4
    for i in range(k):
        assert V[np.argmax(np.abs(V[:, i])), i] > 0
