"""Tile configurations of the tensor-core passes (no paper counterpart: a performance
choice). Every geometry the autotuner can pick (adjoint tap tiles of 128 or 256 columns,
forward channel tiles of 128 or all channels, one or two forward U stages) must give the
oracle's iterate within the BF16 bar, and the autotuner must adopt one of the candidates it
measured."""
import numpy as np
import pytest

from oracle import icnnm_oracle as O
from paper_2604_17001_gb300 import icnnm, synth
from tests.gpu_util import need_gpu, rel

pytestmark = pytest.mark.gpu

KD = (7, 7, 3)
ITERS = 40
# plain BF16 over a fixed 40 iterations of this small, half-observed job sits near 1e-3 from
# FP64 whatever the tiles (the precision tests hold the workloads and served runs to 1e-3);
# the tile geometries are compared with each other to 2e-4
BF16_FIXED_BAR = 1.5e-3


@pytest.fixture(scope="module")
def problem():
    need_gpu()
    V, _ = O.learn_V([synth.video(32, 32, 8, synth.seed_for(5, j)) for j in range(1, 4)], KD)
    H, W, T = 40, 32, 8
    L0 = synth.video(H, W, T, seed=81)
    mask = synth.mask_uniform(H, W, T, 0.5, seed=82)
    M = np.where(mask.astype(bool), L0, 0).astype(np.float32)
    Lo, _ = O.icnnm_solve(M, mask, V, KD, max_iters=ITERS)
    with icnnm.Context(0, tile_table=None) as ctx:
        Ld, _ = ctx.icnnm_solve(M, mask, V, KD, max_iters=ITERS, prec="bf16")      # narrow tiles
    return V, M, mask, Lo, Ld


@pytest.mark.parametrize("adj,fwd,stages", [(128, 128, 2), (256, 128, 2), (128, 256, 2), (256, 256, 1), (0, 0, 0)])
def test_every_tile_geometry_matches_oracle(problem, adj, fwd, stages):
    # within the BF16 bar of the oracle, and close to the narrow tiles' result (the
    # geometries differ only in the order of FP32 additions)
    V, M, mask, Lo, Ld = problem
    with icnnm.Context(0, tile_table=None) as ctx:
        ctx.icnnm_set_tile_config(KD, adj, fwd, stages)
        L, _ = ctx.icnnm_solve(M, mask, V, KD, max_iters=ITERS, prec="bf16")
    assert rel(L, Lo) <= BF16_FIXED_BAR
    assert rel(L, Ld) <= 2e-4
    assert np.array_equal(L[mask.astype(bool)], M[mask.astype(bool)])


def test_autotune_adopts_a_measured_candidate(problem):
    V, M, mask, Lo, _ = problem
    with icnnm.Context(0, tile_table=None) as ctx:
        best, res = ctx.icnnm_autotune([(40, 32, 8), (32, 48, 10)], KD, V, iters=4)
        assert len(res) >= 2 and all(r["ms_per_iter"] > 0 for r in res)
        fastest = min(res, key=lambda r: r["ms_per_iter"])
        assert best["adj_tap_width"] in (128, 256) and best["fwd_u_stages"] in (1, 2)
        # the adopted configuration is used from now on, and still solves correctly
        L, _ = ctx.icnnm_solve(M, mask, V, KD, max_iters=ITERS, prec="bf16")
        assert rel(L, Lo) <= BF16_FIXED_BAR
        assert fastest["ms_per_iter"] <= min(r["ms_per_iter"] for r in res)
        with pytest.raises(icnnm.ICNNMError) as e:
            ctx.icnnm_set_tile_config(KD, 192, 0, 0)
        assert e.value.status == icnnm.EINVAL


def test_nondeterministic_mode_matches_oracle(problem):
    # float atomics and a round-robin tile order: the iterate within the BF16 bar, but not
    # reproducible (two solves of this job have been measured 1.3e-3 apart, the order of
    # the atomic additions amplified by the BF16 iteration)
    V, M, mask, Lo, Ld = problem
    with icnnm.Context(0, tile_table=None) as ctx:
        ctx.icnnm_set_deterministic(False)
        L, _ = ctx.icnnm_solve(M, mask, V, KD, max_iters=ITERS, prec="bf16")
        L2, _ = ctx.icnnm_solve(M, mask, V, KD, max_iters=ITERS, prec="bf16")
    assert rel(L, Lo) <= BF16_FIXED_BAR and rel(L2, Lo) <= BF16_FIXED_BAR
    assert rel(L, Ld) <= 3e-3 and rel(L2, L) <= 3e-3
    assert np.array_equal(L[mask.astype(bool)], M[mask.astype(bool)])


def test_deterministic_mode_repeats_bit_for_bit(problem):
    V, M, mask, Lo, Ld = problem
    with icnnm.Context(0, tile_table=None) as ctx:
        L, _ = ctx.icnnm_solve(M, mask, V, KD, max_iters=ITERS, prec="bf16")
    assert np.array_equal(L, Ld)
