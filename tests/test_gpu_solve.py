"""GPU parity: libicnnm (through the C ABI) against the FP64 oracle on the same seeded
inputs. Tolerances: relative L2 <= 1e-5 for the FP32 path and <= 1e-3 for the BF16
path; observed entries bit-exact (lambda = inf)."""
import math

import numpy as np
import pytest

from oracle import icnnm_oracle as O
from paper_2604_17001_gb300 import icnnm, synth
from tests.gpu_util import need_gpu, rel

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "bf16": 1e-3, "bf16x3": 1e-4}


@pytest.fixture(scope="module")
def ctx():
    need_gpu()
    c = icnnm.Context(0)
    yield c
    c.close()


def case(dims, kdims, frac=None, last=None, seed=7, nref=3, vdims=None):
    H, W, T = dims
    L0 = synth.video(H, W, T, seed=seed)
    if last is not None:
        mask = synth.mask_last_frames(H, W, T, last)
    else:
        mask = synth.mask_uniform(H, W, T, frac, seed=seed + 1)
    M = np.where(mask.astype(bool), L0, 0).astype(np.float32)
    vd = vdims or dims
    refs = [synth.video(vd[0], vd[1], vd[2], seed=seed + 10 + j) for j in range(nref)]
    V, _ = O.learn_V(refs, kdims)
    return M, mask, V, L0


CASES = [
    # (dims H,W,T), kernel, mask, iterations
    ((32, 32, 8), (5, 5, 3), dict(frac=0.5), 100),          # completion workload shape
    ((21, 13, 5), (3, 4, 2), dict(frac=0.6), 40),           # ragged vs the 8x16 tile
    ((24, 16, 10), (9, 9, 5), dict(last=2), 40),            # k = 405, prediction mask
    ((37, 29, 1), (5, 5, 1), dict(frac=0.5), 60),           # 2-D image
    ((16, 40, 6), (7, 7, 3), dict(frac=0.4), 50),           # k = 147
    ((24, 40, 3), (3, 11, 2), dict(frac=0.5), 40),          # k2 = 11 (compile-time col2im, 2 tap rows a group)
    ((4, 4, 4), (4, 4, 4), dict(frac=0.7), 30),             # kernel = the whole tensor
    ((16, 16, 4), (1, 1, 1), dict(frac=0.5), 20),           # k = 1: V = [1]
    ((3, 5, 2), (2, 3, 2), dict(frac=0.6), 30),             # tensor smaller than one 8 x 16 voxel tile
    ((40, 40, 1), (32, 32, 1), dict(frac=0.5), 20),         # k = 1024, the largest kernel the library takes
]


# Where every voxel is coupled to every other within a few iterations (a kernel as large
# as the tensor, a tensor smaller than one voxel tile), the BF16 adjoint's rounding (U and
# V D in BF16; BF16X3 splits only the forward pass) dominates the error: a CPU emulation of
# exactly these roundings gives 1.26e-3 (BF16) and 6.3e-4 (BF16X3) for the whole-tensor
# kernel and 1.3e-4 (BF16X3) for the sub-tile tensor, which the GPU reproduces. Bars:
EDGE_TOL = {((4, 4, 4), (4, 4, 4)): {"bf16": 2e-3, "bf16x3": 1e-3},
            ((3, 5, 2), (2, 3, 2)): {"bf16x3": 2e-4}}


@pytest.mark.parametrize("prec", ["fp32", "bf16", "bf16x3"])
@pytest.mark.parametrize("dims,kdims,mk,iters", CASES)
def test_solve_matches_oracle(ctx, prec, dims, kdims, mk, iters):
    tol = EDGE_TOL.get((dims, kdims), {}).get(prec, TOL[prec])
    M, mask, V, _ = case(dims, kdims, **mk)
    Lo, so = O.icnnm_solve(M, mask, V, kdims, max_iters=iters)
    try:
        L, st = ctx.icnnm_solve(M, mask, V, kdims, max_iters=iters, prec=prec)
    except icnnm.ICNNMError as e:
        if e.status == icnnm.EUNSUPPORTED:
            pytest.skip(str(e))
        raise
    e = rel(L, Lo)
    assert e <= tol, (prec, dims, kdims, e)
    msk = mask.astype(bool)
    assert np.array_equal(L[msk], M[msk])                      # P_Omega(L) = P_Omega(M) exactly
    assert st["iters"] == iters
    assert abs(st["objective"] - so["objective"]) <= 10 * max(tol, 1e-5) * so["objective"]
    assert abs(st["theta"] - so["theta"]) <= 1e-6 * so["theta"]


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_penalised_lambda_1000(ctx, prec):
    # Eq. (admm) with the paper's lambda = 1000: observed entries are not pinned exactly
    M, mask, V, _ = case((24, 24, 6), (5, 5, 3), frac=0.5)
    Lo, _ = O.icnnm_solve(M, mask, V, (5, 5, 3), lam=1000.0, max_iters=60)
    try:
        L, _ = ctx.icnnm_solve(M, mask, V, (5, 5, 3), lam=1000.0, max_iters=60, prec=prec)
    except icnnm.ICNNMError as e:
        if e.status == icnnm.EUNSUPPORTED:
            pytest.skip(str(e))
        raise
    assert rel(L, Lo) <= TOL[prec]


def test_tolerance_stopping_matches_oracle(ctx):
    M, mask, V, _ = case((32, 24, 6), (5, 5, 3), frac=0.5)
    Lo, so = O.icnnm_solve(M, mask, V, (5, 5, 3), max_iters=300, tol=1e-4, check_every=10)
    L, st = ctx.icnnm_solve(M, mask, V, (5, 5, 3), max_iters=300, tol=1e-4, check_every=10, prec="fp32")
    assert st["iters"] == so["iters"] < 300
    assert rel(L, Lo) <= TOL["fp32"]
    assert abs(st["residual"] - so["residual"]) <= 2e-2 * so["residual"]   # FP32 sums of a cancelling quantity


# Every reduction of both paths is grouped by the job alone (the BF16 col2im adds 64-bit
# fixed-point values, whose sum does not depend on the order; the forward pass's column
# partials are kept per fixed chunk of the job's tiles), so a job's result is the same,
# bit for bit, alone, in a batch and in the serving mix.


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_batch_equals_single(ctx, prec):
    # Uneven problems stepped together give, bit for bit, the results of solving each
    # alone.
    # 100 iterations: mid-run the BF16 iterate is still at its transient error (~1e-3).
    kd = (5, 5, 3)
    its = 100
    probs = [case(d, kd, frac=f, seed=s) for d, f, s in [((32, 16, 8), 0.5, 1), ((16, 48, 5), 0.3, 2),
                                                         ((24, 24, 3), 0.7, 3)]]
    V = probs[0][2]
    try:
        outs, stats = ctx.icnnm_solve_batch([p[0] for p in probs], [p[1] for p in probs], V, kd,
                                            max_iters=its, prec=prec)
    except icnnm.ICNNMError as e:
        if e.status == icnnm.EUNSUPPORTED:
            pytest.skip(str(e))
        raise
    for (M, mask, _, _), Lb in zip(probs, outs):
        Ls, _ = ctx.icnnm_solve(M, mask, V, kd, max_iters=its, prec=prec)
        assert np.array_equal(Lb, Ls)
        Lo, _ = O.icnnm_solve(M, mask, V, kd, max_iters=its)
        assert rel(Lb, Lo) <= TOL[prec]


def test_device_pointers_and_torch_tensors(ctx):
    import torch
    M, mask, V, _ = case((32, 32, 4), (3, 3, 2), frac=0.5)
    Lh, _ = ctx.icnnm_solve(M, mask, V, (3, 3, 2), max_iters=20, prec="fp32")
    Md, kd_ = torch.from_numpy(M).cuda(), torch.from_numpy(mask).cuda()
    Ld, _ = ctx.icnnm_solve(Md, kd_, torch.from_numpy(V).cuda(), (3, 3, 2), max_iters=20, prec="fp32")
    assert np.array_equal(Ld.cpu().numpy(), Lh)


def test_invalid_inputs_are_rejected(ctx):
    M, mask, V, _ = case((16, 16, 4), (3, 3, 2), frac=0.5)
    with pytest.raises(icnnm.ICNNMError) as e:
        ctx.icnnm_solve(M, mask, V, (17, 3, 2))                # kernel larger than the tensor
    assert e.value.status == icnnm.EINVAL
    with pytest.raises(icnnm.ICNNMError) as e:
        ctx.icnnm_solve(M, mask, V * 1.01, (3, 3, 2))          # V not orthonormal
    assert e.value.status == icnnm.EINVAL
    with pytest.raises(icnnm.ICNNMError) as e:
        ctx.icnnm_solve(M, np.zeros_like(mask), V, (3, 3, 2))  # empty Omega
    assert e.value.status == icnnm.EINVAL
    Mn = M.copy()
    Mn.reshape(-1)[np.flatnonzero(mask.ravel())[0]] = np.nan
    with pytest.raises(icnnm.ICNNMError) as e:
        ctx.icnnm_solve(Mn, mask, V, (3, 3, 2))                # non-finite observed entry
    assert e.value.status == icnnm.EINVAL
    with pytest.raises(icnnm.ICNNMError) as e:
        ctx.icnnm_solve(M, mask, V, (3, 3, 2), rho=0.5)
    assert e.value.status == icnnm.EINVAL


def test_budget_enforced():
    need_gpu()
    M, mask, V, _ = case((64, 64, 16), (5, 5, 3), frac=0.5)
    with icnnm.Context(0, hbm_budget_bytes=1 << 20) as c:
        with pytest.raises(icnnm.ICNNMError) as e:
            c.icnnm_solve(M, mask, V, (5, 5, 3), max_iters=2, prec="fp32")
        assert e.value.status == icnnm.ENOMEM


def test_learn_V_matches_oracle(ctx):
    kd = (5, 5, 3)
    refs = [synth.video(32, 32, 8, seed=s) for s in range(1001, 1005)] + [synth.video(16, 24, 6, seed=77)]
    Vo, eo = O.learn_V(refs, kd)
    G = O.gram(refs, kd)
    V, e = ctx.icnnm_learn_V(refs, kd)
    k = 75
    assert np.max(np.abs(e - eo)) <= 2e-6 * eo[0]                    # FP32 products, FP64 sums
    np.testing.assert_allclose(V.T @ V, np.eye(k), atol=1e-12)       # FP64 Jacobi
    recon = (V * e[None, :]) @ V.T
    assert np.linalg.norm(recon - G) <= 2e-6 * np.linalg.norm(G)
    # well-separated leading eigenvectors agree up to the canonical sign (identical)
    gaps = np.abs(np.diff(eo))
    for i in range(8):
        gap = min(gaps[i], gaps[i - 1] if i > 0 else np.inf)
        if gap > 1e-3 * eo[0]:
            assert abs(abs(V[:, i] @ Vo[:, i]) - 1) <= 1e-6, i   # the sign rule can tie
    for i in range(k):
        assert V[np.argmax(np.abs(V[:, i])), i] > 0


def test_serving_submit_poll_equals_solve(ctx):
    kd = (5, 5, 3)
    probs = [case(d, kd, frac=f, seed=s) for d, f, s in [((32, 16, 8), 0.5, 11), ((16, 48, 5), 0.3, 12),
                                                         ((24, 24, 3), 0.7, 13), ((32, 32, 6), 0.5, 14)]]
    V = probs[0][2]
    ids = [ctx.icnnm_submit(M, mask, V, kd, max_iters=25, prec="fp32") for M, mask, _, _ in probs]
    for (M, mask, _, _), jid in zip(probs, ids):
        L = np.zeros_like(M)
        st, stats = ctx.icnnm_wait(jid, L_out=L, timeout_ms=120000)
        assert st == icnnm.OK and stats["iters"] == 25
        Ls, _ = ctx.icnnm_solve(M, mask, V, kd, max_iters=25, prec="fp32")
        assert np.array_equal(L, Ls)
    with pytest.raises(icnnm.ICNNMError) as e:
        ctx.icnnm_poll(ids[0])
    assert e.value.status == icnnm.ENOTFOUND


def test_serving_bf16_mix_equals_alone_and_oracle(ctx):
    # Served BF16: jobs of different sizes and masks admitted while others run give, in the
    # mix, bit for bit the result of solving each alone, and the oracle's within 1e-3.
    kd = (5, 5, 3)
    its = 60
    probs = [case(d, kd, frac=f, seed=s) for d, f, s in [((32, 16, 8), 0.5, 21), ((16, 48, 5), 0.3, 22),
                                                         ((24, 24, 3), 0.7, 23), ((40, 32, 6), 0.5, 24),
                                                         ((21, 13, 5), 0.6, 25)]]
    V = probs[0][2]
    ids = [ctx.icnnm_submit(M, mask, V, kd, max_iters=its, prec="bf16") for M, mask, _, _ in probs]
    for (M, mask, _, _), jid in zip(probs, ids):
        L = np.zeros_like(M)
        st, stats = ctx.icnnm_wait(jid, L_out=L, timeout_ms=120000)
        assert st == icnnm.OK and stats["iters"] == its
        msk = mask.astype(bool)
        assert np.array_equal(L[msk], M[msk])
        Ls, _ = ctx.icnnm_solve(M, mask, V, kd, max_iters=its, prec="bf16")
        assert np.array_equal(L, Ls)
        Lo, _ = O.icnnm_solve(M, mask, V, kd, max_iters=its)
        assert rel(L, Lo) <= TOL["bf16"]


@pytest.mark.parametrize("serve", [False, True])
def test_bf16_tolerance_finishes_in_fp32(ctx, serve):
    # U is stored in BF16, so the BF16 residual stalls near 1e-3; with tol = 1e-3 a BF16
    # job finishes its last iterations in FP32 and stops on an exact residual, like the
    # oracle under the same rule.
    kd = (5, 5, 3)
    M, mask, V, _ = case((32, 24, 8), kd, frac=0.5, seed=31)
    kw = dict(max_iters=1000, tol=1e-3, check_every=10)
    Lo, so = O.icnnm_solve(M, mask, V, kd, **kw)
    if serve:
        jid = ctx.icnnm_submit(M, mask, V, kd, prec="bf16", **kw)
        L = np.zeros_like(M)
        r, st = ctx.icnnm_wait(jid, L_out=L, timeout_ms=120000)
        assert r == icnnm.OK
    else:
        L, st = ctx.icnnm_solve(M, mask, V, kd, prec="bf16", **kw)
    assert st["iters"] < 1000 and st["residual"] <= 1e-3
    assert abs(st["iters"] - so["iters"]) <= 30
    msk = mask.astype(bool)
    assert np.array_equal(L[msk], M[msk])
    # the iterate is unique for a given iteration count; the stopping check may land one
    # check apart on the two sides, so compare with the oracle run for the same count
    Lo, _ = O.icnnm_solve(M, mask, V, kd, max_iters=st["iters"])
    assert rel(L, Lo) <= TOL["bf16"]


def test_bf16_tolerance_batch_mixed_phases(ctx):
    # Jobs of one batch reach the FP32 finish at different checks, so BF16 and FP32 lists
    # step side by side. Each job stops on an exact residual <= tol, near the oracle's
    # stopping iteration, equals the same job solved alone (to the BF16 bar), and is
    # within the BF16 bar of the FP64 oracle run for the same iteration count. The
    # residual is checked every iteration, so that the stopping points of the batch and
    # of the single solves are at most an iteration apart.
    kd = (5, 5, 3)
    kw = dict(max_iters=1000, tol=1e-3, check_every=1)
    probs = [case(d, kd, frac=f, seed=s) for d, f, s in [((32, 24, 8), 0.5, 41), ((16, 40, 6), 0.3, 42),
                                                         ((24, 24, 5), 0.7, 43)]]
    V = probs[0][2]
    outs, stats = ctx.icnnm_solve_batch([p[0] for p in probs], [p[1] for p in probs], V, kd, prec="bf16", **kw)
    for (M, mask, _, _), L, st in zip(probs, outs, stats):
        assert st["iters"] < 1000 and st["residual"] <= 1e-3
        _, so = O.icnnm_solve(M, mask, V, kd, **kw)
        assert abs(st["iters"] - so["iters"]) <= 30
        assert np.array_equal(L[mask.astype(bool)], M[mask.astype(bool)])
        Ls, sts = ctx.icnnm_solve(M, mask, V, kd, prec="bf16", **kw)
        assert st["iters"] == sts["iters"] and np.array_equal(L, Ls)
        Lo, _ = O.icnnm_solve(M, mask, V, kd, max_iters=st["iters"])
        assert rel(L, Lo) <= TOL["bf16"], (M.shape, st["iters"], rel(L, Lo))


def test_bf16_batch_with_long_mixed_phase(ctx):
    # Two jobs whose BF16 phases end far apart (the FP64 oracle under the same rule stops
    # them after 32 and 71 iterations): the first finishes in FP32 while the second is
    # still in BF16, so the blocking batch steps a BF16 list and an FP32 list side by side
    # (each with its own device job table). Every job must end as it does alone.
    kd = (5, 5, 3)
    kw = dict(max_iters=1000, tol=1e-4, check_every=1)
    V, _ = O.learn_V([synth.video(32, 24, 8, seed=61 + j) for j in range(3)], kd)
    jobs = []
    for (H, W, T), mk in (((24, 24, 8), lambda: synth.mask_uniform(24, 24, 8, 0.2, seed=61)),
                          ((32, 32, 16), lambda: synth.mask_last_frames(32, 32, 16, 6))):
        L0 = synth.video(H, W, T, seed=60)
        mask = mk()
        jobs.append((np.where(mask.astype(bool), L0, 0).astype(np.float32), mask))
    outs, stats = ctx.icnnm_solve_batch([j[0] for j in jobs], [j[1] for j in jobs], V, kd, prec="bf16", **kw)
    assert stats[1]["iters"] > stats[0]["iters"] + 20
    for (M, mask), L, st in zip(jobs, outs, stats):
        assert st["residual"] <= 1e-4
        assert np.array_equal(L[mask.astype(bool)], M[mask.astype(bool)])
        Ls, sts = ctx.icnnm_solve(M, mask, V, kd, prec="bf16", **kw)
        # the same, bit for bit (stepping the BF16 list with the finishing list's job table
        # once put them 1.4e-4 apart and one iteration off)
        assert st["iters"] == sts["iters"]
        assert np.array_equal(L, Ls)
