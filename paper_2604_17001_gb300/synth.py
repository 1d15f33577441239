"""Seeded synthetic inputs for ICNNM workloads (targets, reference tensors, masks).

This module holds no arithmetic of the completion method itself: it only draws
smooth "video-like" tensors and sampling masks. Both the FP64 oracle tests and the
GPU path take their inputs from here, so that the two sides see identical data.

The paper's experiments use CDNet 2014 (50x50x31 videos, Sec. V-B/C), UCF-101
(256x256x3, Sec. V-D) and Kodak/CSet8 (200x200 images, Sec. V-A). None of those
datasets is available, so these generators stand in for "smooth video": a sum of
translating 2D sinusoids plus linearly moving Gaussian blobs, rescaled to [0, 1].

Layout: a tensor of dims (H, W, T) is stored as a numpy array of shape (T, H, W),
C order, so the linear voxel index is i = (t*H + h)*W + w.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "video", "mask_uniform", "mask_last_frames", "mask_every_other_frame",
    "mask_drop_frames_plus_random", "mask_block_holes", "mask_mixed",
    "workload", "WORKLOADS", "seed_for", "image_jobs", "serving_shapes", "serving_job", "serving_refs",
]


def seed_for(config: int, slot: int) -> int:
    """Seed convention: target = 1000*c + 0, reference tensors 1000*c + 1..b,
    masks 1000*c + 500 (+ job index for multi-job workloads)."""
    return 1000 * config + slot


def video(H: int, W: int, T: int, seed: int, noise_var: float = 0.0,
          n_sines: int = 3, dtype=np.float32) -> np.ndarray:
    """A smooth synthetic video of shape (T, H, W) with values in [0, 1].

    - ``n_sines`` translating plane waves: spatial frequency uniform in the disc of
      radius 4 cycles/frame, phase U(0, 2pi), velocity magnitude U(0, 1) px/frame in
      a random direction, amplitude U(0.2, 1).
    - 2..4 Gaussian blobs: sigma U(3, 6) px, amplitude U(0.2, 1), start uniform in the
      frame, linear velocity of magnitude <= 1 px/frame, wrapped periodically.
    - min-max rescaled to [0, 1]; then, if ``noise_var`` > 0, N(0, noise_var) noise
      is added (the variance is ``noise_var``).
    """
    rng = np.random.default_rng(seed)
    t = np.arange(T, dtype=np.float64)[:, None, None]
    h = np.arange(H, dtype=np.float64)[None, :, None]
    w = np.arange(W, dtype=np.float64)[None, None, :]
    out = np.zeros((T, H, W), dtype=np.float64)
    for _ in range(n_sines):
        r = 4.0 * np.sqrt(rng.uniform())
        ang = rng.uniform(0, 2 * np.pi)
        fh, fw = r * np.sin(ang), r * np.cos(ang)          # cycles per frame
        phase = rng.uniform(0, 2 * np.pi)
        vmag = rng.uniform(0, 1)
        vang = rng.uniform(0, 2 * np.pi)
        vh, vw = vmag * np.sin(vang), vmag * np.cos(vang)  # px per frame
        amp = rng.uniform(0.2, 1.0)
        out += amp * np.sin(2 * np.pi * (fh * (h - vh * t) / H + fw * (w - vw * t) / W) + phase)
    nblobs = int(rng.integers(2, 5))
    for _ in range(nblobs):
        sig = rng.uniform(3, 6)
        amp = rng.uniform(0.2, 1.0)
        h0, w0 = rng.uniform(0, H), rng.uniform(0, W)
        vmag = rng.uniform(0, 1)
        vang = rng.uniform(0, 2 * np.pi)
        vh, vw = vmag * np.sin(vang), vmag * np.cos(vang)
        ch = (h0 + vh * t) % H
        cw = (w0 + vw * t) % W
        dh = np.abs(h - ch)
        dh = np.minimum(dh, H - dh)
        dw = np.abs(w - cw)
        dw = np.minimum(dw, W - dw)
        out += amp * np.exp(-(dh ** 2 + dw ** 2) / (2 * sig * sig))
    lo, hi = out.min(), out.max()
    out = (out - lo) / (hi - lo) if hi > lo else np.zeros_like(out)
    if noise_var > 0:
        out = out + rng.normal(0.0, np.sqrt(noise_var), size=out.shape)
    return out.astype(dtype)


def mask_uniform(H, W, T, observed_frac: float, seed: int) -> np.ndarray:
    """0/1 mask (uint8, shape (T, H, W)) with round(observed_frac*m) observed entries
    chosen uniformly at random."""
    m = H * W * T
    rng = np.random.default_rng(seed)
    idx = rng.permutation(m)[: int(round(observed_frac * m))]
    mask = np.zeros(m, dtype=np.uint8)
    mask[idx] = 1
    return mask.reshape(T, H, W)


def mask_last_frames(H, W, T, n_missing: int) -> np.ndarray:
    """Frames 0..T-n_missing-1 fully observed; the last n_missing frames missing
    (the video-prediction setting)."""
    mask = np.ones((T, H, W), dtype=np.uint8)
    if n_missing > 0:
        mask[T - n_missing:] = 0
    return mask


def mask_every_other_frame(H, W, T) -> np.ndarray:
    """Odd frames missing, even frames observed (frame interpolation)."""
    mask = np.ones((T, H, W), dtype=np.uint8)
    mask[1::2] = 0
    return mask


def mask_drop_frames_plus_random(H, W, T, drop_frac: float, seed: int) -> np.ndarray:
    """Every other frame dropped, plus ``drop_frac`` of the entries of the remaining
    frames dropped uniformly at random."""
    mask = mask_every_other_frame(H, W, T)
    rng = np.random.default_rng(seed)
    keep = mask.astype(bool)
    cand = np.flatnonzero(keep.ravel())
    n_drop = int(round(drop_frac * cand.size))
    drop = rng.permutation(cand)[:n_drop]
    flat = mask.ravel().copy()
    flat[drop] = 0
    return flat.reshape(T, H, W)


def mask_block_holes(H, W, T, seed: int, block: int = 16, hole_frac: float = 0.3) -> np.ndarray:
    """Square ``block``x``block`` holes (all frames of a hole missing at that place
    in a random subset of frames): about ``hole_frac`` of the blocks of each frame
    are missing."""
    rng = np.random.default_rng(seed)
    mask = np.ones((T, H, W), dtype=np.uint8)
    nbh, nbw = max(1, H // block), max(1, W // block)
    for t in range(T):
        sel = rng.uniform(size=(nbh, nbw)) < hole_frac
        for bh in range(nbh):
            for bw in range(nbw):
                if sel[bh, bw]:
                    mask[t, bh * block:(bh + 1) * block, bw * block:(bw + 1) * block] = 0
    if mask.sum() == 0:
        mask[0, 0, 0] = 1
    return mask


def mask_mixed(H, W, T, seed: int) -> tuple[np.ndarray, str]:
    """One of the four mask families, chosen uniformly: 30-70% uniform-random
    observed, last-k frames missing, every other frame missing, 16x16 block holes."""
    rng = np.random.default_rng(seed)
    fam = int(rng.integers(0, 4))
    if fam == 0:
        frac = float(rng.uniform(0.3, 0.7))
        return mask_uniform(H, W, T, frac, seed + 7), f"uniform{frac:.2f}"
    if fam == 1:
        kmiss = int(rng.integers(1, max(2, T // 4) + 1))
        return mask_last_frames(H, W, T, kmiss), f"last{kmiss}"
    if fam == 2:
        return mask_every_other_frame(H, W, T), "every_other"
    return mask_block_holes(H, W, T, seed + 11), "holes16"


# The five workload families (shapes, kernels, masks, reference-tensor counts).
WORKLOADS = {
    1: dict(name="completion_32x32x8_k5x5x3", dims=(32, 32, 8), kdims=(5, 5, 3),
            n_ref=16, iters=100, mask="uniform50"),
    2: dict(name="prediction_128x128x32_k9x9x5", dims=(128, 128, 32), kdims=(9, 9, 5),
            n_ref=64, iters=500, mask="last8"),
    3: dict(name="interpolation_256x256x64_k7x7x5", dims=(256, 256, 64), kdims=(7, 7, 5),
            n_ref=16, iters=100, mask="every_other+20pct", noise_var=0.01),
    4: dict(name="batch64_uneven_k7x7x3", dims=None, kdims=(7, 7, 3), n_ref=32,
            iters=100, mask="mixed", n_jobs=64),
    5: dict(name="serving_poisson2000_k7x7x3", dims=None, kdims=(7, 7, 3), n_ref=32,
            iters=None, mask="mixed", n_jobs=2000),
    # image completion (Sec. V-A): 200x200 images, 13x13 kernel, V from 7 reference
    # images, masks of 4x4 pixel blocks (adjacent pixels tend to be missing together)
    6: dict(name="image_200x200_k13x13", dims=(200, 200, 1), kdims=(13, 13, 1), n_ref=7,
            iters=500, mask="blocks4_50pct", n_images=24),
}


def _mask_for(cfg: int, H, W, T):
    if cfg == 1:
        return mask_uniform(H, W, T, 0.5, seed_for(1, 500))
    if cfg == 2:
        return mask_last_frames(H, W, T, 8 if T >= 16 else max(1, T // 4))
    if cfg == 3:
        return mask_drop_frames_plus_random(H, W, T, 0.2, seed_for(3, 500))
    if cfg == 6:
        return mask_block_holes(H, W, T, seed_for(6, 500), block=4, hole_frac=0.5)
    raise ValueError(cfg)


def workload(cfg: int, dims=None, n_ref=None):
    """Inputs of a single-tensor workload family.

    Returns dict(L0, M, mask, refs, dims, kdims): ``L0`` the clean target, ``M`` the
    observation tensor (target plus noise where the family has noise; entries outside
    the mask are set to 0), ``refs`` the reference tensors for learning V.
    ``dims`` (H, W, T) and ``n_ref`` may be overridden for reduced-size cases.
    """
    spec = WORKLOADS[cfg]
    H, W, T = dims if dims is not None else spec["dims"]
    nref = spec["n_ref"] if n_ref is None else n_ref
    nv = spec.get("noise_var", 0.0)
    L0 = video(H, W, T, seed_for(cfg, 0))
    noisy = video(H, W, T, seed_for(cfg, 0), noise_var=nv) if nv > 0 else L0
    mask = _mask_for(cfg, H, W, T)
    M = np.where(mask.astype(bool), noisy, 0).astype(np.float32)
    refs = [video(H, W, T, seed_for(cfg, j)) for j in range(1, nref + 1)]
    return dict(L0=L0, M=M, mask=mask, refs=refs, dims=(H, W, T), kdims=spec["kdims"])


def batch_shapes(n_jobs: int, seed: int, hw_range=(32, 192), t_range=(8, 48), step=16):
    """Uneven job shapes: H, W uniform in {lo..hi} step ``step``; T uniform in t_range."""
    rng = np.random.default_rng(seed)
    hs = np.arange(hw_range[0], hw_range[1] + 1, step)
    out = []
    for _ in range(n_jobs):
        out.append((int(rng.choice(hs)), int(rng.choice(hs)), int(rng.integers(t_range[0], t_range[1] + 1))))
    return out


def batch_jobs(n_jobs: int, cfg: int = 4, hw_range=(32, 192), t_range=(8, 48)):
    """Jobs of the batching/serving families: list of dict(M, mask, dims, L0, family)."""
    shapes = batch_shapes(n_jobs, seed_for(cfg, 900), hw_range, t_range)
    jobs = []
    for j, (H, W, T) in enumerate(shapes):
        L0 = video(H, W, T, seed_for(cfg, 2000 + j))
        mask, fam = mask_mixed(H, W, T, seed_for(cfg, 500) + 13 * j)
        M = np.where(mask.astype(bool), L0, 0).astype(np.float32)
        jobs.append(dict(L0=L0, M=M, mask=mask, dims=(H, W, T), family=fam))
    return jobs


SERVING_HW = (32, 256)
SERVING_T = (8, 64)


def serving_shapes(n_requests: int):
    """Shapes of the serving stream: H, W uniform in {32..256} step 16, T uniform in
    {8..64} (the batching family's draws with the serving ranges)."""
    return batch_shapes(n_requests, seed_for(5, 900), SERVING_HW, SERVING_T)


def serving_job(j: int, shapes):
    """Request j of the serving stream (shapes from serving_shapes): dict(L0, M, mask,
    dims, family), generated on its own, identical to the j-th entry of
    batch_jobs(n, cfg=5, hw_range=SERVING_HW, t_range=SERVING_T)."""
    H, W, T = shapes[j]
    L0 = video(H, W, T, seed_for(5, 2000 + j))
    mask, fam = mask_mixed(H, W, T, seed_for(5, 500) + 13 * j)
    M = np.where(mask.astype(bool), L0, 0).astype(np.float32)
    return dict(L0=L0, M=M, mask=mask, dims=(H, W, T), family=fam)


def serving_refs():
    """Reference tensors of the serving family's shared V: 32 videos of 64x64x16."""
    return [video(64, 64, 16, seed_for(5, j)) for j in range(1, WORKLOADS[5]["n_ref"] + 1)]


def image_jobs(n_images: int, missing: float = 0.5, dims=(200, 200)):
    """Targets of the image-completion family: n_images smooth images (T = 1) with
    masks of 4x4 pixel blocks, about ``missing`` of them missing. Returns a list of
    dict(L0, M, mask, dims)."""
    H, W = dims
    jobs = []
    for j in range(n_images):
        L0 = video(H, W, 1, seed_for(6, 100 + j))
        mask = mask_block_holes(H, W, 1, seed_for(6, 500) + j, block=4, hole_frac=missing)
        M = np.where(mask.astype(bool), L0, 0).astype(np.float32)
        jobs.append(dict(L0=L0, M=M, mask=mask, dims=(H, W, 1)))
    return jobs
