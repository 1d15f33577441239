"""Writes the FP64 oracle's result for the frame-interpolation workload (256x256x64,
kernel 7x7x5, every other frame dropped plus 20% of the remaining entries, noise
variance 0.01, V learned from 16 reference tensors, 100 ADMM iterations) to
interpolation_256x256x64_k7x7x5.npz. Calls only oracle/ (and the seeded input
generators). The full result is 32 MB in FP64, so the file keeps V (the solve's input),
the values at 65536 voxels drawn with a fixed seed, the norm of the whole result, the
objective and the final penalty.

    python tests/golden/make_interpolation_reference.py [--iters N] [--refs B]
"""
import argparse
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import icnnm_oracle as O  # noqa: E402
from paper_2604_17001_gb300 import synth  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "interpolation_256x256x64_k7x7x5.npz")
NSAMPLE = 65536
SAMPLE_SEED = 3999


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--iters", type=int, default=100)
    ap.add_argument("--refs", type=int, default=16)
    a = ap.parse_args()
    w = synth.workload(3, n_ref=a.refs)
    t0 = time.time()
    V, sig = O.learn_V(w["refs"], w["kdims"])
    print(f"learn_V: {time.time() - t0:.0f} s", flush=True)
    del w["refs"]
    t0 = time.time()
    L, st = O.icnnm_solve(w["M"], w["mask"], V, w["kdims"], max_iters=a.iters)
    print(f"solve: {time.time() - t0:.0f} s, {st}", flush=True)
    rng = np.random.default_rng(SAMPLE_SEED)
    idx = np.sort(rng.choice(L.size, size=NSAMPLE, replace=False))
    np.savez_compressed(OUT, V=V, sigma=sig, sample_idx=idx, L_sample=L.reshape(-1)[idx].astype(np.float64),
                        objective=st["objective"], theta=st["theta"], iters=st["iters"],
                        L_norm=np.linalg.norm(L))
    print("wrote", OUT)


if __name__ == "__main__":
    main()
