"""Writes the FP64 oracle's result for the video-prediction workload (128x128x32,
kernel 9x9x5, frames 24..31 missing, V learned from 64 reference tensors, 500 ADMM
iterations) to prediction_128x128x32_k9x9x5.npz. Calls only oracle/ (and the seeded
input generators). The file holds V (the solve's input), the completed unobserved
frames, the objective and the final penalty.

    python tests/golden/make_prediction_reference.py [--iters N] [--refs B]
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

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "prediction_128x128x32_k9x9x5.npz")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--iters", type=int, default=500)
    ap.add_argument("--refs", type=int, default=64)
    a = ap.parse_args()
    w = synth.workload(2, n_ref=a.refs)
    t0 = time.time()
    V, sig = O.learn_V(w["refs"], w["kdims"])
    print(f"learn_V: {time.time() - t0:.0f} s", flush=True)
    t0 = time.time()
    L, st = O.icnnm_solve(w["M"], w["mask"], V, w["kdims"], max_iters=a.iters)
    print(f"solve: {time.time() - t0:.0f} s, {st}", flush=True)
    miss = ~w["mask"].astype(bool)
    frames = np.flatnonzero(miss.reshape(miss.shape[0], -1).any(axis=1))
    np.savez_compressed(OUT, V=V, sigma=sig, frames=frames, L_missing=L[frames].astype(np.float64),
                        objective=st["objective"], theta=st["theta"], iters=st["iters"],
                        L_norm=np.linalg.norm(L))
    print("wrote", OUT)


if __name__ == "__main__":
    main()
