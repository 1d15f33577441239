"""Writes the FP64 oracle's result for the image-completion workload (200x200 image,
kernel 13x13, 4x4-pixel blocks missing at 50%, V learned from 7 reference images,
500 ADMM iterations, lambda = infinity) to image_200x200_k13x13.npz: V (the solve's
input), the completed image, the objective and the final penalty. Calls only oracle/
(and the seeded input generators).

    python tests/golden/make_image_reference.py [--iters N]
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

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "image_200x200_k13x13.npz")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--iters", type=int, default=500)
    a = ap.parse_args()
    w = synth.workload(6)
    t0 = time.time()
    V, sig = O.learn_V(w["refs"], w["kdims"])
    L, st = O.icnnm_solve(w["M"], w["mask"], V, w["kdims"], max_iters=a.iters)
    print(f"oracle: {time.time() - t0:.0f} s, {st}", flush=True)
    np.savez_compressed(OUT, V=V, sigma=sig, L=L, objective=st["objective"], theta=st["theta"],
                        iters=st["iters"])
    print("wrote", OUT)


if __name__ == "__main__":
    main()
