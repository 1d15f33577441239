"""Writes the FP64 oracle's result for the completion workload (32x32x8, kernel 5x5x3,
50% of the entries observed uniformly at random, V learned from 16 reference tensors,
100 ADMM iterations) to completion_32x32x8_k5x5x3.npz: V (the solve's input), the whole
result, the objective and the final penalty. Calls only oracle/ (and the seeded input
generators).

    python tests/golden/make_completion_reference.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import icnnm_oracle as O  # noqa: E402
from paper_2604_17001_gb300 import synth  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "completion_32x32x8_k5x5x3.npz")


def main():
    w = synth.workload(1)
    V, sig = O.learn_V(w["refs"], w["kdims"])
    L, st = O.icnnm_solve(w["M"], w["mask"], V, w["kdims"], max_iters=synth.WORKLOADS[1]["iters"])
    np.savez_compressed(OUT, V=V, sigma=sig, L=L.astype(np.float64), objective=st["objective"], theta=st["theta"],
                        iters=st["iters"])
    print("wrote", OUT, st)


if __name__ == "__main__":
    main()
