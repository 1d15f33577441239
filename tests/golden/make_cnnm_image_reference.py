"""Writes the FP64 oracle's CNNM result (Eq. cnnm; SVT of A_k(L) - Y/theta every
iteration, dense SVD) for the image-completion inputs (200x200 image, kernel 13x13,
4x4-pixel blocks missing at 50%) after 200 iterations to cnnm_image_200x200_k13x13.npz:
the completed image and its nuclear norm ||A_k(L)||_*. Calls only oracle/ (and the
seeded input generators).

    python tests/golden/make_cnnm_image_reference.py [--iters N]
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

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "cnnm_image_200x200_k13x13.npz")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--iters", type=int, default=200)
    a = ap.parse_args()
    w = synth.workload(6, n_ref=0)
    t0 = time.time()
    L = O.cnnm_solve(w["M"], w["mask"], w["kdims"], max_iters=a.iters)
    nuc = float(np.linalg.svd(O.conv_matrix(L, w["kdims"]), compute_uv=False).sum())
    print(f"oracle CNNM: {time.time() - t0:.0f} s, nuclear norm {nuc}", flush=True)
    np.savez_compressed(OUT, L=L, nuclear_norm=nuc, iters=a.iters)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
