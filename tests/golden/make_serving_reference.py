"""Writes the FP64 oracle's iterates for a fixed sample of requests of the serving stream
(2000 requests, H, W in 32..256 step 16, T in 8..64, kernel 7x7x3, the four mask
families; V learned from the family's 32 reference tensors of 64x64x16) to
serving_k7x7x3_sample.npz. Calls only oracle/ (and the seeded input generators).

Each sampled request is solved with the serving rule (relative residual <= 1e-3 checked
every 10 iterations) and, past its stopping check, for 40 more iterations; the file
holds, for every multiple of 10 iterations, the oracle's L at 4096 seeded unobserved
voxels and its residual, so that a served result that stopped at any of those checks can
be compared with the oracle iterate of the same count.

    python tests/golden/make_serving_reference.py
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import icnnm_oracle as O  # noqa: E402
from paper_2604_17001_gb300 import synth  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "serving_k7x7x3_sample.npz")
N_REQUESTS = 2000
SAMPLE = [1, 26, 60, 66, 69, 73, 94, 109, 129]
N_VOX = 4096
TOL, EVERY, EXTRA = 1e-3, 10, 40


def main():
    kd = synth.WORKLOADS[5]["kdims"]
    t0 = time.time()
    V, sig = O.learn_V(synth.serving_refs(), kd)
    print(f"learn_V: {time.time() - t0:.0f} s", flush=True)
    shapes = synth.serving_shapes(N_REQUESTS)
    out = dict(V=V, sigma=sig, sample=np.array(SAMPLE), tol=TOL, check_every=EVERY)
    for j in SAMPLE:
        job = synth.serving_job(j, shapes)
        t0 = time.time()
        _, st = O.icnnm_solve(job["M"], job["mask"], V, kd, max_iters=1000, tol=TOL, check_every=EVERY)
        stop = st["iters"]
        _, st2 = O.icnnm_solve(job["M"], job["mask"], V, kd, max_iters=stop + EXTRA, record_every=EVERY)
        miss = np.flatnonzero(~job["mask"].astype(bool).ravel())
        rng = np.random.default_rng(synth.seed_for(5, 3000 + j))
        idx = np.sort(rng.choice(miss, size=min(N_VOX, miss.size), replace=False))
        its = sorted(st2["checkpoints"])
        out[f"r{j}_stop"] = stop
        out[f"r{j}_idx"] = idx
        out[f"r{j}_iters"] = np.array(its)
        out[f"r{j}_L"] = np.stack([st2["checkpoints"][i][0].ravel()[idx] for i in its])
        out[f"r{j}_resid"] = np.array([st2["checkpoints"][i][1] for i in its])
        print(f"request {j} {job['dims']} {job['family']}: stop {stop}, {time.time() - t0:.0f} s", flush=True)
        np.savez_compressed(OUT, **out)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
