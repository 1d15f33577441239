"""Wall time of the FP64 oracle (test infrastructure; the CPU baseline) per ADMM
iteration on the workload families, with one BLAS thread and with every host core.
numpy's BLAS thread count is fixed when numpy loads, so each measurement runs in a fresh
interpreter with OPENBLAS_NUM_THREADS / OMP_NUM_THREADS set. Prints one JSON line per
(workload, threads).

    python oracle/time_oracle.py [--budget SECONDS]
"""
import argparse
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import json, os, sys, time
sys.path.insert(0, {root!r})
import numpy as np
from oracle import icnnm_oracle as O
from paper_2604_17001_gb300 import synth
cfg, budget = {cfg}, {budget}
if cfg == 4:
    spec = synth.WORKLOADS[4]
    jobs = synth.batch_jobs(3, cfg=4)
    job = max(jobs, key=lambda j: int(np.prod(j["dims"])))
    M, mask, dims, kd = job["M"], job["mask"], job["dims"], spec["kdims"]
    refs = [synth.video(32, 32, 8, synth.seed_for(4, j)) for j in (1, 2)]
else:
    w = synth.workload(cfg, n_ref=2)
    M, mask, dims, kd = w["M"], w["mask"], w["dims"], w["kdims"]
    refs = w["refs"]
V, _ = O.learn_V(refs, kd)
L, Y, th = O.icnnm_init(M, mask, V, kd)
Q = O.conv_matrix_times(L, V, kd)
L, Y, Z, Q = O.icnnm_iteration(L, Y, th, M, mask, V, kd, np.inf, Q)     # warm-up (index cache)
n, t0 = 0, time.perf_counter()
while n < 1 or time.perf_counter() - t0 < budget:
    L, Y, Z, Q = O.icnnm_iteration(L, Y, th, M, mask, V, kd, np.inf, Q)
    n += 1
sec = (time.perf_counter() - t0) / n
print(json.dumps(dict(workload=synth.WORKLOADS[cfg]["name"], dims=list(dims), kdims=list(kd),
                      seconds_per_iteration=sec, iterations_timed=n)))
'''


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--budget", type=float, default=20.0)
    ap.add_argument("--configs", default="1,2,3,4")
    a = ap.parse_args()
    cores = os.cpu_count() or 1
    for cfg in [int(x) for x in a.configs.split(",")]:
        for threads in (1, cores):
            env = dict(os.environ, OPENBLAS_NUM_THREADS=str(threads), OMP_NUM_THREADS=str(threads),
                       MKL_NUM_THREADS=str(threads))
            r = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT, cfg=cfg, budget=a.budget)],
                               env=env, capture_output=True, text=True)
            if r.returncode != 0:
                print(json.dumps(dict(config=cfg, threads=threads, error=r.stderr[-400:])), flush=True)
                continue
            d = json.loads(r.stdout.strip().splitlines()[-1])
            d.update(threads=threads, host_cores=cores)
            print(json.dumps(d), flush=True)


if __name__ == "__main__":
    main()
