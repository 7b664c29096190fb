"""Write the oracle's level record of the full-size benchmark workload.

Workload (the c3 preset): level 3 (64^3 cells) with its level-2 partner on the
same draw, 256 KL modes of the exponential covariance (correlation length 0.2,
sigma 1), theta 10, alpha 1e-4, seed 0, control z = z_test on the 64^3 grid,
optimisation step 0, samples 0..4095.  The record is the one
mlsgd_level_gradient forms (Algorithm 1, GradientEstimate and PairwiseUpdate;
eq:delta-notation, eq:sec-order-sum): sample count, shift c = max Phi, the
mean of dX~ = X~_3 - X~_2 on the control grid, the mean of dY~ and both
second-order sums, all at the shift c.

The oracle solves every sample to rtol 1e-12 (sparse direct below 32^3,
Galerkin-MG-PCG above; at 64^3 with this coefficient contrast the true residual
FP64 can attain lies near 1e-13 ||b||, so rtol 1e-13 stalls for some samples,
while 1e-12 is six orders below the mixed path's bar of 1e-6).  The 4096 samples are spread over one spawn-started
process per host core in chunks; each chunk's record is kept at its own shift
and the chunks are merged with oracle.mlmc.merge_shifted.  Only oracle/ and the
seeded input module are called.  The sparse solves are memory-bound, so the rate
depends on the host's memory bandwidth: about 10 minutes on 16 Grace cores,
hours on a small x86 host.

    python tests/golden/make_c3_record.py [output.npz]
"""
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(HERE, "c3_level3_record.npz")
ITERATION, LEVEL, SAMPLES, CHUNK = 0, 3, 4096, 16

_STATE = {}


def _workload():
    from oracle import mlmc
    from paper_2606_09291_gb300 import inputs
    p = inputs.PRESETS["c3"]
    return mlmc.Workload(n0=p["n0"], n_levels=p["n_levels"], n_modes=p["n_modes"], corr_len=p["corr_len"],
                         sigma=p["sigma"], theta=p["theta"], alpha=p["alpha"], seed=p["seed"], rtol=1e-12)


def _init():
    os.environ["OMP_NUM_THREADS"] = "1"
    sys.path.insert(0, ROOT)
    from oracle import mlmc
    from paper_2606_09291_gb300 import inputs
    W = _workload()
    W.level(LEVEL), W.level(LEVEL - 1)
    _STATE.update(W=W, z=inputs.z_test(W.Nc), mlmc=mlmc)


def _chunk(first):
    st = _STATE
    r = st["mlmc"].level_batch(st["W"], ITERATION, LEVEL, range(first, min(first + CHUNK, SAMPLES)), st["z"])
    return dict(stats=r["stats"], shift=r["shift"])


def main():
    sys.path.insert(0, ROOT)
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    from oracle import mlmc
    procs = len(os.sched_getaffinity(0))
    t = time.time()
    with mp.get_context("spawn").Pool(procs, initializer=_init) as pool:
        parts = pool.map(_chunk, range(0, SAMPLES, CHUNK), chunksize=1)
    W = _workload()
    rec = mlmc.merge_shifted(parts, W.theta, W.hc3)
    S = rec["stats"]
    assert S.n == SAMPLES
    out = sys.argv[1] if len(sys.argv) > 1 else OUT
    np.savez_compressed(out, count=S.n, shift=rec["shift"], mean_x=S.mean_x, s2_x=S.s2_x, mean_y=S.mean_y,
                        s2_y=S.s2_y, iteration=ITERATION, level=LEVEL, first_sample=0, oracle_rtol=W.rtol)
    print("wrote %s: %d samples in %.0f s on %d processes, shift %.15g" % (out, S.n, time.time() - t, procs,
                                                                           rec["shift"]))


if __name__ == "__main__":
    main()
