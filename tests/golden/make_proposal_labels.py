"""Writes proposal_labels_4096x1024_r16.npz: the crosses that the FP64 oracle selects on
members of the learned proposal's training family (Gaussian-kernel matrices, points in
[0,1]^3, h ~ U[0.1, 0.4], 4096 x 1024, r = 16, 16 row blocks, 4 column blocks, delta =
1e-2). These are the labels the scoring network is trained on (a row is positive when it
is in I, a column when it is in J). Calls only the oracle and the seeded generators.

    python tests/golden/make_proposal_labels.py [--count 2176] [--procs 8]
"""
import argparse
import multiprocessing as mp
import os
import sys

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")          # one BLAS thread per worker process

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import cur_oracle as orc                      # noqa: E402
from paper_2502_11017_gb300 import workloads as wl        # noqa: E402

F = wl.PROPOSAL_FAMILY
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "proposal_labels_4096x1024_r16.npz")


def one(item):
    seed, h = item
    a = wl.gaussian_kernel(F["m"], F["n"], h, seed=seed)
    I, J, info = orc.cross(a, F["r"], F["b_r"], F["b_c"])
    return I, J, info["status"], info["logvol"], sum(info["sweep_swaps"])


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--count", type=int, default=2176)
    ap.add_argument("--procs", type=int, default=os.cpu_count())
    args = ap.parse_args()
    fam = wl.proposal_family(args.count, h_range=F["h_range"])
    res = []
    with mp.get_context("spawn").Pool(args.procs) as pool:
        for r in pool.imap(one, fam, chunksize=4):
            res.append(r)
            if len(res) % 256 == 0:
                print(f"{len(res)} / {len(fam)}", flush=True)
    np.savez_compressed(
        OUT, seed=np.array([s for s, _ in fam], np.int64), h=np.array([h for _, h in fam]),
        I=np.array([r[0] for r in res], np.int32), J=np.array([r[1] for r in res], np.int32),
        status=np.array([r[2] for r in res], np.int32), logvol=np.array([r[3] for r in res]),
        swaps=np.array([r[4] for r in res], np.int32))
    print(f"wrote {OUT}: {args.count} crosses, statuses {np.bincount([r[2] for r in res])}")


if __name__ == "__main__":
    main()
