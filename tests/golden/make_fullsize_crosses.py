"""Writes tests/golden/fullsize_crosses.json: the FP64 oracle's cross on two full-size
seeded workloads, for the GPU parity tests to compare against.

Only the oracle (``oracle/cur_oracle.py``) and the seeded input generators
(``paper_2502_11017_gb300/workloads.py``, inputs only) are called; nothing here runs
the CUDA library. What is stored per workload: J0 (Algorithm 3 on the columns, Section
2.2), the final I and J in submatrix-position order, log|det A(I,J)| (Definition 1),
the sweeps and swaps of the refinement, and the Chebyshev norm max|A - CUR| (Theorem 1)
and relative Frobenius error (Section 3.1) of the assembled cross (Section 1.1).

Workloads:
  lowrank_haar_2000x1500_r16   A = U diag(2^(-k/2)) V^T + noise (std 1e-4), FP64,
                               Haar U, V; r = 16, 8 row and 8 column blocks.
  gaussian_kernel_65536x8192_r64  A_ij = exp(-|x_i - y_j|^2 / 0.04), x, y uniform in
                               [0,1]^3, FP32 (seed 11019); r = 64, 64 row blocks of 1024
                               rows, 8 column blocks.
delta = 1e-2 for both. The 65536 x 8192 cross takes several minutes on 8 host cores.

Usage: python tests/golden/make_fullsize_crosses.py [--only NAME]
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import cur_oracle as orc  # noqa: E402
from paper_2502_11017_gb300 import workloads as wl  # noqa: E402

OUT = os.path.join(HERE, "fullsize_crosses.json")

CASES = {
    "lowrank_haar_2000x1500_r16": dict(
        make=lambda: wl.lowrank_haar(2000, 1500), r=16, b_r=8, b_c=8),
    "gaussian_kernel_65536x8192_r64": dict(
        make=lambda: wl.gaussian_kernel(65536, 8192, 0.2, seed=11019, chunk_rows=4096),
        r=64, b_r=64, b_c=8),
}


def run(name: str) -> dict:
    c = CASES[name]
    a = c["make"]()
    t0 = time.time()
    I, J, info = orc.cross(a, c["r"], c["b_r"], c["b_c"], 1e-2)
    Cm, U, Rm, rcond, used_pinv = orc.assemble(a, I, J)
    cheb, fro = orc.residual(a, Cm, U, Rm)
    return dict(
        workload=name, m=int(a.shape[0]), n=int(a.shape[1]), dtype=str(a.dtype),
        r=c["r"], b_r=c["b_r"], b_c=c["b_c"], delta=1e-2,
        J0=[int(x) for x in info["J0"]], I=[int(x) for x in I], J=[int(x) for x in J],
        logvol=float(info["logvol"]), status=int(info["status"]), sweeps=int(info["sweeps"]),
        sweep_swaps=[int(x) for x in info["sweep_swaps"]],
        cheb=float(cheb), fro_rel=float(fro), norm_cheb=float(np.abs(a).max()),
        rcond=float(rcond), used_pinv=bool(used_pinv),
        oracle_seconds=round(time.time() - t0, 1))


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--only", default=None)
    args = ap.parse_args()
    data = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            data = json.load(f)
    for name in CASES:
        if args.only and name != args.only:
            continue
        data[name] = run(name)
        print(name, data[name]["logvol"], data[name]["sweeps"], data[name]["oracle_seconds"], "s",
              flush=True)
        with open(OUT, "w") as f:
            json.dump(data, f, indent=1)


if __name__ == "__main__":
    main()
