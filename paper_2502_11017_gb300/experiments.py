"""The approximation-error study of Section 3.1, run on the GPU path.

    python -m paper_2502_11017_gb300.experiments [--out results.md]

For Hilbert matrices (256, 512, 1024) and the synthetic low-rank products H = A B
with A(i,j) = B(i,j) = 1/(i+j) (n = 256, 512, 1024; rank 5, 10, 15, 20), it computes
the cross for r = 1..20 selected rows/columns (FP64 data, 4 row and 4 column blocks),
assembles C, U, R and reports the relative Frobenius error ||A - CUR||_F / ||A||_F.
The paper shows these as figures without printed values; the table is the GPU's. An
entry marked * comes from a cross whose intersection A(I,J) is numerically singular
(r above the numerical rank): U is then the pseudo-inverse.
"""
from __future__ import annotations

import argparse
import ctypes

import torch

import paper_2502_11017_gb300 as cur
from paper_2502_11017_gb300 import workloads as wl


def rel_error(A, r: int, hd, blocks: int = 4):
    """(relative Frobenius error, Chebyshev error, cross status, I, J) of the rank-r cross."""
    m, n = A.shape
    dev = A.device
    h = hd.h
    I = torch.empty(r, dtype=torch.int32, device=dev)
    J = torch.empty(r, dtype=torch.int32, device=dev)
    info = torch.zeros(ctypes.sizeof(cur.CurCrossInfo), dtype=torch.uint8, device=dev)
    cur.cur_cross(h, A, r, min(blocks, m // r), min(blocks, n // r), cur.opts(), I, J, info)
    status = cur.cur_sync_status(h)
    if status not in (cur.CUR_OK, cur.CUR_WARN_RANK, cur.CUR_ERR_SINGULAR):
        return None, None, status, I, J
    C = torch.empty((m, r), dtype=A.dtype, device=dev)
    R = torch.empty((r, n), dtype=A.dtype, device=dev)
    U = torch.empty((r, r), dtype=torch.float64, device=dev)
    rc = torch.empty(1, dtype=torch.float64, device=dev)
    cheb = torch.empty(1, dtype=torch.float64, device=dev)
    fro = torch.empty(1, dtype=torch.float64, device=dev)
    cur.cur_assemble(h, A, I, J, r, C, U, R, rc)
    cur.cur_residual_cheb(h, A, C, U, R, r, cheb, fro)
    st2 = cur.cur_sync_status(h)
    if st2 not in (cur.CUR_OK, cur.CUR_WARN_RANK):
        return None, None, st2, I, J
    return fro.item(), cheb.item(), status, I, J


def run(ranks=range(1, 21), sizes=(256, 512, 1024), prod_ranks=(5, 10, 15, 20)):
    dev = torch.device("cuda:0")
    rows = []
    for n in sizes:
        hd = cur.Handle(n, n, 32, cur.CUR_F64)
        mats = [(f"Hilbert {n}", wl.hilbert(n))]
        mats += [(f"1/(i+j) product n={n} rank={k}", wl.cauchy_product(n, k)) for k in prod_ranks]
        for name, a in mats:
            A = torch.from_numpy(a).to(dev)
            vals = []
            for r in ranks:
                e, _, st, _, _ = rel_error(A, r, hd)
                vals.append((e, st))
            rows.append((name, vals))
        hd.close()
    return list(ranks), rows


def to_markdown(ranks, rows) -> str:
    head = "| matrix | " + " | ".join(f"r={r}" for r in ranks) + " |"
    sep = "|---|" + "---|" * len(ranks)
    lines = [head, sep]
    for name, vals in rows:
        cells = []
        for e, st in vals:
            if e is None:
                cells.append(f"({cur.cur_status_string(st)})")
            else:
                cells.append(f"{e:.1e}" + ("*" if st == cur.CUR_ERR_SINGULAR else ""))
        lines.append(f"| {name} | " + " | ".join(cells) + " |")
    return "\n".join(lines) + "\n"


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    ranks, rows = run()
    md = to_markdown(ranks, rows)
    print(md)
    if a.out:
        with open(a.out, "w") as f:
            f.write(md)


if __name__ == "__main__":
    main()
