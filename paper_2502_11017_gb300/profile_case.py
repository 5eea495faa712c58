"""Runs one library call on a Gaussian-kernel matrix for profiling (e.g. under ncu).

    python -m paper_2502_11017_gb300.profile_case --call aca --m 16384 --n 8192 --r 3
    python -m paper_2502_11017_gb300.profile_case --call residual --m 16384 --n 8192 --r 64
    python -m paper_2502_11017_gb300.profile_case --call cross --m 65536 --n 8192 --r 64
    python -m paper_2502_11017_gb300.profile_case --call alg1 --m 65536 --n 8192 --r 64
    python -m paper_2502_11017_gb300.profile_case --call batch --count 4096
    python -m paper_2502_11017_gb300.profile_case --call coef --m 262144 --r 64

(--call coef: B = C M^-1 on the tensor cores for C = the first r columns of the matrix and
M^-1 the inverse of the rows Algorithm 3 picks in C, the product the swap engine's first
cycle takes; prints the HBM rate of its algorithmic bytes, read C + write B.)

The matrix is exp(-|x_i - y_j|^2 / h^2) with uniform points (the generator of the
65536 x 8192 workload, at any size). --reps calls are made after --warmup calls;
each call is timed with CUDA events and printed.
"""
from __future__ import annotations

import argparse
import time

import numpy as np
import torch

import paper_2502_11017_gb300 as cur
from paper_2502_11017_gb300 import workloads as wl


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--call", choices=["aca", "residual", "cross", "rows", "cols", "alg1", "batch", "coef"],
                    required=True)
    ap.add_argument("--count", type=int, default=4096, help="matrices of the batched workload (--call batch)")
    ap.add_argument("--m", type=int, default=16384)
    ap.add_argument("--n", type=int, default=8192)
    ap.add_argument("--r", type=int, default=64)
    ap.add_argument("--b_r", type=int, default=16)
    ap.add_argument("--b_c", type=int, default=8)
    ap.add_argument("--warmup", type=int, default=1)
    ap.add_argument("--bf16", action="store_true", help="CUR_FLAG_PREC_BF16 on the cross / row / column stages")
    ap.add_argument("--reps", type=int, default=1)
    ap.add_argument("--seed", type=int, default=11019)
    ap.add_argument("--data", choices=["gaussian", "bf16product", "haar"], default="gaussian",
                    help="Gaussian kernel (FP32), the rank-r factor product plus noise in BF16, or "
                         "the FP64 low-rank Haar matrix (2000 x 1500, sigma_k = 2^(-k/2))")
    a = ap.parse_args()
    dev = torch.device("cuda:0")
    if a.call == "batch":
        return batch(a)
    if a.call == "coef":
        return coef(a)
    if a.data == "bf16product":
        A = wl.bf16_factor_product(a.m, a.n, a.r, 1e-2, device=dev)
    elif a.data == "haar":
        A = torch.from_numpy(wl.lowrank_haar()).to(dev)
        a.m, a.n = A.shape
    else:
        A = torch.from_numpy(wl.gaussian_kernel(a.m, a.n, 0.2, seed=a.seed, chunk_rows=1024)).to(dev)
    m, n, r = a.m, a.n, a.r
    hd = cur.Handle(m, n, max(r, 64), {"bf16product": cur.CUR_BF16, "haar": cur.CUR_F64}.get(a.data, cur.CUR_F32))
    h = hd.h
    idx = torch.empty(r, dtype=torch.int32, device=dev)
    I = torch.empty(r, dtype=torch.int32, device=dev)
    J = torch.empty(r, dtype=torch.int32, device=dev)
    C = torch.empty((m, r), dtype=A.dtype, device=dev)
    R = torch.empty((r, n), dtype=A.dtype, device=dev)
    U = torch.empty((r, r), dtype=torch.float64, device=dev)
    rc = torch.empty(1, dtype=torch.float64, device=dev)
    cheb = torch.empty(1, dtype=torch.float64, device=dev)
    fro = torch.empty(1, dtype=torch.float64, device=dev)
    o = cur.opts(bf16=a.bf16)
    Rw = torch.empty((m, n), dtype=torch.float64 if A.dtype == torch.float64 else torch.float32,
                     device=dev) if a.call == "alg1" else None
    piv = torch.empty(r, dtype=torch.float64, device=dev)
    if a.call in ("residual", "rows", "cols"):
        cur.cur_cross(h, A, r, a.b_r, a.b_c, o, I, J)
        cur.cur_assemble(h, A, I, J, r, C, U, R, rc)
        cur.cur_aca_select(h, A, 1, r, 1, idx)

    def call():
        if a.call == "aca":
            cur.cur_aca_select(h, A, 1, r, 1, idx)
        elif a.call == "residual":
            cur.cur_residual_cheb(h, A, C, U, R, r, cheb, fro)
        elif a.call == "cross":
            cur.cur_cross(h, A, r, a.b_r, a.b_c, o, I, J)
        elif a.call == "rows":
            cur.cur_maxvol_rows(h, A, idx, r, cur.opts(nblocks=a.b_r, bf16=a.bf16), I)
        elif a.call == "cols":
            cur.cur_maxvol_cols(h, A, I, r, cur.opts(nblocks=a.b_c, bf16=a.bf16), J)
        elif a.call == "alg1":
            cur.cur_aca_full(h, A, r, Rw, I, J, piv)

    for _ in range(a.warmup):
        call()
    torch.cuda.synchronize()
    cur.cur_prof_refactors(h)
    for _ in range(a.reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        e0.record()
        call()
        e1.record()
        torch.cuda.synchronize()
        print(f"{a.call} m={m} n={n} r={r}: {e0.elapsed_time(e1):.3f} ms (host {1e3 * (time.perf_counter() - t0):.3f} ms)")
    if a.call == "alg1":
        # per-step update pass (read + write of the m x n FP32 residual), CUDA events
        cur.cur_prof_enable(h, 1)
        call()
        torch.cuda.synchronize()
        tot_ms, npass, _k = cur.cur_prof_read(h)
        if npass:
            avg = tot_ms / npass
            gbs = 2 * m * n * 4 / (avg * 1e-3) / 1e9
            print(f"alg1 update pass: {npass} launches, {avg:.4f} ms average, {gbs:.0f} GB/s (2 m n 4 bytes)")
    print(f"cycle refactorisations in the timed calls: {cur.cur_prof_refactors(h)}")
    st = cur.cur_sync_status(h)
    if st not in (cur.CUR_OK, cur.CUR_WARN_RANK):
        raise SystemExit(f"device status {st}")
    hd.close()


def coef(a):
    """cur_coef_tf32 on an m x r FP32 basis (the Gaussian kernel's first r columns)."""
    dev = torch.device("cuda:0")
    m, r = a.m, a.r
    C = torch.from_numpy(np.ascontiguousarray(wl.gaussian_kernel(m, r, 0.2, seed=a.seed, chunk_rows=4096))).to(dev)
    hd = cur.Handle(m, r, r, cur.CUR_F32)
    idx = torch.empty(r, dtype=torch.int32, device=dev)
    cur.cur_aca_select(hd.h, C, 0, r, 1, idx)
    # M^-1 = C(S,:)^-1 by the library's assembly of the cross (S, all r columns)
    Mi = torch.empty((r, r), dtype=torch.float64, device=dev)
    rc = torch.empty(1, dtype=torch.float64, device=dev)
    cur.cur_assemble(hd.h, C, idx, torch.arange(r, dtype=torch.int32, device=dev), r, None, Mi, None, rc)
    B = torch.empty((m, r), dtype=torch.float32, device=dev)
    for rep in range(a.warmup + a.reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        cur.cur_coef_tf32(hd.h, C, Mi, B)
        e1.record()
        torch.cuda.synchronize()
        if rep >= a.warmup:
            ms = e0.elapsed_time(e1)
            print(f"coef m={m} r={r}: {ms:.4f} ms, {2 * m * r * 4 / (ms * 1e-3) / 1e9:.0f} GB/s of read C + write B")
    st = cur.cur_sync_status(hd.h)
    if st not in (cur.CUR_OK, cur.CUR_WARN_RANK):
        raise SystemExit(f"device status {st}")
    hd.close()


def batch(a):
    """cur_cross_batched on the uneven batch: m ~ U[256, 4096], n ~ U[128, 1024], r ~ U{8..64}."""
    import ctypes
    dev = torch.device("cuda:0")
    shapes = wl.uneven_batch_shapes(a.count)
    data, offs = wl.uneven_batch_device(shapes, device=dev)
    items = cur.batch_items(shapes, offs)
    hd = cur.Handle(1, 1, 1, workspace_bytes=cur.cur_batch_workspace_size(items))
    total = sum(s[2] for s in shapes)
    IJ = torch.empty(2 * total, dtype=torch.int32, device=dev)
    info = torch.zeros(len(shapes) * ctypes.sizeof(cur.CurCrossInfo), dtype=torch.uint8, device=dev)
    a_bytes = sum(m * n * 4 for (m, n, _r, _b, _c) in shapes)
    a_rounds = sum(m * n * 4 * r for (m, n, r, _b, _c) in shapes)
    for rep in range(a.warmup + a.reps):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        e0.record()
        cur.cur_cross_batched(hd.h, data, items, cur.opts(), IJ, info)
        e1.record()
        torch.cuda.synchronize()
        if rep >= a.warmup:
            ms = e0.elapsed_time(e1)
            print(f"batch of {a.count}: {ms:.3f} ms = {1000.0 * a.count / ms:.1f} crosses/s "
                  f"(host {1e3 * (time.perf_counter() - t0):.3f} ms); A {a_bytes / 1e9:.2f} GB, "
                  f"Algorithm 3 streams {a_rounds / 1e12:.3f} TB -> {a_rounds / (ms * 1e-3) / 1e9:.0f} GB/s if all from HBM")
    st = cur.cur_sync_status(hd.h)
    raw = info.cpu().numpy().tobytes()
    sz = ctypes.sizeof(cur.CurCrossInfo)
    stats = [cur.CurCrossInfo.from_buffer_copy(raw[t * sz:(t + 1) * sz]).status for t in range(len(shapes))]
    print("status", st, "per-matrix statuses", {s: stats.count(s) for s in set(stats)})
    hd.close()


if __name__ == "__main__":
    main()
