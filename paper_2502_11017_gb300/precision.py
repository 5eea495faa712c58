"""The BF16 coefficient phase of the swap iteration against the FP32/FP64 engine, on global
maxvol problems shaped like the polish and sweep stages: a basis of p rows and rank r
(Haar factors, singular values exp(-5 j / r)), started from random rows. Reports time,
swaps (all, and those of the BF16 phase) and the log-volume of each result.

    python -m paper_2502_11017_gb300.precision
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import CUR_F32, Handle, cur_maxvol_global, cur_sync_status, opts
from . import workloads as wl


def basis_device(p: int, r: int, seed: int, device):
    import torch
    rng = np.random.default_rng(seed)
    u = torch.from_numpy(wl.haar(p, r, rng)).to(device)
    v = torch.from_numpy(wl.haar(r, r, rng)).to(device)
    s = torch.exp(-5.0 * torch.arange(r, dtype=torch.float64, device=device) / r)
    return ((u * s) @ v.T * np.sqrt(p)).to(torch.float32).contiguous()


def one(hd, C, S0, r: int, prec: str):
    import torch
    dev = C.device
    S = torch.empty(r, dtype=torch.int32, device=dev)
    lv = torch.empty(1, dtype=torch.float64, device=dev)
    sw = torch.zeros(2, dtype=torch.int32, device=dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    cur_maxvol_global(hd.h, C, S0, r, opts(1e-2, bf16=prec == "bf16", fp8=prec == "fp8"), S, lv, sw)
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1e3
    st = cur_sync_status(hd.h)
    return dict(ms=ms, logvol=lv.item(), swaps=sw.tolist(), status=st)


def main(argv=None):
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=None)
    ap.add_argument("--cases", default="65536x64,262144x64,262144x128,16384x64")
    ap.add_argument("--reps", type=int, default=3)
    args = ap.parse_args(argv)
    dev = torch.device("cuda:0")
    hd = Handle(262144, 4096, 128, CUR_F32)
    res = []
    for case in args.cases.split(","):
        p, r = (int(x) for x in case.split("x"))
        C = basis_device(p, r, p + r, dev)
        for rep in range(args.reps):
            S0 = torch.from_numpy(np.random.default_rng(rep).choice(p, r, replace=False).astype(np.int32)).to(dev)
            one(hd, C, S0, r, "fp32")                  # warm
            a = one(hd, C, S0, r, "fp32")
            b = one(hd, C, S0, r, "bf16")
            c = one(hd, C, S0, r, "fp8")
            res.append(dict(p=p, r=r, start=rep, fp32=a, bf16=b, fp8=c, bf16_logvol_diff=b["logvol"] - a["logvol"],
                            fp8_logvol_diff=c["logvol"] - a["logvol"]))
            print(json.dumps(res[-1]), flush=True)
    hd.close()
    if args.out:
        with open(args.out, "w") as f:
            json.dump(res, f, indent=1)
    return res


if __name__ == "__main__":
    main()
