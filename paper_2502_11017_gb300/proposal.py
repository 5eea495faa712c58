"""Learned proposal for the maxvol cross: a scoring network per axis ranks the rows and
the columns of A from Gaussian sketch features; the r best of each start the sweeps of
global maxvol (cur_cross_from), and the plain cross (cur_cross) takes over when the
proposed A(I0, J0) is singular. Training fits the networks to crosses the FP64 oracle
selected on members of a family of matrices (a row is positive when the oracle put it in
I). Every step runs in libcur (sketch, forward, gradient, Adam, top-r, maxvol); this module
only sequences the calls and holds the tensors.

    python -m paper_2502_11017_gb300.proposal --labels tests/golden/proposal_labels_4096x1024_r16.npz
"""
from __future__ import annotations

import argparse
import ctypes
import json
import time

import numpy as np

from . import workloads as wl
from . import (CUR_ERR_SINGULAR, CUR_F32, CurCrossInfo, Handle, cur_adam_step, cur_cross, cur_cross_from,
               cur_maxvol_cols, cur_maxvol_rows, cur_mlp_forward, cur_mlp_grad, cur_propose, cur_sketch,
               cur_sync_status, info_from_tensor, opts)

K, H = 32, 256


def init_params(seed: int, k: int = K, hdim: int = H):
    """He-initialised W1 (k x H), zero b1, w2 ~ N(0, 1/H), b2 = 0, as one FP32 array."""
    rng = np.random.default_rng(seed)
    w1 = rng.standard_normal((k, hdim)) * np.sqrt(2.0 / k)
    w2 = rng.standard_normal(hdim) / np.sqrt(hdim)
    return np.concatenate([w1.ravel(), np.zeros(hdim), w2, [0.0]]).astype(np.float32)


class Net:
    """One scoring network with its Adam state, on the device."""

    def __init__(self, seed: int, device):
        import torch
        self.p = torch.from_numpy(init_params(seed)).to(device)
        self.g = torch.zeros_like(self.p)
        self.m1 = torch.zeros_like(self.p)
        self.m2 = torch.zeros_like(self.p)
        self.t = 0


def features(hd, A, S, T):
    """Normalised sketch features (Y: m x 32 rows, Zt: n x 32 columns) of A."""
    import torch
    m, n = A.shape
    Y = torch.empty((m, K), dtype=torch.float32, device=A.device)
    Zt = torch.empty((n, K), dtype=torch.float32, device=A.device)
    cur_sketch(hd.h, A, S, T, Y, Zt, True)
    return Y, Zt


def family_features(hd, items, device, family=wl.PROPOSAL_FAMILY):
    """Features of every matrix (seed, h) of `items`, stacked: (Xr, Xc)."""
    import torch
    m, n = family["m"], family["n"]
    Xr = torch.empty((len(items) * m, K), dtype=torch.float32, device=device)
    Xc = torch.empty((len(items) * n, K), dtype=torch.float32, device=device)
    for t, (seed, h) in enumerate(items):
        A = wl.gaussian_kernel_device(m, n, h, seed, device)
        s, tt = wl.sketch_matrices(m, n, K, seed=seed + 1)
        S, T = torch.from_numpy(s).to(device), torch.from_numpy(tt).to(device)
        Xr[t * m:(t + 1) * m], Xc[t * n:(t + 1) * n] = features(hd, A, S, T)
    return Xr, Xc


def labels(I, J, family=wl.PROPOSAL_FAMILY):
    """0/1 labels of the stacked rows and columns from the oracle's sets."""
    m, n = family["m"], family["n"]
    yr = np.zeros(len(I) * m, np.float32)
    yc = np.zeros(len(J) * n, np.float32)
    for t in range(len(I)):
        yr[t * m + np.asarray(I[t])] = 1.0
        yc[t * n + np.asarray(J[t])] = 1.0
    return yr, yc


def train(hd, net: Net, X, y, pos_weight: float, epochs: int, batch: int, lr: float, seed: int):
    """Adam on the weighted cross-entropy over minibatches of a seeded shuffle; returns the
    mean loss of each epoch."""
    import torch
    N = X.shape[0]
    gen = torch.Generator(device=X.device)
    gen.manual_seed(seed)
    loss = torch.zeros(1, dtype=torch.float64, device=X.device)
    hist = []
    for _ in range(epochs):
        perm = torch.randperm(N, generator=gen, device=X.device)
        tot, steps = torch.zeros((), dtype=torch.float64, device=X.device), 0
        for s0 in range(0, N, batch):
            idx = perm[s0:s0 + batch]
            cur_mlp_grad(hd.h, X, y, net.p, net.g, loss, idx=idx, pos_weight=pos_weight)
            net.t += 1
            cur_adam_step(hd.h, net.p, net.g, net.m1, net.m2, net.t, lr=lr)
            tot += loss[0]
            steps += 1
        hist.append(float(tot.item()) / steps)
    return hist


def scores(hd, net: Net, X):
    import torch
    out = torch.empty(X.shape[0], dtype=torch.float32, device=X.device)
    cur_mlp_forward(hd.h, X, net.p, out)
    return out


def _refine(hd, A, r: int, I0, J0, delta: float):
    dev = A.device
    import torch
    I = torch.empty(r, dtype=torch.int32, device=dev)
    J = torch.empty(r, dtype=torch.int32, device=dev)
    info = torch.zeros(ctypes.sizeof(CurCrossInfo), dtype=torch.uint8, device=dev)
    cur_cross_from(hd.h, A, r, I0, J0, opts(delta), I, J, info)
    inf = info_from_tensor(info)
    cur_sync_status(hd.h)          # clears a SINGULAR / NOCONV mark; info carries it
    return I, J, inf


def propose_cross(hd, A, r: int, rows: Net, cols: Net, S, T, b_r: int, b_c: int, delta: float = 1e-2):
    """The learned cross of A: the r best-scored rows and columns, refined by maxvol sweeps;
    the plain cross when the proposal (or its refinement) is singular. Returns
    (I, J, info, fell_back)."""
    import torch
    dev = A.device
    Y, Zt = features(hd, A, S, T)
    I0 = torch.empty(r, dtype=torch.int32, device=dev)
    J0 = torch.empty(r, dtype=torch.int32, device=dev)
    cur_propose(hd.h, scores(hd, rows, Y), r, I0)
    cur_propose(hd.h, scores(hd, cols, Zt), r, J0)
    I, J, inf = _refine(hd, A, r, I0, J0, delta)
    if inf.status == CUR_ERR_SINGULAR:
        I, J, inf = plain_cross(hd, A, r, b_r, b_c, delta)
        return I, J, inf, True
    return I, J, inf, False


def propose_columns_cross(hd, A, r: int, cols: Net, S, T, b_r: int, b_c: int, delta: float = 1e-2):
    """The cross with the learned columns in place of Algorithm 3's J0: blockwise maxvol rows
    on A(:,J0), blockwise columns on A(I,:), then the sweeps. Returns (I, J, info, fell_back)."""
    import torch
    dev = A.device
    Y, Zt = features(hd, A, S, T)
    J0 = torch.empty(r, dtype=torch.int32, device=dev)
    cur_propose(hd.h, scores(hd, cols, Zt), r, J0)
    I1 = torch.empty(r, dtype=torch.int32, device=dev)
    J1 = torch.empty(r, dtype=torch.int32, device=dev)
    cur_maxvol_rows(hd.h, A, J0, r, opts(delta, nblocks=b_r), I1)
    cur_maxvol_cols(hd.h, A, I1, r, opts(delta, nblocks=b_c), J1)
    cur_sync_status(hd.h)
    I, J, inf = _refine(hd, A, r, I1, J1, delta)
    if inf.status == CUR_ERR_SINGULAR:
        I, J, inf = plain_cross(hd, A, r, b_r, b_c, delta)
        return I, J, inf, True
    return I, J, inf, False


def plain_cross(hd, A, r: int, b_r: int, b_c: int, delta: float = 1e-2):
    import torch
    dev = A.device
    I = torch.empty(r, dtype=torch.int32, device=dev)
    J = torch.empty(r, dtype=torch.int32, device=dev)
    info = torch.zeros(ctypes.sizeof(CurCrossInfo), dtype=torch.uint8, device=dev)
    cur_cross(hd.h, A, r, b_r, b_c, opts(delta), I, J, info)
    cur_sync_status(hd.h)
    return I, J, info_from_tensor(info)


def random_cross(hd, A, r: int, seed: int, delta: float = 1e-2):
    """Refinement from a seeded random start (what the sweeps do with no proposal)."""
    import torch
    dev = A.device
    m, n = A.shape
    rng = np.random.default_rng(seed)
    I0 = torch.from_numpy(rng.choice(m, r, replace=False).astype(np.int32)).to(dev)
    J0 = torch.from_numpy(rng.choice(n, r, replace=False).astype(np.int32)).to(dev)
    return _refine(hd, A, r, I0, J0, delta)


def _timed(fn):
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = fn()
    torch.cuda.synchronize()
    return out, (time.perf_counter() - t0) * 1e3


def evaluate(hd, rows: Net, cols: Net, items, m: int, n: int, r: int, b_r: int, b_c: int, device,
             oracle=None):
    """Per matrix: the plain cross, the learned cross, the learned-columns cross and a
    refinement from a random start, with swaps, log-volumes and wall times. oracle: the
    oracle's (I, J, logvol) per matrix, when known."""
    import torch
    out = []
    for t, (seed, h) in enumerate(items):
        A = wl.gaussian_kernel_device(m, n, h, seed, device)
        s, tt = wl.sketch_matrices(m, n, K, seed=seed + 1)
        S, T = torch.from_numpy(s).to(device), torch.from_numpy(tt).to(device)
        plain_cross(hd, A, r, b_r, b_c)                      # warm
        (Ip, Jp, ip), tp = _timed(lambda: plain_cross(hd, A, r, b_r, b_c))
        (_, _, il, fb), tl = _timed(lambda: propose_cross(hd, A, r, rows, cols, S, T, b_r, b_c))
        (_, _, ic, fc), tc = _timed(lambda: propose_columns_cross(hd, A, r, cols, S, T, b_r, b_c))
        (_, _, ir), tr = _timed(lambda: random_cross(hd, A, r, seed + 2))
        row = dict(seed=seed, h=h, plain_logvol=ip.logvol, plain_swaps=ip.swaps_total, plain_ms=tp,
                   learned_logvol=il.logvol, learned_swaps=il.swaps_total, learned_fallback=fb, learned_ms=tl,
                   learned_cols_logvol=ic.logvol, learned_cols_swaps=ic.swaps_total, learned_cols_fallback=fc,
                   learned_cols_ms=tc, random_logvol=ir.logvol, random_swaps=ir.swaps_total,
                   random_singular=ir.status == CUR_ERR_SINGULAR, random_ms=tr)
        if oracle is not None:
            Io, Jo, lvo = oracle[t]
            row["oracle_logvol"] = float(lvo)
            row["plain_is_oracle"] = (sorted(Ip.tolist()) == sorted(Io)) and (sorted(Jp.tolist()) == sorted(Jo))
        out.append(row)
    return out


def time_parts(hd, rows: Net, cols: Net, m: int, n: int, r: int, device, reps: int = 20):
    """CUDA-event times of the proposal's parts on one m x n member of the family: the
    sketch (with the bytes and flops it must move and do), both forward passes, both top-r
    picks."""
    import torch
    seed, h = wl.proposal_family(1, seed=wl.SEED_BASE + 8)[0]
    A = wl.gaussian_kernel_device(m, n, h, seed, device)
    s, tt = wl.sketch_matrices(m, n, K, seed=seed + 1)
    S, T = torch.from_numpy(s).to(device), torch.from_numpy(tt).to(device)
    Y, Zt = features(hd, A, S, T)
    sr, sc = scores(hd, rows, Y), scores(hd, cols, Zt)
    I0 = torch.empty(r, dtype=torch.int32, device=device)

    def ev(fn):
        for _ in range(3):
            fn()
        st = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(st)
        for _ in range(reps):
            fn()
        e1.record(st)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    t_sk = ev(lambda: cur_sketch(hd.h, A, S, T, Y, Zt, True))
    t_fw = ev(lambda: (cur_mlp_forward(hd.h, Y, rows.p, sr), cur_mlp_forward(hd.h, Zt, cols.p, sc)))
    t_pr = ev(lambda: (cur_propose(hd.h, sr, r, I0), cur_propose(hd.h, sc, r, I0)))
    flops = 2.0 * 2 * m * n * K
    return dict(m=m, n=n, sketch_ms=t_sk, sketch_hbm_gbs=m * n * 4 / t_sk / 1e6,
                sketch_tflops=flops / t_sk / 1e9, forward_ms=t_fw, propose_ms=t_pr)


def summarise(rows):
    a = {k: np.array([r[k] for r in rows], dtype=float) for k in rows[0] if k not in ("seed",)}
    s = dict(count=len(rows))
    for v in ("plain", "learned", "learned_cols", "random"):
        s[f"{v}_swaps_mean"] = float(a[f"{v}_swaps"].mean())
        s[f"{v}_ms_median"] = float(np.median(a[f"{v}_ms"]))
        if v != "plain":
            d = a[f"{v}_logvol"] - a["plain_logvol"]
            fin = np.isfinite(d)
            s[f"{v}_minus_plain_logvol_mean"] = float(d[fin].mean()) if fin.any() else None
            s[f"{v}_minus_plain_logvol_max"] = float(d[fin].max()) if fin.any() else None
            s[f"{v}_vol_ratio_ge_0999"] = int((d[fin] >= np.log(0.999)).sum())
    s["learned_fallbacks"] = int(a["learned_fallback"].sum())
    s["learned_cols_fallbacks"] = int(a["learned_cols_fallback"].sum())
    s["random_singular"] = int(a["random_singular"].sum())
    if "oracle_logvol" in a:
        s["plain_minus_oracle_logvol_max_abs"] = float(np.abs(a["plain_logvol"] - a["oracle_logvol"]).max())
        s["plain_sets_equal_oracle"] = int(a["plain_is_oracle"].sum())
    return s


def main(argv=None):
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--labels", required=True)
    ap.add_argument("--train", type=int, default=2048)
    ap.add_argument("--test", type=int, default=128)
    ap.add_argument("--epochs", type=int, default=24)
    ap.add_argument("--batch", type=int, default=65536)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--large", type=int, default=8, help="matrices of 16384 x 4096, r = 64, to evaluate")
    ap.add_argument("--out", default=None)
    args = ap.parse_args(argv)
    dev = torch.device("cuda:0")
    lab = np.load(args.labels)
    F = wl.PROPOSAL_FAMILY
    m, n, r = F["m"], F["n"], F["r"]
    ntr = min(args.train, len(lab["seed"]) - args.test)
    items = list(zip(lab["seed"].tolist(), lab["h"].tolist()))
    tr_items, te_items = items[:ntr], items[len(items) - args.test:]
    hd = Handle(16384, 4096, 64, CUR_F32)
    t0 = time.perf_counter()
    Xr, Xc = family_features(hd, tr_items, dev)
    yr, yc = labels(lab["I"][:ntr], lab["J"][:ntr])
    yr, yc = torch.from_numpy(yr).to(dev), torch.from_numpy(yc).to(dev)
    torch.cuda.synchronize()
    t_feat = time.perf_counter() - t0
    rows, cols = Net(1, dev), Net(2, dev)
    t0 = time.perf_counter()
    hr = train(hd, rows, Xr, yr, (m - r) / r, args.epochs, args.batch, args.lr, seed=3)
    hc = train(hd, cols, Xc, yc, (n - r) / r, args.epochs, args.batch, args.lr, seed=4)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    res = dict(family=dict(F, train=ntr, test=len(te_items)), features_s=t_feat, train_s=t_train,
               loss_rows=hr, loss_cols=hc)
    k0 = len(items) - args.test
    orc_sets = [(lab["I"][k0 + t].tolist(), lab["J"][k0 + t].tolist(), lab["logvol"][k0 + t])
                for t in range(args.test)]
    ev = evaluate(hd, rows, cols, te_items, m, n, r, F["b_r"], F["b_c"], dev, oracle=orc_sets)
    res["heldout"] = summarise(ev)
    res["parts_16384x4096"] = time_parts(hd, rows, cols, 16384, 4096, 64, dev)
    if args.large:
        big = wl.proposal_family(args.large, seed=wl.SEED_BASE + 7, h_range=F["h_range"])
        evb = evaluate(hd, rows, cols, big, 16384, 4096, 64, 64, 16, dev)
        res["large_16384x4096_r64"] = summarise(evb)
    hd.close()
    print(json.dumps(res, indent=1))
    if args.out:
        with open(args.out, "w") as f:
            json.dump(res, f, indent=1)
    return res


if __name__ == "__main__":
    main()
