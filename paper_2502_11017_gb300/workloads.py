"""Seeded synthetic inputs for the CUR cross (inputs only: no step of the method).

Every generator draws from ``numpy.random.default_rng(seed)`` and returns host
arrays, so the CUDA path and the FP64 oracle read identical bytes. The shapes and
spectra follow the workloads the method is measured on:

* ``lowrank_haar``: A = U diag(sigma) V^T + noise with Haar-orthonormal U, V
  (QR of a Gaussian with the sign of R's diagonal fixed), sigma_k = 2^(-k/2),
  noise variance 1e-8 (standard deviation 1e-4). FP64. 2000 x 1500, r = 16.
* ``gaussian_kernel``: A_ij = exp(-|x_i - y_j|^2 / h^2), x_i and y_j uniform in
  the unit cube, h = 0.2, evaluated in FP64 and rounded once to FP32.
  65536 x 8192, r = 64.
* ``hilbert`` and ``cauchy_product``: the two test families of Section 3.1 of
  the paper (Hilbert matrices; H = A B with A(i,j) = B(i,j) = 1/(i+j), indices
  starting at 1).
* ``lowrank_plus_noise``: Haar factors with a chosen spectrum and noise level,
  used for small parity cases with well separated singular values.
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 11017


def haar(rows: int, cols: int, rng: np.random.Generator) -> np.ndarray:
    """rows x cols matrix with orthonormal columns, Haar distributed."""
    g = rng.standard_normal((rows, cols))
    q, rr = np.linalg.qr(g)
    d = np.sign(np.diag(rr))
    d[d == 0] = 1.0
    return q * d[None, :]


def lowrank_haar(m: int = 2000, n: int = 1500, noise_std: float = 1e-4,
                 seed: int = SEED_BASE + 1) -> np.ndarray:
    """U diag(2^(-k/2)) V^T + N(0, noise_std^2) noise, FP64, m x n (m >= n)."""
    rng = np.random.default_rng(seed)
    k = min(m, n)
    u = haar(m, k, rng)
    v = haar(n, k, rng)
    sigma = 2.0 ** (-np.arange(1, k + 1) / 2.0)
    a = (u * sigma[None, :]) @ v.T
    if noise_std > 0:
        a += noise_std * rng.standard_normal((m, n))
    return np.ascontiguousarray(a)


def lowrank_plus_noise(m: int, n: int, sigma: np.ndarray, noise_std: float,
                       seed: int, dtype=np.float64) -> np.ndarray:
    """X diag(sigma) Y^T + noise with Haar X (m x k), Y (n x k)."""
    rng = np.random.default_rng(seed)
    k = len(sigma)
    x = haar(m, k, rng)
    y = haar(n, k, rng)
    a = (x * np.asarray(sigma)[None, :]) @ y.T
    if noise_std > 0:
        a += noise_std * rng.standard_normal((m, n))
    return np.ascontiguousarray(a.astype(dtype))


def gaussian_kernel(m: int = 65536, n: int = 8192, h: float = 0.2,
                    seed: int = SEED_BASE + 2, dtype=np.float32,
                    chunk_rows: int = 4096) -> np.ndarray:
    """exp(-|x_i - y_j|^2 / h^2) for x (m points) and y (n points) in [0,1]^3."""
    rng = np.random.default_rng(seed)
    x = rng.random((m, 3))
    y = rng.random((n, 3))
    out = np.empty((m, n), dtype=dtype)
    inv_h2 = 1.0 / (h * h)
    for s in range(0, m, chunk_rows):
        e = min(s + chunk_rows, m)
        d2 = ((x[s:e, None, :] - y[None, :, :]) ** 2).sum(axis=2)
        out[s:e] = np.exp(-d2 * inv_h2).astype(dtype)
    return out


def gaussian_kernel_device(m: int, n: int, h: float, seed: int, device="cuda"):
    """gaussian_kernel(m, n, h, seed) formed on `device` as an FP32 torch tensor: the same
    points (numpy, seeded), the distances and exp in FP64 on the device, rounded once."""
    import torch
    rng = np.random.default_rng(seed)
    x = torch.from_numpy(rng.random((m, 3))).to(device)
    y = torch.from_numpy(rng.random((n, 3))).to(device)
    d2 = ((x[:, None, :] - y[None, :, :]) ** 2).sum(dim=2)
    return torch.exp(-d2 / (h * h)).to(torch.float32)


# The learned proposal's training family: Gaussian-kernel matrices (points in [0,1]^3) with
# bandwidth h ~ U[0.1, 0.4]; m x n = 4096 x 1024 and r = 16 keep the proportions r/m = 1/256
# and r/n = 1/64 of the 16384 x 4096, r = 64 workload.
PROPOSAL_FAMILY = dict(m=4096, n=1024, r=16, b_r=16, b_c=4, k=32, h_range=(0.1, 0.4))


def proposal_family(count: int, seed: int = SEED_BASE + 5, h_range=(0.1, 0.4)):
    """(matrix seed, h) for `count` members of the Gaussian-kernel family."""
    rng = np.random.default_rng(seed)
    hs = rng.uniform(h_range[0], h_range[1], size=count)
    return [(seed * 1000 + t, float(hs[t])) for t in range(count)]


def sketch_matrices(m: int, n: int, k: int = 32, seed: int = SEED_BASE + 6):
    """Gaussian test matrices S (n x k) and T (m x k), i.i.d. N(0, 1/k), FP32."""
    rng = np.random.default_rng(seed)
    s = (rng.standard_normal((n, k)) / np.sqrt(k)).astype(np.float32)
    t = (rng.standard_normal((m, k)) / np.sqrt(k)).astype(np.float32)
    return s, t


def bf16_factor_product(m: int = 262144, n: int = 16384, k: int = 128, noise_std: float = 1e-2,
                        seed: int = SEED_BASE + 4, device="cuda", chunk_rows: int = 16384):
    """A = X diag(sigma) Y^T + noise rounded once to BF16, as a torch tensor on `device`:
    X (m x k), Y (n x k) i.i.d. N(0,1) from numpy (seeded), sigma_j = exp(-j/20) for
    j = 1..k, noise i.i.d. N(0, noise_std^2) from torch's counter-based generator on the
    device (seeded). The matrix is formed row chunk by row chunk on the device (8.6 GB at
    the default size; the host never holds it)."""
    import torch
    rng = np.random.default_rng(seed)
    x = torch.from_numpy(rng.standard_normal((m, k)).astype(np.float32)).to(device)
    y = torch.from_numpy(rng.standard_normal((n, k)).astype(np.float32)).to(device)
    sig = torch.from_numpy(np.exp(-np.arange(1, k + 1) / 20.0).astype(np.float32)).to(device)
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    out = torch.empty((m, n), dtype=torch.bfloat16, device=device)
    ys = (y * sig).t().contiguous()
    for s in range(0, m, chunk_rows):
        e = min(s + chunk_rows, m)
        blk = x[s:e] @ ys
        blk += noise_std * torch.randn((e - s, n), generator=g, device=device, dtype=torch.float32)
        out[s:e] = blk.to(torch.bfloat16)
    return out


def uneven_batch_shapes(count: int, seed: int = SEED_BASE + 3, m_range=(256, 4096), n_range=(128, 1024),
                        r_range=(8, 64)):
    """Shapes of the batched workload: m ~ U[m_range], n ~ U[n_range], r ~ U{r_range}
    (inclusive), with b_r = ceil(m / 512) row and b_c = ceil(n / 512) column blocks (blocks
    of at most 512 rows or columns)."""
    rng = np.random.default_rng(seed)
    ms = rng.integers(m_range[0], m_range[1] + 1, size=count)
    ns = rng.integers(n_range[0], n_range[1] + 1, size=count)
    rs = rng.integers(r_range[0], r_range[1] + 1, size=count)
    return [(int(m), int(n), int(r), -(-int(m) // 512), -(-int(n) // 512))
            for m, n, r in zip(ms, ns, rs)]


def uneven_batch_matrix(m: int, n: int, seed: int, rank: int = 96, noise_std: float = 1e-6) -> np.ndarray:
    """One matrix of the batched workload (FP32): U diag(sigma) V^T + noise with Haar U
    (m x k), V (n x k), k = min(rank, m, n), sigma_j = j^-2, i.i.d. noise of std noise_std."""
    rng = np.random.default_rng(seed)
    k = min(rank, m, n)
    u = haar(m, k, rng)
    v = haar(n, k, rng)
    s = 1.0 / np.arange(1, k + 1, dtype=np.float64) ** 2
    a = (u * s) @ v.T + noise_std * rng.standard_normal((m, n))
    return a.astype(np.float32)


def uneven_batch(count: int, seed: int = SEED_BASE + 3, **kw):
    """(shapes, matrices) of the batched workload; matrix t uses seed + 1 + t."""
    shapes = uneven_batch_shapes(count, seed, **kw)
    mats = [uneven_batch_matrix(m, n, seed + 1 + t) for t, (m, n, _r, _br, _bc) in enumerate(shapes)]
    return shapes, mats


def uneven_batch_device(shapes, seed: int = SEED_BASE + 3, rank: int = 96, noise_std: float = 1e-6,
                        device="cuda"):
    """The batched workload built on the device (a packed FP32 tensor and the element
    offsets), for batches too large to build on the host in reasonable time: matrix t is
    U diag(j^-2) V^T + noise with U, V from the QR of Gaussian matrices (sign-fixed, i.e.
    Haar), all drawn from torch's counter-based generator seeded with seed + 1 + t."""
    import torch
    offs, total = [], 0
    for (m, n, _r, _br, _bc) in shapes:
        offs.append(total)
        total += m * n
    out = torch.empty(total, dtype=torch.float32, device=device)
    for t, (m, n, _r, _br, _bc) in enumerate(shapes):
        g = torch.Generator(device=device)
        g.manual_seed(seed + 1 + t)
        k = min(rank, m, n)
        fac = []
        for rows in (m, n):
            gm = torch.randn((rows, k), generator=g, device=device, dtype=torch.float64)
            try:
                q, rr = torch.linalg.qr(gm)
            except RuntimeError:    # no device linear-algebra library in this process
                q, rr = torch.linalg.qr(gm.cpu())
                q, rr = q.to(device), rr.to(device)
            d = torch.sign(torch.diagonal(rr))
            d[d == 0] = 1.0
            fac.append(q * d)
        s = 1.0 / torch.arange(1, k + 1, device=device, dtype=torch.float64) ** 2
        a = (fac[0] * s) @ fac[1].t()
        a += noise_std * torch.randn((m, n), generator=g, device=device, dtype=torch.float64)
        out[offs[t]:offs[t] + m * n] = a.reshape(-1).float()
    return out, offs


def graded_basis(p: int, r: int, sigma_min: float, seed: int) -> np.ndarray:
    """A tall basis with a graded column space: X diag(sigma) Q, X (p x r) standard normal,
    sigma geometric from 1 to sigma_min, Q a Haar orthogonal r x r; rounded once to FP32
    (returned as FP32). Its best r x r submatrices have kappa ~ 1/sigma_min, so the swap
    iteration's drift bound (sum over swaps of kappa) runs out within one cycle."""
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((p, r))
    sig = np.geomspace(1.0, sigma_min, r)
    Q = haar(r, r, rng)
    return ((X * sig) @ Q).astype(np.float32)


def hilbert(n: int) -> np.ndarray:
    """H_ij = 1/(i+j-1) with 1-based i, j (Section 3.1, Hilbert experiment)."""
    i = np.arange(1, n + 1, dtype=np.float64)
    return 1.0 / (i[:, None] + i[None, :] - 1.0)


def cauchy_product(n: int, r: int) -> np.ndarray:
    """H = A B with A (n x r), B (r x n), A(i,j) = B(i,j) = 1/(i+j), 1-based
    (Section 3.1, synthetic low-rank experiment)."""
    i = np.arange(1, n + 1, dtype=np.float64)
    k = np.arange(1, r + 1, dtype=np.float64)
    a = 1.0 / (i[:, None] + k[None, :])
    b = 1.0 / (k[:, None] + i[None, :])
    return a @ b


def random_gaussian(m: int, n: int, seed: int, dtype=np.float64) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.standard_normal((m, n)).astype(dtype)


# Named workloads: shape, rank and block counts of each measured configuration.
CONFIGS = {
    "lowrank_haar_2000x1500_r16": dict(kind="lowrank_haar", m=2000, n=1500, r=16,
                                       b_r=8, b_c=8, delta=1e-2, dtype="f64"),
    "gaussian_kernel_65536x8192_r64": dict(kind="gaussian_kernel", m=65536, n=8192,
                                           r=64, b_r=64, b_c=8, delta=1e-2,
                                           dtype="f32"),
}


def make(name: str, **over) -> np.ndarray:
    cfg = dict(CONFIGS[name])
    cfg.update(over)
    if cfg["kind"] == "lowrank_haar":
        return lowrank_haar(cfg["m"], cfg["n"], cfg.get("noise_std", 1e-4),
                            cfg.get("seed", SEED_BASE + 1))
    if cfg["kind"] == "gaussian_kernel":
        return gaussian_kernel(cfg["m"], cfg["n"], cfg.get("h", 0.2),
                               cfg.get("seed", SEED_BASE + 2))
    raise KeyError(name)
