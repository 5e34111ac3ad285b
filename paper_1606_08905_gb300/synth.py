"""Seeded synthetic inputs for the k-means workloads.

This module holds no k-means arithmetic: it only draws points.  The library
and the oracle both consume what it returns (the same array, handed to each),
so a difference between them can never come from the inputs.

The workloads stand in for the paper's datasets (Friendster eigenvectors and
the RM/RU random matrices of the evaluation's dataset table), which are not
available; they keep the shapes (n, d, k) and the kind of structure the paper
describes (natural clusters for the eigenvector data, uniform and
multivariate-normal random matrices for the scaling runs).

Every generator takes a seed and a torch device.  The mixture parameters are
always drawn on the CPU (so they are identical on every device); the points
are drawn on `device` in chunks of at most 2**26 rows.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import torch

CHUNK_ROWS = 1 << 26


def _cpu_gen(seed: int) -> torch.Generator:
    g = torch.Generator(device="cpu")
    g.manual_seed(int(seed))
    return g


def _dev_gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=torch.device(device))
    g.manual_seed(int(seed) ^ 0x5DEECE66D)
    return g


def _dirichlet1(k: int, g: torch.Generator) -> torch.Tensor:
    """Dirichlet(1,...,1) weights as normalised Exp(1) draws (FP64, CPU)."""
    e = -torch.log1p(-torch.rand(k, generator=g, dtype=torch.float64))
    return e / e.sum()


def _labels(n: int, weights: torch.Tensor, g: torch.Generator, device) -> torch.Tensor:
    """Component label of each point: inverse-CDF of the mixture weights."""
    cdf = torch.cumsum(weights, 0).to(device=device, dtype=torch.float64)
    cdf[-1] = 1.0
    r = torch.rand(n, generator=g, device=device, dtype=torch.float64)
    return torch.clamp(torch.searchsorted(cdf, r, right=True), max=weights.numel() - 1)


@dataclass
class Mixture:
    means: torch.Tensor      # k x d, FP64, CPU
    weights: torch.Tensor    # k, FP64, CPU
    # per-component linear map A_j (x = mu_j + A_j z); None for isotropic
    maps: torch.Tensor | None
    sigma: float | torch.Tensor = 1.0   # isotropic std, or k x d diagonal stds


def _draw(mix: Mixture, n: int, seed: int, device, labels_out: bool):
    device = torch.device(device)
    k, d = mix.means.shape
    g = _dev_gen(seed, device)
    X = torch.empty((n, d), dtype=torch.float32, device=device)
    L = torch.empty(n, dtype=torch.int64, device=device) if labels_out else None
    mu = mix.means.to(device=device, dtype=torch.float32)
    maps = mix.maps.to(device=device, dtype=torch.float32) if mix.maps is not None else None
    sig = mix.sigma.to(device=device, dtype=torch.float32) if torch.is_tensor(mix.sigma) else None
    for lo in range(0, n, CHUNK_ROWS):
        hi = min(n, lo + CHUNK_ROWS)
        m = hi - lo
        lab = _labels(m, mix.weights, g, device)
        z = torch.randn((m, d), generator=g, device=device, dtype=torch.float32)
        if maps is not None:
            out = torch.empty_like(z)
            for j in range(k):
                idx = (lab == j).nonzero(as_tuple=True)[0]
                if idx.numel():
                    out[idx] = z[idx] @ maps[j].T + mu[j]
            z = out
        elif sig is not None:
            z = z * sig[lab] + mu[lab]
        else:
            z = z * float(mix.sigma) + mu[lab]
        X[lo:hi] = z
        if L is not None:
            L[lo:hi] = lab
    return (X, L) if labels_out else X


def isotropic_mixture(n: int, d: int, k: int, seed: int, device="cpu", mean_lo=-10.0,
                      mean_hi=10.0, sigma=1.0, equal_weights=True, labels=False):
    """k isotropic Gaussians, means uniform in [mean_lo, mean_hi]^d, std sigma.
    Equal weights (the 100k x 8, k = 10 plain-Lloyd workload) or Dirichlet(1)."""
    g = _cpu_gen(seed)
    means = mean_lo + (mean_hi - mean_lo) * torch.rand((k, d), generator=g, dtype=torch.float64)
    w = torch.full((k,), 1.0 / k, dtype=torch.float64) if equal_weights else _dirichlet1(k, g)
    return _draw(Mixture(means, w, None, float(sigma)), n, seed, device, labels)


def spd_mixture(n: int, d: int, k: int, seed: int, device="cpu", mean_lo=-5.0, mean_hi=5.0,
                lam_lo=0.5, lam_hi=2.0, labels=False):
    """k Gaussians with random SPD covariances Q diag(lam) Q^T (Q from the QR
    of a Gaussian matrix, lam uniform in [lam_lo, lam_hi]), means uniform in
    [mean_lo, mean_hi]^d, Dirichlet(1) weights (the 66M x 32, k = 20 MTI
    workload; also the 1e9 x 16 mixture variant with means in [0, 10]^16)."""
    g = _cpu_gen(seed)
    means = mean_lo + (mean_hi - mean_lo) * torch.rand((k, d), generator=g, dtype=torch.float64)
    w = _dirichlet1(k, g)
    maps = torch.empty((k, d, d), dtype=torch.float64)
    for j in range(k):
        q, r = torch.linalg.qr(torch.randn((d, d), generator=g, dtype=torch.float64))
        q = q * torch.sign(torch.diagonal(r)).unsqueeze(0)
        lam = lam_lo + (lam_hi - lam_lo) * torch.rand(d, generator=g, dtype=torch.float64)
        maps[j] = q * torch.sqrt(lam).unsqueeze(0)
    return _draw(Mixture(means, w, maps), n, seed, device, labels)


def aniso_mixture(n: int, d: int, k: int, seed: int, device="cpu", mean_lo=-5.0, mean_hi=5.0,
                  std_lo=0.5, std_hi=2.0, labels=False):
    """k axis-aligned anisotropic Gaussians: per-component, per-dimension std
    log-uniform in [std_lo, std_hi]; means uniform in [mean_lo, mean_hi]^d;
    Dirichlet(1) weights (the 10M x 128, k = 1024 precision-form workload)."""
    g = _cpu_gen(seed)
    means = mean_lo + (mean_hi - mean_lo) * torch.rand((k, d), generator=g, dtype=torch.float64)
    w = _dirichlet1(k, g)
    ls = math.log(std_lo) + (math.log(std_hi) - math.log(std_lo)) * torch.rand(
        (k, d), generator=g, dtype=torch.float64)
    return _draw(Mixture(means, w, None, torch.exp(ls)), n, seed, device, labels)


def uniform_cube(n: int, d: int, seed: int, device="cpu", lo=0.0, hi=1.0):
    """i.i.d. uniform points in [lo, hi]^d (the 1e9 x 16 scale workload)."""
    device = torch.device(device)
    g = _dev_gen(seed, device)
    X = torch.empty((n, d), dtype=torch.float32, device=device)
    for a in range(0, n, CHUNK_ROWS):
        b = min(n, a + CHUNK_ROWS)
        X[a:b] = lo + (hi - lo) * torch.rand((b - a, d), generator=g, device=device)
    return X


@dataclass
class InstanceSpec:
    n: int
    d: int
    k: int
    seed: int


def batched_specs(m: int, seed: int, n_lo=1e3, n_hi=1e6, dims=(8, 16, 32, 64), k_lo=4,
                  k_hi=256):
    """m independent instances: n log-uniform in [n_lo, n_hi], d uniform over
    `dims`, k uniform on {k_lo..k_hi} (k never above n)."""
    g = _cpu_gen(seed)
    out = []
    for i in range(m):
        e = math.log10(n_lo) + (math.log10(n_hi) - math.log10(n_lo)) * float(
            torch.rand(1, generator=g, dtype=torch.float64))
        n = int(round(10.0 ** e))
        d = int(dims[int(torch.randint(len(dims), (1,), generator=g))])
        k = int(torch.randint(k_lo, k_hi + 1, (1,), generator=g))
        out.append(InstanceSpec(n=n, d=d, k=min(k, n), seed=int(seed) * 100003 + i))
    return out


def batched_instance(spec: InstanceSpec, device="cpu"):
    """One batched-form instance: an isotropic mixture with spec.k components,
    means uniform in [-10, 10]^d, sigma 1, equal weights."""
    return isotropic_mixture(spec.n, spec.d, spec.k, spec.seed, device=device)


# The named workloads, by the shapes they are quoted on.
WORKLOADS = {
    "plain_100k_d8_k10": dict(kind="isotropic", n=100_000, d=8, k=10, data_seed=1001,
                              max_iters=20, prune=False),
    "mti_66m_d32_k20": dict(kind="spd", n=66_000_000, d=32, k=20, data_seed=1002,
                            max_iters=50, prune=True),
    "precision_10m_d128_k1024": dict(kind="aniso", n=10_000_000, d=128, k=1024,
                                     data_seed=1003, max_iters=30, prune=False, precision="fp16"),
    # 512 instances: n log-uniform in [1e3, 1e6], d in {8, 16, 32, 64}, k in
    # {4..256}; n is the total over the instances (batched_specs(512, 1004))
    "batched_512": dict(kind="batched", m=512, n=0, d=0, k=0, data_seed=1004, max_iters=25, prune=True),
    "scale_1b_d16_k100_uniform": dict(kind="uniform", n=1_000_000_000, d=16, k=100,
                                      data_seed=1005, max_iters=20, prune=True),
    "scale_1b_d16_k100_mixture": dict(kind="spd_scaled", n=1_000_000_000, d=16, k=100,
                                      data_seed=1006, max_iters=20, prune=True),
    # Elkan's lower bounds (the ablation of MTI) on the 100k x 8, k = 10
    # workload's points and on a 16M-point slice of the 66M x 32, k = 20 one
    # the 66M x 32, k = 20 workload with the points left in pinned host
    # memory (read in place over the host link; Clause 1 saves the transfers)
    "host_66m_d32_k20": dict(kind="spd", n=66_000_000, d=32, k=20, data_seed=1002,
                             max_iters=50, prune=True, points_in_host=True),
    "elkan_100k_d8_k10": dict(kind="isotropic", n=100_000, d=8, k=10, data_seed=1001,
                              max_iters=20, prune=True, elkan=True),
    "elkan_16m_d32_k20": dict(kind="spd", n=16_000_000, d=32, k=20, data_seed=1002,
                              max_iters=50, prune=True, elkan=True),
}
INIT_SEED = 42
WORKLOADS["batched_512"]["n"] = sum(s.n for s in batched_specs(512, 1004))


def make(kind: str, n: int, d: int, k: int, seed: int, device="cpu"):
    """Points of one workload kind at the given size."""
    if kind == "isotropic":
        return isotropic_mixture(n, d, k, seed, device=device)
    if kind == "spd":
        return spd_mixture(n, d, k, seed, device=device)
    if kind == "spd_scaled":
        return spd_mixture(n, d, k, seed, device=device, mean_lo=0.0, mean_hi=10.0)
    if kind == "aniso":
        return aniso_mixture(n, d, k, seed, device=device)
    if kind == "uniform":
        return uniform_cube(n, d, seed, device=device)
    raise ValueError(kind)
