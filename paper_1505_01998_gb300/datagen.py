"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no arithmetic of the bandwidth-selection method; it only draws
samples.  Both the CUDA path and the FP64 oracle take their inputs from here.

The paper measured on unspecified "random" data (Sec. 7.2) and names no public
dataset, so every workload is synthetic.  All draws use
``numpy.random.Generator(PCG64(seed))``; the seeds are recorded by the callers.
Arrays are returned in the paper's layout: a ``(d, n)`` matrix, one sample per
column (Sec. 4.4.2).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def mixture_1d(n: int, seed: int, weights=(0.5, 0.3, 0.2), means=(-2.0, 0.0, 3.0),
               sds=(0.5, 1.0, 0.8), dtype=np.float64) -> np.ndarray:
    """Univariate Gaussian mixture; the defaults are the n=1,024 workload."""
    g = rng(seed)
    comp = g.choice(len(weights), size=n, p=np.asarray(weights) / np.sum(weights))
    x = g.normal(np.asarray(means)[comp], np.asarray(sds)[comp])
    return x.astype(dtype)[None, :]


def skewed_column(n: int, seed: int, dtype=np.float32) -> np.ndarray:
    """Half lognormal(0, 1), half uniform[0, 100], shuffled: the skewed column
    of the n=65,536 workload."""
    g = rng(seed)
    a = g.lognormal(0.0, 1.0, size=n // 2)
    b = g.uniform(0.0, 100.0, size=n - n // 2)
    x = np.concatenate([a, b])
    g.shuffle(x)
    return x.astype(dtype)[None, :]


def random_spd(d: int, g: np.random.Generator, cond: float = 50.0) -> np.ndarray:
    """Q diag(lam) Q^T with Q from the QR of a Gaussian matrix (sign-fixed) and
    eigenvalues log-uniform on [1, cond], the extremes forced to 1 and cond."""
    q, r = np.linalg.qr(g.normal(size=(d, d)))
    q = q * np.sign(np.diag(r))[None, :]
    lam = np.exp(g.uniform(0.0, math.log(cond), size=d))
    if d >= 2:
        lam[0], lam[-1] = 1.0, cond
    else:
        lam[0] = 1.0
    return (q * lam[None, :]) @ q.T


def correlated_mixture(n: int, d: int, seed: int, k: int = 4, dtype=np.float32) -> np.ndarray:
    """Equal-weight mixture of k correlated Gaussians in d dimensions: means
    U[-4, 4]^d, covariances random SPD with condition number <= 50."""
    g = rng(seed)
    means = g.uniform(-4.0, 4.0, size=(k, d))
    chol = [np.linalg.cholesky(random_spd(d, g)) for _ in range(k)]
    comp = g.integers(0, k, size=n)
    z = g.normal(size=(n, d))
    x = np.empty((n, d))
    for c in range(k):
        m = comp == c
        x[m] = means[c] + z[m] @ chol[c].T
    return np.ascontiguousarray(x.T.astype(dtype))


def batch_dataset(n: int, g: np.random.Generator, dtype=np.float32) -> np.ndarray:
    """One dataset of the 512-dataset batch: with probability 1/2 a mixture of
    1-5 Gaussians (Dirichlet(1) weights, means U[-5, 5], sds log-U[0.2, 2]),
    otherwise lognormal(0, 1)."""
    if g.uniform() < 0.5:
        k = int(g.integers(1, 6))
        w = g.dirichlet(np.ones(k))
        mu = g.uniform(-5.0, 5.0, size=k)
        sd = np.exp(g.uniform(math.log(0.2), math.log(2.0), size=k))
        comp = g.choice(k, size=n, p=w)
        x = g.normal(mu[comp], sd[comp])
    else:
        x = g.lognormal(0.0, 1.0, size=n)
    return x.astype(dtype)[None, :]


def batch_sizes(count: int, seed: int, lo: int = 256, hi: int = 131072) -> np.ndarray:
    g = rng(seed)
    return np.rint(np.exp(g.uniform(math.log(lo), math.log(hi), size=count))).astype(np.int64)


def batch(count: int = 512, seed: int = 4, lo: int = 256, hi: int = 131072, dtype=np.float32):
    """The batched workload: ``count`` univariate datasets, sizes log-uniform."""
    sizes = batch_sizes(count, seed, lo, hi)
    g = rng(seed + 1000)
    return [batch_dataset(int(m), g, dtype) for m in sizes]


@dataclass
class Request:
    """One bandwidth-selection request of the serving workload."""
    arrival_s: float
    n: int
    d: int
    method: str  # "lscv" or "plugin"
    seed: int
    x: np.ndarray = field(repr=False, default=None)


def serving_requests(rate_per_s: float, count: int, seed: int = 5, lo: int = 1024,
                     hi: int = 262144, materialise: bool = True, dtype=np.float32):
    """Poisson arrivals; n log-uniform in [lo, hi]; d = 1 : d = 2 at 4 : 1;
    d = 2 always LSCV; d = 1 draws plug-in with p = 0.625 so the overall mix is
    50/50; samples as in the correlated-mixture workload."""
    g = rng(seed)
    t = 0.0
    out = []
    for k in range(count):
        t += g.exponential(1.0 / rate_per_s)
        n = int(round(math.exp(g.uniform(math.log(lo), math.log(hi)))))
        d = 1 if g.uniform() < 0.8 else 2
        method = "lscv" if d == 2 else ("plugin" if g.uniform() < 0.625 else "lscv")
        rseed = int(g.integers(0, 2**31 - 1))
        r = Request(t, n, d, method, rseed)
        if materialise:
            r.x = correlated_mixture(n, d, rseed, dtype=dtype)
        out.append(r)
    return out


# The paper's toy dataset (Sec. 4.2, the 8-point example behind its KDE figure).
TOY8 = np.array([[0.0, 1.0, 1.1, 1.5, 1.9, 2.8, 2.9, 3.5]])
