"""Seeded synthetic collections and query workloads.

This module only makes inputs; it holds none of the k-NN method's arithmetic.
The tests, the smoke check and the benchmark feed the same tensors to the CUDA
library and to the oracle (the oracle gets host copies).

Shapes and distributions follow the paper's workloads (Sec. 4.1):
  * Synth: random walks, cumulative sums of N(0,1) steps, z-normalised per
    series (population std; a constant series becomes all zeros);
  * Gaussian rows (N(0,1) per point), optionally L2-normalised, standing in
    for embedding collections such as Deep;
  * queries: a series drawn uniformly from the collection plus N(0, sigma^2)
    noise per point, then normalised like the collection (the paper's 1%-10%
    workloads are sigma^2 in [0.01, 0.1]).
Random numbers come from torch generators seeded explicitly; generation is
chunked with a fixed chunk size so the output does not depend on memory.
"""
import torch

CHUNK_ROWS = 1 << 18


def _znorm_(x: torch.Tensor) -> torch.Tensor:
    mu = x.mean(dim=1, keepdim=True)
    x.sub_(mu)
    sd = x.square().mean(dim=1, keepdim=True).sqrt_()
    x.div_(torch.where(sd > 0, sd, torch.ones_like(sd)))
    return x


def _l2norm_(x: torch.Tensor) -> torch.Tensor:
    nrm = x.square().sum(dim=1, keepdim=True).sqrt_()
    x.div_(torch.where(nrm > 0, nrm, torch.ones_like(nrm)))
    return x


def random_walk_chunks(N: int, n: int, seed: int = 0, device="cpu"):
    """The rows of random_walk(N, n, seed) as (first row, float32 block) pairs,
    generated block by block from the same random stream."""
    dev = torch.device(device)
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    for a in range(0, N, CHUNK_ROWS):
        b = min(N, a + CHUNK_ROWS)
        steps = torch.randn((b - a, n), generator=g, device=dev, dtype=torch.float32)
        walk = torch.cumsum(steps.double(), dim=1)
        yield a, _znorm_(walk).float()


def random_walk(N: int, n: int, seed: int = 0, device="cpu", out=None):
    """N z-normalised random walks of length n, float32 [N, n]."""
    if out is None:
        out = torch.empty((N, n), dtype=torch.float32, device=torch.device(device))
    for a, rows in random_walk_chunks(N, n, seed, device):
        out[a:a + rows.shape[0]] = rows
    return out


def gaussian(N: int, n: int, seed: int = 0, device="cpu", l2=False, out=None):
    """N rows of N(0,1) points, float32 [N, n]; L2-normalised if l2."""
    dev = torch.device(device)
    if out is None:
        out = torch.empty((N, n), dtype=torch.float32, device=dev)
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    for a in range(0, N, CHUNK_ROWS):
        b = min(N, a + CHUNK_ROWS)
        rows = torch.randn((b - a, n), generator=g, device=dev, dtype=torch.float32)
        out[a:b] = _l2norm_(rows.double()).float() if l2 else rows
    return out


def queries(X: torch.Tensor, nq: int, sigmas, seed: int = 1, norm="z"):
    """nq queries: uniformly drawn rows of X plus N(0, sigma_i^2) noise.

    sigmas: a float, or a sequence used cyclically (query i gets
    sigmas[i % len(sigmas)]).  norm: 'z' (z-normalise), 'l2' or None.
    Returns (Q [nq, n] float32 on X's device, source row ids [nq] int64).
    """
    dev = X.device
    N, n = X.shape
    g = torch.Generator(device="cpu")
    g.manual_seed(seed)
    src = torch.randint(0, N, (nq,), generator=g)
    if isinstance(sigmas, (int, float)):
        sig = torch.full((nq,), float(sigmas), dtype=torch.float64)
    else:
        s = torch.tensor(list(sigmas), dtype=torch.float64)
        sig = s[torch.arange(nq) % s.numel()]
    noise = torch.randn((nq, n), generator=g, dtype=torch.float64) * sig[:, None]
    q = X[src.to(dev)].double() + noise.to(dev)
    if norm == "z":
        _znorm_(q)
    elif norm == "l2":
        _l2norm_(q)
    return q.float().contiguous(), src


# The served mix: four device-resident collections (name, N, n, kind, leaf
# capacity), standing in for the paper's Deep (n = 96, embeddings), SALD
# (n = 128) and Synth / Seismic (random walks) collections.  Collection i
# uses data seed 10 + i and query seed 20 + i.
SERVED_MIX = [
    ("20M x 96 Gaussian, L2-normalised", 20_000_000, 96, "gauss_l2", 10_000),
    ("10M x 128 Gaussian", 10_000_000, 128, "gauss", 10_000),
    ("10M x 256 random walk", 10_000_000, 256, "rw", 10_000),
    ("2M x 1024 random walk", 2_000_000, 1024, "rw", 10_000),
]


def collection(kind: str, N: int, n: int, seed: int, device="cpu"):
    """A collection of the served mix's kinds: 'rw' (z-normalised random
    walks), 'gauss' (N(0,1) rows) or 'gauss_l2' (the same, L2-normalised)."""
    if kind == "rw":
        return random_walk(N, n, seed=seed, device=device)
    return gaussian(N, n, seed=seed, device=device, l2=(kind == "gauss_l2"))


def query_norm(kind: str):
    """How queries of a collection kind are normalised (as its rows are)."""
    return {"rw": "z", "gauss_l2": "l2", "gauss": None}[kind]


def uniform_sigmas(nq: int, lo: float, hi: float, seed: int = 1):
    """nq noise levels drawn uniformly from [lo, hi]."""
    g = torch.Generator(device="cpu")
    g.manual_seed(seed + 7919)
    return (lo + (hi - lo) * torch.rand((nq,), generator=g, dtype=torch.float64)).tolist()
