"""Seeded synthetic inputs shaped like the paper's workloads.

This module draws data only: it holds none of the clustering method's
arithmetic and imports nothing from the CUDA binding or the oracle, so both
sides of every parity check read the same arrays from here.

The paper's datasets (SIFT1M, GIST1M, VLAD10M; Tab. 1) are not available, so
each workload has a stand-in with the same n, d, value range and a latent
cluster structure:

  gauss_mixture   isotropic Gaussian mixture, centres uniform in [-box, box]^d
  sift_like       SIFT-shaped: non-negative integers 0..255 from a clipped,
                  rounded log-normal around latent centres (mean about 20)
  gist_like       GIST-shaped: values in [0, 1] from Beta draws around latent
                  Beta(2, 8) centres
  deep_like       deep-feature-shaped: unit vectors from von Mises-Fisher
                  components (Wood's 1994 sampler), stored as bfloat16 bits

All draws use numpy's PCG64 generator seeded from the arguments.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 170501813


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def gauss_mixture(n: int, d: int, n_centers: int, seed: int, box: float = 10.0, sigma: float = 1.0,
                  return_components: bool = False):
    """x = c_z + N(0, sigma^2 I), z uniform over n_centers centres drawn U[-box, box]^d."""
    g = _rng(seed)
    centers = g.uniform(-box, box, size=(n_centers, d)).astype(np.float64)
    z = g.integers(0, n_centers, size=n)
    X = np.empty((n, d), np.float32)
    step = 1 << 18
    for s in range(0, n, step):
        e = min(n, s + step)
        X[s:e] = (centers[z[s:e]] + sigma * g.standard_normal((e - s, d))).astype(np.float32)
    return (X, z) if return_components else X


def sift_like(n: int, d: int = 128, n_latent: int = 10000, seed: int = BASE_SEED + 1):
    """Integers in [0, 255] stored as FP32: clip(round(exp(mu_{z,t} + 0.7 e)), 0, 255).

    mu_{c,t} ~ N(ln 20 - 0.37, 0.5) per latent centre and dimension, e ~ N(0, 1);
    the offset 0.37 = (0.5^2 + 0.7^2) / 2 puts the log-normal's mean at 20 (before
    rounding and clipping), with a heavy upper tail.
    """
    g = _rng(seed)
    mu = g.normal(math.log(20.0) - 0.37, 0.5, size=(n_latent, d))
    z = g.integers(0, n_latent, size=n)
    X = np.empty((n, d), np.float32)
    step = 1 << 17
    for s in range(0, n, step):
        e = min(n, s + step)
        v = np.exp(mu[z[s:e]] + 0.7 * g.standard_normal((e - s, d)))
        X[s:e] = np.clip(np.rint(v), 0.0, 255.0).astype(np.float32)
    return X


def gist_like(n: int, d: int = 960, n_latent: int = 1000, seed: int = BASE_SEED + 2, conc: float = 50.0):
    """x_t ~ Beta(conc mu_{z,t}, conc (1 - mu_{z,t})) with latent mu_{c,t} ~ Beta(2, 8)."""
    g = _rng(seed)
    mu = np.clip(g.beta(2.0, 8.0, size=(n_latent, d)), 1e-3, 1 - 1e-3)
    z = g.integers(0, n_latent, size=n)
    X = np.empty((n, d), np.float32)
    step = 1 << 15
    for s in range(0, n, step):
        e = min(n, s + step)
        m = mu[z[s:e]]
        X[s:e] = g.beta(conc * m, conc * (1.0 - m)).astype(np.float32)
    return X


def gamma_device(alpha, g, max_rounds: int = 64):
    """Gamma(alpha, 1) draws, one per element of the tensor alpha (> 0), with the seeded torch generator g:
    Marsaglia and Tsang (2000) rejection for shape >= 1 (d = a - 1/3, c = 1/sqrt(9d), v = (1 + c z)^3,
    accept when log u < z^2/2 + d - d v + d log v), and for shape < 1 the draw at shape + 1 times
    u^(1/shape)."""
    import torch
    a = alpha.to(torch.float64)
    small = a < 1.0
    sh = torch.where(small, a + 1.0, a)
    dd = sh - 1.0 / 3.0
    c = 1.0 / torch.sqrt(9.0 * dd)
    out = torch.empty_like(a)
    todo = torch.arange(a.numel(), device=a.device)
    flat_d, flat_c = dd.reshape(-1), c.reshape(-1)
    for _ in range(max_rounds):
        if todo.numel() == 0:
            break
        z = torch.randn(todo.shape, generator=g, device=a.device, dtype=torch.float64)
        u = torch.rand(todo.shape, generator=g, device=a.device, dtype=torch.float64)
        dq, cq = flat_d[todo], flat_c[todo]
        v = (1.0 + cq * z) ** 3
        ok = (v > 0) & (torch.log(u) < 0.5 * z * z + dq - dq * v + dq * torch.log(torch.clamp(v, min=1e-300)))
        out.view(-1)[todo[ok]] = (dq * v)[ok]
        todo = todo[~ok]
    if todo.numel():
        raise RuntimeError("gamma sampler did not converge")
    u = torch.rand(a.shape, generator=g, device=a.device, dtype=torch.float64)
    return torch.where(small, out * u ** (1.0 / a), out)


def gist_like_device(n: int, d: int = 960, n_latent: int = 1000, seed: int = BASE_SEED + 2, conc: float = 50.0,
                     device="cuda", chunk: int = 1 << 16):
    """The recipe of gist_like drawn on the GPU with a seeded torch generator (same recipe, different stream of
    random numbers): latent mu ~ Beta(2, 8) clipped to [1e-3, 1 - 1e-3], x_t ~ Beta(conc mu, conc (1 - mu)),
    every Beta draw as G_a / (G_a + G_b) of two Gamma draws.  Returns an n x d FP32 tensor on the device."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))

    def beta(a, b):
        ga, gb = gamma_device(a, g), gamma_device(b, g)
        return ga / (ga + gb)

    mu = torch.clamp(beta(torch.full((n_latent, d), 2.0, device=device, dtype=torch.float64),
                          torch.full((n_latent, d), 8.0, device=device, dtype=torch.float64)), 1e-3, 1 - 1e-3)
    z = torch.randint(0, n_latent, (n,), generator=g, device=device)
    X = torch.empty((n, d), dtype=torch.float32, device=device)
    for s in range(0, n, chunk):
        m = mu[z[s:s + chunk]]
        X[s:s + m.shape[0]] = beta(conc * m, conc * (1.0 - m)).to(torch.float32)
    return X


def _vmf_w(g: np.random.Generator, kappa: float, d: int, size: int) -> np.ndarray:
    """Wood (1994) rejection sampler for the cosine w of a vMF draw in d dimensions."""
    b = (-2.0 * kappa + math.sqrt(4.0 * kappa * kappa + (d - 1.0) ** 2)) / (d - 1.0)
    x0 = (1.0 - b) / (1.0 + b)
    c = kappa * x0 + (d - 1.0) * math.log(1.0 - x0 * x0)
    out = np.empty(size)
    filled = 0
    while filled < size:
        m = (size - filled) * 2 + 16
        zb = g.beta((d - 1.0) / 2.0, (d - 1.0) / 2.0, size=m)
        w = (1.0 - (1.0 + b) * zb) / (1.0 - (1.0 - b) * zb)
        u = g.uniform(size=m)
        ok = kappa * w + (d - 1.0) * np.log(1.0 - x0 * w) - c >= np.log(u)
        w = w[ok][: size - filled]
        out[filled:filled + w.shape[0]] = w
        filled += w.shape[0]
    return out


def to_bf16_bits(a: np.ndarray) -> np.ndarray:
    """Round FP32 to bfloat16 (nearest, ties to even) and return the 16-bit patterns."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32)
    r = ((u >> 16) & 1) + 0x7FFF
    return ((u + r) >> 16).astype(np.uint16)


def bf16_bits_to_f32(b: np.ndarray) -> np.ndarray:
    return (np.asarray(b, dtype=np.uint16).astype(np.uint32) << 16).view(np.float32)


def deep_like(n: int, d: int = 512, n_dirs: int = 2_000_000, kappa_vmf: float = 50.0,
              seed: int = BASE_SEED + 3) -> np.ndarray:
    """Unit vectors from a mixture of vMF(mu_c, kappa_vmf); returns bfloat16 bit patterns [n, d]."""
    g = _rng(seed)
    z = g.integers(0, n_dirs, size=n)
    out = np.empty((n, d), np.uint16)
    step = 1 << 14
    for s in range(0, n, step):
        e = min(n, s + step)
        m = e - s
        # mean directions are regenerated from a per-direction seed so that the
        # n_dirs x d table never has to be held in memory
        mu = np.stack([_rng(seed * 1_000_003 + int(c)).standard_normal(d) for c in z[s:e]])
        mu /= np.linalg.norm(mu, axis=1, keepdims=True)
        w = _vmf_w(g, kappa_vmf, d, m)
        v = g.standard_normal((m, d))
        v -= (v * mu).sum(1, keepdims=True) * mu
        v /= np.linalg.norm(v, axis=1, keepdims=True)
        x = w[:, None] * mu + np.sqrt(np.maximum(0.0, 1.0 - w * w))[:, None] * v
        out[s:e] = to_bf16_bits(x.astype(np.float32))
    return out


@dataclass
class Workload:
    """One synthetic clustering workload (sizes and method parameters)."""
    name: str
    n: int
    d: int
    k: int
    kappa: int
    xi: int = 50
    tau: int = 10
    iters: int = 10
    max_cluster: int = 128
    seed: int = BASE_SEED
    storage: str = "f32"
    extra: dict = field(default_factory=dict)

    @property
    def k0(self) -> int:
        return max(1, self.n // self.xi)

    def data(self) -> np.ndarray:
        if self.name.startswith("gauss"):
            return gauss_mixture(self.n, self.d, self.extra.get("n_centers", 200), self.seed)
        if self.name.startswith("sift"):
            return sift_like(self.n, self.d, self.extra.get("n_latent", 10000), self.seed)
        if self.name.startswith("gist"):
            return gist_like(self.n, self.d, self.extra.get("n_latent", 1000), self.seed)
        if self.name.startswith("deep"):
            return deep_like(self.n, self.d, self.extra.get("n_dirs", 2_000_000), 50.0, self.seed)
        raise KeyError(self.name)


WORKLOADS = {
    # plain method, FP32: 200-component Gaussian mixture
    "gauss_n20000_d32_k200": Workload("gauss_n20000_d32_k200", 20_000, 32, 200, 20, seed=BASE_SEED,
                                      extra={"n_centers": 200}),
    # SIFT-shaped
    "sift_n1000000_d128_k10000": Workload("sift_n1000000_d128_k10000", 1_000_000, 128, 10_000, 50,
                                          seed=BASE_SEED + 1, extra={"n_latent": 10000}),
    # GIST-shaped
    "gist_n1000000_d960_k10000": Workload("gist_n1000000_d960_k10000", 1_000_000, 960, 10_000, 50,
                                          seed=BASE_SEED + 2, extra={"n_latent": 1000}),
    # deep-feature-shaped, largest scale, bfloat16 storage
    "deep_n10000000_d512_k1000000": Workload("deep_n10000000_d512_k1000000", 10_000_000, 512, 1_000_000, 40,
                                             seed=BASE_SEED + 3, storage="bf16",
                                             extra={"n_dirs": 2_000_000}),
}


def gauss_mixture_device(n: int, d: int, n_centers: int, seed: int, device, box: float = 10.0, sigma: float = 1.0,
                         out=None, z_out=None):
    """The mixture of gauss_mixture drawn on the GPU with a seeded torch generator (same recipe, different
    stream of random numbers): serving jobs generate their samples where they are clustered.  out (n x d
    float32) and z_out (n int64) may be given so that nothing of size n is allocated."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    centers = (torch.rand((n_centers, d), generator=g, device=device, dtype=torch.float32) * 2.0 - 1.0) * box
    z = torch.empty(n, dtype=torch.int64, device=device) if z_out is None else z_out
    torch.randint(0, n_centers, (n,), generator=g, device=device, out=z)
    X = torch.empty((n, d), dtype=torch.float32, device=device) if out is None else out
    torch.randn((n, d), generator=g, device=device, dtype=torch.float32, out=X)
    X.mul_(sigma)
    step = 1 << 16  # the centres are added in chunks (bounded temporaries)
    for s in range(0, n, step):
        X[s:s + step] += centers[z[s:s + step]]
    return X


def deep_like_device(n: int, d: int = 512, n_dirs: int = 2_000_000, kappa_vmf: float = 50.0,
                     seed: int = BASE_SEED + 3, device="cuda", chunk: int = 1 << 18):
    """The vMF mixture of deep_like drawn on the GPU with a seeded torch generator (same recipe, different
    stream of random numbers); returns an n x d bfloat16 tensor on the device.  The n_dirs x d table of
    mean directions is held on the device (4 GB at 2,000,000 x 512).  The cosine w to the mean direction
    follows Wood (1994), with its Beta((d-1)/2, (d-1)/2) draw taken as a ratio of two chi-square
    variables of d - 1 degrees of freedom (sums of squared normals)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    mu = torch.empty((n_dirs, d), dtype=torch.float32, device=device)
    for s in range(0, n_dirs, chunk):
        blk = torch.randn((min(n_dirs, s + chunk) - s, d), generator=g, device=device)
        mu[s:s + blk.shape[0]] = blk / blk.norm(dim=1, keepdim=True)
    kap = float(kappa_vmf)
    b = (-2.0 * kap + math.sqrt(4.0 * kap * kap + (d - 1.0) ** 2)) / (d - 1.0)
    x0 = (1.0 - b) / (1.0 + b)
    c = kap * x0 + (d - 1.0) * math.log(1.0 - x0 * x0)

    def chi2(m):
        return torch.randn((m, d - 1), generator=g, device=device).double().square().sum(1)

    X = torch.empty((n, d), dtype=torch.bfloat16, device=device)
    for s in range(0, n, chunk):
        m = min(n, s + chunk) - s
        z = torch.randint(0, n_dirs, (m,), generator=g, device=device)
        w = torch.empty(m, dtype=torch.float64, device=device)
        todo = torch.arange(m, device=device)
        while todo.numel():
            r = todo.numel()
            a1, a2 = chi2(r), chi2(r)
            zb = a1 / (a1 + a2)
            ww = (1.0 - (1.0 + b) * zb) / (1.0 - (1.0 - b) * zb)
            u = torch.rand(r, generator=g, device=device, dtype=torch.float64)
            ok = kap * ww + (d - 1.0) * torch.log(1.0 - x0 * ww) - c >= torch.log(u)
            w[todo[ok]] = ww[ok]
            todo = todo[~ok]
        mz = mu[z]
        v = torch.randn((m, d), generator=g, device=device)
        v -= (v * mz).sum(1, keepdim=True) * mz
        v /= v.norm(dim=1, keepdim=True)
        x = w[:, None].float() * mz + torch.sqrt(torch.clamp(1.0 - w * w, min=0.0))[:, None].float() * v
        X[s:s + m] = x.to(torch.bfloat16)
    return X


def serving_jobs(count: int = 512, rate: float = 20.0, seed: int = BASE_SEED + 4):
    """Poisson job stream: arrival times, n log-uniform in [1e4, 1e6], d in {64,128,256}, k = n/100."""
    g = _rng(seed)
    t = np.cumsum(g.exponential(1.0 / rate, size=count))
    n = np.floor(10.0 ** g.uniform(4.0, 6.0, size=count)).astype(np.int64)
    d = g.choice(np.array([64, 128, 256]), size=count)
    return [dict(arrival=float(t[i]), n=int(n[i]), d=int(d[i]), k=max(1, int(n[i]) // 100), kappa=20,
                 seed=int(seed * 1000 + i)) for i in range(count)]
