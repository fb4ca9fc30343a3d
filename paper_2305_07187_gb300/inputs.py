"""Seeded synthetic inputs for the Spring-Ising hot path.

This module only draws numbers: it holds none of the method's arithmetic, so
that the CUDA path and the FP64 oracle can both consume exactly the same
inputs without sharing any computation.  Every generator is a NumPy
``Generator(PCG64(seed))``.

Workload shapes follow the paper's benchmark, K2000 (a complete graph on 2000
vertices, Section "Discussion"): the instance itself is not available, so
seeded complete graphs with +-1 (or Gaussian) couplings stand in for it.
Parameter defaults follow the runs of Fig. 4 / Fig. 5: k = 0.5, Delta = 0.2,
m = 1, zeta ramped from 0.8*zeta0 to 10*zeta0 with zeta0 = 0.05.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

ZETA0 = 0.05
ZETA_START = 0.8 * ZETA0      # 0.04
ZETA_END = 10.0 * ZETA0       # 0.5
DT = 0.2
K_SPRING = 0.5
MASS = 1.0
Q_MAX = math.sqrt(2.0)
P_MAX = 2.0


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def pm1_coupling(n: int, seed: int = 1) -> np.ndarray:
    """Complete graph, J_ij = +-1 iid for i < j, mirrored, zero diagonal (float32)."""
    g = _rng(seed)
    J = np.zeros((n, n), dtype=np.float32)
    iu = np.triu_indices(n, 1)
    J[iu] = g.choice(np.array([-1.0, 1.0], dtype=np.float32), size=iu[0].size)
    J += J.T
    return J


def king_graph_coupling(L: int, seed: int = 5) -> np.ndarray:
    """King graph on an L x L grid with open boundaries (spin index
    i = row * L + col; each spin coupled to its up to 8 neighbours),
    J_ij = +-1 iid on the edges, zero elsewhere (float32, symmetric)."""
    g = _rng(seed)
    n = L * L
    J = np.zeros((n, n), dtype=np.float32)
    rows, cols = [], []
    for r in range(L):
        for c in range(L):
            i = r * L + c
            for dr, dc in ((0, 1), (1, -1), (1, 0), (1, 1)):
                rr, cc = r + dr, c + dc
                if 0 <= rr < L and 0 <= cc < L:
                    rows.append(i)
                    cols.append(rr * L + cc)
    v = g.choice(np.array([-1.0, 1.0], dtype=np.float32), size=len(rows))
    J[rows, cols] = v
    J[cols, rows] = v
    return J


def round_to_bf16(x: np.ndarray) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even), as float32."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).reshape(x.shape)


def gauss_coupling_bf16(n: int, seed: int = 2) -> np.ndarray:
    """Complete graph, J_ij ~ N(0,1) for i < j rounded once to bf16, mirrored."""
    g = _rng(seed)
    J = np.zeros((n, n), dtype=np.float32)
    iu = np.triu_indices(n, 1)
    J[iu] = g.standard_normal(iu[0].size).astype(np.float32)
    J = round_to_bf16(J)
    J = np.triu(J, 1)
    J = J + J.T
    return J


def field(n: int, seed: int = 7, scale: float = 0.5) -> np.ndarray:
    """External field h_i ~ N(0, scale^2) (float32)."""
    return (scale * _rng(seed).standard_normal(n)).astype(np.float32)


def positions(n: int, replicas: int, seed0: int = 100, lo: float = -0.1,
              hi: float = 0.1) -> np.ndarray:
    """Initial positions, replica r ~ U[lo, hi]^n from seed seed0 + r: (R, n) float32."""
    q = np.empty((replicas, n), dtype=np.float32)
    for r in range(replicas):
        q[r] = _rng(seed0 + r).uniform(lo, hi, n).astype(np.float32)
    return q


def zeta_ramp(steps: int, plateau: int = 1, start: float = ZETA_START,
              end: float = ZETA_END) -> np.ndarray:
    """Piecewise-constant linear ramp of the coupling coefficient (float32).

    zeta_n = start + (end - start) * floor(n / L) / (ceil(T / L) - 1), with L
    the plateau length; L = 1 is the pure linear ramp.
    """
    if steps <= 0:
        return np.zeros(0, dtype=np.float32)
    levels = -(-steps // plateau)
    n = np.arange(steps)
    if levels == 1:
        frac = np.zeros(steps)
    else:
        frac = (n // plateau) / (levels - 1)
    return (start + (end - start) * frac).astype(np.float32)


def dt_const(steps: int, dt: float = DT) -> np.ndarray:
    return np.full(steps, dt, dtype=np.float32)


@dataclass
class InstanceSpec:
    index: int
    n: int
    replicas: int
    kind: str          # "pm1" or "gauss"
    seed: int


def uneven_instances(count: int = 256, seed: int = 3000, n_lo: int = 256,
                     n_hi: int = 8192, r_lo: int = 16, r_hi: int = 256):
    """Batch of instances of uneven size: N log-uniform in [n_lo, n_hi],
    R a multiple of 16 drawn log-uniformly in [r_lo, r_hi]; even index +-1
    couplings, odd index Gaussian couplings rounded to bf16."""
    specs = []
    for i in range(count):
        g = _rng(seed + i)
        n = int(round(math.exp(g.uniform(math.log(n_lo), math.log(n_hi)))))
        r = int(16 * round(math.exp(g.uniform(math.log(r_lo), math.log(r_hi))) / 16))
        r = max(16, min(r_hi, r))
        specs.append(InstanceSpec(i, n, r, "pm1" if i % 2 == 0 else "gauss",
                                  seed + 100000 + i))
    return specs


def instance_coupling(spec: InstanceSpec) -> np.ndarray:
    if spec.kind == "pm1":
        return pm1_coupling(spec.n, spec.seed)
    return gauss_coupling_bf16(spec.n, spec.seed)


# ---------------------------------------------------------------- on device
# Seeded generators that draw directly on a CUDA device (torch's Philox
# generator), for workloads whose couplings are too large to draw on the host
# quickly.  Same distributions as the NumPy generators above, different
# streams; tests that check these against the oracle copy the drawn J back.

def pm1_coupling_torch(n: int, seed: int, device="cuda"):
    import torch
    g = torch.Generator(device=device).manual_seed(int(seed))
    u = torch.randint(0, 2, (n, n), generator=g, device=device, dtype=torch.int8)
    J = (2 * u.to(torch.float32) - 1).triu(1)
    return J + J.T


def king_graph_coupling_torch(L: int, seed: int, device="cuda"):
    """King graph as in king_graph_coupling, drawn on the device (torch
    Philox stream, so not the NumPy graph of the same seed)."""
    import torch
    g = torch.Generator(device=device).manual_seed(int(seed))
    n = L * L
    idx = torch.arange(n, device=device)
    r, c = idx // L, idx % L
    J = torch.zeros((n, n), dtype=torch.float32, device=device)
    for dr, dc in ((0, 1), (1, -1), (1, 0), (1, 1)):
        ok = (r + dr < L) & (c + dc >= 0) & (c + dc < L)
        i = idx[ok]
        j = (r[ok] + dr) * L + (c[ok] + dc)
        v = 2 * torch.randint(0, 2, (i.numel(),), generator=g, device=device, dtype=torch.int8).to(torch.float32) - 1
        J[i, j] = v
        J[j, i] = v
    return J


def gauss_coupling_bf16_torch(n: int, seed: int, device="cuda"):
    import torch
    g = torch.Generator(device=device).manual_seed(int(seed))
    J = torch.randn((n, n), generator=g, device=device, dtype=torch.float32)
    J = J.to(torch.bfloat16).to(torch.float32).triu(1)
    return J + J.T


def positions_torch(n: int, replicas: int, seed: int, device="cuda", lo=-0.1, hi=0.1):
    import torch
    g = torch.Generator(device=device).manual_seed(int(seed))
    return (lo + (hi - lo) * torch.rand((replicas, n), generator=g, device=device)).contiguous()


def instance_coupling_torch(spec: InstanceSpec, device="cuda"):
    if spec.kind == "pm1":
        return pm1_coupling_torch(spec.n, spec.seed, device)
    return gauss_coupling_bf16_torch(spec.n, spec.seed, device)
