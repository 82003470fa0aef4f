"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module holds no arithmetic of the method: it only turns (seed, index) into
numbers.  The generator is SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based stream:
the value at index i is the SplitMix64 output for the state seed + (i+1)*gamma,
with gamma = 0x9E3779B97F4A7C15.  A double in [-1, 1) is 2*u - 1 with
u = (z >> 11) * 2^-53.

Indices are canonical (logical, row-major over the tensor's logical axes), so a
tensor stored in any storage order holds the same logical values.

Two implementations are provided: numpy on the host, and torch integer ops on
any device (used to fill multi-GB inputs directly in device memory).  A CPU
test checks that they agree bit for bit.
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
MIX1 = 0xBF58476D1CE4E5B9
MIX2 = 0x94D049BB133111EB
MASK64 = (1 << 64) - 1

# Per-workload seeds: small update chain, size sweep, contraction,
# uneven batch, cost-model request stream.
SEED_CHAIN_SMALL = 0xC1A1
SEED_CHAIN_SWEEP = 0xC1A2
SEED_LTIMES = 0xC1A3
SEED_UNEVEN = 0xC1A4
SEED_REQUESTS = 0xC1A5
SEED_MASS = 0xC1A6

# Sub-stream offsets so that different quantities drawn from one workload seed
# never share indices.
STREAM_A = 0
STREAM_N = 1 << 40
STREAM_T = 2 << 40
STREAM_L = 3 << 40
STREAM_MISC = 4 << 40


def splitmix64_scalar(seed: int, idx: int) -> int:
    """Python-int reference of one draw (used by tests and tiny cases)."""
    z = (seed + (idx + 1) * GAMMA) & MASK64
    z = ((z ^ (z >> 30)) * MIX1) & MASK64
    z = ((z ^ (z >> 27)) * MIX2) & MASK64
    return z ^ (z >> 31)


def _splitmix64_np(seed: int, idx: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = np.uint64(seed & MASK64) + (idx.astype(np.uint64) + np.uint64(1)) * np.uint64(GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(MIX1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(MIX2)
        return z ^ (z >> np.uint64(31))


def uniform_np(seed: int, start: int, count: int, chunk: int = 1 << 22) -> np.ndarray:
    """count doubles in [-1, 1) for indices start .. start+count-1."""
    out = np.empty(count, dtype=np.float64)
    scale = 2.0 ** -53
    for s in range(0, count, chunk):
        e = min(count, s + chunk)
        z = _splitmix64_np(seed, np.arange(start + s, start + e, dtype=np.uint64))
        u = (z >> np.uint64(11)).astype(np.float64) * scale
        out[s:e] = 2.0 * u - 1.0
    return out


def unit_np(seed: int, start: int, count: int) -> np.ndarray:
    """count doubles in [0, 1) (the u above) for indices start .. start+count-1."""
    z = _splitmix64_np(seed, np.arange(start, start + count, dtype=np.uint64))
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


# ---- torch variant (device-side fill) --------------------------------------

def _to_i64(v: int) -> int:
    v &= MASK64
    return v - (1 << 64) if v >= (1 << 63) else v


def _lsr(z, k: int):
    # logical shift right of int64 bit patterns
    import torch
    return torch.bitwise_and(torch.bitwise_right_shift(z, k), (1 << (64 - k)) - 1)


def uniform_torch(seed: int, start: int, count: int, device, chunk: int = 1 << 24):
    """Same values as uniform_np, computed with torch int64 ops on `device`."""
    import torch
    out = torch.empty(count, dtype=torch.float64, device=device)
    g = _to_i64(GAMMA)
    m1 = _to_i64(MIX1)
    m2 = _to_i64(MIX2)
    sd = _to_i64(seed)
    scale = 2.0 ** -53
    for s in range(0, count, chunk):
        e = min(count, s + chunk)
        i = torch.arange(start + s + 1, start + e + 1, dtype=torch.int64, device=device)
        z = i * g + sd
        z = torch.bitwise_xor(z, _lsr(z, 30)) * m1
        z = torch.bitwise_xor(z, _lsr(z, 27)) * m2
        z = torch.bitwise_xor(z, _lsr(z, 31))
        u = _lsr(z, 11).to(torch.float64) * scale
        out[s:e] = 2.0 * u - 1.0
    return out


# ---- workload recipes ------------------------------------------------------

def chain_batch(n: int) -> int:
    """Instances per size in the FP64 size sweep: floor(2^27 / N^2)."""
    return (1 << 27) // (n * n)


def chain_inputs_np(seed: int, batch: int, n: int, layout: int = 0) -> np.ndarray:
    """A[b][i][j] uniform in [-1,1), canonical index b*N*N + i*N + j.

    layout 0 stores each instance row-major, layout 1 column-major; the
    returned array is the physical buffer, shape (batch, n, n).
    """
    a = uniform_np(seed, STREAM_A, batch * n * n).reshape(batch, n, n)
    if layout == 1:
        a = np.ascontiguousarray(a.transpose(0, 2, 1))
    return a


def chain_inputs_torch(seed: int, batch: int, n: int, device, layout: int = 0):
    a = uniform_torch(seed, STREAM_A, batch * n * n, device).view(batch, n, n)
    if layout == 1:
        a = a.transpose(1, 2).contiguous()
    return a


def uneven_sizes(seed: int, count: int, n_lo: int = 2, n_hi: int = 64,
                 t_lo: int = 16, t_hi: int = 128):
    """Per-instance (N, T) for the uneven batch.

    N is a log-uniform integer in [n_lo, n_hi]: floor(exp(U[ln n_lo, ln(n_hi+1))))
    clipped to n_hi; T is uniform in [t_lo, t_hi]: t_lo + floor(u*(t_hi-t_lo+1)).
    """
    un = unit_np(seed, STREAM_N, count)
    ut = unit_np(seed, STREAM_T, count)
    lo, hi = math.log(n_lo), math.log(n_hi + 1)
    n = np.minimum(n_hi, np.floor(np.exp(lo + un * (hi - lo)))).astype(np.int64)
    n = np.maximum(n, n_lo)
    t = (t_lo + np.floor(ut * (t_hi - t_lo + 1))).astype(np.int64)
    t = np.minimum(t, t_hi)
    return n, t


def uneven_inputs_np(seed: int, n: np.ndarray, offsets: np.ndarray | None = None) -> tuple[np.ndarray, np.ndarray]:
    """Pool of all instances' A, row-major, instance k at offsets[k].

    Instance k's entries use canonical indices offsets[k] + i*N_k + j in the
    A stream, so the pool is one contiguous draw.
    """
    sizes = (n.astype(np.int64) ** 2)
    if offsets is None:
        offsets = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
    total = int(offsets[-1] + sizes[-1]) if len(n) else 0
    pool = uniform_np(seed, STREAM_A, total)
    return pool, offsets


# Storage orders of a three-index tensor, slowest -> fastest, over the logical
# axes (0=d or m, 1=g, 2=z).  Enumeration: DGZ, DZG, GDZ, GZD, ZDG, ZGD.
LAYOUT_NAMES = ("DGZ", "DZG", "GDZ", "GZD", "ZDG", "ZGD")
LAYOUT_PERMS = ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0))


def to_layout(canon: np.ndarray, layout: int) -> np.ndarray:
    """Physical buffer of a canonical [x][g][z] array stored in `layout`."""
    return np.ascontiguousarray(canon.transpose(LAYOUT_PERMS[layout]))


def from_layout(phys: np.ndarray, layout: int, shape) -> np.ndarray:
    """Canonical [x][g][z] view of a physical buffer stored in `layout`."""
    perm = LAYOUT_PERMS[layout]
    pshape = tuple(shape[p] for p in perm)
    inv = np.argsort(perm)
    return phys.reshape(pshape).transpose(inv)


def ltimes_inputs_np(seed: int, m: int, d: int, g: int, z: int):
    """L[m][d] and canonical in[d][g][z], both uniform in [-1,1)."""
    L = uniform_np(seed, STREAM_L, m * d).reshape(m, d)
    x = uniform_np(seed, STREAM_A, d * g * z).reshape(d, g, z)
    return L, x


def mass_basis(D: int, Q: int) -> np.ndarray:
    """B1[q][d]: the Lagrange polynomials on D equally spaced nodes of [-1, 1]
    evaluated at the Q Gauss-Legendre points (a finite element's 1-D basis at
    its quadrature points; D = 1 is the constant)."""
    xq, _ = np.polynomial.legendre.leggauss(Q)
    nodes = np.linspace(-1.0, 1.0, D) if D > 1 else np.zeros(1)
    B = np.ones((Q, D))
    for d in range(D):
        for m in range(D):
            if m != d:
                B[:, d] *= (xq - nodes[m]) / (nodes[d] - nodes[m])
    return B


def mass_inputs_np(seed: int, dim: int, D: int, Q: int, ne: int):
    """(B1, op, x) of the mass operator over ne elements: op (quadrature data,
    density x |J| x weight) uniform in [0.5, 1.5), x uniform in [-1, 1), both
    [ne][...] with the first index fastest; canonical element-major indices."""
    B1 = mass_basis(D, Q)
    op = 1.0 + 0.5 * uniform_np(seed, STREAM_L, ne * Q ** dim).reshape(ne, Q ** dim)
    x = uniform_np(seed, STREAM_A, ne * D ** dim).reshape(ne, D ** dim)
    return B1, op, x


def mass_inputs_torch(seed: int, dim: int, D: int, Q: int, ne: int, device):
    """The same values as mass_inputs_np, drawn on the device."""
    B1 = mass_basis(D, Q)
    op = 1.0 + 0.5 * uniform_torch(seed, STREAM_L, ne * Q ** dim, device).view(ne, Q ** dim)
    x = uniform_torch(seed, STREAM_A, ne * D ** dim, device).view(ne, D ** dim)
    return B1, op, x
