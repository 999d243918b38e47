"""Seeded synthetic inputs shared by the CUDA path, the tests and the CPU oracle.

This module holds no arithmetic of the solver: it only draws random numbers
and lays them out.  Everything is counter-based so any slice of a stream can
be produced without generating what precedes it.

Generator: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014).  The n-th output (n = 0, 1, ...) of the
stream with seed s is ``mix(s + (n + 1) * GAMMA)`` where ``mix`` is the
published 64-bit finaliser.

Derived draws:
  * uniform[-1, 1): ``(z >> 40) * 2**-23 - 1`` -- 24 significant bits, so the
    value is exact in float32 and float64 alike (both sides see one number).
  * standard normal: Box-Muller on two 53-bit uniforms in (0, 1].
  * choice among m items: ``((z >> 40) * m) >> 24``.

Workloads (the problem statements of the solver's configurations):
  * ``uniform_rhs(n, seed, offset)``: right-hand side b, i.i.d. uniform[-1,1).
  * ``lognormal_blocks(nbx, nby, nbz, seed)``: k = exp(Z), Z ~ N(0, 1), one
    value per 8^3 block, row-major block order (bx fastest).  Stream draws
    0 .. 2*nblocks-1 (two per block for Box-Muller).
  * ``batch_shapes(nprob, seed, sizes)``: per-axis sizes drawn uniformly from
    ``sizes``; three draws per problem in (nx, ny, nz) order.
  * ``unet_init_weights(seed, layers)``: initial weights of the learned
    preconditioner's convolutions, He-style normals (std sqrt(2 / (27 ci)),
    halved for the last layer), one stream per layer (seed * 1000 + index).
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_CHUNK = 1 << 22


def splitmix64(seed: int, offset: int, count: int) -> np.ndarray:
    """Outputs ``offset .. offset+count-1`` of the SplitMix64 stream ``seed``."""
    if count < 0 or offset < 0:
        raise ValueError("offset and count must be non-negative")
    with np.errstate(over="ignore"):
        n = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + n * GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform_pm1(seed: int, offset: int, count: int, dtype=np.float32) -> np.ndarray:
    """``count`` i.i.d. uniform[-1, 1) values, exact in float32; chunked."""
    out = np.empty(count, dtype=dtype)
    for s in range(0, count, _CHUNK):
        c = min(_CHUNK, count - s)
        z = splitmix64(seed, offset + s, c)
        m = (z >> np.uint64(40)).astype(np.float64)
        out[s:s + c] = (m * (2.0 ** -23) - 1.0).astype(dtype)
    return out


def uniform_rhs(shape, seed: int, offset: int = 0, dtype=np.float32) -> np.ndarray:
    """Right-hand side on a grid of ``shape`` = (nz, ny, nx), x fastest."""
    n = int(np.prod(shape))
    return uniform_pm1(seed, offset, n, dtype).reshape(shape)


def standard_normal(seed: int, offset: int, count: int) -> np.ndarray:
    """Box-Muller normals; draw ``offset+2i`` and ``offset+2i+1`` feed value i."""
    z = splitmix64(seed, offset, 2 * count).reshape(count, 2)
    u = ((z >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)  # (0, 1]
    return np.sqrt(-2.0 * np.log(u[:, 0])) * np.cos(2.0 * np.pi * u[:, 1])


def lognormal_blocks(nbx: int, nby: int, nbz: int, seed: int) -> np.ndarray:
    """k = exp(N(0,1)) per block, float32, shape (nbz, nby, nbx)."""
    nb = nbx * nby * nbz
    return np.exp(standard_normal(seed, 0, nb)).astype(np.float32).reshape(nbz, nby, nbx)


def choice(seed: int, offset: int, count: int, items) -> np.ndarray:
    z = splitmix64(seed, offset, count)
    idx = ((z >> np.uint64(40)) * np.uint64(len(items))) >> np.uint64(24)
    return np.asarray(items)[idx.astype(np.int64)]


def batch_shapes(nprob: int, seed: int, sizes=(48, 64, 96, 128, 160)):
    """List of (nx, ny, nz) for ``nprob`` problems."""
    v = choice(seed, 0, 3 * nprob, sizes).reshape(nprob, 3)
    return [tuple(int(a) for a in row) for row in v]


def batch_rhs(shapes, seed: int, dtype=np.float32):
    """RHS of each batched problem; drawn from ``seed`` after the shape draws."""
    off = 3 * len(shapes)
    out = []
    for (nx, ny, nz) in shapes:
        n = nx * ny * nz
        out.append(uniform_pm1(seed, off, n, dtype).reshape(nz, ny, nx))
        off += n
    return out


def block_counts(nx: int, ny: int, nz: int, kb: int = 8):
    """Number of coefficient blocks per axis for block edge ``kb``."""
    return (-(-nx // kb), -(-ny // kb), -(-nz // kb))


# Named workloads -----------------------------------------------------------

def poisson_problem(n: int, seed: int = 0, dtype=np.float32):
    """Constant-coefficient Poisson, n^3 interior points, b ~ U[-1,1) seed."""
    return uniform_rhs((n, n, n), seed, 0, dtype)


def varcoeff_problem(nx: int, ny: int, nz: int, seed: int = 1, kb: int = 8, dtype=np.float32):
    """Lognormal block coefficient then RHS from the same stream after it."""
    nbx, nby, nbz = block_counts(nx, ny, nz, kb)
    k = lognormal_blocks(nbx, nby, nbz, seed)
    b = uniform_rhs((nz, ny, nx), seed, 2 * k.size, dtype)
    return k, b


def unet_init_weights(seed: int, layers) -> dict:
    """{name: (co, 27, ci) float64} for layers [(name, ci, co), ...]; the last layer's std is halved."""
    ws = {}
    for li, (name, ci, co) in enumerate(layers):
        n = co * 27 * ci
        std = np.sqrt(2.0 / (27 * ci)) * (0.5 if li == len(layers) - 1 else 1.0)
        ws[name] = standard_normal(seed * 1000 + li, 0, n).reshape(co, 27, ci) * std
    return ws
