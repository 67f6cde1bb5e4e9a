"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle's callers.

This module holds no arithmetic of the QS-PIC method.  It builds the initial beam
macroparticles of a workload:

* a quiet lattice of ppc_x * ppc_y * ppc_xi sub-positions per (x, y, xi) cell;
* "random macroparticle weights" (the QuaSSis paragraph of the paper) as a Gaussian relative
  perturbation of std noise_rel, optionally times seeded transverse density modes;
* Gaussian thermal u_x, u_y and a Gaussian relative spread of gamma.

Random numbers come from Philox-4x32-10 (Salmon, Moraes, Dror and Shaw, "Parallel random
numbers: as easy as 1, 2, 3", SC'11), keyed by the run seed and counted by
(particle id, species), and turned into normals by the Box-Muller transform.  The CUDA
initialiser implements the same generator from the same published definition, so that large
runs can be built on the device while small runs are built here and passed to both sides.

Particle id order (also the device order): id = ((k_xi * ny + iy) * nx + ix) * ppc + sub,
sub = (s_xi * ppc_y + s_y) * ppc_x + s_x.
"""
from __future__ import annotations

import math

import numpy as np

PHILOX_M0 = np.uint64(0xD2511F53)
PHILOX_M1 = np.uint64(0xCD9E8D57)
PHILOX_W0 = np.uint32(0x9E3779B9)
PHILOX_W1 = np.uint32(0xBB67AE85)
_MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox-4x32 with 10 rounds on uint32 arrays (counter c0..c3, key k0, k1)."""
    c0 = np.asarray(c0, dtype=np.uint32).copy()
    c1 = np.asarray(c1, dtype=np.uint32).copy()
    c2 = np.asarray(c2, dtype=np.uint32).copy()
    c3 = np.asarray(c3, dtype=np.uint32).copy()
    k0 = np.uint32(k0)
    k1 = np.uint32(k1)
    with np.errstate(over="ignore"):
        for _ in range(10):
            p0 = PHILOX_M0 * c0.astype(np.uint64)
            p1 = PHILOX_M1 * c2.astype(np.uint64)
            hi0 = (p0 >> np.uint64(32)).astype(np.uint32)
            lo0 = (p0 & _MASK32).astype(np.uint32)
            hi1 = (p1 >> np.uint64(32)).astype(np.uint32)
            lo1 = (p1 & _MASK32).astype(np.uint32)
            c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
            k0 = np.uint32(k0 + PHILOX_W0)
            k1 = np.uint32(k1 + PHILOX_W1)
    return c0, c1, c2, c3


def u01(r):
    """uint32 -> uniform in (0, 1): (r + 1/2) / 2^32."""
    return (r.astype(np.float64) + 0.5) * (1.0 / 4294967296.0)


def normals4(ids, species_index, seed):
    """Four standard normals per particle id (two Box-Muller pairs of one Philox call)."""
    ids = np.asarray(ids, dtype=np.uint64)
    c0 = (ids & _MASK32).astype(np.uint32)
    c1 = (ids >> np.uint64(32)).astype(np.uint32)
    c2 = np.full(ids.shape, species_index, dtype=np.uint32)
    c3 = np.zeros(ids.shape, dtype=np.uint32)
    seed = int(seed)
    r0, r1, r2, r3 = philox4x32_10(c0, c1, c2, c3, seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    a = np.sqrt(-2.0 * np.log(u01(r0)))
    b = np.sqrt(-2.0 * np.log(u01(r2)))
    t1 = 2.0 * math.pi * u01(r1)
    t3 = 2.0 * math.pi * u01(r3)
    return a * np.cos(t1), a * np.sin(t1), b * np.cos(t3), b * np.sin(t3)


def beam_extent(p, s):
    """First xi cell and number of xi cells of species s."""
    back = p.Lxi if s.xi_back < 0 else s.xi_back
    k0 = int(round(s.xi_front / p.dxi))
    k1 = int(round(back / p.dxi))
    return k0, max(k1 - k0, 0)


def beam_count(p, si):
    s = p.species[si]
    _, nk = beam_extent(p, s)
    return p.nx * p.ny * nk * s.ppc_x * s.ppc_y * s.ppc_xi


def beam_arrays(p, si, id_lo=0, id_hi=None):
    """Initial beam macroparticles of species si for ids in [id_lo, id_hi), as a dict of fp64
    arrays x, y, xi, ux, uy, uz, w (absolute positions in the box)."""
    s = p.species[si]
    k0, nk = beam_extent(p, s)
    ppc = s.ppc_x * s.ppc_y * s.ppc_xi
    n = p.nx * p.ny * nk * ppc
    if id_hi is None:
        id_hi = n
    ids = np.arange(id_lo, id_hi, dtype=np.int64)
    sub = ids % ppc
    cell = ids // ppc
    ix = cell % p.nx
    iy = (cell // p.nx) % p.ny
    kx = cell // (p.nx * p.ny) + k0
    sx = sub % s.ppc_x
    sy = (sub // s.ppc_x) % s.ppc_y
    sxi = sub // (s.ppc_x * s.ppc_y)
    x = (ix + (sx + 0.5) / s.ppc_x) * p.dx
    y = (iy + (sy + 0.5) / s.ppc_y) * p.dy
    xi = (kx + (sxi + 0.5) / s.ppc_xi) * p.dxi
    n0, n1, n2, n3 = normals4(ids, si, p.seed)
    w = np.full(ids.shape, s.alpha * p.dx * p.dy * p.dxi / ppc)
    w = w * (1.0 + s.noise_rel * n0)
    if s.seeded and p.modes:
        mod = np.ones(ids.shape)
        for m in p.modes:
            kxm = 2 * math.pi * m.mx / p.Lx
            kym = 2 * math.pi * m.my / p.Ly
            mod = mod + m.amplitude * np.cos(kxm * x + kym * y + m.phase)
        w = w * mod
    ux = s.uperp_spread * n1
    uy = s.uperp_spread * n2
    gam = s.gamma_b * (1.0 + s.gamma_spread_rel * n3)
    uz = np.sqrt(gam * gam - 1.0 - ux * ux - uy * uy)
    return dict(x=x, y=y, xi=xi, ux=ux, uy=uy, uz=uz, w=w)


def all_beams(p):
    return [beam_arrays(p, si) for si in range(len(p.species))]
