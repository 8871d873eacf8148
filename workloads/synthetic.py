"""Seeded random sector-blocked superblocks (no physics, matvec workloads).

``random_sectored`` draws ``n_sectors`` sectors with dimensions uniform in
``[dmin, dmax]`` and Kronecker terms that shift the sector index by a fixed
delta (the way an operator such as c^dagger shifts a quantum number, paper
Sec. 3.2).  Blocks are dense N(0, 1/d_inner): the variance is 1/(inner
dimension) of the product they enter, so A @ Psi @ B.T stays O(1).

The 64-sector, 16..512, 12-term instance is the synthetic batched-matvec
workload (4 terms each with delta 0, +1, -1; pairs off either end dropped,
which gives 4*64 + 8*63 = 760 pairs).
"""
from __future__ import annotations

import numpy as np

from .superblock import Pair, Superblock


def random_sectored(seed: int = 0, n_sectors: int = 64, dmin: int = 16,
                    dmax: int = 512, deltas=(0, 0, 0, 0, 1, 1, 1, 1, -1, -1, -1, -1),
                    batch: int = 1, identity_terms: bool = False,
                    coeff_scale: float = 1.0) -> Superblock:
    rng = np.random.default_rng(seed)
    r = rng.integers(dmin, dmax + 1, size=n_sectors)
    c = rng.integers(dmin, dmax + 1, size=n_sectors)
    pairs = []
    names = []
    n_terms = len(deltas)
    for k, dl in enumerate(deltas):
        names.append(f"rand{k}_d{dl:+d}")
        for s_in in range(n_sectors):
            s_out = s_in + dl
            if not (0 <= s_out < n_sectors):
                continue
            A = rng.standard_normal((r[s_out], r[s_in])) / np.sqrt(r[s_in])
            B = rng.standard_normal((c[s_out], c[s_in])) / np.sqrt(c[s_in])
            pairs.append(Pair(k, s_out, s_in, A, B))
    if identity_terms:
        # one system-side and one environment-side block-diagonal term
        kS, kE = n_terms, n_terms + 1
        names += ["id_B(system)", "id_A(environment)"]
        n_terms += 2
        for s in range(n_sectors):
            HS = rng.standard_normal((r[s], r[s])) / np.sqrt(r[s])
            HE = rng.standard_normal((c[s], c[s])) / np.sqrt(c[s])
            pairs.append(Pair(kS, s, s, HS + HS.T, None))
            pairs.append(Pair(kE, s, s, None, HE + HE.T))
    coeffs = coeff_scale * (1.0 + 0.5 * rng.standard_normal((batch, n_terms)))
    sb = Superblock(r, c, coeffs, pairs, names)
    sb.meta.update(kind="random_sectored", seed=seed)
    return sb


def ragged_small(seed: int = 1, batch: int = 1, tiny: bool = False) -> Superblock:
    """A tiny superblock with every degenerate shape the kernels must handle:
    1x1 blocks, r != c, dims that are not multiples of 4 or 8, an empty
    sector (r = 0), a sector with c = 0, a sector no term writes to, and
    identity terms on both sides."""
    rng = np.random.default_rng(seed)
    r = np.array([1, 3, 7, 0, 13, 33, 5, 2, 130, 17])
    c = np.array([1, 5, 2, 4, 0, 9, 21, 1, 70, 150])
    if tiny:
        r = np.array([1, 3, 7, 0, 13, 9, 5, 2, 30, 17])
        c = np.array([1, 5, 2, 4, 0, 9, 21, 1, 20, 15])
    S = len(r)
    pairs = []
    names = ["d0", "d+1", "d-1", "d+2", "HS", "HE"]
    for k, dl in enumerate([0, 1, -1, 2]):
        for s_in in range(S):
            s_out = s_in + dl
            if not (0 <= s_out < S) or s_out == 6:  # sector 6: no Kronecker term writes it
                continue
            if r[s_out] * c[s_out] == 0 or r[s_in] * c[s_in] == 0:
                continue
            A = rng.standard_normal((r[s_out], r[s_in]))
            B = rng.standard_normal((c[s_out], c[s_in]))
            pairs.append(Pair(k, s_out, s_in, A, B))
    for s in range(S):
        if r[s] * c[s] == 0 or s == 6:
            continue
        HS = rng.standard_normal((r[s], r[s]))
        HE = rng.standard_normal((c[s], c[s]))
        pairs.append(Pair(4, s, s, HS + HS.T, None))
        pairs.append(Pair(5, s, s, None, HE + HE.T))
    coeffs = 1.0 + 0.3 * rng.standard_normal((batch, 6))
    sb = Superblock(r, c, coeffs, pairs, names)
    sb.meta.update(kind="ragged_small", seed=seed)
    return sb
