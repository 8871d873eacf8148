"""Isometry-grown Hubbard superblocks at any kept-state count m.

Real DMRG superblocks at m = 1000 need a full DMRG run to produce.  This
generator builds superblocks with the same structure much faster: blocks are
grown one site at a time exactly as in the infinite algorithm (paper Sec. 3.1
and Sec. 3.3: S' = S (x) X_step, E' = Y_step (x) E, every local operator
re-expressed in the product basis, the block Hamiltonian plus the connection
to the added site), but once a block holds more than m states it is projected
with a seeded random isometry W (W^T W = 1) that preserves the quantum numbers
instead of the density-matrix eigenvectors of Eq. (rhoSystem).  The number of
states kept per (N_up, N_dn) sector follows a product of binomial weights
centred on the mean filling, which gives the uneven sector sizes of a real
run.  Because W^T W = 1, the result is an exact Rayleigh-Ritz projection of
the lattice Hamiltonian: Hermitian, with the right sector shifts and fermion
signs, and variational.

Everything here is input generation: block-sparse bookkeeping and Kronecker
products of site operators.  No superblock product and no eigensolver is in
this module.

Conventions (shared with the oracle's own, independent model code):
* Hubbard site basis {e, up, dn, updn}, |updn> = c^dag_up c^dag_dn |e>.
* Jordan-Wigner order by site label; S' holds the lower labels, so a
  fermion operator of E' picks up the parity F_S' of S' (the reading of the
  paper's silent fermion sign).
* H = -t sum_<ij>,sigma (c^dag_i c_j + h.c.) + U sum_i n_up n_dn.
  Coupling classes: ``t`` (every hopping, unit block = -sum(...)) and ``U``.
* Ladder site label i = 2*x + leg (rung-major), one site added per step.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Dict, List, Tuple

import numpy as np

from .superblock import Pair, Superblock, transition

# --------------------------------------------------------------------- site
_E, _UP, _DN, _UD = 0, 1, 2, 3
SITE_QN = [(0, 0), (1, 0), (0, 1), (1, 1)]  # (n_up, n_dn) of e, up, dn, updn


def _site_ops() -> Dict[str, np.ndarray]:
    cu = np.zeros((4, 4))
    cu[_E, _UP] = 1.0
    cu[_DN, _UD] = 1.0
    cd = np.zeros((4, 4))
    cd[_E, _DN] = 1.0
    cd[_UP, _UD] = -1.0
    return dict(c_up=cu, c_dn=cd, F=np.diag([1.0, -1.0, -1.0, 1.0]),
                nn=np.diag([0.0, 0.0, 0.0, 1.0]), I=np.eye(4))


SITE = _site_ops()
SPIN_SHIFT = {"up": (1, 0), "dn": (0, 1)}

Sector = Tuple[int, int]


# -------------------------------------------------------- block-sparse ops
@dataclass
class Basis:
    sectors: List[Sector]           # sorted by q = n_up + Q*n_dn
    dims: List[int]

    def index(self) -> Dict[Sector, int]:
        return {z: i for i, z in enumerate(self.sectors)}


# an operator is {(z_out, z_in): dense block}
Op = Dict[Tuple[Sector, Sector], np.ndarray]


def _dag(op: Op) -> Op:
    return {(zi, zo): b.T.copy() for (zo, zi), b in op.items()}


def _parity(z: Sector) -> float:
    return -1.0 if (z[0] + z[1]) % 2 else 1.0


def _times_F_right(op: Op) -> Op:
    return {(zo, zi): b * _parity(zi) for (zo, zi), b in op.items()}


def _times_F_left(op: Op) -> Op:
    return {(zo, zi): b * _parity(zo) for (zo, zi), b in op.items()}


def _identity(basis: Basis) -> Op:
    return {(z, z): np.eye(d) for z, d in zip(basis.sectors, basis.dims)}


def _F(basis: Basis) -> Op:
    return {(z, z): _parity(z) * np.eye(d) for z, d in zip(basis.sectors, basis.dims)}


@dataclass
class Product:
    """Basis of block (x) site.  Sector z of the product is the concatenation,
    over site states t in order e, up, dn, updn, of the block sector z - qn(t)."""
    basis: Basis
    comps: Dict[Sector, List[Tuple[int, Sector, int]]]  # z -> [(t, block sector, offset)]


def _product_basis(block: Basis, Q: int) -> Product:
    comps: Dict[Sector, List[Tuple[int, Sector, int]]] = {}
    dims_b = dict(zip(block.sectors, block.dims))
    new = set()
    for z in block.sectors:
        for t in range(4):
            new.add((z[0] + SITE_QN[t][0], z[1] + SITE_QN[t][1]))
    order = sorted(new, key=lambda z: (z[0] + Q * z[1]))
    dims = []
    for zn in order:
        off = 0
        lst = []
        for t in range(4):
            za = (zn[0] - SITE_QN[t][0], zn[1] - SITE_QN[t][1])
            if za in dims_b:
                lst.append((t, za, off))
                off += dims_b[za]
        comps[zn] = lst
        dims.append(off)
    return Product(Basis(order, dims), comps)


def _kron(prod: Product, op_block: Op, op_site: np.ndarray) -> Op:
    """<a,t| O_block (x) o_site |a',t'> = O[a,a'] o[t,t'] in the product basis."""
    out: Op = {}
    dims = dict(zip(prod.basis.sectors, prod.basis.dims))
    by_in: Dict[Sector, List] = {}
    for (ao, ai), blk in op_block.items():
        by_in.setdefault(ai, []).append((ao, blk))
    offs = {(z, t): o for z, lst in prod.comps.items() for (t, a, o) in lst}
    for zi, ci in prod.comps.items():
        for (t_in, a_in, off_in) in ci:
            for t_out in range(4):
                v = op_site[t_out, t_in]
                if v == 0.0:
                    continue
                for ao, blk in by_in.get(a_in, ()):
                    zo = (ao[0] + SITE_QN[t_out][0], ao[1] + SITE_QN[t_out][1])
                    off_out = offs.get((zo, t_out))
                    if off_out is None:
                        continue
                    key = (zo, zi)
                    if key not in out:
                        out[key] = np.zeros((dims[zo], dims[zi]))
                    out[key][off_out:off_out + blk.shape[0],
                             off_in:off_in + blk.shape[1]] += v * blk
    return out


def _add(a: Op, b: Op, scale: float = 1.0) -> Op:
    out = {k: v.copy() for k, v in a.items()}
    for k, v in b.items():
        if k in out:
            out[k] = out[k] + scale * v
        else:
            out[k] = scale * v
    return out


def _project(op: Op, W: Dict[Sector, np.ndarray]) -> Op:
    out: Op = {}
    for (zo, zi), b in op.items():
        if zo in W and zi in W:
            out[(zo, zi)] = W[zo].T @ b @ W[zi]
    return out


# ------------------------------------------------------------ the blocks
@dataclass
class Block:
    sites: List[int]
    basis: Basis
    H: Dict[str, Op]                       # coupling class -> block Hamiltonian
    c: Dict[Tuple[int, str], Op] = field(default_factory=dict)  # (site, spin) -> c


def _site_block(site: int, Q: int) -> Block:
    order = sorted(range(4), key=lambda t: SITE_QN[t][0] + Q * SITE_QN[t][1])
    sectors = [SITE_QN[t] for t in order]
    basis = Basis(sectors, [1] * 4)
    def to_op(m):
        op: Op = {}
        for to in range(4):
            for ti in range(4):
                if m[to, ti] != 0.0:
                    op[(SITE_QN[to], SITE_QN[ti])] = np.array([[m[to, ti]]])
        return op
    H = {"t": {}, "U": to_op(SITE["nn"])}
    for z in sectors:
        H["t"][(z, z)] = np.zeros((1, 1))
        H["U"].setdefault((z, z), np.zeros((1, 1)))
    c = {(site, "up"): to_op(SITE["c_up"]), (site, "dn"): to_op(SITE["c_dn"])}
    return Block([site], basis, H, c)


def _allocate(avail: Dict[Sector, int], weight: Dict[Sector, float], m: int) -> Dict[Sector, int]:
    """Split m kept states over sectors in proportion to weight, capped by the
    available count (water filling + largest remainder, ties by sector)."""
    total = sum(avail.values())
    if total <= m:
        return dict(avail)
    keys = sorted(avail, key=lambda z: (z[1], z[0]))
    capped: Dict[Sector, int] = {}
    while True:
        free = [z for z in keys if z not in capped]
        budget = m - sum(capped.values())
        wsum = sum(weight[z] for z in free)
        ideal = {z: budget * weight[z] / wsum if wsum > 0 else 0.0 for z in free}
        newcap = [z for z in free if ideal[z] >= avail[z]]
        if not newcap:
            break
        for z in newcap:
            capped[z] = avail[z]
    out = dict(capped)
    fl = {z: int(np.floor(ideal[z])) for z in free}
    out.update(fl)
    rem = m - sum(out.values())
    frac = sorted(free, key=lambda z: (-(ideal[z] - fl[z]), z[1], z[0]))
    for z in frac[:rem]:
        out[z] += 1
    return {z: k for z, k in out.items() if k > 0}


def _binom_logpmf(k: int, n: int, p: float) -> float:
    from math import lgamma, log
    if k < 0 or k > n:
        return -np.inf
    return (lgamma(n + 1) - lgamma(k + 1) - lgamma(n - k + 1)
            + k * log(p) + (n - k) * log(1 - p))


def _grow(block: Block, site: int, bonds_to_site, Q: int, left: bool) -> Tuple[Block, Product]:
    """S' = S (x) site (left=False, site has the highest label) or
    E' = site (x) E (left=True, site has the lowest label).  In both cases the
    product basis is written block (x) site; only the Jordan-Wigner factor
    differs: for S' the new site's c gets F_S, for E' the old sites' c get
    F_site."""
    prod = _product_basis(block.basis, Q)
    I_b = _identity(block.basis)
    F_b = _F(block.basis)
    H = {}
    for cls, h in block.H.items():
        H[cls] = _kron(prod, h, SITE["I"])
    H["U"] = _add(H["U"], _kron(prod, I_b, SITE["nn"]))
    c_new: Dict[Tuple[int, str], Op] = {}
    for spin, cs in (("up", SITE["c_up"]), ("dn", SITE["c_dn"])):
        if left:
            c_new[(site, spin)] = _kron(prod, I_b, cs)
        else:
            c_new[(site, spin)] = _kron(prod, F_b, cs)
    for (j, spin), op in block.c.items():
        if left:
            c_new[(j, spin)] = _kron(prod, op, SITE["F"])
        else:
            c_new[(j, spin)] = _kron(prod, op, SITE["I"])
    # hopping between the new site and the block sites it bonds to, unit -1
    for j in bonds_to_site:
        for spin in ("up", "dn"):
            ci = c_new[(j, spin)]
            cs = c_new[(site, spin)]
            hop = _mul(_dag(ci), cs)
            H["t"] = _add(H["t"], hop, -1.0)
            H["t"] = _add(H["t"], _dag(hop), -1.0)
    sites = ([site] + block.sites) if left else (block.sites + [site])
    return Block(sites, prod.basis, H, c_new), prod


def _mul(a: Op, b: Op) -> Op:
    out: Op = {}
    bi: Dict[Sector, List] = {}
    for (zo, zi), blk in b.items():
        bi.setdefault(zo, []).append((zi, blk))
    for (zo, zm), ablk in a.items():
        for (zi, bblk) in bi.get(zm, []):
            key = (zo, zi)
            v = ablk @ bblk
            out[key] = out[key] + v if key in out else v
    return out


def _truncate(block: Block, m: int, p: float, keep_sites, rng) -> Block:
    n = len(block.sites)
    avail = dict(zip(block.basis.sectors, block.basis.dims))
    weight = {z: np.exp(_binom_logpmf(z[0], n, p) + _binom_logpmf(z[1], n, p)) for z in avail}
    kept = _allocate(avail, weight, m)
    if sum(kept.values()) == sum(avail.values()):
        W = None
    else:
        W = {}
        for z in block.basis.sectors:
            k = kept.get(z, 0)
            if k == 0:
                continue
            g = rng.standard_normal((avail[z], k))
            qm, rm = np.linalg.qr(g)
            W[z] = qm * np.sign(np.diag(rm))[None, :]
    if W is None:
        c = {key: op for key, op in block.c.items() if key[0] in keep_sites}
        return Block(block.sites, block.basis, block.H, c)
    sectors = [z for z in block.basis.sectors if z in W]
    basis = Basis(sectors, [W[z].shape[1] for z in sectors])
    H = {cls: _project(h, W) for cls, h in block.H.items()}
    c = {key: _project(op, W) for key, op in block.c.items() if key[0] in keep_sites}
    return Block(block.sites, basis, H, c)


# --------------------------------------------------------------- geometry
def ladder_bonds(n_sites: int):
    """Nearest-neighbour bonds (i < j) of a two-leg ladder with site label
    2*x + leg: rungs (2x, 2x+1) and legs (i, i+2)."""
    bonds = []
    for i in range(n_sites):
        if i % 2 == 0 and i + 1 < n_sites:
            bonds.append((i, i + 1))
        if i + 2 < n_sites:
            bonds.append((i, i + 2))
    return bonds


def chain_bonds(n_sites: int):
    return [(i, i + 1) for i in range(n_sites - 1)]


def _grown_blocks(n_sites, geometry, n_up, n_dn, m, cut, seed):
    """S' = sites [0, cut) and E' = sites [cut, n_sites), grown site by site and
    projected to at most m states per step with the (n_up, n_dn) weights."""
    bonds = ladder_bonds(n_sites) if geometry == "ladder" else chain_bonds(n_sites)
    if cut is None:
        cut = n_sites // 2 + (1 if geometry == "ladder" and (n_sites // 2) % 2 == 0 else 0)
    reach = 2 if geometry == "ladder" else 1
    Q = n_sites + 1
    p_up, p_dn = n_up / n_sites, n_dn / n_sites
    p = 0.5 * (p_up + p_dn)
    rng = np.random.default_rng(seed)

    # system: sites 0 .. cut-1, the last one added without truncation
    S = _site_block(0, Q)
    for x in range(1, cut):
        S = _truncate(S, m, p, set(range(x - reach, x)), rng)
        nb = [i for (i, j) in bonds if j == x and i < x]
        S, _ = _grow(S, x, nb, Q, left=False)
    S.c = {k: v for k, v in S.c.items() if k[0] >= cut - reach}
    # environment: sites n_sites-1 .. cut, grown to the left
    E = _site_block(n_sites - 1, Q)
    for y in range(n_sites - 2, cut - 1, -1):
        E = _truncate(E, m, p, set(range(y + 1, y + 1 + reach)), rng)
        nb = [j for (i, j) in bonds if i == y and j > y]
        E, _ = _grow(E, y, nb, Q, left=True)
    E.c = {k: v for k, v in E.c.items() if k[0] < cut + reach}
    return S, E, bonds, cut


def _target_sectors(S, E, n_up, n_dn):
    """S' sectors of the (n_up, n_dn) target with both sides present, and the
    dimensions (r from S', c from the partner sector of E')."""
    e_idx = E.basis.index()
    dims_e = dict(zip(E.basis.sectors, E.basis.dims))
    sec_S, r, c = [], [], []
    for z, d in zip(S.basis.sectors, S.basis.dims):
        ze = (n_up - z[0], n_dn - z[1])
        if ze in e_idx and d > 0 and dims_e[ze] > 0:
            sec_S.append(z)
            r.append(d)
            c.append(dims_e[ze])
    return sec_S, r, c


def _assemble(S, E, bonds, cut, n_up, n_dn, t, U_values, meta) -> Superblock:
    sec_S, r, c = _target_sectors(S, E, n_up, n_dn)
    sidx = {z: i for i, z in enumerate(sec_S)}
    partner = lambda z: (n_up - z[0], n_dn - z[1])

    names, tclass, tmult = [], [], []
    pairs: List[Pair] = []

    def add_term(name, cls, mult, A: Op | None, B: Op | None):
        k = len(names)
        names.append(name)
        tclass.append(cls)
        tmult.append(mult)
        for z_in in sec_S:
            if A is None:
                outs = [z_in]
            else:
                outs = [zo for (zo, zi) in A if zi == z_in]
            for z_out in outs:
                if z_out not in sidx:
                    continue
                a = None if A is None else A[(z_out, z_in)]
                if B is None:
                    if z_out != z_in:
                        continue
                    b = None
                else:
                    key = (partner(z_out), partner(z_in))
                    if key not in B:
                        continue
                    b = B[key]
                if (a is not None and not np.any(a)) or (b is not None and not np.any(b)):
                    continue
                pairs.append(Pair(k, sidx[z_out], sidx[z_in],
                                  None if a is None else np.ascontiguousarray(a),
                                  None if b is None else np.ascontiguousarray(b)))

    for cls in ("t", "U"):
        add_term(f"H_S'[{cls}] x 1", cls, 1.0, S.H[cls], None)
    for cls in ("t", "U"):
        add_term(f"1 x H_E'[{cls}]", cls, 1.0, None, E.H[cls])
    cross = [(i, j) for (i, j) in bonds if i < cut <= j]
    for (i, j) in cross:
        for spin in ("up", "dn"):
            ci = S.c[(i, spin)]
            cj = E.c[(j, spin)]
            # c^dag_i c_j = (c_i^dag F_S') (x) c_j ;  c^dag_j c_i = (F_S' c_i) (x) c_j^dag
            add_term(f"c+_{i}{spin} c_{j}{spin}", "t", -1.0, _times_F_right(_dag(ci)), cj)
            add_term(f"c+_{j}{spin} c_{i}{spin}", "t", -1.0, _times_F_left(ci), _dag(cj))

    classes = ["t", "U"]
    U_values = np.atleast_1d(np.asarray(U_values, dtype=np.float64))
    couplings = np.stack([np.full_like(U_values, t), U_values], axis=1)
    term_class = np.array([classes.index(cl) for cl in tclass])
    term_mult = np.array(tmult)
    coeffs = couplings[:, term_class] * term_mult[None, :]
    sb = Superblock(np.array(r), np.array(c), coeffs, pairs, names, classes,
                    term_class, term_mult, couplings,
                    q_labels=np.array(sec_S, dtype=np.int64))
    sb.meta.update(meta, n_up=n_up, n_dn=n_dn,
                   dim_S=int(sum(S.basis.dims)), dim_E=int(sum(E.basis.dims)))
    return sb


def grown_hubbard_superblock(n_sites: int = 64, geometry: str = "ladder",
                             n_up: int = 28, n_dn: int = 28, m: int = 1000,
                             cut: int | None = None, t: float = 1.0,
                             U_values=(8.0,), seed: int = 0) -> Superblock:
    """Superblock S' = sites [0, cut), E' = sites [cut, n_sites) of the Hubbard
    model, both blocks grown site by site and projected to at most m states
    per step, in the (n_up, n_dn) target sector.  One batch member per U."""
    S, E, bonds, cut = _grown_blocks(n_sites, geometry, n_up, n_dn, m, cut, seed)
    return _assemble(S, E, bonds, cut, n_up, n_dn, t, U_values,
                     dict(kind="grown_hubbard", geometry=geometry, n_sites=n_sites, m=m, cut=cut, seed=seed))


def grown_ldos_inputs(n_sites: int = 64, geometry: str = "ladder", n_up: int = 28, n_dn: int = 28,
                      m: int = 1000, cut: int | None = None, t: float = 1.0, U_values=(8.0,),
                      seed: int = 0, spin: str = "up"):
    """One growth of S', E' (as grown_hubbard_superblock) and, on those
    blocks, the superblocks of the (n_up, n_dn) target and of one particle
    of `spin` less and more, with the transition containers of c (x) 1 and
    c^dag (x) 1 for the last site of S' (block-local operator, Jordan-Wigner
    string inside S'; E' holds the higher labels).  Returns
    {"N": sb, "hole": (sb, trans), "particle": (sb, trans), "site": i}."""
    S, E, bonds, cut = _grown_blocks(n_sites, geometry, n_up, n_dn, m, cut, seed)
    meta = dict(kind="grown_hubbard", geometry=geometry, n_sites=n_sites, m=m, cut=cut, seed=seed)
    site = cut - 1
    d = (1, 0) if spin == "up" else (0, 1)
    batch = len(np.atleast_1d(U_values))
    out = {"N": _assemble(S, E, bonds, cut, n_up, n_dn, t, U_values, meta), "site": site}
    sec_in, r_in, c_in = _target_sectors(S, E, n_up, n_dn)
    c_op = S.c[(site, spin)]
    for part, sgn, op in (("hole", -1, c_op), ("particle", +1, _dag(c_op))):
        nu, nd = n_up + sgn * d[0], n_dn + sgn * d[1]
        sb = _assemble(S, E, bonds, cut, nu, nd, t, U_values, meta)
        sec_out, r_out, c_out = _target_sectors(S, E, nu, nd)
        iin = {z: k for k, z in enumerate(sec_in)}
        blocks = []
        for so, zo in enumerate(sec_out):
            zi = (zo[0] - sgn * d[0], zo[1] - sgn * d[1])
            if zi in iin and (zo, zi) in op and np.any(op[(zo, zi)]):
                si = iin[zi]
                blocks.append((so, si, op[(zo, zi)], np.eye(c_out[so])))
        tr = transition(r_out, c_out, r_in, c_in, blocks, batch=batch,
                        name=("c" if sgn < 0 else "c+") + f"_{site}{spin}")
        out[part] = (sb, tr)
    return out


def ladder_m1000(batch: int = 16, seed: int = 0) -> Superblock:
    """2 x 32 Hubbard ladder, t_leg = t_rung = 1, N_up = N_dn = 28 (1/8 hole
    doping), m = 1000, cut through a rung (three crossing bonds), one batch
    member per U = 4 + 8 i / 15."""
    Us = 4.0 + 8.0 * np.arange(batch) / max(batch - 1, 1)
    return grown_hubbard_superblock(64, "ladder", 28, 28, 1000, cut=33,
                                    U_values=Us, seed=seed)


def ladder_m1000_ldos(batch: int = 16, seed: int = 0, spin: str = "up"):
    """ladder_m1000 (the same growth, the same "N" superblock) with the N - 1
    and N + 1 superblocks and the c (x) 1, c^dag (x) 1 transitions of the last
    system site (grown_ldos_inputs)."""
    Us = 4.0 + 8.0 * np.arange(batch) / max(batch - 1, 1)
    return grown_ldos_inputs(64, "ladder", 28, 28, 1000, cut=33, U_values=Us, seed=seed, spin=spin)
