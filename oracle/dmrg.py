"""Infinite and finite DMRG driver that produces superblocks (oracle).

Follows paper Sec. 1 and Sec. 3.1 (Fig. infiniteloop): S = {0}, E = {L-1},
X_step = {step+1}, Y_step = {L-2-step}; each step grows S' = S (x) X_step
(site to the right) and E' = Y_step (x) E (site to the left), forms the
superblock, finds its ground state with Lanczos, builds the density matrices
rho_S = Psi Psi^T and rho_E = Psi^T Psi (Eqs. rhoSystem, rhoEnviron), keeps
the m eigenvectors of largest eigenvalue, and changes basis with
H <- W^T H W (Eq. transformation; W^T W = 1).  Operators are kept for the
boundary sites only; the block Hamiltonian itself is carried (Sec. 3.3: the
product of transformed operators is not the transformed product).  The
truncation error is eps = sum of discarded eigenvalues (Sec. 2).

Readings where the paper is silent (see the design notes): one-site blocks;
eigenvalues of rho sorted globally in decreasing order, values within tie_tol
(1e-12; rho has trace 1) of their neighbour counted as equal and ordered by
(q, index within the sector), exactly m kept; infinite-phase target N = round(density * L_k) rounded to even with
N_up = N_dn = N/2 for Hubbard and N_up = L_k/2 for Heisenberg; the finite
algorithm (Sec. 2, "not discussed here, see code") is the standard sweep at
fixed L, one sweep = a left-to-right plus a right-to-left pass, starting and
ending at the middle.

Blocks store their sites by distance from their own outer end (left blocks:
position p; right blocks: distance j from the right end), so the same block
serves the infinite phase, where the lattice grows, and the finite phase.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, Dict, List, Optional, Tuple

import numpy as np

from workloads.superblock import Superblock, seeded_normal

from . import lanczos as olz
from . import models
from . import superblock as osb


# ------------------------------------------------------------------ model
@dataclass
class Model:
    kind: str                    # "heisenberg" or "hubbard"
    geometry: Callable[[int], list]  # L -> [(i, j, class)] with i < j
    couplings: Dict[str, float]  # class -> value (hopping classes, 'U', or J classes)
    reach: int                   # longest bond length in site labels
    Q: int = 0                   # base of the effective quantum number
    density: float = 1.0

    def site(self):
        return models.heisenberg_site() if self.kind == "heisenberg" else models.hubbard_site()

    def site_q(self):
        s = self.site()
        if self.kind == "heisenberg":
            return s["n_up"].astype(np.int64)
        return (s["n_up"] + self.Q * s["n_dn"]).astype(np.int64)

    def site_N(self):
        s = self.site()
        return (s["n_up"] + s["n_dn"]).astype(np.int64)

    def target(self, L_k):
        if self.kind == "heisenberg":
            return L_k // 2
        N = int(round(self.density * L_k))
        N -= N % 2
        return N // 2 + self.Q * (N // 2)

    def classes(self):
        return list(self.couplings)


def heisenberg_chain(J1=1.0, J2=0.0, Lmax=64):
    if J2 == 0.0:
        return Model("heisenberg", lambda L: [(i, i + 1, "J1") for i in range(L - 1)],
                     {"J1": J1}, 1, Q=Lmax + 1)
    return Model("heisenberg",
                 lambda L: [(i, i + 1, "J1") for i in range(L - 1)] +
                           [(i, i + 2, "J2") for i in range(L - 2)],
                 {"J1": J1, "J2": J2}, 2, Q=Lmax + 1)


def hubbard_chain(t=1.0, U=4.0, density=1.0, Lmax=64):
    return Model("hubbard", lambda L: [(i, i + 1, "t") for i in range(L - 1)],
                 {"t": t, "U": U}, 1, Q=Lmax + 1, density=density)


def hubbard_ladder(t_leg=1.0, t_rung=1.0, U=8.0, density=1.0, Lmax=64):
    def geom(L):
        return [(i, j, "t_leg" if cls == "leg" else "t_rung")
                for (i, j, cls) in models.ladder_bonds(L)]
    return Model("hubbard", geom, {"t_leg": t_leg, "t_rung": t_rung, "U": U}, 2,
                 Q=Lmax + 1, density=density)


# ------------------------------------------------------------------ block
@dataclass
class DBlock:
    n: int                              # number of sites
    q: np.ndarray                       # effective quantum number per state
    N: np.ndarray                       # particle number per state (parity)
    H: Dict[str, np.ndarray]            # class -> unit-coupling part
    ops: Dict[Tuple[int, str], np.ndarray] = field(default_factory=dict)  # (end distance, name)

    @property
    def dim(self):
        return len(self.q)

    def F(self):
        return np.diag((-1.0) ** self.N)


def site_block(model: Model) -> DBlock:
    s = model.site()
    d = s["d"]
    H = {cls: np.zeros((d, d)) for cls in model.classes()}
    if model.kind == "hubbard":
        H["U"] = s["nn"].copy()
        ops = {(0, "c_up"): s["c_up"], (0, "c_dn"): s["c_dn"]}
    else:
        ops = {(0, "Sz"): s["Sz"], (0, "Sp"): s["Sp"]}
    b = DBlock(1, model.site_q(), model.site_N(), H, ops)
    return _sorted(b)


def _sorted(b: DBlock) -> DBlock:
    """Symmetry ordering (Sec. 3.2): stable sort of the basis by q."""
    P = np.argsort(b.q, kind="stable")
    return DBlock(b.n, b.q[P], b.N[P], {k: v[np.ix_(P, P)] for k, v in b.H.items()},
                  {k: v[np.ix_(P, P)] for k, v in b.ops.items()})


def _bond_h(model: Model, oi: Dict[str, np.ndarray], oj: Dict[str, np.ndarray]):
    """Unit-coupling bond Hamiltonian from block-space operators of sites i < j
    (Jordan-Wigner strings already inside the fermion operators)."""
    if model.kind == "heisenberg":
        return oi["Sz"] @ oj["Sz"] + 0.5 * (oi["Sp"] @ oj["Sp"].T + oi["Sp"].T @ oj["Sp"])
    h = 0
    for spin in ("up", "dn"):
        ci, cj = oi["c_" + spin], oj["c_" + spin]
        hop = ci.T @ cj
        h = h - (hop + hop.T)
    return h


def _ops_of(b: DBlock, key: int):
    return {name: M for (k, name), M in b.ops.items() if k == key}


def grow(model: Model, b: DBlock, side: str) -> DBlock:
    """S' = S (x) site (side 'left' block grows to the right) or
    E' = site (x) E (side 'right' block grows to the left), in the product
    basis, then symmetry ordered.  Old sites keep their end distance; the new
    site gets end distance b.n (for a right block counted from the right end)."""
    s = model.site()
    d = s["d"]
    I_b = np.eye(b.dim)
    I_s = np.eye(d)
    fermion = model.kind == "hubbard"
    new = b.n
    if side == "left":
        q = (b.q[:, None] + model.site_q()[None, :]).ravel()
        N = (b.N[:, None] + model.site_N()[None, :]).ravel()
        H = {cls: np.kron(h, I_s) for cls, h in b.H.items()}
        if fermion:
            H["U"] = H["U"] + np.kron(I_b, s["nn"])
        ops = {k: np.kron(M, I_s) for k, M in b.ops.items()}
        for name in (("c_up", "c_dn") if fermion else ("Sz", "Sp")):
            ops[(new, name)] = np.kron(b.F() if fermion else I_b, s[name])
    else:
        q = (model.site_q()[:, None] + b.q[None, :]).ravel()
        N = (model.site_N()[:, None] + b.N[None, :]).ravel()
        H = {cls: np.kron(I_s, h) for cls, h in b.H.items()}
        if fermion:
            H["U"] = H["U"] + np.kron(s["nn"], I_b)
        ops = {k: np.kron(s["F"] if fermion else I_s, M) for k, M in b.ops.items()}
        for name in (("c_up", "c_dn") if fermion else ("Sz", "Sp")):
            ops[(new, name)] = np.kron(s[name], I_b)
    nb = DBlock(b.n + 1, q, N, H, ops)
    # bonds between the new site and the old ones: in end-distance terms the
    # geometry is mirror symmetric, so use the left-anchored lattice of n+1 sites
    for (i, j, cls) in model.geometry(b.n + 1):
        if j == new and i < new:
            oi = _ops_of(nb, i)
            oj = _ops_of(nb, new)
            if side == "left":
                nb.H[cls] = nb.H[cls] + _bond_h(model, oi, oj)
            else:
                # right block: end distance new is the leftmost (lowest label)
                nb.H[cls] = nb.H[cls] + _bond_h(model, oj, oi)
    return _sorted(nb)


def superblock_terms(model: Model, Sp: DBlock, Ep: DBlock, L_k: int):
    """Kronecker terms of H_super = H_S' (x) 1 + 1 (x) H_E' + connection,
    with coupling classes.  Returns (terms [(A|None, B|None)], names,
    class per term, multiplier per term)."""
    terms, names, tcls, tmult = [], [], [], []
    for cls in model.classes():
        terms.append((Sp.H[cls], None)); names.append(f"H_S'[{cls}]"); tcls.append(cls); tmult.append(1.0)
    for cls in model.classes():
        terms.append((None, Ep.H[cls])); names.append(f"H_E'[{cls}]"); tcls.append(cls); tmult.append(1.0)
    nS = Sp.n
    FS = Sp.F()
    for (i, j, cls) in model.geometry(L_k):
        if not (i < nS <= j):
            continue
        jd = L_k - 1 - j  # end distance inside E'
        oi = _ops_of(Sp, i)
        oj = _ops_of(Ep, jd)
        if model.kind == "heisenberg":
            terms += [(oi["Sz"], oj["Sz"]), (oi["Sp"], oj["Sp"].T), (oi["Sp"].T, oj["Sp"])]
            names += [f"Sz{i}Sz{j}", f"S+{i}S-{j}", f"S-{i}S+{j}"]
            tcls += [cls] * 3
            tmult += [1.0, 0.5, 0.5]
        else:
            for spin in ("up", "dn"):
                ci, cj = oi["c_" + spin], oj["c_" + spin]
                # c^dag_i c_j = (c_i^dag F_S') (x) c_j ; c^dag_j c_i = (F_S' c_i) (x) c_j^dag
                terms += [(ci.T @ FS, cj), (FS @ ci, cj.T)]
                names += [f"c+{i}{spin}c{j}", f"c+{j}{spin}c{i}"]
                tcls += [cls, cls]
                tmult += [-1.0, -1.0]
    return terms, names, tcls, tmult


def make_superblock(model: Model, Sp: DBlock, Ep: DBlock, L_k: int,
                    couplings_batch=None) -> Tuple[Superblock, list]:
    terms, names, tcls, tmult = superblock_terms(model, Sp, Ep, L_k)
    classes = model.classes()
    if couplings_batch is None:
        couplings_batch = [[model.couplings[c] for c in classes]]
    g = np.atleast_2d(np.asarray(couplings_batch, dtype=np.float64))
    tci = np.array([classes.index(c) for c in tcls])
    tm = np.array(tmult)
    coeffs = g[:, tci] * tm[None, :]
    sb = osb.superblock_from_full(Sp.q, Ep.q, model.target(L_k), terms, coeffs[0], names)
    sb.coeffs = coeffs
    sb.class_names = classes
    sb.term_class = tci
    sb.term_mult = tm
    sb.couplings = g
    sb.meta.update(L=L_k, nS=Sp.n, nE=Ep.n, dim_S=Sp.dim, dim_E=Ep.dim)
    return sb, terms


def _truncate(b: DBlock, rho_blocks, m: int, keep_keys, tie_tol: float = 1e-12):
    """Keep the m eigenvectors of the block-diagonal rho with the largest
    eigenvalues, then H <- W^T H W.  Ties: eigenvalues within tie_tol of
    their neighbour in decreasing order count as equal (one cluster), and a
    cluster is taken in the order (q, index within the sector).  Returns
    (block, discarded weight, gap at the cut: the m-th kept value minus the
    first discarded one, 0 when nothing is cut)."""
    cand = []  # (-lambda, q, index, sector indices, vector)
    for q in sorted(set(b.q.tolist())):
        idx = np.nonzero(b.q == q)[0]
        R = rho_blocks.get(q)
        if R is None:
            w = np.zeros(len(idx))
            V = np.eye(len(idx))
        else:
            w, V = np.linalg.eigh(R)
            w, V = w[::-1], V[:, ::-1]
        for a in range(len(idx)):
            cand.append((-w[a], q, a, idx, V[:, a]))
    cand.sort(key=lambda t: (t[0], t[1], t[2]))
    # clusters of equal eigenvalues (equal up to rounding): a new cluster
    # starts where the value drops by more than tie_tol from its predecessor
    clustered, cl = [], 0
    for i, t in enumerate(cand):
        if i > 0 and (-cand[i - 1][0]) - (-t[0]) > tie_tol:
            cl += 1
        clustered.append((cl, t))
    clustered.sort(key=lambda ct: (ct[0], ct[1][1], ct[1][2]))
    cand = [t for _, t in clustered]
    total = sum(-t[0] for t in cand)
    if m >= len(cand):
        keep = cand
        gap = 0.0
    else:
        keep = cand[:m]
        gap = float(-cand[m - 1][0] - (-cand[m][0]))
    eps = max(0.0, total - sum(-t[0] for t in keep))
    keep.sort(key=lambda t: (t[1], t[2]))  # new basis in q order
    W = np.zeros((b.dim, len(keep)))
    for col, (_, q, a, idx, v) in enumerate(keep):
        W[idx, col] = v
    qn = np.array([t[1] for t in keep], dtype=np.int64)
    Nn = np.array([b.N[t[3][0]] for t in keep], dtype=np.int64)
    H = {k: W.T @ h @ W for k, h in b.H.items()}
    ops = {k: W.T @ M @ W for k, M in b.ops.items() if k[0] in keep_keys}
    return DBlock(b.n, qn, Nn, H, ops), eps, gap


def _rho(sb: Superblock, psi, side):
    off = sb.offsets()
    out = {}
    for s in range(sb.n_sectors):
        P = psi[off[s]:off[s + 1]].reshape(sb.r[s], sb.c[s])
        out[s] = P @ P.T if side == "S" else P.T @ P
    return out


@dataclass
class StepResult:
    L: int
    nS: int
    energy: float
    eps_S: float
    eps_E: float
    iters: int
    superblock: Optional[Superblock] = None
    psi: Optional[np.ndarray] = None
    blocks: Optional[tuple] = None  # (S', E') of the step, with keep_superblocks
    gap_S: float = 0.0  # lambda_m - lambda_{m+1} at the cut of each truncated side (0: nothing cut)
    gap_E: float = 0.0


def _solve(model, Sp, Ep, L_k, seed, tol, max_iter, keep_sb):
    sb, _ = make_superblock(model, Sp, Ep, L_k)
    v0 = seeded_normal(seed, sb.dim)
    res = olz.lanczos_ground(lambda v: osb.apply_H(sb, v), v0, tol=tol, max_iter=max_iter)
    return sb, res


def _rho_by_q(sb, psi, blockS: DBlock, blockE: DBlock, Q_t):
    """rho blocks keyed by the block's own q (S side: q_S; E side: Q_t - q_S)."""
    rS = _rho(sb, psi, "S")
    rE = _rho(sb, psi, "E")
    qs = sb.q_labels
    return ({int(qs[s]): rS[s] for s in rS}, {int(Q_t - qs[s]): rE[s] for s in rE})


def infinite_dmrg(model: Model, L: int, m: int, seed: int = 0, tol: float = 1e-12,
                  max_iter: int = 300, keep_superblocks: bool = False, tie_tol: float = 1e-12):
    """Returns (steps, left_blocks, right_blocks); left_blocks[n] is the
    truncated block of the n leftmost sites (n = 1 .. L/2 - 1 plus the
    final untruncated halves are not stored)."""
    S = site_block(model)
    E = site_block(model)
    left = {1: S}
    right = {1: E}
    steps = []
    for step in range(L // 2 - 1):
        Sp = grow(model, S, "left")
        Ep = grow(model, E, "right")
        L_k = Sp.n + Ep.n
        sb, res = _solve(model, Sp, Ep, L_k, seed + step, tol, max_iter, keep_superblocks)
        Q_t = model.target(L_k)
        rS, rE = _rho_by_q(sb, res.psi, Sp, Ep, Q_t)
        keep = set(range(Sp.n - model.reach, Sp.n))
        S, eS, gS = _truncate(Sp, rS, m, keep, tie_tol)
        E, eE, gE = _truncate(Ep, rE, m, keep, tie_tol)
        left[S.n] = S
        right[E.n] = E
        steps.append(StepResult(L_k, Sp.n, res.e0, eS, eE, res.iters,
                                sb if keep_superblocks else None,
                                res.psi if keep_superblocks else None,
                                (Sp, Ep) if keep_superblocks else None, gS, gE))
    return steps, left, right


def finite_dmrg(model: Model, L: int, m: int, n_sweeps: int = 2, seed: int = 0,
                tol: float = 1e-12, max_iter: int = 300, keep_superblocks: bool = False,
                m_infinite: Optional[int] = None, tie_tol: float = 1e-12):
    """Infinite phase to L sites, then n_sweeps sweeps at fixed L.  A step at
    split l has S' = sites [0, l), E' = sites [l, L); S' = left[l-1] (x) site,
    E' = site (x) right[L-l-1]."""
    steps, left, right = infinite_dmrg(model, L, m if m_infinite is None else m_infinite,
                                       seed, tol, max_iter, keep_superblocks, tie_tol)
    out = list(steps)
    half = L // 2
    path = []
    for _ in range(n_sweeps):
        path += [(l, "right") for l in range(half + 1, L - 1)]   # grow S to the right end
        path += [(l, "left") for l in range(L - 2, 1, -1)]       # then E to the left end
        path += [(l, "right") for l in range(2, half + 1)]       # back to the middle
    for k, (l, direction) in enumerate(path):
        Sp = grow(model, left[l - 1], "left")
        Ep = grow(model, right[L - l - 1], "right")
        sb, res = _solve(model, Sp, Ep, L, seed + 1000 + k, tol, max_iter, keep_superblocks)
        Q_t = model.target(L)
        rS, rE = _rho_by_q(sb, res.psi, Sp, Ep, Q_t)
        if direction == "right":
            keepS = set(range(Sp.n - model.reach, Sp.n))
            left[Sp.n], eS, gS = _truncate(Sp, rS, m, keepS, tie_tol)
            eE, gE = 0.0, 0.0
        else:
            keepE = set(range(Ep.n - model.reach, Ep.n))
            right[Ep.n], eE, gE = _truncate(Ep, rE, m, keepE, tie_tol)
            eS, gS = 0.0, 0.0
        out.append(StepResult(L, Sp.n, res.e0, eS, eE, res.iters,
                              sb if keep_superblocks else None,
                              res.psi if keep_superblocks else None, None, gS, gE))
    return out
