"""Plain container for one sector-blocked superblock Hamiltonian, plus npz I/O.

This module holds data only; it does no Hamiltonian arithmetic.  It is the
common input format of the CPU oracle (``oracle/``) and of the GPU library
binding, so both consume exactly the same operator blocks.

Meaning of the container (paper Sec. 3.3, the three tasks of the
``x += H y`` product, and Sec. 3.2 for the symmetry sectors):

* The superblock is S' (x) E'.  Its basis is blocked by the effective quantum
  number q of S'; sector ``s`` pairs the S' states with q_S(s) and the E'
  states with Q_target - q_S(s).  ``r[s]`` and ``c[s]`` are the two dimensions.
* The wavefunction is the concatenation of the row-major blocks Psi_s
  (``r[s] x c[s]``) at ``offsets()[s]``; D = sum_s r[s]*c[s].
* ``H = sum_k coeffs[k] * A_k (x) B_k``.  Each (term, sector pair) with a
  nonzero block is one :class:`Pair`; its action is
  ``Y[s_out] += coeffs[term] * A @ Psi[s_in] @ B.T``,
  with ``A`` of shape ``(r[s_out], r[s_in])`` and ``B`` of shape
  ``(c[s_out], c[s_in])``.  ``A is None`` (or ``B is None``) means the
  identity on that side, which is how H_S' (x) 1 and 1 (x) H_E' enter.
* ``coeffs`` has shape ``(batch, n_terms)``: ``batch`` superblocks that share
  every block and differ only in their coefficients (coupling sweeps).
* Coupling classes: ``coeffs[b, k] = term_mult[k] * couplings[b, term_class[k]]``
  when the superblock was built from a model, so that dE/d(coupling) is a
  chain-rule sum of dE/dc_k.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np


@dataclass
class Pair:
    term: int
    s_out: int
    s_in: int
    A: Optional[np.ndarray]  # (r[s_out], r[s_in]) float64, None = identity
    B: Optional[np.ndarray]  # (c[s_out], c[s_in]) float64, None = identity


@dataclass
class Superblock:
    r: np.ndarray
    c: np.ndarray
    coeffs: np.ndarray
    pairs: List[Pair]
    term_names: List[str] = field(default_factory=list)
    class_names: List[str] = field(default_factory=list)
    term_class: Optional[np.ndarray] = None
    term_mult: Optional[np.ndarray] = None
    couplings: Optional[np.ndarray] = None
    q_labels: Optional[np.ndarray] = None
    meta: dict = field(default_factory=dict)

    def __post_init__(self):
        self.r = np.asarray(self.r, dtype=np.int64)
        self.c = np.asarray(self.c, dtype=np.int64)
        self.coeffs = np.atleast_2d(np.asarray(self.coeffs, dtype=np.float64))

    @property
    def n_sectors(self) -> int:
        return int(self.r.shape[0])

    @property
    def n_terms(self) -> int:
        return int(self.coeffs.shape[1])

    @property
    def batch(self) -> int:
        return int(self.coeffs.shape[0])

    @property
    def dim(self) -> int:
        return int(np.sum(self.r * self.c))

    def offsets(self) -> np.ndarray:
        off = np.zeros(self.n_sectors + 1, dtype=np.int64)
        off[1:] = np.cumsum(self.r * self.c)
        return off

    def with_coeffs(self, coeffs) -> "Superblock":
        """Same blocks, new coefficient table (shape (batch, n_terms))."""
        return Superblock(self.r, self.c, np.atleast_2d(coeffs), self.pairs,
                          self.term_names, self.class_names, self.term_class,
                          self.term_mult, None, self.q_labels, dict(self.meta))

    def coeffs_from_couplings(self, couplings) -> np.ndarray:
        """c_k = term_mult[k] * g[term_class[k]] for a (batch, n_classes) table."""
        g = np.atleast_2d(np.asarray(couplings, dtype=np.float64))
        return g[:, self.term_class] * self.term_mult[None, :]

    def validate(self) -> None:
        S = self.n_sectors
        for i, p in enumerate(self.pairs):
            if not (0 <= p.term < self.n_terms):
                raise ValueError(f"pair {i}: term {p.term} out of range")
            if not (0 <= p.s_out < S and 0 <= p.s_in < S):
                raise ValueError(f"pair {i}: sector out of range")
            if p.A is None and p.B is None:
                raise ValueError(f"pair {i}: both sides identity")
            if p.A is None and self.r[p.s_out] != self.r[p.s_in]:
                raise ValueError(f"pair {i}: identity A needs r_out == r_in")
            if p.B is None and self.c[p.s_out] != self.c[p.s_in]:
                raise ValueError(f"pair {i}: identity B needs c_out == c_in")
            if p.A is not None and p.A.shape != (self.r[p.s_out], self.r[p.s_in]):
                raise ValueError(f"pair {i}: A shape {p.A.shape}")
            if p.B is not None and p.B.shape != (self.c[p.s_out], self.c[p.s_in]):
                raise ValueError(f"pair {i}: B shape {p.B.shape}")

    # ------------------------------------------------------------------ I/O
    def save(self, path: str) -> None:
        arrays = dict(r=self.r, c=self.c, coeffs=self.coeffs)
        meta = np.array([[p.term, p.s_out, p.s_in, p.A is not None, p.B is not None]
                         for p in self.pairs], dtype=np.int64).reshape(-1, 5)
        arrays["pair_meta"] = meta
        for i, p in enumerate(self.pairs):
            if p.A is not None:
                arrays[f"A{i}"] = p.A
            if p.B is not None:
                arrays[f"B{i}"] = p.B
        if self.term_class is not None:
            arrays["term_class"] = self.term_class
            arrays["term_mult"] = self.term_mult
        if self.couplings is not None:
            arrays["couplings"] = self.couplings
        if self.q_labels is not None:
            arrays["q_labels"] = self.q_labels
        arrays["term_names"] = np.array(self.term_names, dtype=object)
        arrays["class_names"] = np.array(self.class_names, dtype=object)
        np.savez_compressed(path, **arrays)

    @staticmethod
    def load(path: str) -> "Superblock":
        z = np.load(path, allow_pickle=True)
        pairs = []
        for i, (t, so, si, ha, hb) in enumerate(z["pair_meta"]):
            pairs.append(Pair(int(t), int(so), int(si),
                              z[f"A{i}"] if ha else None,
                              z[f"B{i}"] if hb else None))
        get = lambda k: z[k] if k in z.files else None
        return Superblock(z["r"], z["c"], z["coeffs"], pairs,
                          list(z["term_names"]), list(z["class_names"]),
                          get("term_class"), get("term_mult"), get("couplings"),
                          get("q_labels"))


def transition(r_out, c_out, r_in, c_in, blocks, batch: int = 1, name: str = "O") -> Superblock:
    """An operator between two target spaces as one container: sectors of the
    output space first, then those of the input space; one term (coefficient
    1 for every member) whose pairs are ``blocks`` = [(s_out, s_in, A, B)]
    with s_out, s_in counted in their own spaces.  Applying it to
    [0 (output space), psi] gives [O psi, 0].  An identity side must be given
    explicitly (the sectors differ)."""
    r_out, c_out = np.asarray(r_out, dtype=np.int64), np.asarray(c_out, dtype=np.int64)
    n_out = len(r_out)
    pairs = [Pair(0, int(so), n_out + int(si), np.ascontiguousarray(A, dtype=np.float64),
                  np.ascontiguousarray(B, dtype=np.float64)) for (so, si, A, B) in blocks]
    sb = Superblock(np.concatenate([r_out, np.asarray(r_in, dtype=np.int64)]),
                    np.concatenate([c_out, np.asarray(c_in, dtype=np.int64)]),
                    np.ones((batch, 1)), pairs, [name])
    sb.meta.update(kind="transition", n_out=n_out, dim_out=int(np.sum(r_out * c_out)))
    return sb


def seeded_normal(seed: int, shape) -> np.ndarray:
    """N(0,1) float64 draws from numpy's PCG64 stream ``seed``.

    Used for Lanczos start vectors and for wavefunction inputs; both the
    oracle and the GPU path receive the same array.
    """
    return np.random.default_rng(seed).standard_normal(shape)
