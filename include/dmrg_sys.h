/*
 * dmrg_sys.h -- C ABI of the DMRG driver around the superblock product:
 * the infinite- and finite-system algorithms with every block operation on
 * the GPU (G. Alvarez, DMRG++ paper, Sec. 3.1 and Fig. infiniteloop).
 *
 * One DMRG step (Sec. 3.1): grow the system S' = S (x) X and the environment
 * E' = Y (x) E by one site, with every kept operator re-expressed in the
 * product basis and the basis ordered by the effective quantum number
 * (Sec. 3.2-3.3: DmrgBasis, DmrgBasisWithOperators, the outer product);
 * form the superblock S' (x) E' of the target sector and find its ground
 * state with the Lanczos solver of dmrg_gb300.h; build the reduced density
 * matrices rho_S = Psi Psi^T and rho_E = Psi^T Psi per symmetry sector
 * (Eqs. rhoSystem, rhoEnviron); keep the m eigenvectors of largest eigenvalue
 * over all sectors; and change the basis of the block Hamiltonian and of the
 * operators still needed, O <- W^T O W (Eq. transformation).  The truncation
 * error is the sum of the discarded eigenvalues.
 *
 * Conventions:
 *  - Blocks carry their sites by distance from their own outer end (the left
 *    block's first site, the right block's last site), so one block serves
 *    the infinite phase, where the lattice grows, and the sweeps at fixed L.
 *  - Fermion signs: Jordan-Wigner order by site label.  Fermionic block
 *    operators carry the string inside their block; a fermionic operator of
 *    E' picks up the parity of S' in the superblock.
 *  - Effective quantum numbers are int64 sums of the site values; a symmetry
 *    sector of a block must have one fermion parity.
 *  - Target of a lattice of L sites: N = round(density * L) rounded down to
 *    even, q = N/2 + Q * N/2 (Hubbard with q = N_up + Q N_dn; with Q = 0 and
 *    density 1, q = L/2 = N_up: S_z = 0 of a spin-1/2 chain).
 *  - Truncation ties: the density-matrix eigenvalues of all sectors are taken
 *    in decreasing order; values within tie_tol of their neighbour form one
 *    cluster, ordered by (sector, index within the sector); exactly m kept.
 *  - Everything runs on the current CUDA device, on the legacy default
 *    stream; the calls synchronise before returning.
 */
#ifndef DMRG_SYS_H
#define DMRG_SYS_H

#include <stdint.h>

#include "dmrg_gb300.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dmrg_sys dmrg_sys;

/* One term of the unit-coupling bond Hamiltonian between sites i < j:
 * coef * op(O_a at i) * op(O_b at j), op = transpose when trans = 1.  Both
 * operators fermionic (the Jordan-Wigner string between them is implied) or
 * both not. */
typedef struct {
  double coef;
  int32_t op_a, trans_a, op_b, trans_b;
} dmrg_bond_term;

/* A model (paper Sec. 4.1, Hubbard and Heisenberg): site basis, the site
 * operators kept at block boundaries, on-site terms, the lattice as bond
 * rules, and the bond Hamiltonian.  Every pointer is host memory, read by
 * dmrg_sys_create and not kept. */
typedef struct {
  int32_t d;                  /* site dimension */
  const int64_t* site_q;      /* [d] effective quantum number of each site state */
  const int32_t* site_parity; /* [d] fermion parity (0 or 1) of each site state */
  int32_t n_ops;              /* site operators (e.g. S^z, S^+ or c_up, c_dn) */
  const double* ops;          /* [n_ops][d][d] row-major, <t|O|t'> */
  const int32_t* op_fermion;  /* [n_ops] 1 for a fermionic (parity-odd) operator */
  int32_t n_classes;          /* coupling classes (J1, J2 or t, U ...) */
  const double* couplings;    /* [n_classes] */
  int32_t n_onsite;           /* on-site terms */
  const int32_t* onsite_class;/* [n_onsite] */
  const double* onsite;       /* [n_onsite][d][d] */
  int32_t n_bond_rules;       /* bonds (p, p + delta) of a class, for every p with p % mod == rem */
  const int32_t* bond_rules;  /* [n_bond_rules][4]: delta (>= 1), class, mod (>= 1), rem */
  int32_t n_bond_terms;
  const dmrg_bond_term* bond_terms; /* [n_bond_terms] */
  double density;             /* particles per site of the target */
  int64_t Q;                  /* base of the effective quantum number (q = N_up + Q N_dn) */
} dmrg_model_desc;

typedef struct {
  double tol;         /* Lanczos residual tolerance of every step (after refinement for a mixed precision) */
  int32_t max_iter;   /* Lanczos cap per step */
  int32_t prec;       /* dmrg_prec of the products */
  int32_t refine;     /* refinement mode of dmrg_lanczos_opts when prec is a tensor-core precision */
  int32_t guess;      /* 0: start every step from a random vector; 1: finite steps start from the
                         previous step's ground state carried to the new basis (wavefunction
                         transformation) */
  double mixed_tol;   /* tolerance of the mixed-precision Lanczos before refinement */
  double tie_tol;     /* truncation tie tolerance (eigenvalues of rho, trace 1) */
  uint64_t seed;      /* random start vectors: uniform(-1, 1) from splitmix64 of (seed, step, index) */
} dmrg_sys_opts;

typedef struct {      /* one per DMRG step */
  int32_t L;          /* lattice size of the step */
  int32_t n_sys;      /* sites of S' */
  int32_t direction;  /* 0 infinite (both blocks truncated), 1 sweep to the right (S' truncated), -1 to the left */
  int32_t status;     /* dmrg_status of the Lanczos solve */
  int64_t dim;        /* superblock target-sector dimension D */
  double energy;      /* ground-state energy of the step */
  double eps_S, eps_E;/* truncation error (discarded weight) of the truncated side(s), else 0 */
  double gap_S, gap_E;/* lambda_m - lambda_{m+1} at the cut of the truncated side(s) (0: nothing cut) */
  int32_t iters;      /* Lanczos iterations */
  int32_t kept_S, kept_E; /* states kept (0 for a side not truncated) */
  int32_t n_terms;    /* superblock terms */
  double ms;          /* wall time of the step */
  double ms_grow, ms_superblock, ms_solve, ms_truncate; /* its parts: growth of S' and E', superblock
                         assembly and creation, the Lanczos solve, density matrices to W^T O W */
  int32_t max_sector; /* largest symmetry sector of the truncated block(s) (eigensolve size) */
  int32_t guessed;    /* 1: the Lanczos solve started from the transformed previous ground state */
  double ms_eig, ms_select, ms_transform; /* parts of ms_truncate: density matrices and their
                         eigensolves; the global choice of the kept states; W^T O W */
} dmrg_step_info;

/* A DMRG run on a lattice of L (even, >= 4) sites keeping m states.  Builds
 * the site blocks on the device.  DMRG_EINVAL for an inconsistent model. */
dmrg_status dmrg_sys_create(const dmrg_model_desc* model, int32_t L, int32_t m, const dmrg_sys_opts* opts,
                            dmrg_sys** out);
void dmrg_sys_destroy(dmrg_sys* sys);
const char* dmrg_sys_last_error(const dmrg_sys* sys);

/* The infinite-system algorithm (Fig. infiniteloop): L/2 - 1 steps from the
 * four-site superblock to L sites, both blocks truncated each step.  steps:
 * host [L/2 - 1]; *n_steps = steps written.  Must be the first run call. */
dmrg_status dmrg_sys_infinite(dmrg_sys* sys, dmrg_step_info* steps, int32_t* n_steps);

/* Finite-system sweeps at fixed L after dmrg_sys_infinite: one sweep moves the
 * split from the middle to the right end, to the left end and back to the
 * middle, 2 (L - 3) steps; the block that grows is truncated.  steps: host
 * [n_sweeps * 2 * (L - 3)]. */
dmrg_status dmrg_sys_sweeps(dmrg_sys* sys, int32_t n_sweeps, dmrg_step_info* steps, int32_t* n_steps);

/* The superblock of the last step as a descriptor of host copies (valid until
 * the next step or dmrg_sys_destroy), with each term's coupling class and
 * multiplier (c_k = term_mult[k] * couplings[term_class[k]]), and its ground
 * state (host [D]; psi may be NULL). */
typedef struct {
  dmrg_sb_desc desc;
  const int32_t* term_class;  /* [n_terms] */
  const double* term_mult;    /* [n_terms] */
  const int64_t* sector_q;    /* [n_sectors] effective quantum number of the S' side */
  int32_t n_sys, L;
} dmrg_sys_superblock_view;
dmrg_status dmrg_sys_last_superblock(dmrg_sys* sys, dmrg_sys_superblock_view* out, double* psi);

/* The batched symmetric eigensolver of the DMRG step (the per-sector
 * eigen-decompositions of rho_S and rho_E, Eqs. rhoSystem, rhoEnviron):
 * for each of `count` symmetric matrices A[i] (device, n[i] x n[i]
 * row-major, not modified) the eigenvalues w[i] (device [n[i]], decreasing)
 * and eigenvectors V[i] (device n[i] x n[i] row-major, column j for w[i][j]),
 * by cyclic Jacobi rotations in float64: one thread block per matrix up to
 * n = 110 (in its shared memory), a cluster of 16 blocks up to n = 448 (in
 * their distributed shared memory), one block over global memory above that
 * (n <= 4096).  n, A, V, w: host arrays of [count]; stream-ordered (workspace
 * is allocated on the stream).  DMRG_EINVAL for n[i] < 0 or > 4096 or NULL
 * pointers. */
dmrg_status dmrg_sym_eig_batched(int32_t count, const int32_t* n, const double* const* A, double* const* V,
                                 double* const* w, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* DMRG_SYS_H */
