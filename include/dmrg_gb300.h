/*
 * dmrg_gb300.h -- C ABI of the GB300 superblock H*psi + Lanczos library.
 *
 * The operation (G. Alvarez, DMRG++ paper, Sec. 3.3): the Lanczos solver
 * needs only x += H y, with the superblock Hamiltonian
 *     H = H_S' (x) 1 + 1 (x) H_E' + sum_k c_k A_k (x) B_k
 * acting on a wavefunction that is blocked by the effective quantum number
 * (Sec. 3.2).  Sector s pairs the S' states of quantum number q_s with the
 * E' states of Q_target - q_s; its block Psi_s is r[s] x c[s], row-major,
 * and the flat vector is the concatenation of the blocks in sector order
 * (D = sum_s r[s] c[s]).  Every (term k, sector pair) with a nonzero block
 * contributes
 *     Y[s_out] += c_k * A[s_out,s_in] * Psi[s_in] * B[s_out,s_in]^T
 * because (A (x) B) vec(Psi) = vec(A Psi B^T).  H_S' (x) 1 and 1 (x) H_E'
 * are pairs whose B (respectively A) is the identity (flags below).
 *
 * Conventions shared by every call:
 *  - All vectors are float64, device pointers, laid out [batch][D]; the
 *    library never keeps or frees caller memory.
 *  - Calls are ordered on the given CUDA stream (a cudaStream_t passed as
 *    void*, NULL = legacy default stream).  Calls that return host scalars
 *    (e0, info) synchronise that stream before returning.
 *  - Errors never cross the ABI as exceptions: every call returns a
 *    dmrg_status; dmrg_last_error gives a message for the superblock.
 *  - A superblock is not thread safe: calls on one dmrg_sb must not overlap
 *    (they share its workspace).
 */
#ifndef DMRG_GB300_H
#define DMRG_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dmrg_sb dmrg_sb;

typedef enum {
  DMRG_OK = 0,
  DMRG_EINVAL = 1,      /* bad argument or descriptor */
  DMRG_ENOMEM = 2,      /* device or host allocation failed */
  DMRG_ECUDA = 3,       /* a CUDA runtime call failed */
  DMRG_ENOCONV = 4,     /* Lanczos hit max_iter before the tolerance */
  DMRG_EBREAKDOWN = 5,  /* (informational) Krylov space became invariant: result exact */
  DMRG_ETIMEOUT = 6,    /* a bounded device-side wait gave up */
  DMRG_ENAN = 7,        /* NaN or Inf met in a Lanczos scalar */
  DMRG_EUNSUPPORTED = 8 /* precision or feature not built for this device */
} dmrg_status;

typedef enum {
  DMRG_FP64 = 0,   /* float64 products on the CUDA cores */
  DMRG_TF32 = 1,   /* tensor cores, TF32 operands, FP32 accumulation */
  DMRG_BF16X3 = 2, /* tensor cores, x = hi + lo in BF16, hi*hi + hi*lo + lo*hi, FP32 accumulation */
  DMRG_DF64 = 3    /* CUDA cores, float64 in and out, double-float arithmetic (pairs of float32:
                      about 2^-46 relative error per multiply-add, 48 significant bits); forward
                      product only (dmrg_apply_H, and the residuals of refine = 3) */
} dmrg_prec;

enum { DMRG_ID_A = 1, /* A is the identity (1 (x) B term; r[s_out] == r[s_in]) */
       DMRG_ID_B = 2  /* B is the identity (A (x) 1 term; c[s_out] == c[s_in]) */ };

/* One (term, sector pair).  A: r[s_out] x r[s_in] row-major with leading
 * dimension lda >= r[s_in]; B: c[s_out] x c[s_in] with ldb >= c[s_in].
 * Pointers are host or device memory (dmrg_sb_desc.blocks_on_device); they
 * are read during dmrg_create_superblock and not kept. */
typedef struct {
  int32_t term, s_out, s_in, flags;
  const double* A;
  int64_t lda;
  const double* B;
  int64_t ldb;
} dmrg_pair;

typedef struct {
  int32_t n_sectors;
  const int32_t* r;        /* host, [n_sectors], >= 0 */
  const int32_t* c;        /* host, [n_sectors], >= 0 */
  int32_t n_terms;
  const double* coeffs;    /* host, [batch][n_terms] */
  int32_t n_pairs;
  const dmrg_pair* pairs;  /* host, [n_pairs] */
  int32_t blocks_on_device;
} dmrg_sb_desc;

typedef struct {
  int64_t dim;              /* D per batch member */
  int32_t batch, n_sectors, n_terms, n_pairs;
  double flops_per_matvec;  /* algorithmic flops of one H*psi, all batch members */
  double op_bytes_f64;      /* bytes of the stored float64 operator blocks */
  double op_bytes_mixed;    /* bytes of the tensor-core operand copies (TF32 layout) */
} dmrg_sb_info;

typedef struct {
  double tol;          /* stop when beta_j |s_j| <= tol * max(1, |theta|) */
  int32_t max_iter;    /* Krylov dimension cap (clamped to 768 and to D) */
  int32_t prec;        /* dmrg_prec of the products in the main solve */
  int32_t refine;      /* after a mixed-precision solve: 0 none; 1 restart FP64 Lanczos from its psi;
                          2 Newton steps: FP64 residual, correction equation by mixed-precision CG
                          preconditioned with diag(H); 3 as 2 with the residual products in
                          DMRG_DF64 (about 2x faster on GB300, residuals accurate to ~1e-13 |H psi|) */
  double refine_tol;   /* residual tolerance of the refinement (float64 or double-float residual), relative to max(1, |theta|) */
  int32_t check_every; /* run the tridiagonal test every this many iterations (>= 1) */
  int32_t graph_iters; /* iterations captured per CUDA graph launch (>= 1) */
} dmrg_lanczos_opts;

typedef struct {     /* one per batch member */
  double e0;
  double residual;        /* beta_j |s_j| at exit */
  int32_t iters;          /* Lanczos iterations of the main solve */
  int32_t refine_iters;   /* FP64 iterations of the refinement */
  int32_t mixed_matvecs;
  int32_t fp64_matvecs;
  int32_t status;         /* dmrg_status of this member */
  int32_t breakdown;
  int32_t kernel_launches; /* kernels the whole call launched (all members, graph nodes counted) */
  int32_t restarts;        /* Lanczos restarts from the Ritz vector: the member passed the float32
                              test but missed the float64 test after the loop, and continued from
                              its Ritz vector with the iterations it had left */
} dmrg_lanczos_info;

/* Sec. 3.2-3.3: build the sector tables, the (term, sector pair) task lists,
 * device copies of every operator block (float64 layout) and the workspace.
 * The operator layouts of the other precisions (the tensor-core panels of
 * DMRG_TF32 and DMRG_BF16X3, the double-float pairs of DMRG_DF64) are built
 * at the first product in that precision: that call allocates and copies, so
 * make it before capturing such products in a CUDA graph of your own.  batch >= 1 superblocks share all blocks and differ only
 * in coeffs.  Returns DMRG_EINVAL for inconsistent shapes (identity flag with
 * r_out != r_in, sector out of range, ld too small, NULL block). */
dmrg_status dmrg_create_superblock(const dmrg_sb_desc* d, int32_t batch, dmrg_sb** out);
void dmrg_destroy_superblock(dmrg_sb* sb);
const char* dmrg_last_error(const dmrg_sb* sb);
dmrg_status dmrg_query(const dmrg_sb* sb, dmrg_sb_info* info);

/* Replace the coefficient table (host, [batch][n_terms]) without rebuilding:
 * coupling sweeps and finite differences.  The device copy is written on
 * `stream` (through a pinned staging copy), after the work already queued on
 * that stream, and the call returns once it is written (it synchronises
 * `stream`).  Work on other streams that reads this superblock must be
 * ordered before the call by the caller. */
dmrg_status dmrg_set_coeffs(dmrg_sb* sb, const double* coeffs, void* stream);

/* Sec. 3.3 x += H y: y = H psi (accumulate = 0) or y += H psi (accumulate =
 * 1) for every batch member.  psi, y: device [batch][D], must not overlap. */
dmrg_status dmrg_apply_H(dmrg_sb* sb, const double* psi, double* y, int32_t accumulate,
                         int32_t prec, void* stream);

/* The float64 product of dmrg_apply_H (FP64 precision) for callers that
 * cannot allocate device memory when they apply H (processes whose device
 * memory belongs to another framework's pool, real-time loops in which an
 * allocation, which can synchronise the device, is not allowed).  Its intermediate
 * workspace is one static buffer of 4 Mi float64 values (32 MiB) per GPU,
 * part of the loaded library and held until the process exits; the call
 * allocates nothing.  The first call on a device looks up the buffer's device
 * address (cudaGetSymbolAddress) and must come before any stream capture.
 * Calls share the buffer, which keeps the last call's contents: calls whose
 * kernels overlap on the GPU race.  Returns DMRG_EINVAL, with a message, when
 * the superblock's forward product needs more intermediate workspace than the
 * buffer holds.  The looked-up address is kept for the life of the process:
 * re-creating a device's primary context (cudaDeviceReset) while the library
 * is loaded is not supported by this call.  The paper has
 * no counterpart to this call. */
dmrg_status dmrg_apply_H_static_scratch(dmrg_sb* sb, const double* psi, double* y, int32_t accumulate,
                                        void* stream);

/* Reverse mode of y = H(c) psi for a cotangent g (device [batch][D]):
 * dpsi = H^T g (device [batch][D]) and dc[b][k] = <g_b, (A_k (x) B_k) psi_b>
 * (device [batch][n_terms]).  Either output may be NULL. */
dmrg_status dmrg_apply_H_backward(dmrg_sb* sb, const double* psi, const double* g,
                                  double* dpsi, double* dc, int32_t prec, void* stream);

/* Sec. 3.3 (diagonalize / Lanczos): lowest eigenpair of every batch member,
 * Lanczos with float64 scalars and full reorthogonalisation (every step
 * against every Krylov vector: the three-term step, one classical
 * Gram-Schmidt pass, and a second pass where the norm fell below 1/sqrt(2)),
 * the iteration captured in CUDA graphs.  A member stops when a float32
 * estimate of its residual passes at half the tolerance; the float64 test
 * after the loop confirms it, and a member that misses it restarts from its
 * Ritz vector with the iterations it has left (DMRG_ENOCONV only at max_iter).
 * Tolerances below 1e-5 are finer than the float32 estimate resolves: near
 * convergence those members are tested in float64 at every check instead.  psi0: device [batch][D] start vectors;
 * psi_out: device [batch][D], normalised; e0: host [batch]; info: host
 * [batch] or NULL.  Returns the worst member status (DMRG_OK if all met the
 * tolerance; DMRG_EBREAKDOWN is reported in info only). */
dmrg_status dmrg_lanczos_ground(dmrg_sb* sb, const double* psi0, double* psi_out, double* e0,
                                const dmrg_lanczos_opts* opts, dmrg_lanczos_info* info,
                                void* stream);

/* dmrg_lanczos_ground, then the Hellmann-Feynman gradient of the returned
 * state, dE_dc[b][k] = <psi_b, (A_k (x) B_k) psi_b> / <psi_b, psi_b> (device
 * [batch][n_terms], as dmrg_energy_grad).  With refine = 2 (3) the
 * refinement's float64 (double-float) residual product that is expected to
 * be the last (the previous step's requested accuracy, or the mixed product's
 * error floor, meets the tolerance for every member) gives H psi and the
 * per-term dots in one pass, so the gradient of the final state costs no
 * extra pass; otherwise (also when a residual meets the tolerance earlier
 * than expected) it is computed after the solve.  Same statuses as
 * dmrg_lanczos_ground; DMRG_EINVAL for dE_dc == NULL. */
dmrg_status dmrg_lanczos_ground_grad(dmrg_sb* sb, const double* psi0, double* psi_out, double* e0,
                                     double* dE_dc, const dmrg_lanczos_opts* opts,
                                     dmrg_lanczos_info* info, void* stream);

/* Sec. 3.3 product with the per-term dots: y = H psi (device [batch][D], y
 * must not overlap psi) and dots[b][k] = <psi_b, (A_k (x) B_k) psi_b> (device
 * [batch][n_terms], no coefficient), in one pass over the pair products;
 * prec DMRG_FP64 (float64 arithmetic) or DMRG_DF64 (double-float products,
 * float64 dots).  Stream-ordered; DMRG_EINVAL for NULL or aliased pointers or
 * another precision. */
dmrg_status dmrg_apply_H_term_dots(dmrg_sb* sb, const double* psi, double* y, double* dots, int32_t prec,
                                   void* stream);

/* Lanczos coefficients for continued fractions (paper: the local density of
 * states from the continued fraction of the Lanczos coefficients of the
 * superblock Hamiltonian started from c_i |psi>).  Runs min(n_max, 768, D)
 * steps of the same Lanczos iteration as dmrg_lanczos_ground (float64
 * scalars, full reorthogonalisation, products in `prec`: DMRG_FP64, TF32 or
 * BF16X3) from phi0 / |phi0| (device [batch][D], not modified) with no
 * convergence test; a member stops early only at an invariant subspace.
 * Writes, for every member b: norm2[b] = |phi0_b|^2 (device [batch]);
 * alpha[b][j] = <v_j, H v_j> and beta[b][j] = |w_j| (the coupling of v_j and
 * v_{j+1}), j < n_out[b], into device arrays [batch][n_max] (row length
 * n_max; entries past n_out[b] are unspecified); n_out[b] (HOST [batch],
 * written after an internal stream synchronisation) = number of coefficients
 * (0 for a member whose phi0 is zero: its continued fraction is 0).
 * DMRG_EINVAL for NULL pointers, n_max < 1 or another precision; DMRG_ENAN
 * when a member with a nonzero phi0 met NaN or Inf. */
dmrg_status dmrg_lanczos_coeffs(dmrg_sb* sb, const double* phi0, int32_t n_max, int32_t prec, double* alpha,
                                double* beta, double* norm2, int32_t* n_out, void* stream);

/* Continued fractions G_b(z) = norm2[b] / (z - alpha[b][0] - beta[b][0]^2 /
 * (z - alpha[b][1] - ... - beta[b][k-2]^2 / (z - alpha[b][k-1]))), k = n[b],
 * at n_z complex points per member: z = z_re + i z_im, device [batch][n_z];
 * the result into g_re, g_im (device [batch][n_z]).  alpha, beta: device
 * [batch][ld] (as written by dmrg_lanczos_coeffs with ld = n_max); n, norm2:
 * device [batch]; n[b] is clamped to [0, ld] (0 gives G = 0).  Points must lie
 * off the spectrum (Im z > 0 for the densities of states: -Im G / pi is then
 * a sum of Lorentzians).  One thread per (member, point), evaluated from the
 * deepest level up in float64.  Stream-ordered; DMRG_EINVAL for NULL
 * pointers, batch < 0, ld < 1 or n_z < 0. */
dmrg_status dmrg_continued_fraction(const double* norm2, const double* alpha, const double* beta, const int32_t* n,
                                    int32_t batch, int32_t ld, const double* z_re, const double* z_im, int32_t n_z,
                                    double* g_re, double* g_im, void* stream);

/* Autotuner of the tensor-core product (no paper counterpart; the paper's
 * block loop has no tuning): times the product of this superblock, `reps`
 * launches per candidate after a warm-up, for every tile width (64, 128,
 * 256), tile order (heaviest first, or as built) and phase-1
 * packing (pairs sharing their wavefunction operand side by side in one
 * tile, or one tile set per pair), keeps the fastest, and also times the
 * baseline that launches one kernel per output block.  Rebuilds task lists and operand panels (allocates); invalidates
 * captured Lanczos graphs.  Synchronises the stream. */
typedef struct {
  double best_ms;        /* median product time with the chosen tuning */
  double default_ms;     /* median product time with the build-time default */
  double per_block_ms;   /* median product time, one launch per output block */
  int32_t best_tile_n;   /* chosen widest MMA N */
  int32_t heavy_first;   /* chosen tile order */
  int32_t candidates;
  int32_t pieces;        /* chosen phase-1 packing (1: pairs side by side) */
} dmrg_tune_info;
dmrg_status dmrg_autotune(dmrg_sb* sb, int32_t prec, int32_t reps, void* stream, dmrg_tune_info* info);

/* Measurement hook (no paper counterpart): event-timed average of `reps`
 * full Gram-Schmidt passes of the Lanczos solver at Krylov index j (dots of w
 * against rows 0..j, their reduction, and the update w -= V h) for every
 * member of this superblock, in the basis storage of `prec` (float64 for
 * DMRG_FP64, double-float pairs otherwise).  Allocates the Lanczos buffers
 * for j + 1 rows if needed; the rows and w hold arbitrary values (the time
 * does not depend on them).  *ms = milliseconds per pass; *bytes = the bytes
 * one pass must move, (2 (j + 1) + 3) D batch 8.  Synchronises the stream.
 * DMRG_EINVAL for j outside [0, 767], reps < 1 or NULL outputs. */
dmrg_status dmrg_time_reorth(dmrg_sb* sb, int32_t prec, int32_t j, int32_t reps, double* ms, double* bytes,
                             void* stream);

/* Synchronise `stream` and report device-side failures of earlier calls on
 * this superblock: DMRG_ETIMEOUT if a bounded wait inside a tensor-core
 * kernel gave up (the kernel then skipped its output and released its
 * resources; the context stays usable).  Clears the flag. */
dmrg_status dmrg_sync_status(dmrg_sb* sb, void* stream);

/* Testing hook (no paper counterpart): what = 1 makes the next tensor-core
 * product's copy warp issue no copies, so that its bounded waits run out and
 * report DMRG_ETIMEOUT through dmrg_sync_status; what = 2 makes the float32
 * convergence test of the next Lanczos solve pass at its first check, so
 * that the float64 test after the loop fails and the restart from the Ritz
 * vector runs; what = 0 clears both.  No memory is touched out of bounds and
 * every wait ends after its limit. */
dmrg_status dmrg_test_inject(dmrg_sb* sb, int32_t what);

/* Hellmann-Feynman: dE0/dc_k = <psi, (A_k (x) B_k) psi> / <psi, psi> for
 * every batch member.  psi: device [batch][D]; dE_dc: device [batch][n_terms]. */
dmrg_status dmrg_energy_grad(dmrg_sb* sb, const double* psi, double* dE_dc, int32_t prec,
                             void* stream);

#ifdef __cplusplus
}
#endif

#endif /* DMRG_GB300_H */
