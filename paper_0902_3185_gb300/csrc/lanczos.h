// Launchers and constants of the float64 Lanczos kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace dmrg {

constexpr int LZ_THREADS = 256;   // threads of the vector kernels
constexpr int LZ_EPT = 4;         // elements per thread
constexpr int LZ_CHUNK = LZ_THREADS * LZ_EPT;
constexpr int LZ_ROWS = 4;        // Krylov rows reduced together in k_multidot
constexpr int LZ_TRI = 32;        // threads of the tridiagonal multisection (one warp)
constexpr int LZ_DOT_EPT = 16;    // elements per thread in the reorthogonalisation dots
constexpr int LZ_DOT_CHUNK = LZ_THREADS * LZ_DOT_EPT;
constexpr int LZ_DOT_WARPS = LZ_THREADS / 32;  // dot partials per chunk (one per warp)

// LZ_CTL_FORCE (testing hook): nonzero makes the float32 test pass at its first check
enum LzCtl : int {
  LZ_CTL_J = 0, LZ_CTL_MAXIT = 1, LZ_CTL_CHECK = 2, LZ_CTL_ALLDONE = 3, LZ_CTL_FORCE = 4, LZ_CTL_MEMBER = 5
};
// LZ_PENDING: stopped on the float32 test, float64 eigenpair not yet computed;
// LZ_RESUME: the float64 test after the loop failed with iterations left (the
// host restarts the member from its Ritz vector); LZ_HOLD: finished in an
// earlier run, skipped by every kernel of a restart
enum LzCode : int {
  LZ_RUNNING = 0, LZ_CONVERGED = 1, LZ_BREAKDOWN = 2, LZ_NAN = 3, LZ_CAP = 4, LZ_PENDING = 5, LZ_RESUME = 6,
  LZ_HOLD = 7
};

inline int lz_nchunk(int64_t D) { return (int)((D + LZ_CHUNK - 1) / LZ_CHUNK); }
inline int lz_dot_nchunk(int64_t D) { return (int)((D + LZ_DOT_CHUNK - 1) / LZ_DOT_CHUNK); }
// dot partials per member and Krylov row written by one k_multidot launch
inline int lz_dot_nparts(int64_t D) { return lz_dot_nchunk(D) * LZ_DOT_WARPS; }

// Gram-Schmidt passes over the Krylov rows first_row(j, win)..j (win = 0: all
// rows); members with gate != NULL and gate[b] == 0 are skipped.
// h_pre / npart_pre: apply the three-term update with coefficients h_pre
// first (written back to w, per-chunk norm partials into npart_pre).
// pair: the Krylov basis V is stored as double-float pairs (mixed-precision
// solves; the passes run in double-float arithmetic), else float64
void lz_launch_multidot(const double* V, double* w, double* partial, const int32_t* ctl, int64_t D,
                        int batch, int cap, int win, const int32_t* gate, cudaStream_t st,
                        const double* h_pre, double* npart_pre, bool pair);
// pass A's dots (w with v_{j-1} and v_j) into the partials of a win = 2 pass
void lz_launch_dots_local(const double* V, const double* w, double* partial, const int32_t* ctl, int64_t D,
                          int batch, int cap, cudaStream_t st, bool pair);
void lz_launch_reduce_rows(const double* partial, double* h, const int32_t* ctl, int nchunk, int cap,
                           int batch, int win, const int32_t* gate, cudaStream_t st);
void lz_launch_multiaxpy(const double* V, double* w, const double* h, double* norm_partial,
                         const int32_t* ctl, int64_t D, int batch, int cap, int nchunk, int win,
                         const int32_t* gate, cudaStream_t st, bool pair);
void lz_launch_dgks(const double* npart_a, const double* npart_b, int32_t* gate, const int32_t* ctl, int batch,
                    int nchunk_a, int nchunk, cudaStream_t st);
void lz_launch_finalize_ab(const double* h, const double* npart_b, const double* npart_c, const int32_t* gate,
                           double* ab, const int32_t* ctl, int batch, int cap, int nchunk, cudaStream_t st);
// continued fractions of Lanczos coefficients at complex points (per member)
void lz_launch_cfrac(const double* norm2, const double* alpha, const double* beta, const int32_t* n, int ld,
                     const double* zr, const double* zi, int n_z, double* gr, double* gi, int batch,
                     cudaStream_t st);
void lz_launch_tridiag(const double* ab, double* s, double* out, int32_t* ctl, const double* tol, int batch,
                       int cap, int64_t D, cudaStream_t st, int final_pass = 0);
void lz_launch_next_vector(const double* w, const double* ab, double* V, double* vcur, const int32_t* ctl,
                           int64_t D, int batch, int cap, cudaStream_t st, bool pair);
void lz_launch_advance(int32_t* ctl, int batch, cudaStream_t st);
void lz_launch_sumsq(const double* x, double* part, int64_t D, int batch, int nchunk, cudaStream_t st);
void lz_launch_dot(const double* x, const double* y, double* part, int64_t D, int batch, int nchunk,
                   cudaStream_t st);
void lz_launch_sum_chunks(const double* part, double* res, int nchunk, int batch, cudaStream_t st);
// y = x / |x| (pair: y is a Krylov row stored as double-float pairs); y2, if
// not NULL, gets the float64 values
void lz_launch_scale_unit(const double* x, const double* nrm2, double* y, double* y2, int64_t D, int batch,
                          cudaStream_t st, bool pair = false);
void lz_launch_ritz(const double* V, const double* s, const int32_t* ctl, double* out, int64_t D, int batch,
                    int cap, cudaStream_t st, bool pair);
void lz_launch_div_rows(double* v, const double* nrm2, int n_terms, int batch, cudaStream_t st);
void lz_launch_reduce_terms(const double* part, const int32_t* ptr, const int32_t* idx, double* out, int n,
                            cudaStream_t st);

}  // namespace dmrg
