// Internal types of the superblock library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "dmrg_gb300.h"

namespace dmrg {

// ---------------------------------------------------------------- FP64 path
// Buffers a task can address.  Offsets are in elements, so one task list
// serves every call whatever the caller's pointers are.
enum BufId : int32_t { BUF_X = 0, BUF_Y = 1, BUF_T = 2, BUF_OPS = 3, BUF_G = 4, NBUF = 5 };

struct Bufs {
  double* p[NBUF];
};

// One product L (M x K) * R (K x N) added into the tile.  Either operand may
// stack the batch members along its outer dimension (rows of L, columns of
// R): element index -> (member, index within the member) with `*_rm` rows
// per member and `*_bs` elements between members.  The coefficient is a
// table index (coef_mode 0, -1 = none) or a term whose member is taken from
// the stacked side (coef_mode 1: rows of L, 2: columns of R).
struct SegF64 {
  int64_t l_off, r_off;
  int64_t l_bs, r_bs;
  int32_t l_buf, r_buf;
  int32_t ldl, ldr;
  int32_t K;
  int32_t l_trans;  // 0: L(m,k) = X[m*ldl + k]; 1: L(m,k) = X[k*ldl + m]
  int32_t r_trans;  // 0: R(k,n) = X[k*ldr + n]; 1: R(k,n) = X[n*ldr + k]
  int32_t l_rm, r_rm;
  int32_t coef;
  int32_t coef_mode;
  int32_t pad;
};

// One output tile C[m0:m0+16*ni, n0:n0+16*nj] of an M x N matrix (ni, nj in
// 1..4, chosen per output to fit its shape); the members may be stacked along
// M (c_axis 0) or N (c_axis 1), c_rm rows per member.
enum TileMode : int32_t { TM_STORE = 0, TM_DOT = 2, TM_STORE_DOTS = 3 };
struct TileF64 {
  int64_t c_off, c_bs;
  int32_t c_buf, ldc;
  int32_t M, N, m0, n0;
  int32_t seg_begin, seg_end;
  int32_t mode;     // TM_STORE: C = acc (C += acc when the launch accumulates or `add`); TM_DOT: sum(acc .* C);
                    // TM_STORE_DOTS: C = sum over segments of c(member, seg) * seg_acc, and per segment
                    // sum(seg_acc .* X) at the same offset of BUF_X (one member per tile)
  int32_t c_rm, c_axis;
  int32_t c_trans;  // 0: C(mm, nn) at [mm*ldc + nn]; 1: at [nn*ldc + mm]
  int32_t add;      // second writer of an output block: always accumulate
  int32_t shape;    // ni | nj << 8
  int32_t member;   // TM_STORE_DOTS: the batch member of the tile
  int32_t dot_base; // TM_STORE_DOTS: partials of segment s at dot_out[(dot_base + s - seg_begin) * 64 + row/col]
};

struct TaskListF64 {
  std::vector<TileF64> h_tiles;
  std::vector<SegF64> h_segs;
  TileF64* d_tiles = nullptr;
  SegF64* d_segs = nullptr;
  int64_t n_tiles = 0;
};

// skip: optional device flag; when *skip != 0 the launch does nothing
void launch_seg_gemm_f64(const TaskListF64& tl, const Bufs& bufs, const double* coef, int n_terms,
                         int accumulate, double* dot_out, const int32_t* skip, cudaStream_t st);
// tiles of mode TM_STORE_DOTS (product and per-segment dots in one pass)
void launch_seg_gemm_f64_dots(const TaskListF64& tl, const Bufs& bufs, const double* coef, int n_terms,
                              int accumulate, double* dot_out, const int32_t* skip, cudaStream_t st);
// the same task lists in double-float arithmetic (matvec_df.cu); buffers whose
// bit is set in pair_mask (1 << BufId) hold float32 pairs (hi, lo) in their
// 8-byte slots: read without splitting, written (TM_STORE) as pairs
void launch_seg_gemm_df(const TaskListF64& tl, const Bufs& bufs, const double* coef, int n_terms, int accumulate,
                        double* dot_out, const int32_t* skip, cudaStream_t st, uint32_t pair_mask = 0);
void launch_seg_gemm_df_dots(const TaskListF64& tl, const Bufs& bufs, const double* coef, int n_terms,
                             int accumulate, double* dot_out, const int32_t* skip, cudaStream_t st,
                             uint32_t pair_mask = 0);
// dst[i] = the double-float pair of src[i] (n elements)
void launch_split_pairs(const double* src, double* dst, int64_t n, cudaStream_t st);

// ------------------------------------------------------------ host pair info
struct PairH {
  int32_t term, s_out, s_in, flags;
  int64_t a_off, b_off;  // element offsets in the FP64 operator arena (ld = cols)
  int32_t order;         // two-GEMM pairs: 0 = (A Psi) B^T first A, 1 = A (Psi B^T)
};

}  // namespace dmrg

// ------------------------------------------------------------ the superblock
struct dmrg_sb {
  int32_t S = 0, n_terms = 0, batch = 0;
  std::vector<int32_t> r, c;
  std::vector<int64_t> off;  // [S+1]
  int64_t D = 0;
  std::vector<double> coeffs;  // host [batch][n_terms]
  double* d_coeffs = nullptr;  // device [batch][n_terms]
  double* h_coeffs_pinned = nullptr;  // pinned staging copy of coeffs for dmrg_set_coeffs
  std::vector<dmrg::PairH> pairs;
  double* d_ops = nullptr;     // FP64 operator arena
  double* d_ops_df = nullptr;  // the same arena as double-float pairs (first double-float product)
  double* d_x_df = nullptr;    // [batch][D] the double-float product's input as pairs
  int64_t ops_elems = 0;
  double flops = 0;            // algorithmic flops of one product, one member

  // FP64 task lists
  dmrg::TaskListF64 f64_fwd1, f64_fwd2, f64_fwd3;  // forward: intermediates, outputs (members along M, along N)
  dmrg::TaskListF64 f64_bwd1, f64_bwd2, f64_bwd3;  // H^T g
  dmrg::TaskListF64 f64_dot1, f64_dot2;   // per-pair <g, A psi B^T>
  dmrg::TaskListF64 f64_pdot2, f64_pdot3; // H psi and per-term <psi, (A_k x B_k) psi> in one pass (after f64_dot1)
  int32_t* d_pdot_ptr = nullptr;          // term reduction of its segment partials, as d_dot_red_*
  int32_t* d_pdot_idx = nullptr;
  double* d_pdot_partial = nullptr;
  double* d_T = nullptr;                  // FP64 intermediate workspace
  int64_t T_elems = 0;
  int64_t T_fwd_elems = 0;               // the part of it the forward product uses
  // term reduction of dot tiles: for (b, k): tile range [dot_red_ptr[bk], dot_red_ptr[bk+1])
  int32_t* d_dot_red_ptr = nullptr;
  int32_t* d_dot_red_idx = nullptr;
  double* d_dot_partial = nullptr;
  double* d_scratch = nullptr;  // small reduction scratch (batch norms)
  double* d_red = nullptr;      // [batch][chunks] reduction partials outside Lanczos

  // Lanczos state (allocated on first use)
  int32_t lz_cap = 0;  // Krylov capacity (max_iter + 1)
  double* lz_V = nullptr;        // [lz_cap][batch][D]
  double* lz_w = nullptr;        // [batch][D]
  double* lz_vcur = nullptr;     // [batch][D]
  double* lz_partial = nullptr;  // [batch][nchunk][lz_cap]
  double* lz_h = nullptr;        // Gram-Schmidt coefficients of passes A, B, C: [3][batch][lz_cap]
  double* lz_npart = nullptr;    // |w|^2 chunk partials after passes A, B, C: [3][batch][nchunk]
  int32_t* lz_gate = nullptr;    // [batch] 1: run the second full pass (C)
  double* lz_ab = nullptr;       // alpha [batch][lz_cap], beta [batch][lz_cap]
  double* lz_s = nullptr;        // Ritz vector [batch][lz_cap]
  double* lz_out = nullptr;      // per member: theta, resid
  int32_t* lz_ctl = nullptr;     // device control words
  int32_t* h_ctl = nullptr;      // pinned host mirror
  int32_t lz_nchunk = 0;
  // float64 refinement (Newton step with mixed CG) buffers, allocated with Lanczos
  float* rf_res = nullptr;       // [batch][D] inner CG vectors (float32)
  float* rf_p = nullptr;
  double* rf_q = nullptr;        // [batch][D] mixed product H p (float64 output)
  float* rf_hp = nullptr;        // (H - theta) p
  float* rf_t = nullptr;
  float* rf_psi32 = nullptr;     // the iterate, rounded for the inner solve
  double* rf_sc = nullptr;       // [batch][8] scalars, then eps
  int32_t* rf_ctl = nullptr;     // [2 batch + 2]
  double* rf_diag = nullptr;     // [batch][D] diag(H) per member (preconditioner)
  float* rf_minv = nullptr;      // [batch][D] 1 / max(diag - theta, delta)
  double* rf_part = nullptr;     // [4][batch][nchunk] reduction partials
  // terms with diagonal blocks (s_out == s_in): their diagonals, [n][D]
  std::vector<int32_t> dg_terms;
  int32_t* d_dg_terms = nullptr;
  double* d_dg = nullptr;
  void* lz_graphs[8] = {};       // cached cudaGraphExec_t per (prec, K) slot
  int32_t lz_graph_key[8] = {};

  void* tc = nullptr;            // tensor-core path state (matvec_tc.cu)
  int32_t* d_tc_err = nullptr;   // set by a tensor-core kernel whose bounded wait gave up
  int32_t test_stall = 0;        // testing hook: the next tensor-core product issues no copies
  int32_t test_force_pending = 0;  // testing hook: the next Lanczos solve's float32 test passes at its first check
  std::vector<double> h_ops;     // host copy of the float64 arena during creation only

  std::string err;
};
