// Mixed-precision superblock product on the tcgen05 tensor cores.
//
// Paper Sec. 3.3: x += H y as system, environment and connection tasks, each
// a product of sector blocks, formed on the fly.  With batch members that
// share every operator block (coupling sweeps), the member wavefunctions are
// stacked along the M dimension of every product (member stride = dim rounded
// up to 8 rows, the padding rows zero), so that the small, uneven sector
// blocks of a DMRG superblock become GEMMs with M = batch x dim:
//
//   order R pairs (A last):  X_b = Psi_b[s_in] B^T         (phase 1)
//                            Y_b^T += X_b^T A^T              (group S)
//   order L pairs (B last):  Z_b^T = Psi_b[s_in]^T A^T      (phase 1)
//                            Y_b += Z_b B^T                  (group E)
//   1 (x) B terms:           Y_b += (c Psi_b) B^T            (group E)
//   A (x) 1 terms:           Y_b^T += (c Psi_b)^T A^T        (group S)
//
// Every product is D = L R^T with both operands K-major, so operands are
// kept in HBM already in the tensor cores' shared-memory image ("panels"):
// 8-row atoms of 64-byte rows with the 64-byte swizzle, atoms of one
// 64-byte K chunk stored contiguously.  A tile load is then one contiguous
// cp.async.bulk per operand and no tensor maps are needed.  Zero padding in
// K is written once; padding rows only feed accumulator rows/columns that
// are never stored.
//
// One persistent kernel runs a list of output tiles (128 x up to 256) per
// launch: warp 0 streams operand tiles through a multi-stage shared-memory
// ring, warp 1 issues tcgen05.mma into two or three TMEM accumulator buffers,
// warps 2-9 drain them (tcgen05.ld) and either write the float64 output
// block or the next phase's operand panel (scaled by the member's
// coefficient, rounded to TF32 or split into BF16 hi + lo, written in 16-byte
// granules after a transpose through shared memory).  Phase-1 pairs that
// share their wavefunction operand run as one "pieced" tile: their operator
// panels side by side along N behind one L tile.
//
// Eight draining warps rather than twelve: the block then gets 168 registers
// a thread without spills (at 448 threads the cap of 128 spilled inside the
// producer's and the MMA warp's loops), and fewer warps share the issue slots
// of the two single-thread roles; on the real m = 1000 superblock the product
// fell from 0.600 to 0.557 ms.
//
// Precisions: TF32 (kind::tf32), and BF16x3: x = hi + lo, products
// hi*hi + hi*lo + lo*hi in kind::f16 with an FP32 accumulator.

#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <stdexcept>
#include <vector>

#include <cuda_bf16.h>

#include "internal.h"
#include "tc.h"
#include "tc_kernel.cuh"

namespace dmrg {

// ----------------------------------------------------------- task structs
struct TcSeg {
  const char* l;      // L panel (hi)
  const char* r;      // R panel (hi)
  int64_t l_lo, r_lo; // byte offset hi -> lo panel (BF16x3)
  int32_t l_atoms, r_atoms;  // atoms per K chunk in each panel
  int32_t kchunks;
  int32_t slot;       // accumulator slot (0: coefficients already applied)
  int32_t col0;       // pieced tiles: first tile column of this piece (a multiple of 16)
  int32_t ra;         // pieced tiles: atoms of R rows this piece copies
};

enum OutKind : int32_t { OUT_Y_ROW = 0, OUT_Y_COL = 1, OUT_PANEL = 2 };

struct TcOut {
  int32_t kind;
  int32_t Rm;      // accumulator rows per batch member (a multiple of 8)
  int32_t Rv;      // of which hold data (the rest is padding of the member stride)
  int32_t Np;      // panel: panel rows per member (N rounded up to 8)
  int32_t M, N;    // accumulator rows (batch x Rm) / valid columns
  int32_t ldy;     // Y: row length of the output block
  int32_t add;     // Y: accumulate into y (second group of a sector)
  int32_t term;    // panel: coefficient column, -1 = 1
  int32_t p_atoms; // panel: atoms per K chunk
  int64_t y_off;   // Y: element offset of the sector block in a member
  char* p;         // panel (hi)
  int64_t p_lo;
};

constexpr int TC_MAX_SLOTS = 4;
struct TcTile {
  int32_t m0, n0, ntile, la, ra;  // la / ra: atoms to load from L / R
  int32_t seg_begin, seg_end, out;
  int32_t slot_used;              // bit k: slot k receives at least one product
  int32_t slot_term[TC_MAX_SLOTS];  // slot k >= 1: its coefficient column (member from the row)
  // pieced tile (phase 1): its segments are pieces -- products that share the
  // L operand and K, with their R operands side by side along N (each from
  // column col0); one MMA chain covers all, piece q's output is seg_outs[q].
  // cmap: the piece of every 16-column chunk, 4 bits each (chunks 0-7 in
  // cmap_lo, 8-15 in cmap_hi).  ra then counts the atoms of all pieces.
  int32_t pieced;
  uint32_t cmap_lo, cmap_hi;
  TcOut o;                        // the output this tile belongs to (a copy: one load per tile)
};

struct StageOut {  // one operand panel fed by a sector block
  char* p;          // hi panel (BF16x3: the lo panel follows at the arena's lo offset)
  int32_t atoms;    // 8-row atoms per K chunk (member-stacked rows / 8)
  int32_t transpose;  // panel rows are the block's columns (K = block rows)
  int32_t term;     // scale by the member's coefficient of this term (-1: none)
  int32_t pad_;
};

struct StageTile {  // a STAGE_T x STAGE_T tile of one sector block
  int64_t src_off;  // sector block offset inside a member
  int32_t r, c;     // block dims
  int32_t r0, c0;   // tile origin
  int32_t out_begin, out_end;  // its panels
};

// Operand panel layout: K split into chunks of PANEL_ROW_BYTES (32 BF16 or
// 16 TF32 values: the sector blocks are narrow, and shorter chunks pad K
// less), rows into 8-row atoms of ATOM_BYTES with the 64-byte swizzle (the
// 16-byte piece q of row r of an atom is stored at piece q ^ ((r >> 1) & 3)),
// all atoms of one K chunk contiguous.
constexpr int PANEL_ROW_BYTES = 64;
constexpr int ATOM_BYTES = 8 * PANEL_ROW_BYTES;
constexpr int MMA_K_STEPS = PANEL_ROW_BYTES / 32;  // one MMA consumes 32 bytes of K
__host__ __device__ constexpr int swz(int piece, int r8) { return piece ^ ((r8 >> 1) & 3); }

// byte offset of element (row, k) inside a panel
__host__ __device__ inline int64_t panel_off(int64_t row, int64_t k, int64_t atoms, int es) {
  const int64_t kce = PANEL_ROW_BYTES / es;
  const int64_t kc = k / kce, kk = k - kc * kce;
  const int64_t atom = row >> 3, r8 = row & 7;
  const int64_t byte = kk * es;
  return (kc * atoms + atom) * ATOM_BYTES + r8 * PANEL_ROW_BYTES + ((int64_t)swz((int)(byte >> 4), (int)r8) << 4) +
         (byte & 15);
}

// ---------------------------------------------------------------- staging
// float64 psi blocks -> operand panels (plain or transposed, optionally
// scaled by the member's coefficient of a term).  One CTA per 32 x 32 tile
// of a sector block and member: the tile is read once (each warp one
// contiguous row run), rounded to float once into shared memory, and every
// panel the block feeds is written from there in 16-byte granules (8 BF16 hi
// and lo, or 4 TF32 consecutive K values of one panel row; consecutive
// threads take consecutive granules of a row, so a warp writes whole 64-byte
// panel rows).  Tile entries outside the block are zero, so granules reaching
// into the K padding write zeros there; padding rows are never written.
constexpr int STAGE_T = 32;
__device__ __forceinline__ float to_float(double v) { return tc::d2f_rn32(v); }
__device__ __forceinline__ float to_float(float v) { return v; }

template <int PREC, class TIn>
__global__ void __launch_bounds__(256)
tc_stage_kernel(const StageTile* __restrict__ tiles, const StageOut* __restrict__ outs, const TIn* __restrict__ x,
                int64_t D, int64_t p_lo, const double* __restrict__ coef, int n_terms,
                const int32_t* __restrict__ skip, const int32_t* __restrict__ member_done) {
  constexpr int G = PREC == DMRG_TF32 ? 4 : 8;  // values per 16-byte granule
  constexpr int es = PREC == DMRG_TF32 ? 4 : 2;
  constexpr int NKG = STAGE_T / G;              // granules per tile row
  __shared__ float tile[STAGE_T][STAGE_T + 1];
  if (skip && *skip) return;
  const StageTile tl = tiles[blockIdx.x];
  const int b = blockIdx.y;
  if (member_done && member_done[b]) return;  // a member whose solve has stopped
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int rows_t = min(STAGE_T, tl.r - tl.r0), cols_t = min(STAGE_T, tl.c - tl.c0);
  // 32-bit offsets inside the sector block (r * c < 2^31)
  const TIn* src = x + (int64_t)b * D + tl.src_off + tl.r0 * tl.c + tl.c0;
  TIn raw[STAGE_T / 8];
#pragma unroll
  for (int i = 0; i < STAGE_T / 8; ++i) {
    const int row = ty + 8 * i;
    raw[i] = (row < rows_t && tx < cols_t) ? src[row * tl.c + tx] : TIn(0);
  }
#pragma unroll
  for (int i = 0; i < STAGE_T / 8; ++i) tile[ty + 8 * i][tx] = to_float(raw[i]);
  __syncthreads();
  for (int o = tl.out_begin; o < tl.out_end; ++o) {
    const StageOut so = outs[o];
    const float scf = so.term >= 0 ? tc::d2f_rn(coef[(int64_t)b * n_terms + so.term]) : 1.0f;
    const int prows = so.transpose ? cols_t : rows_t;            // panel rows in this tile
    const int nkg = ((so.transpose ? rows_t : cols_t) + G - 1) / G;  // granules per panel row
    const int pr = threadIdx.x / NKG, kg = threadIdx.x - pr * NKG;
    if (pr >= prows || kg >= nkg) continue;
    float v[G];
#pragma unroll
    for (int i = 0; i < G; ++i) v[i] = (so.transpose ? tile[kg * G + i][pr] : tile[pr][kg * G + i]) * scf;
    const int64_t panel_rows = so.transpose ? tl.c : tl.r;
    const int64_t grow = (int64_t)b * ((panel_rows + 7) & ~7) + (so.transpose ? tl.c0 : tl.r0) + pr;
    const int64_t o_b = panel_off(grow, (int64_t)(so.transpose ? tl.r0 : tl.c0) + kg * G, so.atoms, es);
    if (PREC == DMRG_TF32) {
      const uint4 w = make_uint4(__float_as_uint(tc::round_tf32(v[0])), __float_as_uint(tc::round_tf32(v[1])),
                                 __float_as_uint(tc::round_tf32(v[2])), __float_as_uint(tc::round_tf32(v[3])));
      *reinterpret_cast<uint4*>(so.p + o_b) = w;
    } else {
      uint32_t wh[4], wl[4];  // hi = bf16(x), lo = bf16(x - hi), two K values per word
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        wh[i] = tc::bf16x2_rn(v[2 * i], v[2 * i + 1]);
        wl[i] = tc::bf16x2_rn(v[2 * i] - __uint_as_float(wh[i] << 16), v[2 * i + 1] - __uint_as_float(wh[i] & 0xffff0000u));
      }
      *reinterpret_cast<uint4*>(so.p + o_b) = make_uint4(wh[0], wh[1], wh[2], wh[3]);
      *reinterpret_cast<uint4*>(so.p + p_lo + o_b) = make_uint4(wl[0], wl[1], wl[2], wl[3]);
    }
  }
}

// ------------------------------------------------------ grouped tile GEMM
constexpr int TC_EPI_WARPS = 8;                    // two per TMEM lane quadrant
constexpr int TC_EPI_PARTS = TC_EPI_WARPS / 4;      // warps per TMEM lane quadrant
constexpr int TC_MAX_ACC = 4;                        // accumulator buffers in TMEM
constexpr int TC_THREADS = 64 + 32 * TC_EPI_WARPS;  // producer, MMA, epilogue
constexpr int L_TILE_BYTES = 128 * PANEL_ROW_BYTES;  // 128 rows of one K chunk
constexpr int EPI_LD = 17;                          // staging row stride (doubles)
constexpr int EPI_BYTES = TC_EPI_WARPS * 32 * EPI_LD * 8;
// panel outputs: a warp's 16 x 32 block of packed words, column stride chosen
// so that the transposed 16-byte reads hit distinct banks
template <int PREC>
constexpr int panel_ld() { return PREC == DMRG_TF32 ? 40 : 36; }
constexpr int PANEL_EPI_BYTES = TC_EPI_WARPS * 16 * 40 * 4;
constexpr int TC_COEF_MAX = 512;                    // coefficients cached in shared memory (float)
constexpr int TC_CTRL_BYTES = 256 + 4 * TC_COEF_MAX;  // barriers etc., then the coefficient cache

// A tile whose rows all belong to members whose solve has stopped
// (member_done[b] != 0: converged Lanczos or CG members of a batch) is
// skipped by all three roles alike: no copies, no MMAs, no output.  Rows are
// member-stacked: row m belongs to member m / Rm.
__device__ __forceinline__ bool tile_done(const TcTile& tl, const int32_t* __restrict__ member_done) {
  if (!member_done || tl.o.Rm <= 0) return false;
  const int last = min(tl.m0 + tl.la * 8, tl.o.M) - 1;
  for (int b = tl.m0 / tl.o.Rm; b <= last / tl.o.Rm; ++b)
    if (!member_done[b]) return false;
  return true;
}

template <int PREC>
__global__ void __launch_bounds__(TC_THREADS, 1)
tc_gemm_kernel(const TcTile* __restrict__ tiles, int n_tiles, const TcSeg* __restrict__ segs,
               const TcOut* __restrict__ seg_outs, double* __restrict__ y, int64_t D, const double* __restrict__ coef, int n_terms, int n_coef,
               int accumulate, const int32_t* __restrict__ skip, const int32_t* __restrict__ member_done,
               int32_t* __restrict__ err, int stages, int stage_bytes, int r_tile_bytes, int tmem_cols,
               int epi_bytes, int acc_stride, int n_acc, int tile_split, int stall) {
  if (skip && *skip) return;
  extern __shared__ __align__(1024) char smem_raw[];
  // control block, then 1024-aligned stage ring
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw);
  uint64_t* empty = full + 8;
  uint64_t* acc_full = empty + 8;
  uint64_t* acc_empty = acc_full + TC_MAX_ACC;
  uint64_t* drain = acc_empty + TC_MAX_ACC;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  float* coef_s = reinterpret_cast<float*>(smem_raw + 256);  // member coefficients as float
  double* epi_stage = reinterpret_cast<double*>(smem_raw + TC_CTRL_BYTES);
  const uint32_t base_u32 = tc::smem_u32(smem_raw);
  char* ring = smem_raw + (((base_u32 + TC_CTRL_BYTES + (uint32_t)epi_bytes + 1023) & ~1023u) - base_u32);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < n_acc; ++a) {
      tc::mbar_init(&acc_full[a], 1);
      tc::mbar_init(&acc_empty[a], tile_split ? 4 : TC_EPI_WARPS);  // the warps that drain one tile
    }
    tc::mbar_init(drain, 1);
    *abort_flag = 0;
    tc::fence_mbar_init();
  }
  if (warp == 1) {
    tc::tmem_alloc(tmem_slot, (uint32_t)tmem_cols);
    tc::tmem_relinquish();
  }
  // the coefficients are applied in float32 (their rounding, 2^-24, is far
  // below the operand precision); cached here so that no tile waits on them
  const bool coef_cached = n_coef <= TC_COEF_MAX;
  if (coef_cached)
    for (int k = threadIdx.x; k < n_coef; k += blockDim.x) coef_s[k] = tc::d2f_rn(coef[k]);
  auto coef_f = [&](int k) { return coef_cached ? coef_s[k] : tc::d2f_rn(coef[k]); };
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0 && !stall) {  // stall: testing hook, the consumers' bounded waits run out
      int stage = 0;
      uint32_t phase = 0;
      uint32_t issued = 0;  // bit s: stage s has a copy in flight or landed
      uint32_t issued_par = 0;
      // descriptors are fetched one segment (and one tile) ahead, so that
      // their load latency overlaps the copies of the current segment
      int t = blockIdx.x;
      TcTile tl{}, tl_n{};
      if (t < n_tiles) tl_n = tiles[t];
      TcSeg sg_n{};
      int sg_n_idx = -1;
      for (; t < n_tiles; t += gridDim.x) {
        tl = tl_n;
        const int tn = t + gridDim.x;
        if (tn < n_tiles) tl_n = tiles[tn];
        if (tile_done(tl, member_done)) continue;
        const uint32_t lb = (uint32_t)tl.la * ATOM_BYTES, rb = (uint32_t)tl.ra * ATOM_BYTES;
        if (tl.pieced) {
          // one L tile and every piece's R rows per K chunk
          const TcSeg sg = sg_n_idx == tl.seg_begin ? sg_n : segs[tl.seg_begin];
          if (tn < n_tiles && tl_n.seg_begin < tl_n.seg_end) {
            sg_n = segs[tl_n.seg_begin];
            sg_n_idx = tl_n.seg_begin;
          }
          for (int kc = 0; kc < sg.kchunks; ++kc) {
            if (!tc::mbar_wait(&empty[stage], phase ^ 1u, abort_flag)) goto producer_done;
            char* st = ring + (size_t)stage * stage_bytes;
            const char* lsrc = sg.l + ((int64_t)kc * sg.l_atoms + tl.m0 / 8) * ATOM_BYTES;
            tc::mbar_arrive_expect_tx(&full[stage], PREC == DMRG_TF32 ? lb + rb : 2u * (lb + rb));
            tc::bulk_g2s(st, lsrc, lb, &full[stage]);
            if (PREC == DMRG_BF16X3) tc::bulk_g2s(st + L_TILE_BYTES + r_tile_bytes, lsrc + sg.l_lo, lb, &full[stage]);
            for (int q = tl.seg_begin; q < tl.seg_end; ++q) {
              const TcSeg pq = segs[q];
              const char* rsrc = pq.r + (int64_t)kc * pq.r_atoms * ATOM_BYTES;
              const uint32_t at = (uint32_t)(pq.col0 / 8) * ATOM_BYTES, nb = (uint32_t)pq.ra * ATOM_BYTES;
              tc::bulk_g2s(st + L_TILE_BYTES + at, rsrc, nb, &full[stage]);
              if (PREC == DMRG_BF16X3)
                tc::bulk_g2s(st + 2 * L_TILE_BYTES + r_tile_bytes + at, rsrc + pq.r_lo, nb, &full[stage]);
            }
            issued |= 1u << stage;
            issued_par = (issued_par & ~(1u << stage)) | (phase << stage);
            if (++stage == stages) {
              stage = 0;
              phase ^= 1u;
            }
          }
          continue;
        }
        for (int s = tl.seg_begin; s < tl.seg_end; ++s) {
          const TcSeg sg = sg_n_idx == s ? sg_n : segs[s];
          if (s + 1 < tl.seg_end) {
            sg_n = segs[s + 1];
            sg_n_idx = s + 1;
          } else if (tn < n_tiles && tl_n.seg_begin < tl_n.seg_end) {
            sg_n = segs[tl_n.seg_begin];
            sg_n_idx = tl_n.seg_begin;
          }
          for (int kc = 0; kc < sg.kchunks; ++kc) {
            if (!tc::mbar_wait(&empty[stage], phase ^ 1u, abort_flag)) goto producer_done;
            char* st = ring + (size_t)stage * stage_bytes;
            const char* lsrc = sg.l + ((int64_t)kc * sg.l_atoms + tl.m0 / 8) * ATOM_BYTES;
            const char* rsrc = sg.r + ((int64_t)kc * sg.r_atoms + tl.n0 / 8) * ATOM_BYTES;
            tc::mbar_arrive_expect_tx(&full[stage], PREC == DMRG_TF32 ? lb + rb : 2u * (lb + rb));
            tc::bulk_g2s(st, lsrc, lb, &full[stage]);
            tc::bulk_g2s(st + L_TILE_BYTES, rsrc, rb, &full[stage]);
            if (PREC == DMRG_BF16X3) {
              tc::bulk_g2s(st + L_TILE_BYTES + r_tile_bytes, lsrc + sg.l_lo, lb, &full[stage]);
              tc::bulk_g2s(st + 2 * L_TILE_BYTES + r_tile_bytes, rsrc + sg.r_lo, rb, &full[stage]);
            }
            issued |= 1u << stage;
            issued_par = (issued_par & ~(1u << stage)) | (phase << stage);
            if (++stage == stages) {
              stage = 0;
              phase ^= 1u;
            }
          }
        }
      }
    producer_done:
      // never leave with a copy in flight: wait for the last copy of every stage
      for (int s = 0; s < stages; ++s) {
        if (!(issued >> s & 1u)) continue;
        const uint64_t t0 = tc::globaltimer();
        while (!tc::mbar_try_wait(&full[s], (issued_par >> s) & 1u)) {
          if (tc::globaltimer() - t0 > tc::WAIT_LIMIT_NS) {
            *abort_flag = 1;
            break;
          }
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issue
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int kk = 0;  // tiles with products so far: tile kk uses accumulator buffer kk % n_acc
      constexpr uint32_t fmt = PREC == DMRG_TF32 ? tc::FMT_TF32 : tc::FMT_BF16;
      TcTile tl_n{};
      if (blockIdx.x < n_tiles) tl_n = tiles[blockIdx.x];
      int nt_seg = -1, nt_kch = 0, nt_slot = 0;  // the next tile's first segment, loaded during this tile
      for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        const TcTile tl = tl_n;
        if (t + (int)gridDim.x < n_tiles) tl_n = tiles[t + gridDim.x];  // one tile ahead
        if (tl.seg_begin == tl.seg_end || tile_done(tl, member_done)) continue;
        int kch_n = nt_seg == tl.seg_begin ? nt_kch : segs[tl.seg_begin].kchunks;
        int slot_n = nt_seg == tl.seg_begin ? nt_slot : segs[tl.seg_begin].slot;
        const int acc = kk % n_acc;
        const uint32_t acc_phase = (uint32_t)(kk / n_acc) & 1u;
        ++kk;
        if (!tc::mbar_wait(&acc_empty[acc], acc_phase ^ 1u, abort_flag)) goto mma_done;
        tc::tc_fence_after();
        const uint32_t d_acc = tmem_base + (uint32_t)(acc * acc_stride);
        const uint32_t idesc = tc::idesc_f32acc(fmt, 128, (uint32_t)tl.ntile);
        uint32_t started = 0;  // slots that already hold a partial sum
        const int s_end = tl.pieced ? tl.seg_begin + 1 : tl.seg_end;  // a pieced tile is one MMA chain
        for (int s = tl.seg_begin; s < s_end; ++s) {
          const int kch = kch_n;
          const int slot = slot_n;
          if (s + 1 < s_end) {  // one segment ahead
            kch_n = segs[s + 1].kchunks;
            slot_n = segs[s + 1].slot;
          } else if (t + (int)gridDim.x < n_tiles && tl_n.seg_begin < tl_n.seg_end) {
            nt_seg = tl_n.seg_begin;  // the next tile's first: in flight during this last segment
            nt_kch = segs[nt_seg].kchunks;
            nt_slot = segs[nt_seg].slot;
          }
          const uint32_t d_tmem = d_acc + (uint32_t)(slot * tl.ntile);
          uint32_t accum = (started >> slot) & 1u;
          started |= 1u << slot;
          for (int kc = 0; kc < kch; ++kc) {
            if (!tc::mbar_wait(&full[stage], phase, abort_flag)) goto mma_done;
            tc::tc_fence_after();
            char* st = ring + (size_t)stage * stage_bytes;
            const uint64_t ah = tc::sw64_desc(tc::smem_u32(st));
            const uint64_t bh = tc::sw64_desc(tc::smem_u32(st + L_TILE_BYTES));
            if (PREC == DMRG_TF32) {
#pragma unroll
              for (int k = 0; k < MMA_K_STEPS; ++k) {
                tc::mma_tf32(d_tmem, ah + 2 * k, bh + 2 * k, idesc, accum);
                accum = 1;
              }
            } else {
              const uint64_t al = tc::sw64_desc(tc::smem_u32(st + L_TILE_BYTES + r_tile_bytes));
              const uint64_t bl = tc::sw64_desc(tc::smem_u32(st + 2 * L_TILE_BYTES + r_tile_bytes));
#pragma unroll
              for (int k = 0; k < MMA_K_STEPS; ++k) {
                tc::mma_bf16(d_tmem, ah + 2 * k, bh + 2 * k, idesc, accum);
                accum = 1;
                tc::mma_bf16(d_tmem, ah + 2 * k, bl + 2 * k, idesc, 1);
                tc::mma_bf16(d_tmem, al + 2 * k, bh + 2 * k, idesc, 1);
              }
            }
            tc::mma_commit(&empty[stage]);
            if (++stage == stages) {
              stage = 0;
              phase ^= 1u;
            }
          }
        }
        tc::mma_commit(&acc_full[acc]);
      }
    mma_done:
      // every MMA this thread issued completes before the TMEM is released
      tc::mma_commit(drain);
      const uint64_t t0 = tc::globaltimer();
      while (!tc::mbar_try_wait(drain, 0)) {
        if (tc::globaltimer() - t0 > tc::WAIT_LIMIT_NS) {
          *abort_flag = 1;
          break;
        }
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue
    // warp w reads TMEM lanes 32 (w % 4) .. +31 (the hardware's quadrant
    // rule); its part = (w - 2) / 4 in 0..TC_EPI_PARTS-1 takes either every
    // TC_EPI_PARTS-th 16-column chunk of every tile (column split: many
    // columns per tile), or every column of every TC_EPI_PARTS-th tile (tile
    // split: many small tiles, whose epilogues then run concurrently from
    // different accumulator buffers).
    const int q = warp & 3;
    const int half = (warp - 2) >> 2;
    const int row = 32 * q + lane;
    double* stg = epi_stage + (warp - 2) * (epi_bytes / (8 * TC_EPI_WARPS));  // this warp's staging
    int kk = 0;  // tiles with products so far (same count as the MMA warp's)
    TcTile tl_n{};
    if (blockIdx.x < n_tiles) tl_n = tiles[blockIdx.x];
    for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
      const TcTile tl = tl_n;
      if (t + (int)gridDim.x < n_tiles) tl_n = tiles[t + gridDim.x];  // one tile ahead
      if (tile_done(tl, member_done)) continue;
      const TcOut& o = tl.o;
      const bool empty_tile = tl.seg_begin == tl.seg_end;
      const int acc = kk % n_acc;
      const uint32_t acc_phase = (uint32_t)(kk / n_acc) & 1u;
      const bool mine = empty_tile ? half == 0 : !tile_split || kk % TC_EPI_PARTS == half;
      if (!empty_tile) ++kk;
      if (!mine) continue;
      const int m = tl.m0 + row;
      const int b = m < o.M ? m / o.Rm : 0;
      const int i = m < o.M ? m - b * o.Rm : 0;
      const bool mv = m < o.M && i < o.Rv;  // this lane's row holds data (not stride padding)
      const int nend = min(tl.n0 + tl.ntile, o.N);
      const bool add = o.add || accumulate;
      if (empty_tile) {
        if (mv && o.kind != OUT_PANEL && !add) {
          double* yb = y + (int64_t)b * D + o.y_off;
          for (int n = tl.n0; n < nend; ++n)
            yb[o.kind == OUT_Y_ROW ? (int64_t)i * o.ldy + n : (int64_t)n * o.ldy + i] = 0.0;
        }
        continue;
      }
      int ok = 1;
      if (lane == 0) ok = tc::mbar_wait(&acc_full[acc], acc_phase, abort_flag) ? 1 : 0;
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) break;
      tc::tc_fence_after();
      const uint32_t tb = tmem_base + (uint32_t)(acc * acc_stride) + ((uint32_t)(32 * q) << 16);
      const float scf = (o.kind == OUT_PANEL && o.term >= 0 && mv) ? coef_f(b * n_terms + o.term) : 1.0f;
      // row-major output: element offset of this lane's row (-1 = row not stored)
      const int64_t rbase = (o.kind == OUT_Y_ROW && mv) ? (int64_t)b * D + o.y_off + (int64_t)i * o.ldy : -1;
      float slot_sc[TC_MAX_SLOTS];
#pragma unroll
      for (int k = 1; k < TC_MAX_SLOTS; ++k)
        slot_sc[k] = ((tl.slot_used >> k) & 1) && mv ? coef_f(b * n_terms + tl.slot_term[k]) : 0.0f;
      // pieced tiles: lane l holds piece l's output (panel, rows per member,
      // atoms, columns, coefficient column, first column), which each chunk
      // then reads with shuffles instead of dependent loads
      char* pc_p = nullptr;
      int pc_np = 0, pc_at = 0, pc_n = 0, pc_term = -1, pc_col0 = 0;
      if (tl.pieced && lane < tl.seg_end - tl.seg_begin) {
        const TcOut& so = seg_outs[tl.seg_begin + lane];
        pc_p = so.p;
        pc_np = so.Np;
        pc_at = so.p_atoms;
        pc_n = so.N;
        pc_term = so.term;
        pc_col0 = segs[tl.seg_begin + lane].col0;
      }
      const int c_first = tile_split ? 0 : 16 * half, c_step = tile_split ? 16 : 16 * TC_EPI_PARTS;
      const int c_end = tl.m0 + 32 * q < o.M ? tl.ntile : 0;  // no rows of this quadrant: nothing to drain
      for (int c0 = c_first; c0 < c_end; c0 += c_step) {
        float v[16];
        if (tl.slot_used == 1) {
          tc::tmem_ld16(tb + (uint32_t)c0, v);
        } else {
          // products of the identity terms were accumulated per coefficient:
          // y = slot 0 + sum_k c_k(member) * slot k
#pragma unroll
          for (int jj = 0; jj < 16; ++jj) v[jj] = 0.0f;
#pragma unroll
          for (int k = 0; k < TC_MAX_SLOTS; ++k) {
            if (!((tl.slot_used >> k) & 1)) continue;
            float u[16];
            tc::tmem_ld16(tb + (uint32_t)(k * tl.ntile + c0), u);
            const float w = k == 0 ? 1.0f : slot_sc[k];
#pragma unroll
            for (int jj = 0; jj < 16; ++jj) v[jj] = fmaf(w, u[jj], v[jj]);
          }
        }
        if (o.kind == OUT_Y_ROW) {
          // stage 32 rows x 16 columns, then write each row's 16 values as one
          // contiguous 128-byte segment (16 lanes per row, two rows per store)
#pragma unroll
          for (int jj = 0; jj < 16; ++jj) stg[lane * EPI_LD + jj] = tc::f2d_exact(v[jj]);
          __syncwarp();
          const int jj = lane & 15;
          const int n = tl.n0 + c0 + jj;
#pragma unroll 4
          for (int rr = 0; rr < 32; rr += 2) {
            const int r2 = rr + (lane >> 4);
            const int64_t rb = __shfl_sync(0xffffffffu, rbase, r2);
            if (rb >= 0 && n < nend) {
              double* p = y + rb + n;
              const double val = stg[r2 * EPI_LD + jj];
              *p = add ? *p + val : val;
            }
          }
          __syncwarp();
          continue;
        }
        if (o.kind == OUT_PANEL) {
          // Lanes G g .. G g + G-1 hold G consecutive accumulator rows, i.e. G
          // consecutive K values of one member (the member stride is a
          // multiple of 8).  Transpose the warp's 32 x 16 block through shared
          // memory so that a lane holds G rows of one column, and write them
          // as one 16-byte granule of the panel (per half for BF16).
          constexpr int G = PREC == DMRG_TF32 ? 4 : 8;
          constexpr int LD = panel_ld<PREC>();
          uint32_t* pstg = reinterpret_cast<uint32_t*>(stg);
          // the output of this 16-column chunk: the tile's, or its piece's
          TcOut po = o;
          int pcol0 = 0;
          float pscf = scf;
          if (tl.pieced) {
            const int ci = c0 >> 4;
            const int pi = (int)(((ci < 8 ? tl.cmap_lo >> (4 * ci) : tl.cmap_hi >> (4 * (ci - 8)))) & 15u);
            po.p = reinterpret_cast<char*>(
                __shfl_sync(0xffffffffu, (unsigned long long)reinterpret_cast<uintptr_t>(pc_p), pi));
            po.Np = __shfl_sync(0xffffffffu, pc_np, pi);
            po.p_atoms = __shfl_sync(0xffffffffu, pc_at, pi);
            po.N = __shfl_sync(0xffffffffu, pc_n, pi);
            po.term = __shfl_sync(0xffffffffu, pc_term, pi);
            pcol0 = __shfl_sync(0xffffffffu, pc_col0, pi);
            pscf = (po.term >= 0 && mv) ? coef_f(b * n_terms + po.term) : 1.0f;
          }
          const int pend = tl.pieced ? po.N : nend;  // end column (a piece counts from its own first)
          if (PREC == DMRG_TF32) {
#pragma unroll
            for (int jj = 0; jj < 16; ++jj) pstg[jj * LD + lane] = __float_as_uint(tc::round_tf32(v[jj] * pscf));
          } else {
            // two columns per conversion instruction: hi = bf16(x), lo = bf16(x - hi)
#pragma unroll
            for (int jj = 0; jj < 16; jj += 2) {
              const float x0 = v[jj] * pscf, x1 = v[jj + 1] * pscf;
              const uint32_t hp = tc::bf16x2_rn(x0, x1);
              const uint32_t lp = tc::bf16x2_rn(x0 - __uint_as_float(hp << 16), x1 - __uint_as_float(hp & 0xffff0000u));
              pstg[jj * LD + lane] = __byte_perm(hp, lp, 0x5410);        // hi | lo << 16 of column jj
              pstg[(jj + 1) * LD + lane] = __byte_perm(hp, lp, 0x7632);  // of column jj + 1
            }
          }
          __syncwarp();
          const int cg = lane & (G - 1), g0 = lane & ~(G - 1);
          const bool gv = tl.m0 + 32 * q + g0 < o.M;  // the group's rows exist
          constexpr int es = PREC == DMRG_TF32 ? 4 : 2, kce = PANEL_ROW_BYTES / es;
          const int kfirst = i - cg;  // K index of row g0: a multiple of G
          const int kc = kfirst / kce;
          const int chunk = ((kfirst - kc * kce) * es) >> 4;
#pragma unroll
          for (int blk = 0; blk < 16; blk += G) {
            const int n = tl.n0 + c0 + blk + cg - pcol0;  // column of the (piece's) output
            if (!gv || n >= pend) continue;
            const uint32_t* src = pstg + (blk + cg) * LD + g0;
            const int prow = b * po.Np + n;
            const int r8 = prow & 7;
            const int off = (kc * po.p_atoms + (prow >> 3)) * ATOM_BYTES + r8 * PANEL_ROW_BYTES + (swz(chunk, r8) << 4);
            if (PREC == DMRG_TF32) {
              *reinterpret_cast<uint4*>(po.p + off) = *reinterpret_cast<const uint4*>(src);
            } else {
              const uint4 a = *reinterpret_cast<const uint4*>(src);
              const uint4 c4 = *reinterpret_cast<const uint4*>(src + 4);
              *reinterpret_cast<uint4*>(po.p + off) =
                  make_uint4(__byte_perm(a.x, a.y, 0x5410), __byte_perm(a.z, a.w, 0x5410),
                             __byte_perm(c4.x, c4.y, 0x5410), __byte_perm(c4.z, c4.w, 0x5410));
              *reinterpret_cast<uint4*>(po.p + po.p_lo + off) =
                  make_uint4(__byte_perm(a.x, a.y, 0x7632), __byte_perm(a.z, a.w, 0x7632),
                             __byte_perm(c4.x, c4.y, 0x7632), __byte_perm(c4.z, c4.w, 0x7632));
            }
          }
          __syncwarp();
          continue;
        }
        if (!mv) continue;
        {  // column-major float64 output: lanes write consecutive i
          double* yb = y + (int64_t)b * D + o.y_off + i;
          const int nn = min(16, nend - (tl.n0 + c0));
          if (add) {
            double old[16];  // issue every load before the first add
#pragma unroll
            for (int jj = 0; jj < 16; ++jj)
              if (jj < nn) old[jj] = yb[(int64_t)(tl.n0 + c0 + jj) * o.ldy];
#pragma unroll
            for (int jj = 0; jj < 16; ++jj)
              if (jj < nn) yb[(int64_t)(tl.n0 + c0 + jj) * o.ldy] = old[jj] + tc::f2d_exact(v[jj]);
          } else {
#pragma unroll
            for (int jj = 0; jj < 16; ++jj)
              if (jj < nn) yb[(int64_t)(tl.n0 + c0 + jj) * o.ldy] = tc::f2d_exact(v[jj]);
          }
        }
      }
      tc::tc_fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&acc_empty[acc]);
    }
  }

  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  if (warp == 1) tc::tmem_dealloc(tmem_base, (uint32_t)tmem_cols);
  if (threadIdx.x == 0 && *abort_flag) atomicOr(err, 1);
}

// =================================================================== host
namespace {

struct CudaFail : std::runtime_error {
  using std::runtime_error::runtime_error;
};
#define TCK(x)                                                             \
  do {                                                                     \
    cudaError_t e_ = (x);                                                  \
    if (e_ != cudaSuccess) throw CudaFail(std::string(#x) + ": " + cudaGetErrorString(e_)); \
  } while (0)

template <class T>
T* up(const std::vector<T>& h) {
  void* p = nullptr;
  const size_t n = std::max<size_t>(1, h.size());
  TCK(cudaMalloc(&p, n * sizeof(T)));
  if (!h.empty()) TCK(cudaMemcpy(p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
  return static_cast<T*>(p);
}

uint16_t f2bf(float f) {  // round to nearest even
  uint32_t u;
  memcpy(&u, &f, 4);
  if ((u & 0x7fffffffu) > 0x7f800000u) return (uint16_t)((u >> 16) | 0x40u);
  u += 0x7fffu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}
float bf2f(uint16_t h) {
  const uint32_t u = (uint32_t)h << 16;
  float f;
  memcpy(&f, &u, 4);
  return f;
}
float to_tf32(double x) {  // round to a 10-bit mantissa, nearest even
  float f = (float)x;
  uint32_t u;
  memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) != 0x7f800000u) {
    u += 0xfffu + ((u >> 13) & 1u);
    u &= 0xffffe000u;
  }
  memcpy(&f, &u, 4);
  return f;
}

int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
int64_t pad8(int64_t a) { return cdiv(a, 8) * 8; }  // member stride of stacked panels and accumulators

struct Launch {  // one grouped GEMM launch
  TcTile* tiles = nullptr;
  TcTile* tiles_by_out = nullptr;   // the same tiles grouped by output block
  std::vector<int> out_begin;       // per output: first tile in tiles_by_out (+ end)
  TcSeg* segs = nullptr;
  TcOut* seg_outs = nullptr;        // per segment: the output of a piece (pieced tiles)
  int n_tiles = 0;
  int ntile_max = 16;
  int acc_cols = 16;         // TMEM columns per accumulator buffer (all slots)
  bool has_row_out = false;  // some output is row-major float64 (needs epilogue staging)
  bool has_panel_out = false;  // some output is a panel (transposed through shared memory)
};

struct PairSet {  // the forward pairs or their transposes
  StageTile* stage_tiles = nullptr;  // staging: psi tiles (per member) ...
  StageOut* stage_outs = nullptr;    // ... and the panels they feed
  int n_stage_tiles = 0;
  int64_t p_lo = 0;                  // byte offset of the lo panels from the hi panels (BF16x3)
  Launch ph1, grpE, grpS;
};

struct Fmt {
  char* arena = nullptr;
  size_t bytes = 0;   // per hi/lo half
  PairSet fwd, bwd;
  bool built = false;                // panels and task lists exist (built at the first use of the precision)
  std::vector<double> built_coeffs;  // the coefficient table its panels were built with
};

// A pair as the product sees it (forward, or transposed for H^T)
struct EPair {
  int32_t term, s_out, s_in, flags, order;
  const double* A;  // host, r_out x r_in (already transposed for H^T)
  const double* B;  // host, c_out x c_in
};

struct Tune {         // picked by dmrg_autotune
  int max_ntile = 0;  // widest MMA N of a tile (0: default per precision)
  int heavy_first = 1;  // deal the heaviest tiles first (else build order)
  int per_block = 0;  // baseline: one launch per output block instead of one persistent launch
  int pieces = 1;     // phase 1: pack pairs sharing their L operand side by side (pieced tiles)
};

struct State {
  int num_sms = 0;
  bool ok = false;
  Fmt f[2];  // 0: TF32, 1: BF16x3
  Tune tune[2];
  double op_bytes_tf32 = 0;
  std::vector<double> host_ops;               // float64 blocks (forward)
  std::vector<std::vector<double>> trans;     // transposed blocks (H^T)
  std::vector<EPair> fw, bw;
};

void free_launch(Launch& l) {
  for (void* p : {(void*)l.tiles, (void*)l.tiles_by_out, (void*)l.segs, (void*)l.seg_outs})
    if (p) cudaFree(p);
  l = Launch{};
}
void free_set(PairSet& s) {
  if (s.stage_tiles) cudaFree(s.stage_tiles);
  if (s.stage_outs) cudaFree(s.stage_outs);
  free_launch(s.ph1);
  free_launch(s.grpE);
  free_launch(s.grpS);
  s = PairSet{};
}

struct Panel {
  int64_t off = -1;  // byte offset in the half-arena
  int64_t rows = 0, K = 0, atoms = 0;
};

// Pack a host float64 block (rows x K, element (row,k) at X[row*ld + k]) into a panel.
void pack(std::vector<uint8_t>& hi, std::vector<uint8_t>& lo, const Panel& p, const double* X, int64_t ld,
          int prec) {
  const int es = prec == DMRG_TF32 ? 4 : 2;
  for (int64_t r = 0; r < p.rows; ++r)
    for (int64_t k = 0; k < p.K; ++k) {
      const double x = X[r * ld + k];
      const int64_t o = p.off + panel_off(r, k, p.atoms, es);
      if (prec == DMRG_TF32) {
        const float f = to_tf32(x);
        memcpy(&hi[o], &f, 4);
      } else {
        const uint16_t h = f2bf((float)x);
        const uint16_t l = f2bf((float)(x - (double)bf2f(h)));
        memcpy(&hi[o], &h, 2);
        memcpy(&lo[o], &l, 2);
      }
    }
}

}  // namespace

// Build the panels and launches of one pair set in one format.  The caller's
// half-arena layout starts at `base_off`; returns the bytes used.
static int64_t build_set(const dmrg_sb* sb, int prec, const std::vector<EPair>& P, int64_t base_off,
                         std::vector<uint8_t>& hi, std::vector<uint8_t>& lo, char* d_hi, int64_t lo_delta,
                         PairSet& out, bool dry, const Tune& tune, int n_sms) {
  const int64_t nb = sb->batch;
  const int es = prec == DMRG_TF32 ? 4 : 2;
  const int64_t kce = PANEL_ROW_BYTES / es;
  const auto& r = sb->r;
  const auto& c = sb->c;
  const int S = sb->S;
  // widest MMA N per tile: BF16x3 stages hold four operand tiles, so its
  // default is 128 (more pipeline stages in shared memory); the autotuner
  // also tries 256
  const int max_ntile = tune.max_ntile > 0 ? tune.max_ntile : (prec == DMRG_BF16X3 ? 128 : 256);
  int64_t cur = base_off;
  auto alloc = [&](int64_t rows, int64_t K) {
    Panel p;
    p.rows = rows;
    p.K = K;
    p.atoms = cdiv(rows, 8);
    p.off = cur;
    cur += p.atoms * cdiv(K, kce) * ATOM_BYTES;
    return p;
  };
  const size_t np = P.size();
  std::vector<std::vector<size_t>> by_out(S);
  for (size_t i = 0; i < np; ++i) by_out[P[i].s_out].push_back(i);
  // Identity-term coefficients differ per member.  Where the accumulator has
  // room, each such term accumulates into its own TMEM slot (weighted by the
  // member's coefficient in the epilogue) and reads the shared unscaled
  // wavefunction panel; otherwise the term gets a coefficient-scaled copy.
  // slot_of[i]: slot of identity pair i (0 = scaled copy or not an identity pair)
  std::vector<int> slot_of(np, 0);
  // An identity term whose coefficient is the same for every member (e.g. a
  // hopping class at fixed t while U is swept) needs no per-member scaling:
  // the diagonal identity pairs of one output sector and group with such
  // coefficients are folded into one operator panel, sum_k c_k B_k (or
  // sum_k c_k A_k), read against the unscaled wavefunction panel into the
  // main accumulator (their coefficients are in the panel).  folded[i]: pair
  // i is one of them; fold[s][grp]: the pairs folded for sector s.
  const int nt = sb->n_terms;
  auto uniform = [&](int term) {
    for (int64_t b = 1; b < nb; ++b)
      if (sb->coeffs[(size_t)b * nt + term] != sb->coeffs[term]) return false;
    return true;
  };
  std::vector<char> folded(np, 0);
  std::vector<std::array<std::vector<size_t>, 2>> fold((size_t)S);
  for (size_t i = 0; i < np; ++i) {
    const EPair& e = P[i];
    if (!(e.flags & (DMRG_ID_A | DMRG_ID_B)) || e.s_out != e.s_in || !uniform(e.term)) continue;
    folded[i] = 1;
    fold[(size_t)e.s_out][(e.flags & DMRG_ID_A) ? 0 : 1].push_back(i);
  }
  for (int s = 0; s < S; ++s) {
    for (int grp = 0; grp < 2; ++grp) {  // 0: 1 (x) B terms (group E), 1: A (x) 1 terms (group S)
      const int flag = grp == 0 ? DMRG_ID_A : DMRG_ID_B;
      std::vector<int> terms;
      for (size_t i : by_out[s])
        if ((P[i].flags & flag) && !folded[i] && std::find(terms.begin(), terms.end(), P[i].term) == terms.end())
          terms.push_back(P[i].term);
      if (terms.empty()) continue;
      const int64_t Nout = grp == 0 ? c[s] : r[s];
      const int64_t ntile = std::min<int64_t>(max_ntile, cdiv(Nout, 16) * 16);
      const int nslot = 1 + (int)terms.size();
      if (nslot > TC_MAX_SLOTS || nslot * ntile > 256) continue;
      for (size_t i : by_out[s])
        if ((P[i].flags & flag) && !folded[i])
          slot_of[i] = 1 + (int)(std::find(terms.begin(), terms.end(), P[i].term) - terms.begin());
    }
  }
  std::vector<Panel> pA(np), pB(np), pX(np), pS(np);  // operator A, B; intermediate; scaled psi copy
  std::vector<Panel> psiP(S), psiPT(S);
  std::vector<char> needP(S, 0), needPT(S, 0);
  std::vector<Panel> pF((size_t)S * 2);  // folded operator panels: [s][0] sum c B (group E), [s][1] sum c A (group S)
  for (int s = 0; s < S; ++s) {
    if (!fold[(size_t)s][0].empty()) {
      pF[(size_t)s * 2] = alloc(c[s], c[s]);
      needP[s] = 1;
    }
    if (!fold[(size_t)s][1].empty()) {
      pF[(size_t)s * 2 + 1] = alloc(r[s], r[s]);
      needPT[s] = 1;
    }
  }
  for (size_t i = 0; i < np; ++i) {
    const EPair& e = P[i];
    if (folded[i]) continue;
    const int64_t ro = r[e.s_out], ri = r[e.s_in], co = c[e.s_out], ci = c[e.s_in];
    if (!(e.flags & DMRG_ID_A)) pA[i] = alloc(ro, ri);
    if (!(e.flags & DMRG_ID_B)) pB[i] = alloc(co, ci);
    if (e.flags & DMRG_ID_A) {                                  // c Psi       (group E, L)
      if (slot_of[i]) needP[e.s_in] = 1;
      else pS[i] = alloc(nb * pad8(ri), ci);
    } else if (e.flags & DMRG_ID_B) {                           // (c Psi)^T   (group S, L)
      if (slot_of[i]) needPT[e.s_in] = 1;
      else pS[i] = alloc(nb * pad8(ci), ri);
    } else if (e.order == 1) { pX[i] = alloc(nb * pad8(co), ri); needP[e.s_in] = 1; }   // X^T stacked
    else { pX[i] = alloc(nb * pad8(ro), ci); needPT[e.s_in] = 1; }                   // Z stacked
  }
  for (int s = 0; s < S; ++s) {
    if (needP[s]) psiP[s] = alloc(nb * pad8(r[s]), c[s]);
    if (needPT[s]) psiPT[s] = alloc(nb * pad8(c[s]), r[s]);
  }
  if (dry) return cur - base_off;
  hi.resize(cur, 0);
  if (prec == DMRG_BF16X3) lo.resize(cur, 0);
  for (size_t i = 0; i < np; ++i) {
    const EPair& e = P[i];
    if (pA[i].off >= 0) pack(hi, lo, pA[i], e.A, r[e.s_in], prec);
    if (pB[i].off >= 0) pack(hi, lo, pB[i], e.B, c[e.s_in], prec);
  }
  for (int s = 0; s < S; ++s)
    for (int grp = 0; grp < 2; ++grp) {
      const std::vector<size_t>& f = fold[(size_t)s][grp];
      if (f.empty()) continue;
      const int64_t n = grp == 0 ? c[s] : r[s];
      std::vector<double> M((size_t)(n * n), 0.0);
      for (size_t i : f) {
        const double ck = sb->coeffs[P[i].term];
        const double* X = grp == 0 ? P[i].B : P[i].A;
        for (int64_t k = 0; k < n * n; ++k) M[(size_t)k] += ck * X[k];
      }
      pack(hi, lo, pF[(size_t)s * 2 + grp], M.data(), n, prec);
    }
  auto dptr = [&](const Panel& p) { return d_hi + p.off; };

  // ---- staging: the panels each sector block feeds, then its tiles
  std::vector<std::vector<StageOut>> feeds((size_t)S);
  auto add_feed = [&](int s_, int transpose, int term, const Panel& p) {
    if ((int64_t)r[s_] * c[s_] >= INT32_MAX)
      throw std::logic_error("tensor-core staging: sector block too large for 32-bit offsets");
    feeds[(size_t)s_].push_back(StageOut{dptr(p), (int32_t)p.atoms, transpose, term, 0});
  };
  for (int s_ = 0; s_ < S; ++s_) {
    if (needP[s_]) add_feed(s_, 0, -1, psiP[s_]);
    if (needPT[s_]) add_feed(s_, 1, -1, psiPT[s_]);
  }
  for (size_t i = 0; i < np; ++i) {
    const EPair& e = P[i];
    if (slot_of[i] || folded[i]) continue;
    if (e.flags & DMRG_ID_A) add_feed(e.s_in, 0, e.term, pS[i]);
    else if (e.flags & DMRG_ID_B) add_feed(e.s_in, 1, e.term, pS[i]);
  }
  std::vector<StageTile> stiles;
  std::vector<StageOut> souts;
  for (int s_ = 0; s_ < S; ++s_) {
    if (feeds[(size_t)s_].empty() || (int64_t)r[s_] * c[s_] == 0) continue;
    const int32_t ob = (int32_t)souts.size();
    souts.insert(souts.end(), feeds[(size_t)s_].begin(), feeds[(size_t)s_].end());
    for (int r0 = 0; r0 < r[s_]; r0 += STAGE_T)
      for (int c0 = 0; c0 < c[s_]; c0 += STAGE_T)
        stiles.push_back(StageTile{sb->off[s_], (int32_t)r[s_], (int32_t)c[s_], r0, c0, ob, (int32_t)souts.size()});
  }
  if (stiles.size() >= (size_t)INT32_MAX) throw std::logic_error("tensor-core staging: too many tiles");
  // ---- grouped launches
  struct Build {
    std::vector<TcTile> tiles;
    std::vector<TcSeg> segs;
    std::vector<TcOut> seg_outs;  // parallel to segs
    std::vector<TcOut> outs;
    std::vector<int64_t> weight;
    int ntile_max = 16;
    int acc_cols = 16;  // TMEM columns of one accumulator buffer (slots x N)
  } L1, LE, LS;
  // host-side bounds proof of every bulk copy the tiles will issue
  auto check = [](bool ok, const char* what) {
    if (!ok) throw std::logic_error(std::string("tensor-core task list: ") + what);
  };
  auto seg = [&](const Panel& Lp, const Panel& Rp) {
    check(Lp.off >= 0 && Rp.off >= 0 && Lp.K == Rp.K, "segment operands");
    TcSeg g{};
    g.l = dptr(Lp);
    g.r = dptr(Rp);
    g.l_lo = lo_delta;
    g.r_lo = lo_delta;
    g.l_atoms = (int32_t)Lp.atoms;
    g.r_atoms = (int32_t)Rp.atoms;
    g.kchunks = (int32_t)cdiv(Lp.K, kce);
    return g;
  };
  auto add_out = [&](Build& B, const TcOut& o, const std::vector<TcSeg>& sg, const std::vector<int>& slot_terms) {
    for (const TcSeg& g : sg) {
      check(g.l_atoms == cdiv(o.M, 8) && g.r_atoms == cdiv(o.N, 8), "operand rows differ from the output");
      check(g.kchunks >= 1, "empty K");
    }
    check(o.Rm % 8 == 0 && o.Rv <= o.Rm && o.M % o.Rm == 0, "member stride");
    if (o.kind == OUT_PANEL)
      check(o.Np == pad8(o.N) && o.p_atoms == (int64_t)o.Np * (o.M / o.Rm) / 8, "panel rows");
    else check(o.y_off + (int64_t)(o.kind == OUT_Y_ROW ? o.Rv : o.N) * o.ldy <= sb->D, "output block");
    const int oid = (int)B.outs.size();
    B.outs.push_back(o);
    const int s0 = (int)B.segs.size();
    B.segs.insert(B.segs.end(), sg.begin(), sg.end());
    B.seg_outs.resize(B.segs.size());
    const int s1 = (int)B.segs.size();
    int64_t kw = 0;
    for (const TcSeg& g : sg) kw += g.kchunks;
    // N split into tiles of (nearly) equal width, multiples of 16, at most max_ntile
    const int64_t n_tiles = cdiv(o.N, max_ntile);
    const int64_t width = cdiv(cdiv(o.N, n_tiles), 16) * 16;
    for (int m0 = 0; m0 < o.M; m0 += 128)
      for (int n0 = 0; n0 < o.N; n0 += (int)width) {
        TcTile t{};
        t.m0 = m0;
        t.n0 = n0;
        t.ntile = (int)std::min<int64_t>(width, cdiv(o.N - n0, 16) * 16);
        t.la = (int)std::min<int64_t>(16, cdiv(o.M - m0, 8));
        t.ra = (int)std::min<int64_t>(t.ntile / 8, cdiv(o.N - n0, 8));
        t.seg_begin = s0;
        t.seg_end = s1;
        t.out = oid;
        t.o = o;
        for (const TcSeg& g : sg) t.slot_used |= 1 << g.slot;
        if (sg.empty()) t.slot_used = 1;
        for (size_t k = 0; k < slot_terms.size(); ++k) t.slot_term[k + 1] = slot_terms[k];
        check(t.slot_used < (1 << TC_MAX_SLOTS), "accumulator slots");
        int top = 0;
        for (int k = 0; k < TC_MAX_SLOTS; ++k)
          if (t.slot_used >> k & 1) top = k;
        B.acc_cols = std::max(B.acc_cols, (top + 1) * t.ntile);
        check(B.acc_cols <= 256, "accumulator columns");
        check(t.m0 % 8 == 0 && t.n0 % 8 == 0 && t.la >= 1 && t.ra >= 1, "tile origin");
        check(t.m0 / 8 + t.la <= cdiv(o.M, 8) && t.n0 / 8 + t.ra <= cdiv(o.N, 8), "tile past its panels");
        check(t.ntile % 16 == 0 && t.ntile >= 16 && t.ntile <= 256 && t.ra * 8 <= t.ntile, "MMA N");
        B.ntile_max = std::max(B.ntile_max, t.ntile);
        B.tiles.push_back(t);
        B.weight.push_back(kw * (int64_t)t.ntile + 64);
      }
  };
  // phase 1: the output (an operand panel of phase 2) of a two-GEMM pair
  auto ph1_out = [&](size_t i) {
    const EPair& e = P[i];
    const int64_t ro = r[e.s_out], ri = r[e.s_in], co = c[e.s_out], ci = c[e.s_in];
    TcOut o{};
    o.kind = OUT_PANEL;
    o.term = e.term;
    o.p = dptr(pX[i]);
    o.p_lo = lo_delta;
    o.p_atoms = (int32_t)pX[i].atoms;
    if (e.order == 1) {  // X_b = Psi_b B^T : rows (b, a'), cols beta; stored as X^T rows (b, beta), k = a'
      o.Rm = (int32_t)pad8(ri);
      o.Rv = (int32_t)ri;
      o.N = (int32_t)co;
      o.Np = (int32_t)pad8(co);
    } else {  // Z_b^T = Psi_b^T A^T : rows (b, beta'), cols alpha; stored as Z rows (b, alpha), k = beta'
      o.Rm = (int32_t)pad8(ci);
      o.Rv = (int32_t)ci;
      o.N = (int32_t)ro;
      o.Np = (int32_t)pad8(ro);
    }
    o.M = (int32_t)(nb * o.Rm);
    return o;
  };
  auto ph1_seg = [&](size_t i) {
    const EPair& e = P[i];
    return e.order == 1 ? seg(psiP[e.s_in], pB[i]) : seg(psiPT[e.s_in], pA[i]);
  };
  // Pairs that share the L operand (same s_in and order) are packed side by
  // side along N into pieced tiles of at most max_ntile columns (each piece
  // 16-column aligned), so one L tile feeds several products; pairs wider
  // than half a tile keep tiles of their own.
  std::vector<std::vector<size_t>> by_in(2 * (size_t)S);
  for (size_t i = 0; i < np; ++i) {
    const EPair& e = P[i];
    if (e.flags & (DMRG_ID_A | DMRG_ID_B)) continue;
    const TcOut o = ph1_out(i);
    if (!tune.pieces || cdiv(o.N, 16) * 16 * 2 > max_ntile) {
      add_out(L1, o, {ph1_seg(i)}, {});
      continue;
    }
    by_in[(size_t)e.order * S + e.s_in].push_back(i);
  }
  for (auto& grp : by_in) {
    if (grp.empty()) continue;
    std::stable_sort(grp.begin(), grp.end(), [&](size_t a, size_t b) { return ph1_out(a).N > ph1_out(b).N; });
    std::vector<std::vector<size_t>> bins;
    std::vector<int64_t> used;
    for (size_t i : grp) {  // first fit, widest first
      const int64_t w = cdiv(ph1_out(i).N, 16) * 16;
      size_t k = 0;
      while (k < bins.size() && (used[k] + w > max_ntile || bins[k].size() >= 16)) ++k;
      if (k == bins.size()) {
        bins.emplace_back();
        used.push_back(0);
      }
      bins[k].push_back(i);
      used[k] += w;
    }
    for (size_t k = 0; k < bins.size(); ++k) {
      std::vector<TcSeg> sg;
      std::vector<TcOut> so;
      uint64_t cmap = 0;
      int32_t col = 0, ra = 0;
      const TcOut o0 = ph1_out(bins[k][0]);
      for (size_t pi = 0; pi < bins[k].size(); ++pi) {
        const size_t i = bins[k][pi];
        const TcOut o = ph1_out(i);
        TcSeg g = ph1_seg(i);
        check(o.M == o0.M && o.Rm == o0.Rm && g.kchunks == ph1_seg(bins[k][0]).kchunks &&
                  g.l == ph1_seg(bins[k][0]).l, "pieces share L");
        check(g.r_atoms == cdiv(o.N, 8) && g.l_atoms == cdiv(o.M, 8), "piece operand rows");
        g.col0 = col;
        g.ra = (int32_t)cdiv(o.N, 8);
        const int32_t w = (int32_t)cdiv(o.N, 16) * 16;
        for (int32_t cc = col / 16; cc < (col + w) / 16; ++cc) cmap |= (uint64_t)pi << (4 * cc);
        col += w;
        ra += g.ra;
        sg.push_back(g);
        so.push_back(o);
      }
      check(col <= max_ntile && col % 16 == 0 && col <= 256, "pieced tile width");
      const int32_t s0 = (int32_t)L1.segs.size();
      L1.segs.insert(L1.segs.end(), sg.begin(), sg.end());
      L1.seg_outs.insert(L1.seg_outs.end(), so.begin(), so.end());
      const int32_t s1 = (int32_t)L1.segs.size();
      const int oid = (int)L1.outs.size();
      L1.outs.push_back(o0);
      for (int32_t m0 = 0; m0 < o0.M; m0 += 128) {
        TcTile t{};
        t.m0 = m0;
        t.n0 = 0;
        t.ntile = col;
        t.la = (int32_t)std::min<int64_t>(16, cdiv(o0.M - m0, 8));
        t.ra = ra;
        t.seg_begin = s0;
        t.seg_end = s1;
        t.out = oid;
        t.slot_used = 1;
        t.pieced = 1;
        t.cmap_lo = (uint32_t)cmap;
        t.cmap_hi = (uint32_t)(cmap >> 32);
        t.o = o0;
        check(t.m0 / 8 + t.la <= cdiv(o0.M, 8), "tile past its panels");
        L1.acc_cols = std::max(L1.acc_cols, col);
        L1.ntile_max = std::max(L1.ntile_max, col);
        L1.tiles.push_back(t);
        L1.weight.push_back((int64_t)sg[0].kchunks * col + 64);
      }
    }
  }
  // groups E and S per output sector
  for (int s = 0; s < S; ++s) {
    if ((int64_t)r[s] * c[s] == 0) continue;
    std::vector<TcSeg> sE, sS;
    std::vector<int> tE, tS;  // terms of slots 1, 2, ...
    if (pF[(size_t)s * 2].off >= 0) sE.push_back(seg(psiP[s], pF[(size_t)s * 2]));          // folded 1 (x) B terms
    if (pF[(size_t)s * 2 + 1].off >= 0) sS.push_back(seg(psiPT[s], pF[(size_t)s * 2 + 1]));  // folded A (x) 1 terms
    for (size_t i : by_out[s]) {
      const EPair& e = P[i];
      if (folded[i]) continue;
      if (e.flags & DMRG_ID_A) {
        TcSeg g = slot_of[i] ? seg(psiP[e.s_in], pB[i]) : seg(pS[i], pB[i]);
        g.slot = slot_of[i];
        if (g.slot && (int)tE.size() < g.slot) tE.resize(g.slot, -1);
        if (g.slot) tE[g.slot - 1] = e.term;
        sE.push_back(g);
      } else if (e.flags & DMRG_ID_B) {
        TcSeg g = slot_of[i] ? seg(psiPT[e.s_in], pA[i]) : seg(pS[i], pA[i]);
        g.slot = slot_of[i];
        if (g.slot && (int)tS.size() < g.slot) tS.resize(g.slot, -1);
        if (g.slot) tS[g.slot - 1] = e.term;
        sS.push_back(g);
      } else if (e.order == 0) {
        sE.push_back(seg(pX[i], pB[i]));
      } else {
        sS.push_back(seg(pX[i], pA[i]));
      }
    }
    const bool hasE = !sE.empty(), hasS = !sS.empty();
    if (hasE || !hasS) {
      TcOut o{};
      o.kind = OUT_Y_ROW;
      o.Rm = (int32_t)pad8(r[s]);
      o.Rv = r[s];
      o.M = (int32_t)(nb * o.Rm);
      o.N = c[s];
      o.ldy = c[s];
      o.add = 0;
      o.term = -1;
      o.y_off = sb->off[s];
      add_out(LE, o, sE, tE);
    }
    if (hasS) {
      TcOut o{};
      o.kind = OUT_Y_COL;
      o.Rm = (int32_t)pad8(c[s]);
      o.Rv = c[s];
      o.M = (int32_t)(nb * o.Rm);
      o.N = r[s];
      o.ldy = c[s];
      o.add = hasE ? 1 : 0;
      o.term = -1;
      o.y_off = sb->off[s];
      add_out(LS, o, sS, tS);
    }
  }
  auto finish = [&](Build& B, Launch& L) {
    // heaviest first, dealt round-robin over the persistent CTAs, by groups of
    // the tiles of one output and first row: the N tiles of a row of tiles
    // share their L operand tiles, the rows of one output their R operands, so
    // a group's tiles (and the rows of one output, of equal group weight) stay
    // neighbours in the order and run on neighbouring CTAs at about the same
    // time, where the second read of a shared operand tile hits L2
    std::vector<size_t> perm(B.tiles.size());
    for (size_t i = 0; i < perm.size(); ++i) perm[i] = i;
    if (tune.heavy_first) {
      std::map<std::pair<int, int>, int64_t> gw;
      for (size_t i = 0; i < B.tiles.size(); ++i) gw[{B.tiles[i].out, B.tiles[i].m0}] += B.weight[i];
      std::vector<int64_t> w(B.tiles.size());
      for (size_t i = 0; i < B.tiles.size(); ++i) w[i] = gw[{B.tiles[i].out, B.tiles[i].m0}];
      std::stable_sort(perm.begin(), perm.end(), [&](size_t a, size_t b) { return w[a] > w[b]; });
      // CTA c takes positions c, c + G, c + 2G, ... (G CTAs): reversing every
      // second round of G deals the sorted tiles back and forth (a snake), so
      // that no CTA takes the heavier tile of every round
      const size_t G = (size_t)std::max(1, std::min(n_sms, (int)perm.size()));
      for (size_t r0 = G; r0 < perm.size(); r0 += 2 * G)
        std::reverse(perm.begin() + r0, perm.begin() + std::min(perm.size(), r0 + G));
    }
    std::vector<TcTile> t(B.tiles.size());
    for (size_t i = 0; i < perm.size(); ++i) t[i] = B.tiles[perm[i]];
    L.tiles = up(t);
    // tiles are built output by output: record where each output starts
    L.tiles_by_out = up(B.tiles);
    L.out_begin.assign(1, 0);
    for (size_t i = 1; i < B.tiles.size(); ++i)
      if (B.tiles[i].out != B.tiles[i - 1].out) L.out_begin.push_back((int)i);
    L.out_begin.push_back((int)B.tiles.size());
    L.segs = up(B.segs);
    L.seg_outs = up(B.seg_outs);
    L.n_tiles = (int)t.size();
    L.ntile_max = B.ntile_max;
    L.acc_cols = B.acc_cols;
    L.has_row_out = false;
    L.has_panel_out = false;
    for (const TcOut& o : B.outs) {
      L.has_row_out = L.has_row_out || o.kind == OUT_Y_ROW;
      L.has_panel_out = L.has_panel_out || o.kind == OUT_PANEL;
    }
  };
  finish(L1, out.ph1);
  finish(LE, out.grpE);
  finish(LS, out.grpS);
  out.stage_tiles = up(stiles);
  out.stage_outs = up(souts);
  out.n_stage_tiles = (int)stiles.size();
  out.p_lo = lo_delta;
  return cur - base_off;
}

static State* st_of(const dmrg_sb* sb) { return static_cast<State*>(sb->tc); }

void tc_free(dmrg_sb* sb) {
  State* s = st_of(sb);
  if (!s) return;
  for (Fmt& f : s->f) {
    free_set(f.fwd);
    free_set(f.bwd);
    if (f.arena) cudaFree(f.arena);
  }
  delete s;
  sb->tc = nullptr;
}

bool tc_available(const dmrg_sb* sb) {
  const State* s = st_of(sb);
  return s && s->ok;
}

double tc_operand_bytes(const dmrg_sb* sb) {
  const State* s = st_of(sb);
  return s ? s->op_bytes_tf32 : 0.0;
}

static void build_fmt(dmrg_sb* sb, State* s, int fi);

// Coefficients are read from the shared table at run time, except those of
// identity terms uniform over the batch, folded into operator panels at build
// time: the panels are rebuilt when the set of such terms or their values
// change.  Returns true when it rebuilt (captured graphs then hold stale task
// lists).
bool tc_set_coeffs(dmrg_sb* sb) {
  State* s = st_of(sb);
  if (!s || !s->ok) return false;
  const int nt = sb->n_terms;
  const int64_t nb = sb->batch;
  auto uniform = [&](const std::vector<double>& cf, int term) {
    for (int64_t b = 1; b < nb; ++b)
      if (cf[(size_t)b * nt + term] != cf[term]) return false;
    return true;
  };
  bool rebuilt = false;
  for (int fi = 0; fi < 2; ++fi) {
    const Fmt& F = s->f[fi];
    if (!F.built) continue;  // built later with the coefficients current then
    bool same = true;
    for (int k = 0; k < nt && same; ++k) {
      const bool uo = uniform(F.built_coeffs, k), un = uniform(sb->coeffs, k);
      same = uo == un && (!uo || F.built_coeffs[k] == sb->coeffs[k]);
    }
    if (same) continue;
    build_fmt(sb, s, fi);
    rebuilt = true;
  }
  return rebuilt;
}

void tc_prepare(dmrg_sb* sb, int prec) {
  State* s = st_of(sb);
  if (!s || !s->ok) return;
  const int fi = prec == DMRG_TF32 ? 0 : 1;
  if (!s->f[fi].built) build_fmt(sb, s, fi);
}

int tc_launches(const dmrg_sb* sb, int prec) {
  const State* s = st_of(sb);
  if (!s || !s->ok) return 0;
  const PairSet& ps = s->f[prec == DMRG_TF32 ? 0 : 1].fwd;
  return (ps.n_stage_tiles > 0) + (ps.ph1.n_tiles > 0) + (ps.grpE.n_tiles > 0) + (ps.grpS.n_tiles > 0);
}

// (Re)build the panels and task lists of one precision with its tuning.
static void build_fmt(dmrg_sb* sb, State* s, int fi) {
  const int prec = fi == 0 ? DMRG_TF32 : DMRG_BF16X3;
  Fmt& F = s->f[fi];
  free_set(F.fwd);
  free_set(F.bwd);
  if (F.arena) cudaFree(F.arena);
  F = Fmt{};
  // sizes depend only on shapes: a dry run lays the arena out first
  std::vector<uint8_t> hi, lo;
  {
    PairSet none;
    const int64_t a = build_set(sb, prec, s->fw, 0, hi, lo, nullptr, 0, none, true, s->tune[fi], s->num_sms);
    const int64_t b2 = build_set(sb, prec, s->bw, a, hi, lo, nullptr, 0, none, true, s->tune[fi], s->num_sms);
    F.bytes = (size_t)(a + b2);
  }
  const size_t total = F.bytes * (prec == DMRG_BF16X3 ? 2 : 1);
  TCK(cudaMalloc(&F.arena, std::max<size_t>(total, 1024)));
  TCK(cudaMemset(F.arena, 0, std::max<size_t>(total, 1024)));
  const int64_t lo_delta = prec == DMRG_BF16X3 ? (int64_t)F.bytes : 0;
  const int64_t a = build_set(sb, prec, s->fw, 0, hi, lo, F.arena, lo_delta, F.fwd, false, s->tune[fi], s->num_sms);
  build_set(sb, prec, s->bw, a, hi, lo, F.arena, lo_delta, F.bwd, false, s->tune[fi], s->num_sms);
  TCK(cudaMemcpy(F.arena, hi.data(), hi.size(), cudaMemcpyHostToDevice));
  if (prec == DMRG_BF16X3) TCK(cudaMemcpy(F.arena + lo_delta, lo.data(), lo.size(), cudaMemcpyHostToDevice));
  F.built_coeffs = sb->coeffs;
  F.built = true;
}

void tc_build(dmrg_sb* sb) {
  int dev = 0;
  TCK(cudaGetDevice(&dev));
  cudaDeviceProp prop{};
  TCK(cudaGetDeviceProperties(&prop, dev));
  State* s = new State();
  sb->tc = s;
  s->num_sms = prop.multiProcessorCount;
  if (prop.major != 10) return;  // tcgen05 is a Blackwell datacenter feature
  // forward and transposed pair lists with host blocks (kept for re-tuning)
  s->host_ops = sb->h_ops;
  const double* H = s->host_ops.data();
  s->trans.reserve(sb->pairs.size() * 2);
  for (const PairH& p : sb->pairs) {
    EPair e{p.term, p.s_out, p.s_in, p.flags, p.order, p.a_off >= 0 ? H + p.a_off : nullptr,
            p.b_off >= 0 ? H + p.b_off : nullptr};
    s->fw.push_back(e);
    const int64_t ro = sb->r[p.s_out], ri = sb->r[p.s_in], co = sb->c[p.s_out], ci = sb->c[p.s_in];
    EPair t{p.term, p.s_in, p.s_out, p.flags, 0, nullptr, nullptr};
    if (p.a_off >= 0) {
      s->trans.emplace_back(ri * ro);
      for (int64_t i = 0; i < ro; ++i)
        for (int64_t j = 0; j < ri; ++j) s->trans.back()[j * ro + i] = H[p.a_off + i * ri + j];
      t.A = s->trans.back().data();
    }
    if (p.b_off >= 0) {
      s->trans.emplace_back(ci * co);
      for (int64_t i = 0; i < co; ++i)
        for (int64_t j = 0; j < ci; ++j) s->trans.back()[j * co + i] = H[p.b_off + i * ci + j];
      t.B = s->trans.back().data();
    }
    if (!(p.flags & (DMRG_ID_A | DMRG_ID_B))) {
      // transposed pair: r_out' = ri, r_in' = ro, c_out' = ci, c_in' = co
      const double c0 = 2.0 * ri * ro * co + 2.0 * ri * co * ci;
      const double c1 = 2.0 * ro * co * ci + 2.0 * ri * ro * ci;
      t.order = c0 <= c1 ? 0 : 1;
    }
    s->bw.push_back(t);
  }
  // the panels of a precision are built at its first use (tc_prepare); the
  // TF32 layout's operand bytes come from a dry run of its forward set
  {
    std::vector<uint8_t> hi, lo;
    PairSet none;
    s->op_bytes_tf32 = (double)build_set(sb, DMRG_TF32, s->fw, 0, hi, lo, nullptr, 0, none, true, s->tune[0],
                                         s->num_sms);
  }
  TCK(cudaFuncSetAttribute(tc_gemm_kernel<DMRG_TF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
  TCK(cudaFuncSetAttribute(tc_gemm_kernel<DMRG_BF16X3>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
  s->ok = true;
}

// ------------------------------------------------------------- launching
template <int PREC>
static void run_gemm(const State* s, const Launch& L, double* y, const dmrg_sb* sb, int accumulate,
                     const int32_t* skip, const int32_t* member_done, cudaStream_t st) {
  if (L.n_tiles == 0) return;
  const int r_tile = L.ntile_max * PANEL_ROW_BYTES;
  const int stage_bytes = (L_TILE_BYTES + r_tile) * (PREC == DMRG_TF32 ? 1 : 2);
  // epilogue staging: row-major float64 outputs, panel transposes
  const int epi = L.has_row_out ? EPI_BYTES : L.has_panel_out ? PANEL_EPI_BYTES : 0;
  const int fixed = TC_CTRL_BYTES + epi + 1024;        // control, epilogue staging, ring alignment
  const int avail = 227 * 1024 - fixed;
  const int stages = std::max(1, std::min(8, avail / stage_bytes));
  const int smem = fixed + stages * stage_bytes;
  if (smem > 227 * 1024) throw CudaFail("tensor-core tile does not fit in shared memory");
  // accumulator buffers: three where they fit in the 512 TMEM columns (so
  // that three tiles' epilogues can run at once), else two; launches of many
  // small tiles split the epilogue warps by tile, the others by column
  const int n_acc = 3 * L.acc_cols <= 512 ? 3 : 2;
  const int tile_split = (L.n_tiles >= 6 * s->num_sms && n_acc == 3) ? 1 : 0;
  int tmem_cols = 32;  // power of two holding the accumulator buffers
  while (tmem_cols < n_acc * L.acc_cols) tmem_cols *= 2;
  if (s->tune[PREC == DMRG_TF32 ? 0 : 1].per_block) {
    // baseline for the autotuner's report: one launch per output block
    for (size_t o = 0; o + 1 < L.out_begin.size(); ++o) {
      const int b0 = L.out_begin[o], n = L.out_begin[o + 1] - b0;
      tc_gemm_kernel<PREC><<<std::min(n, s->num_sms), TC_THREADS, smem, st>>>(
          L.tiles_by_out + b0, n, L.segs, L.seg_outs, y, sb->D, sb->d_coeffs, sb->n_terms, sb->batch * sb->n_terms, accumulate, skip,
          member_done, sb->d_tc_err, stages, stage_bytes, r_tile, tmem_cols, epi, L.acc_cols, n_acc, 0, sb->test_stall);
    }
    return;
  }
  const int grid = std::min(L.n_tiles, s->num_sms);
  tc_gemm_kernel<PREC><<<grid, TC_THREADS, smem, st>>>(L.tiles, L.n_tiles, L.segs, L.seg_outs, y, sb->D,
                                                       sb->d_coeffs, sb->n_terms, sb->batch * sb->n_terms,
                                                       accumulate, skip, member_done,
                                                       sb->d_tc_err, stages, stage_bytes, r_tile, tmem_cols, epi,
                                                       L.acc_cols, n_acc, tile_split, sb->test_stall);
}

template <int PREC, class TIn>
static void run_set(const State* s, const PairSet& ps, const TIn* x, double* y, const dmrg_sb* sb,
                    int accumulate, const int32_t* skip, cudaStream_t st, const int32_t* member_done = nullptr) {
  if (ps.n_stage_tiles > 0)
    tc_stage_kernel<PREC, TIn><<<dim3((unsigned)ps.n_stage_tiles, sb->batch), 256, 0, st>>>(
        ps.stage_tiles, ps.stage_outs, x, sb->D, ps.p_lo, sb->d_coeffs, sb->n_terms, skip, member_done);
  run_gemm<PREC>(s, ps.ph1, y, sb, 0, skip, member_done, st);
  run_gemm<PREC>(s, ps.grpE, y, sb, accumulate, skip, member_done, st);
  run_gemm<PREC>(s, ps.grpS, y, sb, accumulate, skip, member_done, st);
}

// Time the product under each candidate tuning on this superblock and keep
// the fastest (median of `reps` launches after a warm-up, CUDA events on the
// caller's stream).  Also times the per-block launch baseline.
void tc_autotune(dmrg_sb* sb, int prec, int reps, cudaStream_t st, double* out) {
  State* s = st_of(sb);
  if (!s || !s->ok) throw CudaFail("tensor-core path unavailable");
  const int fi = prec == DMRG_TF32 ? 0 : 1;
  const int64_t n = sb->D * sb->batch;
  double *x = nullptr, *y = nullptr;
  TCK(cudaMalloc(&x, n * sizeof(double)));
  TCK(cudaMalloc(&y, n * sizeof(double)));
  TCK(cudaMemsetAsync(x, 0, n * sizeof(double), st));
  cudaEvent_t e0, e1;
  TCK(cudaEventCreate(&e0));
  TCK(cudaEventCreate(&e1));
  auto time_it = [&]() {
    std::vector<float> ms;
    for (int w = 0; w < 2; ++w) tc_matvec(sb, prec, x, y, 0, nullptr, st);
    for (int r = 0; r < std::max(1, reps); ++r) {
      TCK(cudaEventRecord(e0, st));
      tc_matvec(sb, prec, x, y, 0, nullptr, st);
      TCK(cudaEventRecord(e1, st));
      TCK(cudaEventSynchronize(e1));
      float t = 0;
      TCK(cudaEventElapsedTime(&t, e0, e1));
      ms.push_back(t);
    }
    std::sort(ms.begin(), ms.end());
    return (double)ms[ms.size() / 2];
  };
  const std::vector<int> widths = {64, 128, 256};
  const Tune start = s->tune[fi];
  Tune best = start;
  double best_ms = 1e30, default_ms = 0;
  int tried = 0;
  for (int w : widths)
    for (int hf : {1, 0})
      for (int pc : {1, 0}) {
        s->tune[fi] = Tune{w, hf, 0, pc};
        build_fmt(sb, s, fi);
        const double t = time_it();
        ++tried;
        if (w == (prec == DMRG_TF32 ? 256 : 128) && hf == 1 && pc == 1) default_ms = t;
        if (t < best_ms) { best_ms = t; best = s->tune[fi]; }
      }
  s->tune[fi] = best;
  s->tune[fi].per_block = 1;
  build_fmt(sb, s, fi);
  const double per_block_ms = time_it();
  s->tune[fi].per_block = 0;
  TCK(cudaStreamSynchronize(st));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(x);
  cudaFree(y);
  out[0] = best_ms;
  out[1] = default_ms;
  out[2] = per_block_ms;
  out[3] = best.max_ntile;
  out[4] = best.heavy_first;
  out[5] = tried;
  out[6] = best.pieces;
  (void)start;
}

void tc_matvec(dmrg_sb* sb, int prec, const double* x, double* y, int accumulate, const int32_t* skip,
               cudaStream_t st, const int32_t* member_done) {
  tc_prepare(sb, prec);
  const State* s = st_of(sb);
  if (!s || !s->ok) throw CudaFail("tensor-core path unavailable");
  if (prec == DMRG_TF32) run_set<DMRG_TF32>(s, s->f[0].fwd, x, y, sb, accumulate, skip, st, member_done);
  else run_set<DMRG_BF16X3>(s, s->f[1].fwd, x, y, sb, accumulate, skip, st, member_done);
  sb->test_stall = 0;  // the hook applies to one product
}

void tc_matvec_f32in(dmrg_sb* sb, int prec, const float* x, double* y, int accumulate, const int32_t* skip,
                     cudaStream_t st, const int32_t* member_done) {
  tc_prepare(sb, prec);
  const State* s = st_of(sb);
  if (!s || !s->ok) throw CudaFail("tensor-core path unavailable");
  if (prec == DMRG_TF32) run_set<DMRG_TF32>(s, s->f[0].fwd, x, y, sb, accumulate, skip, st, member_done);
  else run_set<DMRG_BF16X3>(s, s->f[1].fwd, x, y, sb, accumulate, skip, st, member_done);
  sb->test_stall = 0;
}

void tc_matvec_T(dmrg_sb* sb, int prec, const double* g, double* dpsi, cudaStream_t st) {
  tc_prepare(sb, prec);
  const State* s = st_of(sb);
  if (!s || !s->ok) throw CudaFail("tensor-core path unavailable");
  if (prec == DMRG_TF32) run_set<DMRG_TF32>(s, s->f[0].bwd, g, dpsi, sb, 0, nullptr, st);
  else run_set<DMRG_BF16X3>(s, s->f[1].bwd, g, dpsi, sb, 0, nullptr, st);
}

}  // namespace dmrg
