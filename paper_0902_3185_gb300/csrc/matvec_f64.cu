// Grouped FP64 sector GEMM: every (term, sector pair) product of the
// superblock Hamiltonian in one launch, on the CUDA cores in float64.
//
// Paper Sec. 3.3: the product x += H y is done per symmetry block, on the
// fly, as system, environment and connection parts.  Here each output tile
// of a block Y_s (or of an intermediate A Psi / Psi B^T) walks over a list of
// segments, each a plain product L (M x K) * R (K x N) with its own layout
// and coefficient, and accumulates them in registers.  One tile writes each
// output element exactly once, so results do not depend on scheduling.
//
// Tiles of 16*ni x 16*nj (ni, nj in 1..4, chosen per output so that the
// sector blocks -- 1..80 wide in a DMRG superblock -- fill them), K step 16
// with the last step cut to the true K, 256 threads with an ni x nj register
// block each (rows ty + 16 i, cols tx + 16 j).  GB300 runs float64 at 1/64 of
// its FP32 rate (2 DFMA per clock per SM), so this kernel is bound by DFMA
// issue, not by memory, and the FMAs it spends on padding are the loss to
// avoid; batch members that share operator blocks are stacked along M or N.

#include "internal.h"

namespace dmrg {

constexpr int F64_BMAX = 64, F64_BK = 16, F64_THREADS = 256;

struct F64Smem {
  double L[F64_BK][F64_BMAX + 1];
  double R[F64_BK][F64_BMAX + 1];
  double red[F64_THREADS / 32];
};
struct F64DotSmem {  // column partials of TM_STORE_DOTS tiles with members along N
  double col[16][F64_BMAX + 1];
};

template <int NI, int NJ, bool DOTS>
__device__ __forceinline__ void f64_tile(const TileF64& t, const SegF64* __restrict__ segs, const Bufs& bufs,
                                         const double* __restrict__ coef, int n_terms, int accumulate,
                                         double* __restrict__ dot_out, F64Smem& sm, F64DotSmem* dsm) {
  constexpr int BM = 16 * NI, BN = 16 * NJ;
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  double acc[NI][NJ];
#pragma unroll
  for (int i = 0; i < NI; ++i)
#pragma unroll
    for (int j = 0; j < NJ; ++j) acc[i][j] = 0.0;
  // element offset of C(m, n) with the members stacked along M or N
  auto coff = [&](int m, int n) -> int64_t {
    int b = 0;
    if (t.c_rm) {
      if (t.c_axis == 0) { b = m / t.c_rm; m -= b * t.c_rm; }
      else { b = n / t.c_rm; n -= b * t.c_rm; }
    }
    return (int64_t)b * t.c_bs + (t.c_trans ? (int64_t)n * t.ldc + m : (int64_t)m * t.ldc + n);
  };
  // TM_STORE_DOTS: each segment accumulates alone (sacc), is dotted with the
  // wavefunction at the output's place (xo) -- per tile row, or per tile
  // column when the members are stacked along N -- and is then added with
  // the coefficient of each element's member
  const bool by_col = t.c_rm && t.c_axis == 1;
  double sacc[DOTS ? NI : 1][DOTS ? NJ : 1];
  // member of each of this thread's rows / columns, and the offsets of its
  // output elements split as roff[i] + coffj[j] (-1: outside the output)
  int mrow[DOTS ? NI : 1], mcol[DOTS ? NJ : 1];
  int64_t roff[DOTS ? NI : 1], coffj[DOTS ? NJ : 1];
  const double* X = bufs.p[BUF_X] + t.c_off;
  if (DOTS) {
#pragma unroll
    for (int i = 0; i < NI; ++i) {
      const int m = t.m0 + ty + 16 * i;
      const int b = (t.c_rm && t.c_axis == 0) ? m / t.c_rm : 0;
      mrow[DOTS ? i : 0] = t.c_rm ? b : t.member;
      roff[DOTS ? i : 0] = m < t.M ? (int64_t)b * t.c_bs + (int64_t)(m - b * t.c_rm) * t.ldc : -1;
    }
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      const int n = t.n0 + tx + 16 * j;
      const int b = by_col ? n / t.c_rm : 0;
      mcol[DOTS ? j : 0] = b;
      coffj[DOTS ? j : 0] = n < t.N ? (int64_t)b * t.c_bs + (n - b * t.c_rm) : -1;
    }
  }
  // the wavefunction at this thread's output element (i, j), 0 outside
  auto xo = [&](int i, int j) -> double {
    const int64_t r = roff[DOTS ? i : 0], c = coffj[DOTS ? j : 0];
    return (r >= 0 && c >= 0) ? X[r + c] : 0.0;
  };

  for (int sg = t.seg_begin; sg < t.seg_end; ++sg) {
    const SegF64 s = segs[sg];
    if (DOTS) {
#pragma unroll
      for (int i = 0; i < NI; ++i)
#pragma unroll
        for (int j = 0; j < NJ; ++j) sacc[DOTS ? i : 0][DOTS ? j : 0] = 0.0;
    }
    const double* L = bufs.p[s.l_buf] + s.l_off;
    const double* R = bufs.p[s.r_buf] + s.r_off;
    const double uscale = (s.coef_mode == 0 && s.coef >= 0) ? coef[s.coef] : 1.0;
    for (int k0 = 0; k0 < s.K; k0 += F64_BK) {
#pragma unroll
      for (int e = 0; e < NI; ++e) {  // BM x BK elements, 256 per pass
        const int idx = tid + e * F64_THREADS;
        int m, k;
        if (s.l_trans) { k = idx / BM; m = idx % BM; }
        else { m = idx / F64_BK; k = idx % F64_BK; }
        const int gm = t.m0 + m, gk = k0 + k;
        double v = 0.0;
        if (gm < t.M && gk < s.K) {
          int bl = 0, mm = gm;
          if (s.l_rm) { bl = gm / s.l_rm; mm = gm - bl * s.l_rm; }
          const double* Lb = L + (int64_t)bl * s.l_bs;
          v = s.l_trans ? Lb[(int64_t)gk * s.ldl + mm] : Lb[(int64_t)mm * s.ldl + gk];
          v *= s.coef_mode == 1 ? coef[bl * n_terms + s.coef] : uscale;
        }
        sm.L[k][m] = v;
      }
#pragma unroll
      for (int e = 0; e < NJ; ++e) {  // BN x BK elements
        const int idx = tid + e * F64_THREADS;
        int n, k;
        if (s.r_trans) { n = idx / F64_BK; k = idx % F64_BK; }
        else { k = idx / BN; n = idx % BN; }
        const int gn = t.n0 + n, gk = k0 + k;
        double v = 0.0;
        if (gn < t.N && gk < s.K) {
          int br = 0, nn = gn;
          if (s.r_rm) { br = gn / s.r_rm; nn = gn - br * s.r_rm; }
          const double* Rb = R + (int64_t)br * s.r_bs;
          v = s.r_trans ? Rb[(int64_t)nn * s.ldr + gk] : Rb[(int64_t)gk * s.ldr + nn];
          if (s.coef_mode == 2) v *= coef[br * n_terms + s.coef];
        }
        sm.R[k][n] = v;
      }
      __syncthreads();
      const int kmax = min(F64_BK, s.K - k0);
      auto step = [&](int k) {
        double a[NI], b[NJ];
#pragma unroll
        for (int i = 0; i < NI; ++i) a[i] = sm.L[k][ty + 16 * i];
#pragma unroll
        for (int j = 0; j < NJ; ++j) b[j] = sm.R[k][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < NI; ++i)
#pragma unroll
          for (int j = 0; j < NJ; ++j) {
            if (DOTS) sacc[DOTS ? i : 0][DOTS ? j : 0] = fma(a[i], b[j], sacc[DOTS ? i : 0][DOTS ? j : 0]);
            else acc[i][j] = fma(a[i], b[j], acc[i][j]);
          }
      };
      if (kmax == F64_BK) {
#pragma unroll
        for (int k = 0; k < F64_BK; ++k) step(k);
      } else {
        for (int k = 0; k < kmax; ++k) step(k);  // no FMAs on the zero padding of K
      }
      __syncthreads();
    }
    if (DOTS) {  // this segment's dots with the wavefunction, then its coefficients
      const int ql = sg - t.seg_begin;
      double* out = dot_out + (int64_t)(t.dot_base + ql) * F64_BMAX;
      if (!by_col) {
        // row partials: the 16 threads of a row are 16 consecutive lanes
#pragma unroll
        for (int i = 0; i < NI; ++i) {
          double part = 0.0;
#pragma unroll
          for (int j = 0; j < NJ; ++j) part = fma(sacc[DOTS ? i : 0][DOTS ? j : 0], xo(i, j), part);
#pragma unroll
          for (int o = 8; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
          if (tx == 0) out[ty + 16 * i] = part;
          const double cf = coef[mrow[DOTS ? i : 0] * n_terms + s.coef];
#pragma unroll
          for (int j = 0; j < NJ; ++j) acc[i][j] = fma(cf, sacc[DOTS ? i : 0][DOTS ? j : 0], acc[i][j]);
        }
      } else {
        // column partials: the 16 threads of a column sit in different warps
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
          double part = 0.0;
#pragma unroll
          for (int i = 0; i < NI; ++i) part = fma(sacc[DOTS ? i : 0][DOTS ? j : 0], xo(i, j), part);
          dsm->col[ty][tx + 16 * j] = part;
          const double cf = coef[mcol[DOTS ? j : 0] * n_terms + s.coef];
#pragma unroll
          for (int i = 0; i < NI; ++i) acc[i][j] = fma(cf, sacc[DOTS ? i : 0][DOTS ? j : 0], acc[i][j]);
        }
        __syncthreads();
        if (tid < BN) {
          double tot = 0.0;
#pragma unroll
          for (int y2 = 0; y2 < 16; ++y2) tot += dsm->col[y2][tid];
          out[tid] = tot;
        }
        __syncthreads();
      }
    }
  }

  double* C = bufs.p[t.c_buf] + t.c_off;
  if (t.mode == TM_STORE || t.mode == TM_STORE_DOTS) {
    const bool add = accumulate || t.add;
#pragma unroll
    for (int i = 0; i < NI; ++i) {
      const int m = t.m0 + ty + 16 * i;
      if (m >= t.M) continue;
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        const int n = t.n0 + tx + 16 * j;
        if (n >= t.N) continue;
        double* p = C + coff(m, n);
        *p = add ? *p + acc[i][j] : acc[i][j];
      }
    }
  } else {  // TM_DOT: sum over the tile of acc .* C, fixed-order block reduction
    double part = 0.0;
#pragma unroll
    for (int i = 0; i < NI; ++i) {
      const int m = t.m0 + ty + 16 * i;
      if (m >= t.M) continue;
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        const int n = t.n0 + tx + 16 * j;
        if (n >= t.N) continue;
        part = fma(acc[i][j], C[coff(m, n)], part);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
    if ((tid & 31) == 0) sm.red[tid >> 5] = part;
    __syncthreads();
    if (tid == 0) {
      double tot = 0.0;
      for (int w = 0; w < F64_THREADS / 32; ++w) tot += sm.red[w];
      dot_out[blockIdx.x] = tot;
    }
  }
}

__global__ void __launch_bounds__(F64_THREADS, 3)
seg_gemm_f64_kernel(const TileF64* __restrict__ tiles, const SegF64* __restrict__ segs,
                    Bufs bufs, const double* __restrict__ coef, int n_terms, int accumulate,
                    double* __restrict__ dot_out, const int32_t* __restrict__ skip) {
  __shared__ F64Smem sm;
  if (skip && *skip) return;
  const TileF64 t = tiles[blockIdx.x];
#define F64_CASE(I, J) \
  case (I) | ((J) << 8): f64_tile<I, J, false>(t, segs, bufs, coef, n_terms, accumulate, dot_out, sm, nullptr); break;
  switch (t.shape) {
    F64_CASE(1, 1) F64_CASE(1, 2) F64_CASE(1, 3) F64_CASE(1, 4)
    F64_CASE(2, 1) F64_CASE(2, 2) F64_CASE(2, 3) F64_CASE(2, 4)
    F64_CASE(3, 1) F64_CASE(3, 2) F64_CASE(3, 3) F64_CASE(3, 4)
    F64_CASE(4, 1) F64_CASE(4, 2) F64_CASE(4, 3) F64_CASE(4, 4)
    default: break;  // the host builds only the shapes above
  }
#undef F64_CASE
}

// Product and per-segment dots in one pass (mode TM_STORE_DOTS): partials
// per (tile, segment, tile row) -- or tile column when the members are
// stacked along N -- at dot_out[(dot_base + segment) * 64 + row or column].
// Three accumulator sets per thread, so fewer blocks per SM.
__global__ void __launch_bounds__(F64_THREADS, 2)
seg_gemm_f64_dots_kernel(const TileF64* __restrict__ tiles, const SegF64* __restrict__ segs, Bufs bufs,
                         const double* __restrict__ coef, int n_terms, int accumulate, double* __restrict__ dot_out,
                         const int32_t* __restrict__ skip) {
  __shared__ F64Smem sm;
  __shared__ F64DotSmem dsm;
  if (skip && *skip) return;
  const TileF64 t = tiles[blockIdx.x];
#define F64_CASE(I, J) \
  case (I) | ((J) << 8): f64_tile<I, J, true>(t, segs, bufs, coef, n_terms, accumulate, dot_out, sm, &dsm); break;
  switch (t.shape) {
    F64_CASE(1, 1) F64_CASE(1, 2) F64_CASE(1, 3) F64_CASE(1, 4)
    F64_CASE(2, 1) F64_CASE(2, 2) F64_CASE(2, 3) F64_CASE(2, 4)
    F64_CASE(3, 1) F64_CASE(3, 2) F64_CASE(3, 3) F64_CASE(3, 4)
    F64_CASE(4, 1) F64_CASE(4, 2) F64_CASE(4, 3) F64_CASE(4, 4)
    default: break;
  }
#undef F64_CASE
}

void launch_seg_gemm_f64_dots(const TaskListF64& tl, const Bufs& bufs, const double* coef, int n_terms,
                              int accumulate, double* dot_out, const int32_t* skip, cudaStream_t st) {
  if (tl.n_tiles == 0) return;
  seg_gemm_f64_dots_kernel<<<(unsigned)tl.n_tiles, F64_THREADS, 0, st>>>(tl.d_tiles, tl.d_segs, bufs, coef, n_terms,
                                                                        accumulate, dot_out, skip);
}

void launch_seg_gemm_f64(const TaskListF64& tl, const Bufs& bufs, const double* coef, int n_terms,
                         int accumulate, double* dot_out, const int32_t* skip, cudaStream_t st) {
  if (tl.n_tiles == 0) return;
  seg_gemm_f64_kernel<<<(unsigned)tl.n_tiles, F64_THREADS, 0, st>>>(
      tl.d_tiles, tl.d_segs, bufs, coef, n_terms, accumulate, dot_out, skip);
}

}  // namespace dmrg
