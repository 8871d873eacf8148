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

template <int NI, int NJ, bool DOTS>
__device__ __forceinline__ void f64_tile(const TileF64& t, const SegF64* __restrict__ segs, const Bufs& bufs,
                                         const double* __restrict__ coef, int n_terms, int accumulate,
                                         double* __restrict__ dot_out, F64Smem& sm) {
  constexpr int BM = 16 * NI, BN = 16 * NJ;
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  double acc[NI][NJ];
#pragma unroll
  for (int i = 0; i < NI; ++i)
#pragma unroll
    for (int j = 0; j < NJ; ++j) acc[i][j] = 0.0;
  // TM_STORE_DOTS: each segment accumulates alone (sacc), is dotted with the
  // wavefunction block at the output's place (xo), then added with its
  // member's coefficient
  double sacc[DOTS ? NI : 1][DOTS ? NJ : 1];
  double xo[DOTS ? NI : 1][DOTS ? NJ : 1];
  if (DOTS) {
    const double* X = bufs.p[BUF_X] + t.c_off;
#pragma unroll
    for (int i = 0; i < NI; ++i)
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        const int m = t.m0 + ty + 16 * i, n = t.n0 + tx + 16 * j;
        xo[DOTS ? i : 0][DOTS ? j : 0] = (m < t.M && n < t.N) ? X[(int64_t)m * t.ldc + n] : 0.0;
      }
  }

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
    if (DOTS) {  // this segment's dot with the wavefunction, then its coefficient
      const double cf = coef[t.member * n_terms + s.coef];
      double part = 0.0;
#pragma unroll
      for (int i = 0; i < NI; ++i)
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
          part = fma(sacc[DOTS ? i : 0][DOTS ? j : 0], xo[DOTS ? i : 0][DOTS ? j : 0], part);
          acc[i][j] = fma(cf, sacc[DOTS ? i : 0][DOTS ? j : 0], acc[i][j]);
        }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
      if ((tid & 31) == 0) sm.red[tid >> 5] = part;
      __syncthreads();
      if (tid == 0) {
        double tot = 0.0;
        for (int w = 0; w < F64_THREADS / 32; ++w) tot += sm.red[w];
        dot_out[t.dot_base + (sg - t.seg_begin)] = tot;
      }
      __syncthreads();
    }
  }

  double* C = bufs.p[t.c_buf] + t.c_off;
  // element offset of C(m, n) with the members stacked along M or N
  auto coff = [&](int m, int n) -> int64_t {
    int b = 0;
    if (t.c_rm) {
      if (t.c_axis == 0) { b = m / t.c_rm; m -= b * t.c_rm; }
      else { b = n / t.c_rm; n -= b * t.c_rm; }
    }
    return (int64_t)b * t.c_bs + (t.c_trans ? (int64_t)n * t.ldc + m : (int64_t)m * t.ldc + n);
  };
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
  case (I) | ((J) << 8): f64_tile<I, J, false>(t, segs, bufs, coef, n_terms, accumulate, dot_out, sm); break;
  switch (t.shape) {
    F64_CASE(1, 1) F64_CASE(1, 2) F64_CASE(1, 3) F64_CASE(1, 4)
    F64_CASE(2, 1) F64_CASE(2, 2) F64_CASE(2, 3) F64_CASE(2, 4)
    F64_CASE(3, 1) F64_CASE(3, 2) F64_CASE(3, 3) F64_CASE(3, 4)
    F64_CASE(4, 1) F64_CASE(4, 2) F64_CASE(4, 3) F64_CASE(4, 4)
    default: break;  // the host builds only the shapes above
  }
#undef F64_CASE
}

// Product and per-segment dots in one pass (tiles of one member, mode
// TM_STORE_DOTS); three accumulator sets per thread, so fewer blocks per SM.
__global__ void __launch_bounds__(F64_THREADS, 2)
seg_gemm_f64_dots_kernel(const TileF64* __restrict__ tiles, const SegF64* __restrict__ segs, Bufs bufs,
                         const double* __restrict__ coef, int n_terms, double* __restrict__ dot_out,
                         const int32_t* __restrict__ skip) {
  __shared__ F64Smem sm;
  if (skip && *skip) return;
  const TileF64 t = tiles[blockIdx.x];
#define F64_CASE(I, J) \
  case (I) | ((J) << 8): f64_tile<I, J, true>(t, segs, bufs, coef, n_terms, 0, dot_out, sm); break;
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
                              double* dot_out, const int32_t* skip, cudaStream_t st) {
  if (tl.n_tiles == 0) return;
  seg_gemm_f64_dots_kernel<<<(unsigned)tl.n_tiles, F64_THREADS, 0, st>>>(tl.d_tiles, tl.d_segs, bufs, coef, n_terms,
                                                                        dot_out, skip);
}

void launch_seg_gemm_f64(const TaskListF64& tl, const Bufs& bufs, const double* coef, int n_terms,
                         int accumulate, double* dot_out, const int32_t* skip, cudaStream_t st) {
  if (tl.n_tiles == 0) return;
  seg_gemm_f64_kernel<<<(unsigned)tl.n_tiles, F64_THREADS, 0, st>>>(
      tl.d_tiles, tl.d_segs, bufs, coef, n_terms, accumulate, dot_out, skip);
}

}  // namespace dmrg
