// Grouped sector GEMM in double-float arithmetic: the float64 product's task
// lists (same tiles, segments and outputs as matvec_f64.cu), with every
// multiply-add done on float32 pairs.
//
// A double-float number is an unevaluated pair hi + lo of float32 values
// (about 48 significant bits).  Inputs are float64; each is split into
// hi = RN24(v) and lo = RN24(v - hi) with integer instructions, products use
// Dekker's splitting-free form with a fused multiply-add (the error of
// hi_a * hi_b is exact, the cross terms are added to it, lo_a * lo_b -- 2^-46
// relative -- is dropped), and sums use Knuth's two-sum, so one multiply-add
// costs 12 float32 operations and has a relative error near 2^-46; the pair
// is renormalised after every K tile of 16 (without it the low sum's own
// rounding grows like K 2^-48: 1e-12 at K = 200).  GB300
// runs float64 at 1/64 of its float32 rate (2 DFMA per clock per SM against
// 128 FFMA), so the arithmetic alone allows five times the float64 kernel's
// rate; with the input splits, the shared-memory tiles and their barriers the
// superblock product runs about twice as fast as the float64 kernel, at an
// accuracy enough for residuals r = H psi - theta psi down to |r| ~ 1e-12 |H psi|.  Outputs are written as
// float64 (hi + lo).  Paper Sec. 3.3: the product x += H y, system,
// environment and connection parts, on the fly.
//
// Buffers flagged in the pair mask hold every element as a float32 pair
// (hi, lo) in its 8-byte slot, already split: the operator arena (split once
// per superblock), the wavefunction (split once per product) and the
// intermediates, which phase 1 writes as its renormalised (s, c) sums (48
// bits, no rounding to float64 between the two GEMMs).  Loads from them skip
// the integer split, which otherwise costs about 28 instructions per loaded
// element per K tile.

#include <algorithm>

#include "df.cuh"
#include "internal.h"
#include "tc_kernel.cuh"

namespace dmrg {

constexpr int DF_BMAX = 64, DF_BK = 16, DF_THREADS = 256;

struct DFSmem {
  float2 L[DF_BK][DF_BMAX + 1];
  float2 R[DF_BK][DF_BMAX + 1];
  double red[DF_THREADS / 32];
};
struct DFDotSmem {
  double col[16][DF_BMAX + 1];
};



// the 8 bytes of a pair slot as (hi, lo): hi is the low word (float2 layout)
__device__ __forceinline__ float2 df_bits(double v) {
  return make_float2(__int_as_float(__double2loint(v)), __int_as_float(__double2hiint(v)));
}
__device__ __forceinline__ double df_slot(float s, float c) {  // (s, c) renormalised into one slot
  const float hi = __fadd_rn(s, c);
  const float lo = __fsub_rn(c, __fsub_rn(hi, s));
  return __hiloint2double(__float_as_int(lo), __float_as_int(hi));
}

template <int NI, int NJ, bool DOTS>
__device__ __forceinline__ void df_tile(const TileF64& t, const SegF64* __restrict__ segs, const Bufs& bufs,
                                        const double* __restrict__ coef, int n_terms, int accumulate,
                                        double* __restrict__ dot_out, DFSmem& sm, DFDotSmem* dsm, uint32_t pm) {
  constexpr int BM = 16 * NI, BN = 16 * NJ;
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  // double-float sums: of the whole tile, or (DOTS) of the current segment
  float s_[NI][NJ], c_[NI][NJ];
#pragma unroll
  for (int i = 0; i < NI; ++i)
#pragma unroll
    for (int j = 0; j < NJ; ++j) s_[i][j] = c_[i][j] = 0.0f;
  auto coff = [&](int m, int n) -> int64_t {
    int b = 0;
    if (t.c_rm) {
      if (t.c_axis == 0) { b = m / t.c_rm; m -= b * t.c_rm; }
      else { b = n / t.c_rm; n -= b * t.c_rm; }
    }
    return (int64_t)b * t.c_bs + (t.c_trans ? (int64_t)n * t.ldc + m : (int64_t)m * t.ldc + n);
  };
  const bool by_col = t.c_rm && t.c_axis == 1;
  const double* X = bufs.p[BUF_X] + t.c_off;
  // DOTS, computed where needed (registers go to the double-float sums): the
  // member of row i / column j and the wavefunction at output element (i, j)
  auto mrow = [&](int i) -> int {
    const int m = t.m0 + ty + 16 * i;
    return (t.c_rm && t.c_axis == 0) ? m / t.c_rm : (t.c_rm ? 0 : t.member);
  };
  auto mcol = [&](int j) -> int { return by_col ? (t.n0 + tx + 16 * j) / t.c_rm : 0; };
  const bool x_pairs = (pm >> BUF_X) & 1u;
  auto xo = [&](int i, int j) -> double {
    const int m = t.m0 + ty + 16 * i, n = t.n0 + tx + 16 * j;
    if (m >= t.M || n >= t.N) return 0.0;
    const double v = X[coff(m, n)];
    if (!x_pairs) return v;
    const float2 p = df_bits(v);
    return df_value(p.x, p.y);
  };

  // DOTS: each segment's coefficient-weighted sum goes straight to the
  // output (written by the first segment, added by the others), which keeps
  // the registers of a float64 accumulator free for the load pipeline
  auto put = [&](int i, int j, double v, bool first) {
    const int m = t.m0 + ty + 16 * i, n = t.n0 + tx + 16 * j;
    if (m >= t.M || n >= t.N) return;
    double* p = bufs.p[t.c_buf] + t.c_off + coff(m, n);
    *p = (first && !(accumulate || t.add)) ? v : *p + v;
  };
  for (int sg = t.seg_begin; sg < t.seg_end; ++sg) {
    const SegF64 s = segs[sg];
    if (DOTS) {
#pragma unroll
      for (int i = 0; i < NI; ++i)
#pragma unroll
        for (int j = 0; j < NJ; ++j) s_[i][j] = c_[i][j] = 0.0f;
    }
    const double* L = bufs.p[s.l_buf] + s.l_off;
    const double* R = bufs.p[s.r_buf] + s.r_off;
    const bool l_pairs = (pm >> s.l_buf) & 1u, r_pairs = (pm >> s.r_buf) & 1u;
    const bool uscaled = s.coef_mode == 0 && s.coef >= 0;
    const float2 uscale = df_split(uscaled ? coef[s.coef] : 1.0);
    // this thread's load slots, fixed over the segment: tile row / column,
    // local k, element offset at k = 0 (-1: outside the output), the K stride
    // and the (member) coefficient as a double-float pair
    constexpr int HI = NI, HJ = NJ;
    int lm[HI], lk[HI], loff[HI];
    float2 lcf[HI];
    const int lks = s.l_trans ? s.ldl : 1;
    int rn_[HJ], rk[HJ], roff_[HJ];
    float2 rcf[HJ];
    const int rks = s.r_trans ? 1 : s.ldr;
    {
#pragma unroll
      for (int e = 0; e < NI; ++e) {
        const int idx = tid + e * DF_THREADS;
        if (s.l_trans) { lk[e] = idx / BM; lm[e] = idx % BM; }
        else { lm[e] = idx / DF_BK; lk[e] = idx % DF_BK; }
        const int gm = t.m0 + lm[e];
        int bl = 0, mm = gm;
        if (s.l_rm) { bl = gm / s.l_rm; mm = gm - bl * s.l_rm; }
        loff[e] = gm < t.M ? (int)((int64_t)bl * s.l_bs + (s.l_trans ? (int64_t)mm : (int64_t)mm * s.ldl)) : -1;
        lcf[e] = s.coef_mode == 1 && gm < t.M ? df_split(coef[bl * n_terms + s.coef]) : uscale;
      }
#pragma unroll
      for (int e = 0; e < NJ; ++e) {
        const int idx = tid + e * DF_THREADS;
        if (s.r_trans) { rn_[e] = idx / DF_BK; rk[e] = idx % DF_BK; }
        else { rk[e] = idx / BN; rn_[e] = idx % BN; }
        const int gn = t.n0 + rn_[e];
        int br = 0, nn = gn;
        if (s.r_rm) { br = gn / s.r_rm; nn = gn - br * s.r_rm; }
        roff_[e] = gn < t.N ? (int)((int64_t)br * s.r_bs + (s.r_trans ? (int64_t)nn * s.ldr : (int64_t)nn)) : -1;
        rcf[e] = s.coef_mode == 2 && gn < t.N ? df_split(coef[br * n_terms + s.coef]) : make_float2(1.0f, 0.0f);
      }
    }
    const bool lscaled = s.coef_mode == 1 || uscaled, rscaled = s.coef_mode == 2;
    // the raw float64 values of the next K tile are loaded before the
    // current tile's multiply-adds (software prefetch)
    double pl[HI], pr[HJ];
    auto fetch = [&](int k0) {
#pragma unroll
      for (int e = 0; e < HI; ++e) {
        const int gk = k0 + lk[e];
        pl[e] = (loff[e] >= 0 && gk < s.K) ? L[loff[e] + (int64_t)gk * lks] : 0.0;
      }
#pragma unroll
      for (int e = 0; e < HJ; ++e) {
        const int gk = k0 + rk[e];
        pr[e] = (roff_[e] >= 0 && gk < s.K) ? R[roff_[e] + (int64_t)gk * rks] : 0.0;
      }
    };
    fetch(0);
    for (int k0 = 0; k0 < s.K; k0 += DF_BK) {
      {
#pragma unroll
        for (int e = 0; e < NI; ++e) {  // BM x BK elements, 256 per pass
          float2 v = l_pairs ? df_bits(pl[e]) : df_split(pl[e]);
          if (lscaled) v = df_mul(v, lcf[e]);
          sm.L[lk[e]][lm[e]] = v;
        }
#pragma unroll
        for (int e = 0; e < NJ; ++e) {  // BN x BK elements
          float2 v = r_pairs ? df_bits(pr[e]) : df_split(pr[e]);
          if (rscaled) v = df_mul(v, rcf[e]);
          sm.R[rk[e]][rn_[e]] = v;
        }
        if (k0 + DF_BK < s.K) fetch(k0 + DF_BK);
      }
      __syncthreads();
      const int kmax = min(DF_BK, s.K - k0);
      auto step = [&](int k) {
        float2 a[NI], b[NJ];
#pragma unroll
        for (int i = 0; i < NI; ++i) a[i] = sm.L[k][ty + 16 * i];
#pragma unroll
        for (int j = 0; j < NJ; ++j) b[j] = sm.R[k][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < NI; ++i)
#pragma unroll
          for (int j = 0; j < NJ; ++j) df_fma(a[i], b[j], s_[i][j], c_[i][j]);
      };
      if (kmax == DF_BK) {
#pragma unroll
        for (int k = 0; k < DF_BK; ++k) step(k);
      } else {
        for (int k = 0; k < kmax; ++k) step(k);  // no work on the zero padding of K
      }
      // renormalise (fast two-sum, |c| << |s|): c restarts near ulp(s) / 2,
      // so its own rounding stays near 2^-48 |s| per K step of the next tile
#pragma unroll
      for (int i = 0; i < NI; ++i)
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
          const float t2 = __fadd_rn(s_[i][j], c_[i][j]);
          c_[i][j] = __fsub_rn(c_[i][j], __fsub_rn(t2, s_[i][j]));
          s_[i][j] = t2;
        }
      __syncthreads();
    }
    if (DOTS) {  // this segment's dots with the wavefunction (float64), then its coefficients
      const int ql = sg - t.seg_begin;
      double* out = dot_out + (int64_t)(t.dot_base + ql) * DF_BMAX;
      if (!by_col) {
#pragma unroll
        for (int i = 0; i < NI; ++i) {
          double part = 0.0;
          const double cf = coef[mrow(i) * n_terms + s.coef];
#pragma unroll
          for (int j = 0; j < NJ; ++j) {
            const double v = df_value(s_[i][j], c_[i][j]);
            part = fma(v, xo(i, j), part);
            put(i, j, cf * v, sg == t.seg_begin);
          }
#pragma unroll
          for (int o = 8; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
          if (tx == 0) out[ty + 16 * i] = part;
        }
      } else {
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
          double part = 0.0;
          const double cf = coef[mcol(j) * n_terms + s.coef];
#pragma unroll
          for (int i = 0; i < NI; ++i) {
            const double v = df_value(s_[i][j], c_[i][j]);
            part = fma(v, xo(i, j), part);
            put(i, j, cf * v, sg == t.seg_begin);
          }
          dsm->col[ty][tx + 16 * j] = part;
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

  if (DOTS && t.seg_begin == t.seg_end) {  // an output no segment writes
#pragma unroll
    for (int i = 0; i < NI; ++i)
#pragma unroll
      for (int j = 0; j < NJ; ++j) put(i, j, 0.0, true);
  }
  double* C = bufs.p[t.c_buf] + t.c_off;
  if (t.mode == TM_STORE && ((pm >> t.c_buf) & 1u)) {  // a pair buffer: (s, c) kept as the pair
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
        float s = s_[i][j], c = c_[i][j];
        if (add) {  // two-sum of the stored pair's high parts, the low parts into c
          const float2 o = df_bits(*p);
          const float tt = __fadd_rn(s, o.x);
          const float bv = __fsub_rn(tt, s);
          c = __fadd_rn(c, __fadd_rn(__fadd_rn(__fsub_rn(s, __fsub_rn(tt, bv)), __fsub_rn(o.x, bv)), o.y));
          s = tt;
        }
        *p = df_slot(s, c);
      }
    }
  } else if (t.mode == TM_STORE) {
    const bool add = accumulate || t.add;
#pragma unroll
    for (int i = 0; i < NI; ++i) {
      const int m = t.m0 + ty + 16 * i;
      if (m >= t.M) continue;
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        const int n = t.n0 + tx + 16 * j;
        if (n >= t.N) continue;
        const double v = df_value(s_[i][j], c_[i][j]);
        double* p = C + coff(m, n);
        *p = add ? *p + v : v;
      }
    }
  } else if (t.mode == TM_DOT) {  // sum over the tile of acc .* C, fixed-order block reduction
    double part = 0.0;
#pragma unroll
    for (int i = 0; i < NI; ++i) {
      const int m = t.m0 + ty + 16 * i;
      if (m >= t.M) continue;
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        const int n = t.n0 + tx + 16 * j;
        if (n >= t.N) continue;
        part = fma(df_value(s_[i][j], c_[i][j]), C[coff(m, n)], part);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
    if ((tid & 31) == 0) sm.red[tid >> 5] = part;
    __syncthreads();
    if (tid == 0) {
      double tot = 0.0;
      for (int w = 0; w < DF_THREADS / 32; ++w) tot += sm.red[w];
      dot_out[blockIdx.x] = tot;
    }
  }
}

#define DF_SHAPES(CASE)                                         \
  CASE(1, 1) CASE(1, 2) CASE(1, 3) CASE(1, 4) CASE(2, 1) CASE(2, 2) \
  CASE(2, 3) CASE(2, 4) CASE(3, 1) CASE(3, 2) CASE(3, 3) CASE(3, 4) \
  CASE(4, 1) CASE(4, 2) CASE(4, 3) CASE(4, 4)

__global__ void __launch_bounds__(DF_THREADS, 2)
seg_gemm_df_kernel(const TileF64* __restrict__ tiles, const SegF64* __restrict__ segs, Bufs bufs,
                   const double* __restrict__ coef, int n_terms, int accumulate, double* __restrict__ dot_out,
                   const int32_t* __restrict__ skip, uint32_t pm) {
  __shared__ DFSmem sm;
  if (skip && *skip) return;
  const TileF64 t = tiles[blockIdx.x];
#define DF_CASE(I, J) \
  case (I) | ((J) << 8): df_tile<I, J, false>(t, segs, bufs, coef, n_terms, accumulate, dot_out, sm, nullptr, pm); break;
  switch (t.shape) {
    DF_SHAPES(DF_CASE)
    default: break;  // the host builds only the shapes above
  }
#undef DF_CASE
}

__global__ void __launch_bounds__(DF_THREADS, 2)
seg_gemm_df_dots_kernel(const TileF64* __restrict__ tiles, const SegF64* __restrict__ segs, Bufs bufs,
                        const double* __restrict__ coef, int n_terms, int accumulate, double* __restrict__ dot_out,
                        const int32_t* __restrict__ skip, uint32_t pm) {
  __shared__ DFSmem sm;
  __shared__ DFDotSmem dsm;
  if (skip && *skip) return;
  const TileF64 t = tiles[blockIdx.x];
#define DF_CASE(I, J) \
  case (I) | ((J) << 8): df_tile<I, J, true>(t, segs, bufs, coef, n_terms, accumulate, dot_out, sm, &dsm, pm); break;
  switch (t.shape) {
    DF_SHAPES(DF_CASE)
    default: break;
  }
#undef DF_CASE
}
#undef DF_SHAPES

void launch_seg_gemm_df(const TaskListF64& tl, const Bufs& bufs, const double* coef, int n_terms, int accumulate,
                        double* dot_out, const int32_t* skip, cudaStream_t st, uint32_t pair_mask) {
  if (tl.n_tiles == 0) return;
  seg_gemm_df_kernel<<<(unsigned)tl.n_tiles, DF_THREADS, 0, st>>>(tl.d_tiles, tl.d_segs, bufs, coef, n_terms,
                                                                  accumulate, dot_out, skip, pair_mask);
}

// dst[i] = the pair (hi, lo) of src[i] in its 8-byte slot
__global__ void k_split_pairs(const double* __restrict__ src, double* __restrict__ dst, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float2 p = df_split(src[i]);
    dst[i] = __hiloint2double(__float_as_int(p.y), __float_as_int(p.x));
  }
}

void launch_split_pairs(const double* src, double* dst, int64_t n, cudaStream_t st) {
  if (n <= 0) return;
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, 4096);  // grid-stride beyond
  k_split_pairs<<<(unsigned)blocks, 256, 0, st>>>(src, dst, n);
}

void launch_seg_gemm_df_dots(const TaskListF64& tl, const Bufs& bufs, const double* coef, int n_terms,
                             int accumulate, double* dot_out, const int32_t* skip, cudaStream_t st,
                             uint32_t pair_mask) {
  if (tl.n_tiles == 0) return;
  seg_gemm_df_dots_kernel<<<(unsigned)tl.n_tiles, DF_THREADS, 0, st>>>(tl.d_tiles, tl.d_segs, bufs, coef, n_terms,
                                                                       accumulate, dot_out, skip, pair_mask);
}

}  // namespace dmrg
