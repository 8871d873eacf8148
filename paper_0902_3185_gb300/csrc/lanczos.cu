// Float64 Lanczos kernels: Krylov scalars, full reorthogonalisation, the
// tridiagonal eigenproblem and the Ritz vector.
//
// Reorthogonalisation of w = H v_j, every iteration against every Krylov
// vector, in three classical Gram-Schmidt passes: (A) the three-term step
// against v_{j-1}, v_j (alpha_j is its v_j coefficient); (B) one pass against
// v_0..v_j; (C) a second full pass for the members whose norm fell below
// 1/sqrt(2) of its value before pass B (the Daniel-Gragg-Kaufman-Stewart
// test).  After the three-term step the remaining components along the basis
// are small, so pass B rarely shrinks w and pass C is rarely run; each full
// pass costs 2 (j+1) D float64 FMAs per member.
//
// Storage of the Krylov basis: float64 for float64 solves; for the
// mixed-precision solves each element is stored as a double-float pair
// (hi, lo) of float32 values in the same 8 bytes (about 48 significant bits,
// split once when the vector is written), and the full Gram-Schmidt passes
// run in double-float arithmetic on the float32 pipes: reading a pair needs
// no split, so a pass is bound by HBM instead of GB300's float64 issue rate
// (2 fused multiply-adds per clock per SM, about 5 TB/s of 8-byte operands).
//
// Paper Sec. 3.3: each targeted symmetry block is diagonalised with Lanczos,
// which needs only x += H y.  Everything here runs on the device for all batch
// members at once and reads the iteration index from device memory, so one
// captured CUDA graph replays any iteration without host round trips.
//
// Control words (int32, device): [0] j = index of the current Krylov vector,
// [1] max_iter, [2] check_every, [3] all members done, [4] testing hook (the
// float32 test passes at its first check), then per member b:
// [5 + b] done code (0 running, 1 converged, 2 breakdown, 3 NaN, 4 cap hit,
// 5 pending: stopped on the float32 test, float64 check after the loop;
// 6 resume: that check failed with iterations left, the host restarts the
// member from its Ritz vector; 7 hold: done in an earlier run, skipped)
// and [5 + batch + b] number of Lanczos vectors in its tridiagonal matrix.

#include <cfloat>

#include "df.cuh"
#include "internal.h"
#include "lanczos.h"

namespace dmrg {

__device__ __forceinline__ double block_sum(double v, double* red) {
  // fixed-order reduction over a 256-thread block; result valid in thread 0
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
  return t;
}

__device__ __forceinline__ bool member_done(const int32_t* ctl, int b) {
  return ctl[LZ_CTL_ALLDONE] != 0 || ctl[LZ_CTL_MEMBER + b] != 0;
}

// skip a member: finished, or gated off (gate != NULL and gate[b] == 0)
__device__ __forceinline__ bool member_skip(const int32_t* ctl, const int32_t* gate, int b) {
  return member_done(ctl, b) || (gate && gate[b] == 0);
}

// a Krylov element stored as a double-float pair
__device__ __forceinline__ float2 ld_pair(const double* p) { return *reinterpret_cast<const float2*>(p); }
// the pair held in the 8 bytes of a loaded element (hi in the low word)
__device__ __forceinline__ float2 pair_bits(double v) {
  return make_float2(__int_as_float(__double2loint(v)), __int_as_float(__double2hiint(v)));
}
__device__ __forceinline__ void st_pair(double* p, double v) { *reinterpret_cast<float2*>(p) = df_split(v); }
__device__ __forceinline__ double pair_value(float2 a) { return tc::f2d_exact(a.x) + tc::f2d_exact(a.y); }
// element d of Krylov row i in either storage
template <bool PAIR>
__device__ __forceinline__ double v_value(const double* p) {
  return PAIR ? pair_value(ld_pair(p)) : *p;
}

// first Krylov row of a pass: the last `win` rows, or all (win = 0)
__device__ __forceinline__ int first_row(int j, int win) { return win ? max(0, j - win + 1) : 0; }

// partial[(b*cap + i)*nparts + chunk*LZ_DOT_WARPS + warp] = sum over the warp's
// elements d of the chunk of V[i][b][d] * w[b][d], i0 <= i <= j (i0 =
// first_row(j, win), nparts = nchunk * LZ_DOT_WARPS): one partial per warp,
// so that no block barrier stands between the row groups and the other warps
// keep loading while one reduces; a row's partials are contiguous for the
// reduction.
// GB300 issues float64 at 1/64 of the float32 rate, so the reduction must not
// cost more float64 work than the dot products: every thread keeps
// LZ_DOT_EPT elements of w in registers, takes 8 rows at a time, and the 8
// row sums are reduced across the warp by a butterfly that halves the values
// per lane at each step (4+2+1+1+1 shuffle-adds for 8 rows, not 8 x 5).
// With h_pre != NULL the previous pass's update (the three-term step,
// w -= h_pre[j-1] v_{j-1} + h_pre[j] v_j, in that order) is applied first,
// written back to w, and its per-chunk sum of squares stored in npart_pre:
// one sweep instead of an update sweep followed by a dot sweep.
template <bool PAIR>
__global__ void __launch_bounds__(LZ_THREADS, PAIR ? 2 : 3)
k_multidot(const double* __restrict__ V, double* __restrict__ w, double* __restrict__ partial,
           const int32_t* __restrict__ ctl, int64_t D, int batch, int cap, int nchunk, int win,
           const int32_t* __restrict__ gate, const double* __restrict__ h_pre, double* __restrict__ npart_pre) {
  __shared__ double red[LZ_THREADS / 32][8];
  const int b = blockIdx.y, chunk = blockIdx.x;
  if (member_skip(ctl, gate, b)) return;
  const int j = ctl[LZ_CTL_J];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double wv[LZ_DOT_EPT];  // w (float64 basis)
  float2 wf[LZ_DOT_EPT];  // w split into double-float pairs (pair basis)
  const int64_t base = (int64_t)chunk * LZ_DOT_CHUNK + threadIdx.x;
  // the pre-update's rows (j - 1 when it exists, then j) and coefficients
  const bool two = j >= 1;
  const double* v0 = V + ((int64_t)(two ? j - 1 : j) * batch + b) * D;
  const double* v1 = V + ((int64_t)j * batch + b) * D;
  const double h0 = h_pre && two ? h_pre[(int64_t)b * cap + j - 1] : 0.0;
  const double h1 = h_pre ? h_pre[(int64_t)b * cap + j] : 0.0;
  double nrm = 0.0;
#pragma unroll
  for (int e = 0; e < LZ_DOT_EPT; ++e) {
    const int64_t d = base + e * LZ_THREADS;
    double x = 0.0;
    if (d < D) {
      x = w[(int64_t)b * D + d];
      if (h_pre) {
        if (two) x = fma(-v_value<PAIR>(v0 + d), h0, x);
        x = fma(-v_value<PAIR>(v1 + d), h1, x);
        w[(int64_t)b * D + d] = x;
        nrm = fma(x, x, nrm);
      }
    }
    if (PAIR) wf[e] = df_split(x);
    else wv[e] = x;
  }
  if (h_pre) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nrm += __shfl_down_sync(0xffffffffu, nrm, o);
    if (lane == 0) red[wid][0] = nrm;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w2 = 0; w2 < LZ_THREADS / 32; ++w2) t += red[w2][0];
      npart_pre[(int64_t)b * nchunk + chunk] = t;
    }
  }
  const bool full = base + (LZ_DOT_EPT - 1) * LZ_THREADS < D;
  for (int i0 = first_row(j, win); i0 <= j; i0 += 8) {
    // per-thread sums of 8 rows: float64, or double-float pairs (pair basis)
    double p[8];
    float2 p2[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int i = i0 + q;
      const double* v = V + ((int64_t)i * batch + b) * D + base;
      if (PAIR) {  // double-float dot of the stored pairs with the split w
        float ps = 0.0f, pc = 0.0f;
        if (i <= j) {
          if (full) {
#pragma unroll
            for (int e = 0; e < LZ_DOT_EPT; ++e) df_fma(ld_pair(v + e * LZ_THREADS), wf[e], ps, pc);
          } else {
#pragma unroll
            for (int e = 0; e < LZ_DOT_EPT; ++e)
              if (base + e * LZ_THREADS < D) df_fma(ld_pair(v + e * LZ_THREADS), wf[e], ps, pc);
          }
        }
        p2[q] = df_pair(ps, pc);
      } else {
        p[q] = 0.0;
        if (i <= j) {
          if (full) {
#pragma unroll
            for (int e = 0; e < LZ_DOT_EPT; ++e) p[q] = fma(v[e * LZ_THREADS], wv[e], p[q]);
          } else {
#pragma unroll
            for (int e = 0; e < LZ_DOT_EPT; ++e)
              if (base + e * LZ_THREADS < D) p[q] = fma(v[e * LZ_THREADS], wv[e], p[q]);
          }
        }
      }
    }
    // butterfly: after the step with offset 16 a lane holds 4 partial rows,
    // after 8 two rows, after 4 one row; offsets 2 and 1 finish that row.
    // The pair basis adds pairs (float32 work: float64 issues at 1/64 of the
    // float32 rate, and float64 adds here had cost a third of the sweep).
    const int row = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
    if (PAIR) {
#pragma unroll
      for (int h = 4; h >= 1; h >>= 1) {  // offsets 16, 8, 4: halve the rows held
        const int off = 4 * h;
        const bool up = lane & off;
#pragma unroll
        for (int q = 0; q < h; ++q) {
          const float2 send = up ? p2[q] : p2[q + h];
          const float2 keep = up ? p2[q + h] : p2[q];
          const float2 got = make_float2(__shfl_xor_sync(0xffffffffu, send.x, off),
                                         __shfl_xor_sync(0xffffffffu, send.y, off));
          p2[q] = df_add(keep, got);
        }
      }
#pragma unroll
      for (int off = 2; off >= 1; off >>= 1)
        p2[0] = df_add(p2[0], make_float2(__shfl_xor_sync(0xffffffffu, p2[0].x, off),
                                          __shfl_xor_sync(0xffffffffu, p2[0].y, off)));
    } else {
      {
        const bool up = lane & 16;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const double send = up ? p[q] : p[q + 4];
          const double keep = up ? p[q + 4] : p[q];
          p[q] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
        }
      }
      {
        const bool up = lane & 8;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const double send = up ? p[q] : p[q + 2];
          const double keep = up ? p[q + 2] : p[q];
          p[q] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
        }
      }
      {
        const bool up = lane & 4;
        const double send = up ? p[0] : p[1];
        const double keep = up ? p[1] : p[0];
        p[0] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
      }
      p[0] += __shfl_xor_sync(0xffffffffu, p[0], 2);
      p[0] += __shfl_xor_sync(0xffffffffu, p[0], 1);
    }
    if ((lane & 3) == 0 && i0 + row <= j)
      partial[((int64_t)b * cap + i0 + row) * ((int64_t)nchunk * LZ_DOT_WARPS) + chunk * LZ_DOT_WARPS + wid] =
          PAIR ? df_value(p2[0].x, p2[0].y) : p[0];
  }
}

// Pass A's dots: w with v_{j-1} and v_j (v_0 alone at j = 0), in the
// partial layout of k_multidot with win = 2.  A pass over two rows does too
// little arithmetic to hide memory latency behind it, so every thread issues
// all of its loads -- its LZ_DOT_EPT elements of w and of both rows -- before
// any arithmetic: one memory round trip per block instead of one for w
// followed by one for the rows.
template <bool PAIR>
__global__ void __launch_bounds__(LZ_THREADS, 2)
k_dots_local(const double* __restrict__ V, const double* __restrict__ w, double* __restrict__ partial,
             const int32_t* __restrict__ ctl, int64_t D, int batch, int cap, int nchunk) {
  const int b = blockIdx.y, chunk = blockIdx.x;
  if (member_done(ctl, b)) return;
  const int j = ctl[LZ_CTL_J];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t base = (int64_t)chunk * LZ_DOT_CHUNK + threadIdx.x;
  const bool two = j >= 1;
  const double* wb = w + (int64_t)b * D + base;
  const double* r0 = V + ((int64_t)(two ? j - 1 : j) * batch + b) * D + base;
  const double* r1 = V + ((int64_t)j * batch + b) * D + base;
  double x[LZ_DOT_EPT], a0[LZ_DOT_EPT], a1[LZ_DOT_EPT];  // w, rows j-1 and j (pairs in their 8 bytes)
#pragma unroll
  for (int e = 0; e < LZ_DOT_EPT; ++e) {
    const bool in = base + e * LZ_THREADS < D;
    x[e] = in ? wb[e * LZ_THREADS] : 0.0;
    a0[e] = in && two ? r0[e * LZ_THREADS] : 0.0;
    a1[e] = in ? r1[e * LZ_THREADS] : 0.0;
  }
  double d0, d1;
  if (PAIR) {
    float s0 = 0.0f, c0 = 0.0f, s1 = 0.0f, c1 = 0.0f;
#pragma unroll
    for (int e = 0; e < LZ_DOT_EPT; ++e) {
      const float2 wf = df_split(x[e]);
      df_fma(pair_bits(a0[e]), wf, s0, c0);
      df_fma(pair_bits(a1[e]), wf, s1, c1);
    }
    // fixed butterfly over the warp in double-float adds (deterministic)
    float2 p0 = df_pair(s0, c0), p1 = df_pair(s1, c1);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      p0 = df_add(p0, make_float2(__shfl_xor_sync(0xffffffffu, p0.x, o), __shfl_xor_sync(0xffffffffu, p0.y, o)));
      p1 = df_add(p1, make_float2(__shfl_xor_sync(0xffffffffu, p1.x, o), __shfl_xor_sync(0xffffffffu, p1.y, o)));
    }
    d0 = df_value(p0.x, p0.y);
    d1 = df_value(p1.x, p1.y);
  } else {
    double q0 = 0.0, q1 = 0.0;
#pragma unroll
    for (int e = 0; e < LZ_DOT_EPT; ++e) {
      q0 = fma(a0[e], x[e], q0);
      q1 = fma(a1[e], x[e], q1);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      q0 += __shfl_xor_sync(0xffffffffu, q0, o);
      q1 += __shfl_xor_sync(0xffffffffu, q1, o);
    }
    d0 = q0;
    d1 = q1;
  }
  if (lane == 0) {
    const int64_t nparts = (int64_t)nchunk * LZ_DOT_WARPS;
    const int64_t slot = (int64_t)chunk * LZ_DOT_WARPS + wid;
    if (two) partial[((int64_t)b * cap + j - 1) * nparts + slot] = d0;
    partial[((int64_t)b * cap + j) * nparts + slot] = d1;
  }
}

// h[b*cap + i] = sum of row i's nparts partials, first_row(j, win) <= i <= j:
// one warp per row (8 rows per block), lane l summing partials l, l + 32, ...
// in four interleaved accumulators (loads in flight), then a fixed shuffle
// tree: the same order on every call (deterministic).
__global__ void __launch_bounds__(256)
k_reduce_rows(const double* __restrict__ partial, double* __restrict__ h, const int32_t* __restrict__ ctl,
              int nparts, int cap, int win, const int32_t* __restrict__ gate) {
  const int b = blockIdx.x;
  if (member_skip(ctl, gate, b)) return;
  const int j = ctl[LZ_CTL_J];
  const int lane = threadIdx.x & 31;
  const int i = first_row(j, win) + blockIdx.y * 8 + (int)(threadIdx.x >> 5);
  if (i > j) return;
  const double* row = partial + ((int64_t)b * cap + i) * nparts;
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  int s = lane;
  for (; s + 96 < nparts; s += 128) {
    a0 += row[s];
    a1 += row[s + 32];
    a2 += row[s + 64];
    a3 += row[s + 96];
  }
  for (; s < nparts; s += 32) a0 += row[s];
  double t = (a0 + a1) + (a2 + a3);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if (lane == 0) h[(int64_t)b * cap + i] = t;
}

// w[b] -= sum_{i0<=i<=j} V[i][b] h[b][i] (i0 = first_row(j, win)); with
// norm_partial != NULL also the per-chunk sum of squares of the new w.
template <bool PAIR>
__global__ void __launch_bounds__(LZ_THREADS)
k_multiaxpy(const double* __restrict__ V, double* __restrict__ w, const double* __restrict__ h,
            double* __restrict__ norm_partial, const int32_t* __restrict__ ctl, int64_t D, int batch,
            int cap, int nchunk, int win, const int32_t* __restrict__ gate) {
  extern __shared__ double sh[];  // the coefficients (pair basis: split into double-float pairs)
  float2* shf = reinterpret_cast<float2*>(sh);
  __shared__ double red[LZ_THREADS / 32];
  const int b = blockIdx.y, chunk = blockIdx.x;
  if (member_skip(ctl, gate, b)) return;
  const int j = ctl[LZ_CTL_J];
  const int i0 = first_row(j, win);
  for (int i = i0 + threadIdx.x; i <= j; i += blockDim.x) {
    if (PAIR) shf[i] = df_split(h[(int64_t)b * cap + i]);
    else sh[i] = h[(int64_t)b * cap + i];
  }
  __syncthreads();
  // the rows in the outer loop and the thread's LZ_EPT elements inside it:
  // independent accumulators, so every row issues LZ_EPT loads at once
  const int64_t d0 = (int64_t)chunk * LZ_CHUNK + threadIdx.x;
  const bool full = d0 + (LZ_EPT - 1) * LZ_THREADS < D;
  double acc[LZ_EPT], wv[LZ_EPT];
  float ss[LZ_EPT], sc[LZ_EPT];
#pragma unroll
  for (int e = 0; e < LZ_EPT; ++e) {
    acc[e] = 0.0;
    ss[e] = sc[e] = 0.0f;
    // w is loaded before the rows, so that its memory round trip overlaps theirs
    const int64_t d = d0 + e * LZ_THREADS;
    wv[e] = d < D ? w[(int64_t)b * D + d] : 0.0;
  }
#pragma unroll 2
  for (int i = i0; i <= j; ++i) {
    const double* vi = V + ((int64_t)i * batch + b) * D + d0;
    if (PAIR) {  // sum_i V[i] h[i] in double-float arithmetic
      const float2 hi = shf[i];
#pragma unroll
      for (int e = 0; e < LZ_EPT; ++e)
        if (full || d0 + e * LZ_THREADS < D) df_fma(ld_pair(vi + e * LZ_THREADS), hi, ss[e], sc[e]);
    } else {
      const double hi = sh[i];
#pragma unroll
      for (int e = 0; e < LZ_EPT; ++e)
        if (full || d0 + e * LZ_THREADS < D) acc[e] = fma(vi[e * LZ_THREADS], hi, acc[e]);
    }
  }
  double nrm = 0.0;
#pragma unroll
  for (int e = 0; e < LZ_EPT; ++e) {
    const int64_t d = d0 + e * LZ_THREADS;
    if (d >= D) continue;
    const double x = wv[e] - (PAIR ? df_value(ss[e], sc[e]) : acc[e]);
    w[(int64_t)b * D + d] = x;
    nrm = fma(x, x, nrm);
  }
  if (norm_partial) {
    const double t = block_sum(nrm, red);
    if (threadIdx.x == 0) norm_partial[(int64_t)b * nchunk + chunk] = t;
  }
}

// sum of a member's norm partials: lane-strided sums, then a fixed shuffle tree
__device__ __forceinline__ double warp_sum_chunks(const double* __restrict__ part, int nchunk) {
  double t = 0.0;
  for (int ch = threadIdx.x; ch < nchunk; ch += 32) t += part[ch];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  return t;
}

// Daniel-Gragg-Kaufman-Stewart test after pass B: gate[b] = 1 (run pass C)
// unless |w_B|^2 >= |w_A|^2 / 2.  One warp per member.
__global__ void k_dgks(const double* __restrict__ npart_a, const double* __restrict__ npart_b,
                       int32_t* __restrict__ gate, const int32_t* __restrict__ ctl, int nchunk_a, int nchunk) {
  const int b = blockIdx.x;
  if (member_done(ctl, b)) return;
  const double na = warp_sum_chunks(npart_a + (int64_t)b * nchunk_a, nchunk_a);
  const double nb = warp_sum_chunks(npart_b + (int64_t)b * nchunk, nchunk);
  if (threadIdx.x == 0) gate[b] = (nb >= 0.5 * na) ? 0 : 1;  // NaN: run pass C, then the NaN check stops it
}

// alpha_j = sum of the v_j coefficients of the passes that ran, beta_j = |w|
// after the last pass.  One warp per member (deterministic).
__global__ void k_finalize_ab(const double* __restrict__ h, const double* __restrict__ npart_b,
                              const double* __restrict__ npart_c, const int32_t* __restrict__ gate,
                              double* __restrict__ ab, const int32_t* __restrict__ ctl, int batch, int cap,
                              int nchunk) {
  const int b = blockIdx.x;
  if (member_done(ctl, b)) return;
  const int j = ctl[LZ_CTL_J];
  const bool c = gate[b] != 0;
  const double t = warp_sum_chunks((c ? npart_c : npart_b) + (int64_t)b * nchunk, nchunk);
  if (threadIdx.x == 0) {
    double a = h[(int64_t)b * cap + j] + h[((int64_t)batch + b) * cap + j];
    if (c) a += h[(2 * (int64_t)batch + b) * cap + j];
    ab[(int64_t)b * cap + j] = a;
    ab[((int64_t)batch + b) * cap + j] = sqrt(t);
  }
}

// Sign and zero test of a float / double from its bit pattern (integer
// instructions: GB300's float64 pipe is narrow), and its biased exponent.
__device__ __forceinline__ bool is_neg(float v) { return __float_as_int(v) < 0; }
__device__ __forceinline__ bool is_neg(double v) { return __double2hiint(v) < 0; }
__device__ __forceinline__ bool is_zero(float v) { return (__float_as_int(v) & 0x7fffffff) == 0; }
__device__ __forceinline__ bool is_zero(double v) {
  return ((__double2hiint(v) & 0x7fffffff) | __double2loint(v)) == 0;
}
__device__ __forceinline__ int bexp(float v) { return (__float_as_int(v) >> 23) & 0xff; }
__device__ __forceinline__ int bexp(double v) { return (__double2hiint(v) >> 20) & 0x7ff; }
// 2^(bias - e) for a biased exponent e: the factor that brings e to the bias
__device__ __forceinline__ float pow2_to_one(int e, float) { return __int_as_float((254 - e) << 23); }
__device__ __forceinline__ double pow2_to_one(int e, double) { return __hiloint2double((2046 - e) << 20, 0); }
template <class T> struct SturmWindow;  // rescale when the larger minor leaves 2^(+-W)
template <> struct SturmWindow<float> { static constexpr int bias = 127, W = 30; };
template <> struct SturmWindow<double> { static constexpr int bias = 1023, W = 400; };

// Power of two s with s * scale in [1/2, 1) (scale >= 1): Sturm counts are
// evaluated on s (T - x I), whose entries are then O(1).
__device__ __forceinline__ double sturm_scale(double scale) {
  return __hiloint2double((2046 - bexp(scale) - 1) << 20, 0);
}

// Number of eigenvalues of T (diagonal a, off-diagonal squares e2) below x.
// The leading principal minors p_i of s (T - x I) obey p_0 = 1,
// p_1 = s (a_0 - x), p_{i+1} = s (a_i - x) p_i - s^2 e2_{i-1} p_{i-1}; each
// sign change between consecutive minors is a negative pivot of the L D L^T
// factorisation, and by Sylvester's law of inertia their number is the
// count.  The recurrence needs no division (one fused multiply-add on its
// dependency chain per step); rounding each term is a relative perturbation
// of a_i - x or e2_{i-1}, as in the pivot form.  When the larger of the last
// two minors leaves the exponent window both are scaled by the same power of
// two (exact); a zero minor takes its predecessor's sign, which puts the
// sign change on the next minor.
template <class T>
__device__ int sturm_count(const T* a, const T* e2, int n, T x, T s) {
  constexpr int bias = SturmWindow<T>::bias, W = SturmWindow<T>::W;
  const T s2 = s * s;
  T pm = T(1);
  T p = (a[0] - x) * s;
  bool neg = is_neg(p) && !is_zero(p);
  int cnt = neg ? 1 : 0;
  for (int i = 1; i < n; ++i) {
    const T t = (a[i] - x) * s;
    const T q = (e2[i - 1] * s2) * pm;
    const T pn = fma(t, p, -q);
    const bool nn = is_zero(pn) ? neg : is_neg(pn);
    cnt += nn != neg;
    neg = nn;
    pm = p;
    p = pn;
    const int em = max(bexp(p), bexp(pm));
    if (em > bias + W || (em < bias - W && em > 0)) {
      const T f = pow2_to_one(em, T(0));
      p *= f;
      pm *= f;
    }
  }
  return cnt;
}

// Multisection by one warp: the 32 lanes evaluate Sturm counts at evenly
// spaced points of [lo, hi] (count(lo) = 0 <= 1 <= count(hi) ... holds for
// the lowest eigenvalue) and keep the sub-interval that holds it.
template <class T>
__device__ void multisection(const T* a, const T* e2, int n, T& lo, T& hi, T rel, int max_rounds, T s) {
  const int lane = threadIdx.x & 31;
  for (int round = 0; round < max_rounds; ++round) {
    const T w = hi - lo;
    if (!(w > rel * fmax(fabs(lo), fabs(hi))) || !(w > T(0))) break;
    const T step = w / T(33);
    const T x = lo + step * T(lane + 1);
    const int cnt = sturm_count<T>(a, e2, n, x, s);
    const unsigned ball = __ballot_sync(0xffffffffu, cnt >= 1);
    const int f = ball ? __ffs(ball) - 1 : 32;  // first point with an eigenvalue below it
    const T nlo = lo + step * T(f);
    const T nhi = f < 32 ? lo + step * T(f + 1) : hi;
    lo = nlo;
    hi = nhi;
  }
}

// Inverse iteration with a shift below lambda_min: T - sigma I is positive
// definite, so its L D L^T factorisation needs no pivoting.  Lane 0 factors
// once (reciprocal pivots rpiv, multipliers lm) and solves `solves` times,
// from z = 1 or, with `given`, from the z passed in; returns in z the
// normalised eigenvector estimate with z[0] >= 0.  Each solve is one forward
// sweep (L y = z, then D^-1) and one backward sweep (L^T) that also
// accumulates |z|^2.
template <class T>
__device__ void inverse_iteration(const T* a, const T* e, int n, T sigma, T* z, T* rpiv, T* lm, int solves, T tiny,
                                  bool given) {
  if ((threadIdx.x & 31) != 0) return;
  T dp = a[0] - sigma;
  rpiv[0] = T(1) / (dp == T(0) ? tiny : dp);
  for (int i = 1; i < n; ++i) {
    const T l = e[i - 1] * rpiv[i - 1];
    lm[i - 1] = l;
    dp = (a[i] - sigma) - l * e[i - 1];
    rpiv[i] = T(1) / (dp == T(0) ? tiny : dp);
  }
  if (!given)
    for (int i = 0; i < n; ++i) z[i] = T(1);
  for (int it = 0; it < solves; ++it) {
    T y = z[0];
    z[0] = y * rpiv[0];
    for (int i = 1; i < n; ++i) {
      y = fma(-lm[i - 1], y, z[i]);
      z[i] = y * rpiv[i];
    }
    T zn = z[n - 1];
    T nz = zn * zn;
    for (int i = n - 2; i >= 0; --i) {
      zn = fma(-lm[i], zn, z[i]);
      z[i] = zn;
      nz = fma(zn, zn, nz);
    }
    const T inv = (zn < T(0) ? T(-1) : T(1)) / sqrt(nz);  // zn = z[0]
    for (int i = 0; i < n; ++i) z[i] *= inv;
  }
}

// Lowest eigenpair of the (j+1) x (j+1) tridiagonal matrix of each member and
// the convergence test.  One warp per member.
//  - every check: float32 multisection and float32 inverse iteration give
//    theta and the last Ritz-vector component to a few digits, enough for the
//    test beta_j |s_j| <= tol max(1, |theta|);
//  - when the float32 test passes with a factor 2 to spare, the member stops
//    as LZ_PENDING; after the iteration loop one launch (final_pass) redoes
//    the float32 step for every pending member at its own length, computes
//    the eigenpair in float64 (multisection from the float32 bracket, widened
//    by its rounding bound, then inverse iteration), repeats the test with
//    the float64 values (a member that then misses the tolerance ends as
//    LZ_RESUME, or LZ_CAP at max_iter; the host restarts a resumed member from
//    its Ritz vector) and stores s for the Ritz vector: the members' float64 solves
//    run side by side in one launch instead of each in the launch where its
//    member converged;
//  - at breakdown or the cap the float64 eigenpair is computed at once;
//  - tolerances below 1e-5 are beyond the float32 estimate's resolution:
//    near convergence (estimate <= 1e-2 |T|) those members take the float64
//    eigenpair and test at every check instead of stopping as pending.
// GB300 issues float64 at 1/64 of the float32 rate, which is why the per-
// iteration test runs in float32.
__global__ void __launch_bounds__(32)
k_tridiag(const double* __restrict__ ab, double* __restrict__ s_out, double* __restrict__ out,
          int32_t* __restrict__ ctl, const double* __restrict__ tolp, int batch, int cap, int64_t D,
          int final_pass) {
  extern __shared__ double sm[];
  double* a = sm;
  double* e = sm + cap;
  double* e2 = sm + 2 * cap;
  double* z = sm + 3 * cap;
  double* rp = sm + 4 * cap;
  float* a32 = reinterpret_cast<float*>(sm + 5 * cap);
  float* e32 = a32 + cap;
  float* e232 = e32 + cap;
  float* z32 = e232 + cap;
  float* rp32 = z32 + cap;
  const int b = blockIdx.x;
  const int lane = threadIdx.x;
  if (final_pass ? ctl[LZ_CTL_MEMBER + b] != LZ_PENDING : member_done(ctl, b)) return;
  const int n = final_pass ? ctl[LZ_CTL_MEMBER + batch + b] : ctl[LZ_CTL_J] + 1;
  const int max_iter = ctl[LZ_CTL_MAXIT];
  const int check_every = ctl[LZ_CTL_CHECK];
  const double tol = *tolp;
  for (int i = lane; i < n; i += 32) {
    const double ai = ab[(int64_t)b * cap + i], ei = ab[((int64_t)batch + b) * cap + i];
    a[i] = ai;
    e[i] = ei;  // e[n-1] = beta_j, the residual factor
    e2[i] = ei * ei;
    a32[i] = (float)ai;
    e32[i] = (float)ei;
    e232[i] = (float)(ei * ei);
  }
  __syncwarp();
  const double beta = e[n - 1];
  // Gershgorin bounds (float64, lane-parallel), amax for the scales
  double glo = 1e300, ghi = 1e300, amax = 0.0;
  for (int i = lane; i < n; i += 32) {
    const double rad = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i < n - 1 ? fabs(e[i]) : 0.0);
    glo = fmin(glo, a[i] - rad);
    ghi = fmin(ghi, a[i]);
    amax = fmax(amax, fabs(a[i]) + rad);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    glo = fmin(glo, __shfl_xor_sync(0xffffffffu, glo, o));
    ghi = fmin(ghi, __shfl_xor_sync(0xffffffffu, ghi, o));
    amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  }
  const double scale_t = fmax(1.0, amax);
  const bool bad = !isfinite(a[n - 1]) || !isfinite(beta);
  const bool small_beta = beta < 1e-14 * scale_t;
  const bool last = n >= max_iter || (int64_t)n >= D;
  if (bad) {
    if (lane == 0) {
      ctl[LZ_CTL_MEMBER + b] = LZ_NAN;
      ctl[LZ_CTL_MEMBER + batch + b] = n;
    }
    return;
  }
  if (!final_pass && !((n % check_every == 0) || last || small_beta)) return;

  // ---- float32 estimate
  const float eps32 = 1.2e-7f;
  const float slack = (float)(8.0 * n * 6e-8 * scale_t);  // rounding of T to float32, Sturm backward error
  float lo = (float)glo - slack, hi = (float)ghi + slack;
  const double ssc = sturm_scale(scale_t);
  multisection<float>(a32, e232, n, lo, hi, 4.0f * eps32, 12, (float)ssc);
  const float th32 = 0.5f * (lo + hi);
  // the multipliers overwrite e2 (the Sturm counts are done)
  inverse_iteration<float>(a32, e32, n, lo - 2.0f * slack - 1e-6f * (float)scale_t, z32, rp32, e232, 3, 1e-30f,
                           false);
  __syncwarp();
  const double est = beta * fabs((double)z32[n - 1]);
  const bool force = ctl[LZ_CTL_FORCE] != 0;
  const bool pass32 = est <= 0.5 * tol * fmax(1.0, fabs((double)th32)) || force;
  // The float32 last component is accurate only to about eps32 |T| / gap
  // (absolute), so the float32 estimate cannot resolve tolerances much below
  // 1e-5: such solves take the float64 eigenpair at every check once the
  // estimate has come within 1e-2 |T|, and stop on the float64 test.
  const bool check64 = !final_pass && tol < 1e-5 && !force && est <= 1e-2 * scale_t;
  if (!final_pass && !(small_beta || last) && !check64) {
    if (lane == 0) {
      out[b * 4 + 0] = th32;
      out[b * 4 + 1] = est;
      out[b * 4 + 2] = beta;
      if (pass32) {
        ctl[LZ_CTL_MEMBER + b] = LZ_PENDING;
        ctl[LZ_CTL_MEMBER + batch + b] = n;
      }
    }
    return;
  }

  // ---- float64 eigenpair
  double lo64 = (double)lo - 2.0 * slack, hi64 = (double)hi + 2.0 * slack;
  lo64 = fmax(lo64, glo - 1e-300);
  {  // the bracket must hold lambda_min: lane 0 counts at lo64, lane 1 at hi64
    const int c = sturm_count<double>(a, e2, n, lane == 0 ? lo64 : hi64, ssc);
    const int c_lo = __shfl_sync(0xffffffffu, c, 0), c_hi = __shfl_sync(0xffffffffu, c, 1);
    if (c_lo != 0) lo64 = glo - 1e-300;
    if (c_hi == 0) hi64 = ghi + 1e-12 * scale_t;
  }
  multisection<double>(a, e2, n, lo64, hi64, 4.0 * 2.2e-16, 64, ssc);
  const double theta = 0.5 * (lo64 + hi64);
  // one solve from the float32 eigenvector: the shift is within a few ulps of
  // lambda_min, so a solve reduces the error by (lambda_1 - sigma) / gap
  for (int i = lane; i < n; i += 32) z[i] = isfinite(z32[i]) ? (double)z32[i] : 1.0;
  __syncwarp();
  inverse_iteration<double>(a, e, n, lo64 - 4.0 * 2.2e-16 * scale_t, z, rp, e2, 1, 1e-300, true);
  __syncwarp();
  if (lane == 0) {
    const double resid = beta * fabs(z[n - 1]);
    const double scale = fmax(1.0, fabs(theta));
    int code = 0;
    if (!isfinite(theta) || !isfinite(resid)) code = LZ_NAN;
    else if (small_beta || beta < 1e-14 * scale || (int64_t)n >= D) code = LZ_BREAKDOWN;
    else if (resid <= tol * scale) code = LZ_CONVERGED;
    else if (n >= max_iter) code = LZ_CAP;
    else if (final_pass) code = LZ_RESUME;
    out[b * 4 + 0] = theta;
    out[b * 4 + 1] = resid;
    out[b * 4 + 2] = beta;
    for (int i = 0; i < n; ++i) s_out[(int64_t)b * cap + i] = z[i];
    if (code) {
      ctl[LZ_CTL_MEMBER + b] = code;
      ctl[LZ_CTL_MEMBER + batch + b] = n;
    }
  }
}

// v_{j+1} = w / beta_j for running members (into the basis and the current vector)
template <bool PAIR>
__global__ void k_next_vector(const double* __restrict__ w, const double* __restrict__ ab,
                              double* __restrict__ V, double* __restrict__ vcur,
                              const int32_t* __restrict__ ctl, int64_t D, int batch, int cap) {
  __shared__ double s_inv;
  const int b = blockIdx.y;
  if (member_done(ctl, b)) return;
  const int j = ctl[LZ_CTL_J];
  // one float64 division per block, not per element (GB300's float64 pipe is narrow)
  if (threadIdx.x == 0) s_inv = 1.0 / ab[((int64_t)batch + b) * cap + j];
  __syncthreads();
  const double inv = s_inv;
  double* vn = V + ((int64_t)(j + 1) * batch + b) * D;
  for (int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; d < D; d += (int64_t)gridDim.x * blockDim.x) {
    const double v = w[(int64_t)b * D + d] * inv;
    if (PAIR) st_pair(vn + d, v);
    else vn[d] = v;
    vcur[(int64_t)b * D + d] = v;
  }
}

__global__ void k_advance(int32_t* ctl, int batch) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (ctl[LZ_CTL_ALLDONE]) return;
  int all = 1;
  for (int b = 0; b < batch; ++b) all &= (ctl[LZ_CTL_MEMBER + b] != 0);
  if (all) ctl[LZ_CTL_ALLDONE] = 1;
  else ctl[LZ_CTL_J] += 1;
}

// ----------------------------------------------------------- vector helpers
// per-chunk sum of squares of x[b] (no control words)
__global__ void __launch_bounds__(LZ_THREADS)
k_sumsq(const double* __restrict__ x, double* __restrict__ part, int64_t D, int nchunk) {
  __shared__ double red[LZ_THREADS / 32];
  const int b = blockIdx.y, chunk = blockIdx.x;
  double t = 0.0;
#pragma unroll
  for (int e = 0; e < LZ_EPT; ++e) {
    const int64_t d = (int64_t)chunk * LZ_CHUNK + e * LZ_THREADS + threadIdx.x;
    if (d < D) { const double v = x[(int64_t)b * D + d]; t = fma(v, v, t); }
  }
  t = block_sum(t, red);
  if (threadIdx.x == 0) part[(int64_t)b * nchunk + chunk] = t;
}

// per-chunk <x[b], y[b]>
__global__ void __launch_bounds__(LZ_THREADS)
k_dot(const double* __restrict__ x, const double* __restrict__ y, double* __restrict__ part, int64_t D,
      int nchunk) {
  __shared__ double red[LZ_THREADS / 32];
  const int b = blockIdx.y, chunk = blockIdx.x;
  double t = 0.0;
#pragma unroll
  for (int e = 0; e < LZ_EPT; ++e) {
    const int64_t d = (int64_t)chunk * LZ_CHUNK + e * LZ_THREADS + threadIdx.x;
    if (d < D) t = fma(x[(int64_t)b * D + d], y[(int64_t)b * D + d], t);
  }
  t = block_sum(t, red);
  if (threadIdx.x == 0) part[(int64_t)b * nchunk + chunk] = t;
}

// res[b] = sum over chunks of part[b][chunk] (fixed order)
__global__ void k_sum_chunks(const double* __restrict__ part, double* __restrict__ res, int nchunk, int batch) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch) return;
  double t = 0.0;
  for (int ch = 0; ch < nchunk; ++ch) t += part[(int64_t)b * nchunk + ch];
  res[b] = t;
}

// y[b] = x[b] / sqrt(nrm2[b]); also into y2 if given
template <bool PAIR>
__global__ void k_scale_unit(const double* __restrict__ x, const double* __restrict__ nrm2,
                             double* __restrict__ y, double* __restrict__ y2, int64_t D) {
  __shared__ double s_inv;
  const int b = blockIdx.y;
  if (threadIdx.x == 0) s_inv = 1.0 / sqrt(nrm2[b]);
  __syncthreads();
  const double inv = s_inv;
  for (int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; d < D; d += (int64_t)gridDim.x * blockDim.x) {
    const double v = x[(int64_t)b * D + d] * inv;
    if (PAIR) st_pair(y + (int64_t)b * D + d, v);  // y is a Krylov row
    else y[(int64_t)b * D + d] = v;
    if (y2) y2[(int64_t)b * D + d] = v;
  }
}

// out[b] = sum_{i < n_b} s[b][i] V[i][b]
template <bool PAIR>
__global__ void k_ritz(const double* __restrict__ V, const double* __restrict__ s,
                       const int32_t* __restrict__ ctl, double* __restrict__ out, int64_t D, int batch,
                       int cap) {
  const int b = blockIdx.y;
  if (ctl[LZ_CTL_MEMBER + b] == LZ_HOLD) return;  // its result came from an earlier run
  const int n = ctl[LZ_CTL_MEMBER + batch + b];
  for (int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; d < D; d += (int64_t)gridDim.x * blockDim.x) {
    if (PAIR) {  // double-float sum of the stored pairs
      float ts = 0.0f, tc2 = 0.0f;
      for (int i = 0; i < n; ++i)
        df_fma(ld_pair(V + ((int64_t)i * batch + b) * D + d), df_split(s[(int64_t)b * cap + i]), ts, tc2);
      out[(int64_t)b * D + d] = df_value(ts, tc2);
    } else {
      double t = 0.0;
      for (int i = 0; i < n; ++i) t = fma(s[(int64_t)b * cap + i], V[((int64_t)i * batch + b) * D + d], t);
      out[(int64_t)b * D + d] = t;
    }
  }
}

// dE_dc[b][k] = dots[b][k] / nrm2[b]
__global__ void k_div_rows(double* __restrict__ v, const double* __restrict__ nrm2, int n_terms, int batch) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_terms * batch) return;
  v[i] /= nrm2[i / n_terms];
}

// dc[b*n_terms + k] = sum of the dot-tile partials of (b, k): one block per
// (b, k), thread-strided sums over its list, then a fixed-order block
// reduction (deterministic)
__global__ void __launch_bounds__(256)
k_reduce_terms(const double* __restrict__ part, const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
               double* __restrict__ out, int n) {
  __shared__ double red[256 / 32];
  const int i = blockIdx.x;
  if (i >= n) return;
  double t = 0.0;
  for (int q = ptr[i] + threadIdx.x; q < ptr[i + 1]; q += blockDim.x) t += part[idx[q]];
  t = block_sum(t, red);
  if (threadIdx.x == 0) out[i] = t;
}

// G_b(z) = norm2_b / (z - a_0 - b_0^2 / (z - a_1 - ... - b_{n-2}^2 / (z - a_{n-1})))
// for complex z, one thread per (member, z), evaluated from the deepest level
// up (paper: the local density of states by the continued-fraction method)
__global__ void k_cfrac(const double* __restrict__ norm2, const double* __restrict__ alpha,
                        const double* __restrict__ beta, const int32_t* __restrict__ n, int ld,
                        const double* __restrict__ zr, const double* __restrict__ zi, int n_z,
                        double* __restrict__ gr, double* __restrict__ gi) {
  const int b = blockIdx.y;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_z) return;
  const int64_t at = (int64_t)b * n_z + k;
  const double xr = zr[at], xi = zi[at];
  const int nb = min(max(n[b], 0), ld);  // a count beyond the row length is clamped, never read past
  const double* a = alpha + (int64_t)b * ld;
  const double* bb = beta + (int64_t)b * ld;
  double tr = 0.0, ti = 0.0;  // t = z - a_j - b_j^2 / t_{j+1}
  if (nb > 0) {
    tr = xr - a[nb - 1];
    ti = xi;
    for (int j = nb - 2; j >= 0; --j) {
      const double d = tr * tr + ti * ti;   // b_j^2 / t = b_j^2 conj(t) / |t|^2
      const double f = bb[j] * bb[j] / d;
      tr = xr - a[j] - f * tr;
      ti = xi + f * ti;
    }
  }
  const double d = tr * tr + ti * ti;
  const double s = nb > 0 ? norm2[b] / d : 0.0;  // norm2 / t
  gr[at] = s * tr;
  gi[at] = -s * ti;
}

// ------------------------------------------------------------- launchers
void lz_launch_cfrac(const double* norm2, const double* alpha, const double* beta, const int32_t* n, int ld,
                     const double* zr, const double* zi, int n_z, double* gr, double* gi, int batch,
                     cudaStream_t st) {
  if (n_z <= 0 || batch <= 0) return;
  k_cfrac<<<dim3((n_z + 127) / 128, batch), 128, 0, st>>>(norm2, alpha, beta, n, ld, zr, zi, n_z, gr, gi);
}
void lz_launch_multidot(const double* V, double* w, double* partial, const int32_t* ctl, int64_t D,
                        int batch, int cap, int win, const int32_t* gate, cudaStream_t st, const double* h_pre,
                        double* npart_pre, bool pair) {
  const dim3 g(lz_dot_nchunk(D), batch);
  if (pair)
    k_multidot<true><<<g, LZ_THREADS, 0, st>>>(V, w, partial, ctl, D, batch, cap, lz_dot_nchunk(D), win, gate, h_pre,
                                               npart_pre);
  else
    k_multidot<false><<<g, LZ_THREADS, 0, st>>>(V, w, partial, ctl, D, batch, cap, lz_dot_nchunk(D), win, gate,
                                                h_pre, npart_pre);
}
void lz_launch_dots_local(const double* V, const double* w, double* partial, const int32_t* ctl, int64_t D,
                          int batch, int cap, cudaStream_t st, bool pair) {
  const dim3 g(lz_dot_nchunk(D), batch);
  if (pair)
    k_dots_local<true><<<g, LZ_THREADS, 0, st>>>(V, w, partial, ctl, D, batch, cap, lz_dot_nchunk(D));
  else
    k_dots_local<false><<<g, LZ_THREADS, 0, st>>>(V, w, partial, ctl, D, batch, cap, lz_dot_nchunk(D));
}
void lz_launch_reduce_rows(const double* partial, double* h, const int32_t* ctl, int nchunk, int cap,
                           int batch, int win, const int32_t* gate, cudaStream_t st) {
  const int rows = win ? win : cap;
  k_reduce_rows<<<dim3(batch, (rows + 7) / 8), 256, 0, st>>>(partial, h, ctl, nchunk, cap, win, gate);
}
void lz_launch_multiaxpy(const double* V, double* w, const double* h, double* norm_partial,
                         const int32_t* ctl, int64_t D, int batch, int cap, int nchunk, int win,
                         const int32_t* gate, cudaStream_t st, bool pair) {
  if (pair)
    k_multiaxpy<true><<<dim3(nchunk, batch), LZ_THREADS, cap * sizeof(double), st>>>(V, w, h, norm_partial, ctl, D,
                                                                                   batch, cap, nchunk, win, gate);
  else
    k_multiaxpy<false><<<dim3(nchunk, batch), LZ_THREADS, cap * sizeof(double), st>>>(V, w, h, norm_partial, ctl,
                                                                                    D, batch, cap, nchunk, win, gate);
}
void lz_launch_dgks(const double* npart_a, const double* npart_b, int32_t* gate, const int32_t* ctl, int batch,
                    int nchunk_a, int nchunk, cudaStream_t st) {
  k_dgks<<<batch, 32, 0, st>>>(npart_a, npart_b, gate, ctl, nchunk_a, nchunk);
}
void lz_launch_finalize_ab(const double* h, const double* npart_b, const double* npart_c, const int32_t* gate,
                           double* ab, const int32_t* ctl, int batch, int cap, int nchunk, cudaStream_t st) {
  k_finalize_ab<<<batch, 32, 0, st>>>(h, npart_b, npart_c, gate, ab, ctl, batch, cap, nchunk);
}
void lz_launch_tridiag(const double* ab, double* s, double* out, int32_t* ctl, const double* tol, int batch,
                       int cap, int64_t D, cudaStream_t st, int final_pass) {
  k_tridiag<<<batch, 32, (5 * cap * sizeof(double) + 5 * cap * sizeof(float)), st>>>(ab, s, out, ctl, tol, batch,
                                                                                   cap, D, final_pass);
}
static int vec_blocks(int64_t D) {
  int64_t nb = (D + 255) / 256;
  return (int)(nb < 2048 ? (nb < 1 ? 1 : nb) : 2048);
}
void lz_launch_next_vector(const double* w, const double* ab, double* V, double* vcur, const int32_t* ctl,
                           int64_t D, int batch, int cap, cudaStream_t st, bool pair) {
  if (pair) k_next_vector<true><<<dim3(vec_blocks(D), batch), 256, 0, st>>>(w, ab, V, vcur, ctl, D, batch, cap);
  else k_next_vector<false><<<dim3(vec_blocks(D), batch), 256, 0, st>>>(w, ab, V, vcur, ctl, D, batch, cap);
}
void lz_launch_advance(int32_t* ctl, int batch, cudaStream_t st) { k_advance<<<1, 32, 0, st>>>(ctl, batch); }
void lz_launch_sumsq(const double* x, double* part, int64_t D, int batch, int nchunk, cudaStream_t st) {
  k_sumsq<<<dim3(nchunk, batch), LZ_THREADS, 0, st>>>(x, part, D, nchunk);
}
void lz_launch_dot(const double* x, const double* y, double* part, int64_t D, int batch, int nchunk,
                   cudaStream_t st) {
  k_dot<<<dim3(nchunk, batch), LZ_THREADS, 0, st>>>(x, y, part, D, nchunk);
}
void lz_launch_sum_chunks(const double* part, double* res, int nchunk, int batch, cudaStream_t st) {
  k_sum_chunks<<<(batch + 127) / 128, 128, 0, st>>>(part, res, nchunk, batch);
}
void lz_launch_scale_unit(const double* x, const double* nrm2, double* y, double* y2, int64_t D, int batch,
                          cudaStream_t st, bool pair) {
  if (pair) k_scale_unit<true><<<dim3(vec_blocks(D), batch), 256, 0, st>>>(x, nrm2, y, y2, D);
  else k_scale_unit<false><<<dim3(vec_blocks(D), batch), 256, 0, st>>>(x, nrm2, y, y2, D);
}
void lz_launch_ritz(const double* V, const double* s, const int32_t* ctl, double* out, int64_t D, int batch,
                    int cap, cudaStream_t st, bool pair) {
  if (pair) k_ritz<true><<<dim3(vec_blocks(D), batch), 256, 0, st>>>(V, s, ctl, out, D, batch, cap);
  else k_ritz<false><<<dim3(vec_blocks(D), batch), 256, 0, st>>>(V, s, ctl, out, D, batch, cap);
}
void lz_launch_div_rows(double* v, const double* nrm2, int n_terms, int batch, cudaStream_t st) {
  const int n = n_terms * batch;
  k_div_rows<<<(n + 127) / 128, 128, 0, st>>>(v, nrm2, n_terms, batch);
}
void lz_launch_reduce_terms(const double* part, const int32_t* ptr, const int32_t* idx, double* out, int n,
                            cudaStream_t st) {
  if (n == 0) return;
  k_reduce_terms<<<n, 256, 0, st>>>(part, ptr, idx, out, n);
}

}  // namespace dmrg
