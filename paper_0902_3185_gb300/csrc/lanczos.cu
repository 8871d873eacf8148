// Float64 Lanczos kernels: Krylov scalars, full reorthogonalisation (classical
// Gram-Schmidt applied twice), the tridiagonal eigenproblem and the Ritz vector.
//
// Paper Sec. 3.3: each targeted symmetry block is diagonalised with Lanczos,
// which needs only x += H y.  Everything here runs on the device for all batch
// members at once and reads the iteration index from device memory, so one
// captured CUDA graph replays any iteration without host round trips.
//
// Control words (int32, device): [0] j = index of the current Krylov vector,
// [1] max_iter, [2] check_every, [3] all members done, then per member b:
// [4 + b] done code (0 running, 1 converged, 2 breakdown, 3 NaN, 4 cap hit)
// and [4 + batch + b] number of Lanczos vectors in its tridiagonal matrix.

#include <cfloat>

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

// partial[(b*nchunk + chunk)*cap + i] = sum_{d in chunk} V[i][b][d] * w[b][d], i <= j
__global__ void __launch_bounds__(LZ_THREADS)
k_multidot(const double* __restrict__ V, const double* __restrict__ w, double* __restrict__ partial,
           const int32_t* __restrict__ ctl, int64_t D, int batch, int cap, int nchunk) {
  __shared__ double red[LZ_THREADS / 32 * LZ_ROWS];
  const int b = blockIdx.y, chunk = blockIdx.x;
  if (member_done(ctl, b)) return;
  const int j = ctl[LZ_CTL_J];
  double wv[LZ_EPT];
  int64_t dd[LZ_EPT];
#pragma unroll
  for (int e = 0; e < LZ_EPT; ++e) {
    dd[e] = (int64_t)chunk * LZ_CHUNK + e * LZ_THREADS + threadIdx.x;
    wv[e] = dd[e] < D ? w[(int64_t)b * D + dd[e]] : 0.0;
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int i0 = 0; i0 <= j; i0 += LZ_ROWS) {
    double p[LZ_ROWS];
#pragma unroll
    for (int q = 0; q < LZ_ROWS; ++q) {
      p[q] = 0.0;
      const int i = i0 + q;
      if (i <= j) {
        const double* v = V + ((int64_t)i * batch + b) * D;
#pragma unroll
        for (int e = 0; e < LZ_EPT; ++e)
          if (dd[e] < D) p[q] = fma(v[dd[e]], wv[e], p[q]);
      }
    }
#pragma unroll
    for (int q = 0; q < LZ_ROWS; ++q) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) p[q] += __shfl_down_sync(0xffffffffu, p[q], o);
    }
    __syncthreads();
    if (lane == 0)
#pragma unroll
      for (int q = 0; q < LZ_ROWS; ++q) red[q * (LZ_THREADS / 32) + wid] = p[q];
    __syncthreads();
    if (threadIdx.x < LZ_ROWS && i0 + (int)threadIdx.x <= j) {
      double t = 0.0;
      for (int w2 = 0; w2 < LZ_THREADS / 32; ++w2) t += red[threadIdx.x * (LZ_THREADS / 32) + w2];
      partial[((int64_t)b * nchunk + chunk) * cap + i0 + threadIdx.x] = t;
    }
  }
}

// h[b*cap + i] = sum over chunks (in order) of the partials, i <= j
__global__ void k_reduce_rows(const double* __restrict__ partial, double* __restrict__ h,
                              const int32_t* __restrict__ ctl, int nchunk, int cap) {
  const int b = blockIdx.x;
  if (member_done(ctl, b)) return;
  const int j = ctl[LZ_CTL_J];
  for (int i = threadIdx.x; i <= j; i += blockDim.x) {
    double t = 0.0;
    for (int ch = 0; ch < nchunk; ++ch) t += partial[((int64_t)b * nchunk + ch) * cap + i];
    h[(int64_t)b * cap + i] = t;
  }
}

// w[b] -= sum_{i<=j} V[i][b] h[b][i]; with norm_partial != NULL also the
// per-chunk sum of squares of the new w.
__global__ void __launch_bounds__(LZ_THREADS)
k_multiaxpy(const double* __restrict__ V, double* __restrict__ w, const double* __restrict__ h,
            double* __restrict__ norm_partial, const int32_t* __restrict__ ctl, int64_t D, int batch,
            int cap, int nchunk) {
  extern __shared__ double sh[];
  __shared__ double red[LZ_THREADS / 32];
  const int b = blockIdx.y, chunk = blockIdx.x;
  if (member_done(ctl, b)) return;
  const int j = ctl[LZ_CTL_J];
  for (int i = threadIdx.x; i <= j; i += blockDim.x) sh[i] = h[(int64_t)b * cap + i];
  __syncthreads();
  double nrm = 0.0;
#pragma unroll
  for (int e = 0; e < LZ_EPT; ++e) {
    const int64_t d = (int64_t)chunk * LZ_CHUNK + e * LZ_THREADS + threadIdx.x;
    if (d >= D) continue;
    double acc = w[(int64_t)b * D + d];
    for (int i = 0; i <= j; ++i) acc = fma(-V[((int64_t)i * batch + b) * D + d], sh[i], acc);
    w[(int64_t)b * D + d] = acc;
    nrm = fma(acc, acc, nrm);
  }
  if (norm_partial) {
    const double t = block_sum(nrm, red);
    if (threadIdx.x == 0) norm_partial[(int64_t)b * nchunk + chunk] = t;
  }
}

// alpha_j = h1[j] + h2[j], beta_j = sqrt(sum of norm partials)
__global__ void k_finalize_ab(const double* __restrict__ h, const double* __restrict__ norm_partial,
                              double* __restrict__ ab, const int32_t* __restrict__ ctl, int batch,
                              int cap, int nchunk) {
  const int b = blockIdx.x;
  if (threadIdx.x != 0 || member_done(ctl, b)) return;
  const int j = ctl[LZ_CTL_J];
  double t = 0.0;
  for (int ch = 0; ch < nchunk; ++ch) t += norm_partial[(int64_t)b * nchunk + ch];
  ab[(int64_t)b * cap + j] = h[(int64_t)b * cap + j] + h[((int64_t)batch + b) * cap + j];
  ab[((int64_t)batch + b) * cap + j] = sqrt(t);
}

// number of eigenvalues of T (diag a, off-diagonal e) below x: signs of the
// LDL^T pivots (Sylvester), with a zero pivot nudged off zero
__device__ int sturm_count(const double* a, const double* e, int n, double x) {
  int cnt = 0;
  double d = a[0] - x;
  if (d < 0) ++cnt;
  for (int i = 1; i < n; ++i) {
    if (d == 0.0) d = DBL_MIN;
    d = (a[i] - x) - e[i - 1] * e[i - 1] / d;
    if (d < 0) ++cnt;
  }
  return cnt;
}

// Lowest eigenpair of the (j+1) x (j+1) tridiagonal matrix of each member,
// convergence test, and the Ritz coefficients s.  One block per member.
//  - multisection: the LZ_TRI threads evaluate Sturm counts at evenly spaced
//    points of the bracket [lo, hi] that holds the lowest eigenvalue, until
//    the bracket is as narrow as float64 resolves;
//  - inverse iteration with the shift lo < lambda_min: T - lo I is positive
//    definite, so its LDL^T solve (one thread, O(n)) is stable, and two
//    solves give the eigenvector to working precision.
__global__ void __launch_bounds__(LZ_TRI)
k_tridiag(const double* __restrict__ ab, double* __restrict__ s_out, double* __restrict__ out,
          int32_t* __restrict__ ctl, const double* __restrict__ tolp, int batch, int cap, int64_t D) {
  extern __shared__ double sm[];
  double* a = sm;
  double* e = sm + cap;
  double* z = sm + 2 * cap;
  double* dpiv = sm + 3 * cap;
  __shared__ double s_lo, s_hi, s_scale;
  __shared__ int s_first;
  __shared__ int s_do;
  const int b = blockIdx.x;
  if (member_done(ctl, b)) return;
  const int j = ctl[LZ_CTL_J];
  const int n = j + 1;
  const int max_iter = ctl[LZ_CTL_MAXIT];
  const int check_every = ctl[LZ_CTL_CHECK];
  const double tol = *tolp;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    a[i] = ab[(int64_t)b * cap + i];
    e[i] = ab[((int64_t)batch + b) * cap + i];  // e[n-1] = beta_j (the residual factor)
  }
  __syncthreads();
  const double beta = e[n - 1];
  if (threadIdx.x == 0) {
    double amax = 0.0;
    for (int i = 0; i < n; ++i) amax = fmax(amax, fabs(a[i]));
    s_scale = fmax(1.0, amax);
    const bool bad = !isfinite(a[n - 1]) || !isfinite(beta);
    const bool small_beta = beta < 1e-14 * s_scale;
    s_do = bad ? 2 : ((n % check_every == 0) || n >= max_iter || (int64_t)n >= D || small_beta) ? 1 : 0;
  }
  __syncthreads();
  if (s_do == 0) return;
  if (s_do == 2) {
    if (threadIdx.x == 0) {
      ctl[LZ_CTL_MEMBER + b] = LZ_NAN;
      ctl[LZ_CTL_MEMBER + batch + b] = n;
    }
    return;
  }
  // Gershgorin bracket for the lowest eigenvalue, hi = min diagonal
  if (threadIdx.x == 0) {
    double lo = DBL_MAX, hi = DBL_MAX;
    for (int i = 0; i < n; ++i) {
      const double r = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i < n - 1 ? fabs(e[i]) : 0.0);
      lo = fmin(lo, a[i] - r);
      hi = fmin(hi, a[i]);
    }
    s_lo = lo - 1e-300;
    s_hi = hi;
  }
  __syncthreads();
  for (int round = 0; round < 64; ++round) {
    const double lo = s_lo, hi = s_hi;
    if (!(hi - lo > 4.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi))) || hi <= lo) break;
    const double x = lo + (hi - lo) * (double)(threadIdx.x + 1) / (double)(blockDim.x + 1);
    const int cnt = sturm_count(a, e, n, x);
    if (threadIdx.x == 0) s_first = blockDim.x;
    __syncthreads();
    if (cnt >= 1) atomicMin(&s_first, (int)threadIdx.x);
    __syncthreads();
    if (threadIdx.x == 0) {
      const int f = s_first;
      const double step = (hi - lo) / (double)(blockDim.x + 1);
      s_hi = (f < (int)blockDim.x) ? lo + step * (f + 1) : hi;
      s_lo = lo + step * f;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    // shift strictly below lambda_min so that T - lo I is positive definite
    const double lo = s_lo - 4.0 * DBL_EPSILON * s_scale;
    const double theta = 0.5 * (s_lo + s_hi);
    // inverse iteration with shift lo
    for (int i = 0; i < n; ++i) z[i] = 1.0;
    for (int it = 0; it < 3; ++it) {
      // LDL^T: dpiv[i] pivots, forward then backward substitution
      dpiv[0] = a[0] - lo;
      for (int i = 1; i < n; ++i) {
        double dp = dpiv[i - 1];
        if (dp == 0.0) dp = DBL_MIN;
        const double l = e[i - 1] / dp;
        dpiv[i] = (a[i] - lo) - l * e[i - 1];
        z[i] -= l * z[i - 1];
      }
      for (int i = 0; i < n; ++i) z[i] /= (dpiv[i] == 0.0 ? DBL_MIN : dpiv[i]);
      for (int i = n - 2; i >= 0; --i) {
        double dp = dpiv[i];
        if (dp == 0.0) dp = DBL_MIN;
        z[i] -= (e[i] / dp) * z[i + 1];
      }
      double nz = 0.0;
      for (int i = 0; i < n; ++i) nz = fma(z[i], z[i], nz);
      nz = sqrt(nz);
      const double sg = z[0] < 0.0 ? -1.0 : 1.0;
      for (int i = 0; i < n; ++i) z[i] = sg * z[i] / nz;
    }
    const double resid = beta * fabs(z[n - 1]);
    const double scale = fmax(1.0, fabs(theta));
    int code = 0;
    if (!isfinite(theta) || !isfinite(resid)) code = LZ_NAN;
    else if (beta < 1e-14 * scale || (int64_t)n >= D) code = LZ_BREAKDOWN;
    else if (resid <= tol * scale) code = LZ_CONVERGED;
    else if (n >= max_iter) code = LZ_CAP;
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
__global__ void k_next_vector(const double* __restrict__ w, const double* __restrict__ ab,
                              double* __restrict__ V, double* __restrict__ vcur,
                              const int32_t* __restrict__ ctl, int64_t D, int batch, int cap) {
  const int b = blockIdx.y;
  if (member_done(ctl, b)) return;
  const int j = ctl[LZ_CTL_J];
  const double inv = 1.0 / ab[((int64_t)batch + b) * cap + j];
  double* vn = V + ((int64_t)(j + 1) * batch + b) * D;
  for (int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; d < D; d += (int64_t)gridDim.x * blockDim.x) {
    const double v = w[(int64_t)b * D + d] * inv;
    vn[d] = v;
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
__global__ void k_scale_unit(const double* __restrict__ x, const double* __restrict__ nrm2,
                             double* __restrict__ y, double* __restrict__ y2, int64_t D) {
  const int b = blockIdx.y;
  const double inv = 1.0 / sqrt(nrm2[b]);
  for (int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; d < D; d += (int64_t)gridDim.x * blockDim.x) {
    const double v = x[(int64_t)b * D + d] * inv;
    y[(int64_t)b * D + d] = v;
    if (y2) y2[(int64_t)b * D + d] = v;
  }
}

// out[b] = sum_{i < n_b} s[b][i] V[i][b]
__global__ void k_ritz(const double* __restrict__ V, const double* __restrict__ s,
                       const int32_t* __restrict__ ctl, double* __restrict__ out, int64_t D, int batch,
                       int cap) {
  const int b = blockIdx.y;
  const int n = ctl[LZ_CTL_MEMBER + batch + b];
  for (int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; d < D; d += (int64_t)gridDim.x * blockDim.x) {
    double t = 0.0;
    for (int i = 0; i < n; ++i) t = fma(s[(int64_t)b * cap + i], V[((int64_t)i * batch + b) * D + d], t);
    out[(int64_t)b * D + d] = t;
  }
}

// dE_dc[b][k] = dots[b][k] / nrm2[b]
__global__ void k_div_rows(double* __restrict__ v, const double* __restrict__ nrm2, int n_terms, int batch) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_terms * batch) return;
  v[i] /= nrm2[i / n_terms];
}

// dc[b*n_terms + k] = sum of the dot-tile partials of (b, k), in list order
__global__ void k_reduce_terms(const double* __restrict__ part, const int32_t* __restrict__ ptr,
                               const int32_t* __restrict__ idx, double* __restrict__ out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double t = 0.0;
  for (int q = ptr[i]; q < ptr[i + 1]; ++q) t += part[idx[q]];
  out[i] = t;
}

// ------------------------------------------------------------- launchers
void lz_launch_multidot(const double* V, const double* w, double* partial, const int32_t* ctl, int64_t D,
                        int batch, int cap, int nchunk, cudaStream_t st) {
  k_multidot<<<dim3(nchunk, batch), LZ_THREADS, 0, st>>>(V, w, partial, ctl, D, batch, cap, nchunk);
}
void lz_launch_reduce_rows(const double* partial, double* h, const int32_t* ctl, int nchunk, int cap,
                           int batch, cudaStream_t st) {
  k_reduce_rows<<<batch, 128, 0, st>>>(partial, h, ctl, nchunk, cap);
}
void lz_launch_multiaxpy(const double* V, double* w, const double* h, double* norm_partial,
                         const int32_t* ctl, int64_t D, int batch, int cap, int nchunk, cudaStream_t st) {
  k_multiaxpy<<<dim3(nchunk, batch), LZ_THREADS, cap * sizeof(double), st>>>(V, w, h, norm_partial, ctl, D,
                                                                            batch, cap, nchunk);
}
void lz_launch_finalize_ab(const double* h, const double* norm_partial, double* ab, const int32_t* ctl,
                           int batch, int cap, int nchunk, cudaStream_t st) {
  k_finalize_ab<<<batch, 32, 0, st>>>(h, norm_partial, ab, ctl, batch, cap, nchunk);
}
void lz_launch_tridiag(const double* ab, double* s, double* out, int32_t* ctl, const double* tol, int batch,
                       int cap, int64_t D, cudaStream_t st) {
  k_tridiag<<<batch, LZ_TRI, 4 * cap * sizeof(double), st>>>(ab, s, out, ctl, tol, batch, cap, D);
}
static int vec_blocks(int64_t D) {
  int64_t nb = (D + 255) / 256;
  return (int)(nb < 2048 ? (nb < 1 ? 1 : nb) : 2048);
}
void lz_launch_next_vector(const double* w, const double* ab, double* V, double* vcur, const int32_t* ctl,
                           int64_t D, int batch, int cap, cudaStream_t st) {
  k_next_vector<<<dim3(vec_blocks(D), batch), 256, 0, st>>>(w, ab, V, vcur, ctl, D, batch, cap);
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
                          cudaStream_t st) {
  k_scale_unit<<<dim3(vec_blocks(D), batch), 256, 0, st>>>(x, nrm2, y, y2, D);
}
void lz_launch_ritz(const double* V, const double* s, const int32_t* ctl, double* out, int64_t D, int batch,
                    int cap, cudaStream_t st) {
  k_ritz<<<dim3(vec_blocks(D), batch), 256, 0, st>>>(V, s, ctl, out, D, batch, cap);
}
void lz_launch_div_rows(double* v, const double* nrm2, int n_terms, int batch, cudaStream_t st) {
  const int n = n_terms * batch;
  k_div_rows<<<(n + 127) / 128, 128, 0, st>>>(v, nrm2, n_terms, batch);
}
void lz_launch_reduce_terms(const double* part, const int32_t* ptr, const int32_t* idx, double* out, int n,
                            cudaStream_t st) {
  if (n == 0) return;
  k_reduce_terms<<<(n + 127) / 128, 128, 0, st>>>(part, ptr, idx, out, n);
}

}  // namespace dmrg
