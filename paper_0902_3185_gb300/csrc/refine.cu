// Float64 refinement of a mixed-precision ground state (batched, on device).
//
// Given psi from the mixed-precision Lanczos, each outer step computes the
// float64 residual r = H psi - theta psi (theta = <psi, H psi>, psi
// normalised) with one float64 product, then solves the projected correction
// equation
//     P (H - theta) P t = -r,   P = 1 - psi psi^T,   t orthogonal to psi,
// by conjugate gradients whose products are the tensor-core (mixed) ones, and
// updates psi <- (psi + t) / |psi + t|.  For theta below the second
// eigenvalue, P (H - theta) P is positive definite on the complement of psi,
// so CG applies.  CG is preconditioned with the diagonal of H (as in
// Davidson's method): M = max(diag(H) - theta, delta) elementwise, applied on
// the complement of psi as
//     z = M^-1 r - gamma M^-1 psi,   gamma = <psi, M^-1 r> / <psi, M^-1 psi>,
// which is symmetric, positive semidefinite and maps into psi's complement.  Each outer step shrinks the eigenvector error by about
// (mixed product error) * |H| / gap, so a few float64 products replace a
// float64 Lanczos run.  All vectors and scalars are float64; reductions are
// two-stage and fixed-order (deterministic).
//
// Per-member scalars (float64, device): [0] theta, [1] |b|, [2] rr, [3] pq,
// [4] s1 = <psi, q>, [5] alpha, [6] beta, [7] rr_new, [8] rho = <r, z>,
// [9] gamma, [10] mu = <psi, M^-1 psi>, [11..12] <psi, M^-1 r>, <r, M^-1 r>;
// control (int32):
// [b] done flag of the inner solve, [B + b] inner iterations, [2B] all
// done, [2B + 1] inner iteration cap.

#include "internal.h"
#include "lanczos.h"
#include "refine.h"

namespace dmrg {

__device__ __forceinline__ double rf_block_sum(double v, double* red) {
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

#define RF_LOOP(body)                                                                  \
  _Pragma("unroll") for (int e = 0; e < LZ_EPT; ++e) {                               \
    const int64_t d = (int64_t)chunk * LZ_CHUNK + e * LZ_THREADS + threadIdx.x;      \
    if (d >= D) continue;                                                            \
    const int64_t i = (int64_t)b * D + d;                                            \
    body                                                                             \
  }

// partials of <psi, q>, <p, q>, <p, p>, <p, psi> for q = H p (rows 0..3);
// the projected operator's q = H p - theta p - s1 psi is formed in the update
__global__ void __launch_bounds__(LZ_THREADS)
k_rf_dots4(const double* __restrict__ q, const double* __restrict__ p, const double* __restrict__ psi,
           const int32_t* __restrict__ ctl, double* __restrict__ part, int64_t D, int nchunk, int batch,
           const int32_t* __restrict__ stop) {
  __shared__ double red[LZ_THREADS / 32];
  const int b = blockIdx.y, chunk = blockIdx.x;
  if ((stop && *stop) || ctl[b]) return;
  double a[4] = {0.0, 0.0, 0.0, 0.0};
  RF_LOOP({
    const double qi = q[i];
    const double pi = p[i];
    const double si = psi[i];
    a[0] = fma(si, qi, a[0]);
    a[1] = fma(pi, qi, a[1]);
    a[2] = fma(pi, pi, a[2]);
    a[3] = fma(pi, si, a[3]);
  })
  const int64_t stride = (int64_t)batch * nchunk, at = (int64_t)b * nchunk + chunk;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const double s = rf_block_sum(a[k], red);
    if (threadIdx.x == 0) part[k * stride + at] = s;
  }
}

// s1 = <psi, Hp> - theta <psi, p>; pq = <p, Hp> - theta <p, p> - s1 <p, psi>;
// alpha = rho / pq (a non-positive pq ends the member's solve).  One warp per
// member: lane-strided chunk sums, then a fixed shuffle tree.
__global__ void k_rf_alpha4(const double* __restrict__ part, double* __restrict__ sc, int32_t* __restrict__ ctl,
                            int nchunk, int batch, const int32_t* __restrict__ stop) {
  const int b = blockIdx.x;
  if ((stop && *stop) || ctl[b]) return;
  double v[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const double* row = part + ((int64_t)k * batch + b) * nchunk;
    double t = 0.0;
    for (int ch = threadIdx.x; ch < nchunk; ch += 32) t += row[ch];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    v[k] = t;
  }
  if (threadIdx.x != 0) return;
  double* s = sc + b * RF_NSC;
  const double th = s[RF_THETA];
  const double s1 = v[0] - th * v[3];
  const double pq = v[1] - th * v[2] - s1 * v[3];
  s[RF_S1] = s1;
  s[RF_PQ] = pq;
  if (!(pq > 0.0) || !isfinite(pq)) {
    ctl[b] = 2;
    s[RF_ALPHA] = 0.0;
    return;
  }
  s[RF_ALPHA] = s[RF_RHO] / pq;
}

// t += alpha p ; res -= alpha (q - theta p - s1 psi) with q = H p ; partials
// of <res, res>, <psi, M^-1 res>, <res, M^-1 res> at part + k B nchunk,
// k = 0..2 (<res, M^-1 psi> equals <psi, M^-1 res>: M is diagonal)
__global__ void __launch_bounds__(LZ_THREADS)
k_rf_update(double* __restrict__ t, double* __restrict__ res, const double* __restrict__ p,
            const double* __restrict__ q, const double* __restrict__ psi, const double* __restrict__ minv,
            const double* __restrict__ sc, const int32_t* __restrict__ ctl, double* __restrict__ part, int64_t D,
            int nchunk, int batch, const int32_t* __restrict__ stop) {
  __shared__ double red[LZ_THREADS / 32];
  const int b = blockIdx.y, chunk = blockIdx.x;
  if ((stop && *stop) || ctl[b]) return;
  const double al = sc[b * RF_NSC + RF_ALPHA];
  const double th = sc[b * RF_NSC + RF_THETA], s1 = sc[b * RF_NSC + RF_S1];
  double rr = 0.0, a1 = 0.0, a2 = 0.0;
  RF_LOOP({
    const double pi = p[i];
    t[i] = fma(al, pi, t[i]);
    const double qp = fma(-s1, psi[i], fma(-th, pi, q[i]));  // (P (H - theta) P p)_i
    const double v = fma(-al, qp, res[i]);
    res[i] = v;
    const double mv = minv[i] * v;
    rr = fma(v, v, rr);
    a1 = fma(psi[i], mv, a1);
    a2 = fma(v, mv, a2);
  })
  const int64_t stride = (int64_t)batch * nchunk, at = (int64_t)b * nchunk + chunk;
  rr = rf_block_sum(rr, red);
  if (threadIdx.x == 0) part[at] = rr;
  a1 = rf_block_sum(a1, red);
  if (threadIdx.x == 0) part[stride + at] = a1;
  a2 = rf_block_sum(a2, red);
  if (threadIdx.x == 0) part[2 * stride + at] = a2;
}

// p = M^-1 (res - gamma psi) + beta p  (first: beta = 0)
__global__ void __launch_bounds__(LZ_THREADS)
k_rf_dir(double* __restrict__ p, const double* __restrict__ res, const double* __restrict__ psi,
         const double* __restrict__ minv, const double* __restrict__ sc, const int32_t* __restrict__ ctl, int64_t D,
         int first, const int32_t* __restrict__ stop) {
  const int b = blockIdx.y, chunk = blockIdx.x;
  if ((stop && *stop) || (ctl && ctl[b])) return;
  const double be = first ? 0.0 : sc[b * RF_NSC + RF_BETA];
  const double ga = sc[b * RF_NSC + RF_GAMMA];
  RF_LOOP({
    const double z = minv[i] * fma(-ga, psi[i], res[i]);
    p[i] = first ? z : fma(be, p[i], z);
  })
}

// per member: diag(H) = sum over terms with diagonal blocks of c_k diag_k
__global__ void k_rf_diag(const double* __restrict__ dterm, const int32_t* __restrict__ terms, int nd,
                          const double* __restrict__ coef, int n_terms, double* __restrict__ diag, int64_t D) {
  const int b = blockIdx.y;
  for (int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; d < D; d += (int64_t)gridDim.x * blockDim.x) {
    double v = 0.0;
    for (int k = 0; k < nd; ++k) v = fma(coef[(int64_t)b * n_terms + terms[k]], dterm[(int64_t)k * D + d], v);
    diag[(int64_t)b * D + d] = v;
  }
}

// M^-1 = 1 / max(diag - theta, delta max(1, |theta|))
__global__ void k_rf_minv(const double* __restrict__ diag, const double* __restrict__ sc, double* __restrict__ minv,
                          int64_t D) {
  const int b = blockIdx.y;
  const double th = sc[b * RF_NSC + RF_THETA];
  const double delta = RF_DELTA * fmax(1.0, fabs(th));
  for (int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; d < D; d += (int64_t)gridDim.x * blockDim.x)
    minv[(int64_t)b * D + d] = 1.0 / fmax(diag[(int64_t)b * D + d] - th, delta);
}

// sc[b][RR_NEW, A1, A2 (, MU)] = sums of the partial rows 0..2 (and 3 when
// with_mu), fixed order
__global__ void k_rf_sum4(const double* __restrict__ part, double* __restrict__ sc, int nchunk, int batch,
                          int with_mu, const int32_t* __restrict__ ctl, const int32_t* __restrict__ stop) {
  const int b = blockIdx.x, k = threadIdx.x;
  if (k >= 3 + with_mu || (stop && *stop) || (ctl && ctl[b])) return;
  const double* row = part + ((int64_t)k * batch + b) * nchunk;
  double t = 0.0;
  for (int ch = 0; ch < nchunk; ++ch) t += row[ch];
  const int slot[4] = {RF_RRNEW, RF_A1, RF_A2, RF_MU};
  sc[b * RF_NSC + slot[k]] = t;
}

// start of an outer step: gamma = a1 / mu, rho = a2 - gamma a3 from the
// start kernel's sums (rr in RF_RRNEW)
__global__ void k_rf_rho0(double* __restrict__ sc, int batch) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch) return;
  double* s = sc + b * RF_NSC;
  s[RF_RR] = s[RF_RRNEW];
  s[RF_BNORM] = sqrt(s[RF_RRNEW]);
  s[RF_GAMMA] = s[RF_A1] / s[RF_MU];
  s[RF_RHO] = s[RF_A2] - s[RF_GAMMA] * s[RF_A1];
}

// gamma, rho = <res, z>, beta = rho_new / rho; stop a member at
// |res| <= eps |b|, the cap, or a non-positive rho (preconditioned residual
// vanished); one thread per member, the block-wide AND gives the "all done" flag
__global__ void k_rf_beta(double* __restrict__ sc, int32_t* __restrict__ ctl, const double* __restrict__ eps,
                          int batch, int32_t* __restrict__ stop) {
  if (blockIdx.x != 0 || *stop) return;  // uniform over the block
  const int max_inner = ctl[2 * batch + 1];
  int all = 1;
  for (int b = threadIdx.x; b < batch; b += blockDim.x) {  // one thread per member
    if (!ctl[b]) {
      double* s = sc + b * RF_NSC;
      const double rn = s[RF_RRNEW];
      s[RF_RR] = rn;
      s[RF_GAMMA] = s[RF_A1] / s[RF_MU];
      const double rho = s[RF_A2] - s[RF_GAMMA] * s[RF_A1];
      s[RF_BETA] = rho / s[RF_RHO];
      s[RF_RHO] = rho;
      const int it = ++ctl[batch + b];
      if (sqrt(rn) <= (*eps) * s[RF_BNORM] || it >= max_inner || !isfinite(rn) || !(rho > 0.0)) ctl[b] = 1;
    }
    all &= ctl[b] != 0;
  }
  if (__syncthreads_and(all) && threadIdx.x == 0) *stop = 1;
}

// outer step: r = w - theta psi into res (negated: the CG right-hand side is
// -r), t = 0; partials of <res, res>, <psi, M^-1 res>, <res, M^-1 res>,
// <psi, M^-1 psi> (rows 0..3)
__global__ void __launch_bounds__(LZ_THREADS)
k_rf_start(const double* __restrict__ w, const double* __restrict__ psi, const double* __restrict__ minv,
           double* __restrict__ res, double* __restrict__ t, const double* __restrict__ sc, double* __restrict__ part,
           int64_t D, int nchunk, int batch) {
  __shared__ double red[LZ_THREADS / 32];
  const int b = blockIdx.y, chunk = blockIdx.x;
  const double th = sc[b * RF_NSC + RF_THETA];
  double a[4] = {0.0, 0.0, 0.0, 0.0};
  RF_LOOP({
    const double v = th * psi[i] - w[i];
    res[i] = v;
    t[i] = 0.0;
    const double mv = minv[i] * v;
    const double mp = minv[i] * psi[i];
    a[0] = fma(v, v, a[0]);
    a[1] = fma(psi[i], mv, a[1]);
    a[2] = fma(v, mv, a[2]);
    a[3] = fma(mp, psi[i], a[3]);
  })
  const int64_t stride = (int64_t)batch * nchunk, at = (int64_t)b * nchunk + chunk;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const double s = rf_block_sum(a[k], red);
    if (threadIdx.x == 0) part[k * stride + at] = s;
  }
}

// per member: theta from <psi, w>; sets |b| and rr from |res|^2 afterwards
__global__ void k_rf_set(double* __restrict__ sc, const double* __restrict__ src, int slot, int batch, int sqrt_too) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch) return;
  sc[b * RF_NSC + slot] = src[b];
  if (sqrt_too) {
    sc[b * RF_NSC + RF_RR] = src[b];
    sc[b * RF_NSC + RF_BNORM] = sqrt(src[b]);
  }
}

// psi += t for members flagged active (mask[b] != 0)
__global__ void k_rf_apply(double* __restrict__ psi, const double* __restrict__ t, const int32_t* __restrict__ mask,
                           int64_t D) {
  const int b = blockIdx.y;
  if (!mask[b]) return;
  for (int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; d < D; d += (int64_t)gridDim.x * blockDim.x)
    psi[(int64_t)b * D + d] += t[(int64_t)b * D + d];
}

// ------------------------------------------------------------- launchers
static dim3 vgrid(int64_t D, int batch) { return dim3(lz_nchunk(D), batch); }

void rf_launch_dots4(const double* q, const double* p, const double* psi, const int32_t* ctl, double* part,
                     int64_t D, int B, const int32_t* stop, cudaStream_t st) {
  k_rf_dots4<<<vgrid(D, B), LZ_THREADS, 0, st>>>(q, p, psi, ctl, part, D, lz_nchunk(D), B, stop);
}
void rf_launch_alpha4(const double* part, double* sc, int32_t* ctl, int64_t D, int B, const int32_t* stop,
                      cudaStream_t st) {
  k_rf_alpha4<<<B, 32, 0, st>>>(part, sc, ctl, lz_nchunk(D), B, stop);
}
void rf_launch_update(double* t, double* res, const double* p, const double* q, const double* psi,
                      const double* minv, const double* sc, const int32_t* ctl, double* part, int64_t D, int B,
                      const int32_t* stop, cudaStream_t st) {
  k_rf_update<<<vgrid(D, B), LZ_THREADS, 0, st>>>(t, res, p, q, psi, minv, sc, ctl, part, D, lz_nchunk(D), B,
                                                  stop);
}
void rf_launch_dir(double* p, const double* res, const double* psi, const double* minv, const double* sc,
                   const int32_t* ctl, int64_t D, int B, int first, const int32_t* stop, cudaStream_t st) {
  k_rf_dir<<<vgrid(D, B), LZ_THREADS, 0, st>>>(p, res, psi, minv, sc, ctl, D, first, stop);
}
void rf_launch_sum4(const double* part, double* sc, int64_t D, int B, int with_mu, const int32_t* ctl,
                    const int32_t* stop, cudaStream_t st) {
  k_rf_sum4<<<B, 32, 0, st>>>(part, sc, lz_nchunk(D), B, with_mu, ctl, stop);
}
static int rf_vec_blocks(int64_t D) {
  const int64_t nb = (D + 255) / 256;
  return (int)(nb > 2048 ? 2048 : (nb < 1 ? 1 : nb));
}
void rf_launch_diag(const double* dterm, const int32_t* terms, int nd, const double* coef, int n_terms,
                    double* diag, int64_t D, int B, cudaStream_t st) {
  k_rf_diag<<<dim3(rf_vec_blocks(D), B), 256, 0, st>>>(dterm, terms, nd, coef, n_terms, diag, D);
}
void rf_launch_minv(const double* diag, const double* sc, double* minv, int64_t D, int B, cudaStream_t st) {
  k_rf_minv<<<dim3(rf_vec_blocks(D), B), 256, 0, st>>>(diag, sc, minv, D);
}
void rf_launch_rho0(double* sc, int B, cudaStream_t st) { k_rf_rho0<<<(B + 63) / 64, 64, 0, st>>>(sc, B); }
void rf_launch_beta(double* sc, int32_t* ctl, const double* eps, int B, int32_t* stop, cudaStream_t st) {
  const int threads = B >= 1024 ? 1024 : ((B + 31) / 32) * 32;
  k_rf_beta<<<1, threads < 32 ? 32 : threads, 0, st>>>(sc, ctl, eps, B, stop);
}
void rf_launch_start(const double* w, const double* psi, const double* minv, double* res, double* t,
                     const double* sc, double* part, int64_t D, int B, cudaStream_t st) {
  k_rf_start<<<vgrid(D, B), LZ_THREADS, 0, st>>>(w, psi, minv, res, t, sc, part, D, lz_nchunk(D), B);
}
void rf_launch_set(double* sc, const double* src, int slot, int B, int sqrt_too, cudaStream_t st) {
  k_rf_set<<<(B + 63) / 64, 64, 0, st>>>(sc, src, slot, B, sqrt_too);
}
void rf_launch_apply(double* psi, const double* t, const int32_t* mask, int64_t D, int B, cudaStream_t st) {
  int64_t nb = (D + 255) / 256;
  if (nb > 2048) nb = 2048;
  k_rf_apply<<<dim3((unsigned)nb, B), 256, 0, st>>>(psi, t, mask, D);
}

}  // namespace dmrg
