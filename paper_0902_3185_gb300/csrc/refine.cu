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
// float64 Lanczos run.  The outer quantities are float64: the iterate, the
// residual r (one float64 product, the difference H psi - theta psi taken in
// float64), theta, |r| and the update psi + t.  The inner solve only has to
// reach the mixed product's own accuracy (relative 1e-5 at best), so its
// vectors (t, res, p, (H - theta) p, psi, M^-1) are float32, with the
// difference H p - theta p again taken in float64 and every scalar and
// reduction in float64 (float32 partials over 4 x 32 elements, then
// two-stage fixed-order float64 sums: deterministic).  GB300 issues float64
// at 1/64 of the float32 rate; this leaves one float64 operation per element
// and CG iteration.
//
// Per-member scalars (float64, device): [0] theta, [1] |b|, [2] rr, [3] pq,
// [4] s1 = <psi, (H - theta) p>, [5] alpha, [6] beta, [7] rr_new, [8] rho = <r, z>,
// [9] gamma, [10] mu = <psi, M^-1 psi>, [11..12] <psi, M^-1 r>, <r, M^-1 r>;
// control (int32):
// [b] done flag of the inner solve, [B + b] inner iterations, [2B] all
// done, [2B + 1] inner iteration cap.

#include "internal.h"
#include "lanczos.h"
#include "refine.h"
#include "tc_kernel.cuh"

namespace dmrg {

// Block sum of float32 partials: a fixed shuffle tree in float32 within each
// warp, the warp sums converted exactly to float64 (integer instructions) and
// added in warp order in float64; the result is valid in thread 0.
__device__ __forceinline__ double rf_block_sum(float v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = tc::f2d_exact(v);
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

// hp = (H - theta) p, formed in float64 from the float64 product q = H p and
// stored in float32 (the one cancellation of the step is taken in float64);
// partials of <psi, hp>, <p, hp>, <p, psi> (rows 0..2)
__global__ void __launch_bounds__(LZ_THREADS)
k_rf_dots4(const double* __restrict__ q, const float* __restrict__ p, const float* __restrict__ psi,
           float* __restrict__ hp, const double* __restrict__ sc, const int32_t* __restrict__ ctl,
           double* __restrict__ part, int64_t D, int nchunk, int batch, const int32_t* __restrict__ stop) {
  __shared__ double red[LZ_THREADS / 32];
  const int b = blockIdx.y, chunk = blockIdx.x;
  if ((stop && *stop) || ctl[b]) return;
  const double th = sc[b * RF_NSC + RF_THETA];
  float a[3] = {0.f, 0.f, 0.f};
  RF_LOOP({
    const float pi = p[i];
    const float si = psi[i];
    const float h = tc::d2f_rn32(fma(-th, tc::f2d_exact(pi), q[i]));
    hp[i] = h;
    a[0] = fmaf(si, h, a[0]);
    a[1] = fmaf(pi, h, a[1]);
    a[2] = fmaf(pi, si, a[2]);
  })
  const int64_t stride = (int64_t)batch * nchunk, at = (int64_t)b * nchunk + chunk;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double s = rf_block_sum(a[k], red);
    if (threadIdx.x == 0) part[k * stride + at] = s;
  }
}

// s1 = <psi, (H - theta) p>; pq = <p, (H - theta) p> - s1 <p, psi> = <p, P (H - theta) P p>
// (p is orthogonal to psi up to rounding); alpha = rho / pq (a non-positive pq
// ends the member's solve).  One warp per member: lane-strided chunk sums,
// then a fixed shuffle tree.
__global__ void k_rf_alpha4(const double* __restrict__ part, double* __restrict__ sc, int32_t* __restrict__ ctl,
                            int nchunk, int batch, const int32_t* __restrict__ stop) {
  const int b = blockIdx.x;
  if ((stop && *stop) || ctl[b]) return;
  double v[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double* row = part + ((int64_t)k * batch + b) * nchunk;
    double t = 0.0;
    for (int ch = threadIdx.x; ch < nchunk; ch += 32) t += row[ch];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    v[k] = t;
  }
  if (threadIdx.x != 0) return;
  double* s = sc + b * RF_NSC;
  const double s1 = v[0];
  const double pq = v[1] - s1 * v[2];
  s[RF_S1] = s1;
  s[RF_PQ] = pq;
  if (!(pq > 0.0) || !isfinite(pq)) {
    ctl[b] = 2;
    s[RF_ALPHA] = 0.0;
    return;
  }
  s[RF_ALPHA] = s[RF_RHO] / pq;
}

// t += alpha p ; res -= alpha (hp - s1 psi) = alpha P (H - theta) P p ;
// partials of <res, res>, <psi, M^-1 res>, <res, M^-1 res> at part + k B nchunk,
// k = 0..2 (<res, M^-1 psi> equals <psi, M^-1 res>: M is diagonal)
__global__ void __launch_bounds__(LZ_THREADS)
k_rf_update(float* __restrict__ t, float* __restrict__ res, const float* __restrict__ p,
            const float* __restrict__ hp, const float* __restrict__ psi, const float* __restrict__ minv,
            const double* __restrict__ sc, const int32_t* __restrict__ ctl, double* __restrict__ part, int64_t D,
            int nchunk, int batch, const int32_t* __restrict__ stop) {
  __shared__ double red[LZ_THREADS / 32];
  const int b = blockIdx.y, chunk = blockIdx.x;
  if ((stop && *stop) || ctl[b]) return;
  const float al = tc::d2f_rn(sc[b * RF_NSC + RF_ALPHA]);
  const float s1 = tc::d2f_rn(sc[b * RF_NSC + RF_S1]);
  float rr = 0.f, a1 = 0.f, a2 = 0.f;
  RF_LOOP({
    const float pi = p[i];
    t[i] = fmaf(al, pi, t[i]);
    const float si = psi[i];
    const float v = fmaf(-al, fmaf(-s1, si, hp[i]), res[i]);
    res[i] = v;
    const float mv = minv[i] * v;
    rr = fmaf(v, v, rr);
    a1 = fmaf(si, mv, a1);
    a2 = fmaf(v, mv, a2);
  })
  const int64_t stride = (int64_t)batch * nchunk, at = (int64_t)b * nchunk + chunk;
  const double r0 = rf_block_sum(rr, red);
  if (threadIdx.x == 0) part[at] = r0;
  const double r1 = rf_block_sum(a1, red);
  if (threadIdx.x == 0) part[stride + at] = r1;
  const double r2 = rf_block_sum(a2, red);
  if (threadIdx.x == 0) part[2 * stride + at] = r2;
}

// p = M^-1 (res - gamma psi) + beta p  (first: beta = 0)
__global__ void __launch_bounds__(LZ_THREADS)
k_rf_dir(float* __restrict__ p, const float* __restrict__ res, const float* __restrict__ psi,
         const float* __restrict__ minv, const double* __restrict__ sc, const int32_t* __restrict__ ctl, int64_t D,
         int first, const int32_t* __restrict__ stop) {
  const int b = blockIdx.y, chunk = blockIdx.x;
  if ((stop && *stop) || (ctl && ctl[b])) return;
  const float be = first ? 0.f : tc::d2f_rn(sc[b * RF_NSC + RF_BETA]);
  const float ga = tc::d2f_rn(sc[b * RF_NSC + RF_GAMMA]);
  RF_LOOP({
    const float z = minv[i] * fmaf(-ga, psi[i], res[i]);
    p[i] = first ? z : fmaf(be, p[i], z);
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

// M^-1 = 1 / max(diag - theta, delta max(1, |theta|)): the difference in
// float64, the reciprocal in float32
__global__ void k_rf_minv(const double* __restrict__ diag, const double* __restrict__ sc, float* __restrict__ minv,
                          int64_t D) {
  const int b = blockIdx.y;
  const double th = sc[b * RF_NSC + RF_THETA];
  const double delta = RF_DELTA * fmax(1.0, fabs(th));
  for (int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; d < D; d += (int64_t)gridDim.x * blockDim.x)
    minv[(int64_t)b * D + d] = 1.0f / tc::d2f_rn32(fmax(diag[(int64_t)b * D + d] - th, delta));
}

// sc[b][RR_NEW, A1, A2 (, MU)] = sums of the partial rows 0..2 (and 3 when
// with_mu), fixed order; one warp per row
__global__ void k_rf_sum4(const double* __restrict__ part, double* __restrict__ sc, int nchunk, int batch,
                          int with_mu, const int32_t* __restrict__ ctl, const int32_t* __restrict__ stop) {
  const int b = blockIdx.x, k = threadIdx.x >> 5, lane = threadIdx.x & 31;  // one warp per row
  if (k >= 3 + with_mu || (stop && *stop) || (ctl && ctl[b])) return;
  const double* row = part + ((int64_t)k * batch + b) * nchunk;
  double t = 0.0;
  for (int ch = lane; ch < nchunk; ch += 32) t += row[ch];  // lane-strided, then a fixed shuffle tree
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  const int slot[4] = {RF_RRNEW, RF_A1, RF_A2, RF_MU};
  if (lane == 0) sc[b * RF_NSC + slot[k]] = t;
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

// outer step: r = w - theta psi, negated (the CG right-hand side is -r) in
// float64 and stored in float32 in res; psi in float32 for the inner
// solve; t = 0; partials of <res, res>, <psi, M^-1 res>, <res, M^-1 res>,
// <psi, M^-1 psi> (rows 0..3)
__global__ void __launch_bounds__(LZ_THREADS)
k_rf_start(const double* __restrict__ w, const double* __restrict__ psi, const float* __restrict__ minv,
           float* __restrict__ res, float* __restrict__ t, float* __restrict__ psi32, const double* __restrict__ sc,
           double* __restrict__ part, int64_t D, int nchunk, int batch) {
  __shared__ double red[LZ_THREADS / 32];
  const int b = blockIdx.y, chunk = blockIdx.x;
  const double th = sc[b * RF_NSC + RF_THETA];
  float a[4] = {0.f, 0.f, 0.f, 0.f};
  RF_LOOP({
    const float v = tc::d2f_rn32(fma(th, psi[i], -w[i]));
    const float si = tc::d2f_rn32(psi[i]);
    res[i] = v;
    t[i] = 0.f;
    psi32[i] = si;
    const float m = minv[i];
    const float mv = m * v;
    a[0] = fmaf(v, v, a[0]);
    a[1] = fmaf(si, mv, a[1]);
    a[2] = fmaf(v, mv, a[2]);
    a[3] = fmaf(m * si, si, a[3]);
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
__global__ void k_rf_apply(double* __restrict__ psi, const float* __restrict__ t, const int32_t* __restrict__ mask,
                           int64_t D) {
  const int b = blockIdx.y;
  if (!mask[b]) return;
  for (int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; d < D; d += (int64_t)gridDim.x * blockDim.x)
    psi[(int64_t)b * D + d] += tc::f2d_exact(t[(int64_t)b * D + d]);
}

// ------------------------------------------------------------- launchers
static dim3 vgrid(int64_t D, int batch) { return dim3(lz_nchunk(D), batch); }

void rf_launch_dots4(const double* q, const float* p, const float* psi, float* hp, const double* sc,
                     const int32_t* ctl, double* part, int64_t D, int B, const int32_t* stop, cudaStream_t st) {
  k_rf_dots4<<<vgrid(D, B), LZ_THREADS, 0, st>>>(q, p, psi, hp, sc, ctl, part, D, lz_nchunk(D), B, stop);
}
void rf_launch_alpha4(const double* part, double* sc, int32_t* ctl, int64_t D, int B, const int32_t* stop,
                      cudaStream_t st) {
  k_rf_alpha4<<<B, 32, 0, st>>>(part, sc, ctl, lz_nchunk(D), B, stop);
}
void rf_launch_update(float* t, float* res, const float* p, const float* hp, const float* psi, const float* minv,
                      const double* sc, const int32_t* ctl, double* part, int64_t D, int B, const int32_t* stop,
                      cudaStream_t st) {
  k_rf_update<<<vgrid(D, B), LZ_THREADS, 0, st>>>(t, res, p, hp, psi, minv, sc, ctl, part, D, lz_nchunk(D), B,
                                                  stop);
}
void rf_launch_dir(float* p, const float* res, const float* psi, const float* minv, const double* sc,
                   const int32_t* ctl, int64_t D, int B, int first, const int32_t* stop, cudaStream_t st) {
  k_rf_dir<<<vgrid(D, B), LZ_THREADS, 0, st>>>(p, res, psi, minv, sc, ctl, D, first, stop);
}
void rf_launch_sum4(const double* part, double* sc, int64_t D, int B, int with_mu, const int32_t* ctl,
                    const int32_t* stop, cudaStream_t st) {
  k_rf_sum4<<<B, 128, 0, st>>>(part, sc, lz_nchunk(D), B, with_mu, ctl, stop);
}
static int rf_vec_blocks(int64_t D) {
  const int64_t nb = (D + 255) / 256;
  return (int)(nb > 2048 ? 2048 : (nb < 1 ? 1 : nb));
}
void rf_launch_diag(const double* dterm, const int32_t* terms, int nd, const double* coef, int n_terms,
                    double* diag, int64_t D, int B, cudaStream_t st) {
  k_rf_diag<<<dim3(rf_vec_blocks(D), B), 256, 0, st>>>(dterm, terms, nd, coef, n_terms, diag, D);
}
void rf_launch_minv(const double* diag, const double* sc, float* minv, int64_t D, int B, cudaStream_t st) {
  k_rf_minv<<<dim3(rf_vec_blocks(D), B), 256, 0, st>>>(diag, sc, minv, D);
}
void rf_launch_rho0(double* sc, int B, cudaStream_t st) { k_rf_rho0<<<(B + 63) / 64, 64, 0, st>>>(sc, B); }
void rf_launch_beta(double* sc, int32_t* ctl, const double* eps, int B, int32_t* stop, cudaStream_t st) {
  const int threads = B >= 1024 ? 1024 : ((B + 31) / 32) * 32;
  k_rf_beta<<<1, threads < 32 ? 32 : threads, 0, st>>>(sc, ctl, eps, B, stop);
}
void rf_launch_start(const double* w, const double* psi, const float* minv, float* res, float* t, float* psi32,
                     const double* sc, double* part, int64_t D, int B, cudaStream_t st) {
  k_rf_start<<<vgrid(D, B), LZ_THREADS, 0, st>>>(w, psi, minv, res, t, psi32, sc, part, D, lz_nchunk(D), B);
}
void rf_launch_set(double* sc, const double* src, int slot, int B, int sqrt_too, cudaStream_t st) {
  k_rf_set<<<(B + 63) / 64, 64, 0, st>>>(sc, src, slot, B, sqrt_too);
}
void rf_launch_apply(double* psi, const float* t, const int32_t* mask, int64_t D, int B, cudaStream_t st) {
  int64_t nb = (D + 255) / 256;
  if (nb > 2048) nb = 2048;
  k_rf_apply<<<dim3((unsigned)nb, B), 256, 0, st>>>(psi, t, mask, D);
}

}  // namespace dmrg
