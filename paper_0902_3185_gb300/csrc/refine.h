// Launchers of the refinement kernels (refine.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace dmrg {

// per-member scalar slots
enum RfSlot : int { RF_THETA = 0, RF_BNORM = 1, RF_RR = 2, RF_PQ = 3, RF_S1 = 4, RF_ALPHA = 5, RF_BETA = 6,
                    RF_RRNEW = 7, RF_RHO = 8, RF_GAMMA = 9, RF_MU = 10, RF_A1 = 11, RF_A2 = 12, RF_NSC = 13 };

// Diagonal preconditioner M = max(diag(H) - theta, delta), delta = RF_DELTA max(1, |theta|)
constexpr double RF_DELTA = 1e-2;

// inner CG: float32 vectors (t, res, p, hp = (H - theta) p, psi and M^-1 in
// float32), float64 scalars and reductions
void rf_launch_dots4(const double* q, const float* p, const float* psi, float* hp, const double* sc,
                     const int32_t* ctl, double* part, int64_t D, int B, const int32_t* stop, cudaStream_t st);
void rf_launch_alpha4(const double* part, double* sc, int32_t* ctl, int64_t D, int B, const int32_t* stop,
                      cudaStream_t st);
void rf_launch_update(float* t, float* res, const float* p, const float* hp, const float* psi, const float* minv,
                      const double* sc, const int32_t* ctl, double* part, int64_t D, int B, const int32_t* stop,
                      cudaStream_t st);
void rf_launch_dir(float* p, const float* res, const float* psi, const float* minv, const double* sc,
                   const int32_t* ctl, int64_t D, int B, int first, const int32_t* stop, cudaStream_t st);
void rf_launch_sum4(const double* part, double* sc, int64_t D, int B, int with_mu, const int32_t* ctl,
                    const int32_t* stop, cudaStream_t st);
void rf_launch_diag(const double* dterm, const int32_t* terms, int nd, const double* coef, int n_terms,
                    double* diag, int64_t D, int B, cudaStream_t st);
void rf_launch_minv(const double* diag, const double* sc, float* minv, int64_t D, int B, cudaStream_t st);
void rf_launch_rho0(double* sc, int B, cudaStream_t st);
void rf_launch_beta(double* sc, int32_t* ctl, const double* eps, int B, int32_t* stop, cudaStream_t st);
void rf_launch_start(const double* w, const double* psi, const float* minv, float* res, float* t, float* psi32,
                     const double* sc, double* part, int64_t D, int B, cudaStream_t st);
void rf_launch_set(double* sc, const double* src, int slot, int B, int sqrt_too, cudaStream_t st);
void rf_launch_apply(double* psi, const float* t, const int32_t* mask, int64_t D, int B, cudaStream_t st);

}  // namespace dmrg
