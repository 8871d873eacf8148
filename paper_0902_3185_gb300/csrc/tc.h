// Tensor-core (tcgen05) path of the superblock product: mixed precision.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

struct dmrg_sb;

namespace dmrg {

void tc_build(dmrg_sb* sb);      // pair lists (no-op when unsupported); panels are built per precision at first use
// build the operand panels and task lists of `prec` now if they do not exist
// (allocates and copies: call it before a stream capture that runs products)
void tc_prepare(dmrg_sb* sb, int prec);
void tc_free(dmrg_sb* sb);
bool tc_available(const dmrg_sb* sb);
bool tc_set_coeffs(dmrg_sb* sb);  // true: operand panels rebuilt (captured graphs are stale)
double tc_operand_bytes(const dmrg_sb* sb);
int tc_launches(const dmrg_sb* sb, int prec);  // kernels one product launches
// member_done (device [batch], may be null): members whose flag is nonzero are
// skipped entirely (their rows of y are left as they are)
void tc_matvec(dmrg_sb* sb, int prec, const double* x, double* y, int accumulate, const int32_t* skip,
               cudaStream_t st, const int32_t* member_done = nullptr);
// the same product of a float32 x (the mixed products round x to float32 first anyway)
void tc_matvec_f32in(dmrg_sb* sb, int prec, const float* x, double* y, int accumulate, const int32_t* skip,
                     cudaStream_t st, const int32_t* member_done = nullptr);
void tc_matvec_T(dmrg_sb* sb, int prec, const double* g, double* dpsi, cudaStream_t st);
// out: best ms, default ms, per-block baseline ms, best tile N, heavy-first flag, candidates
void tc_autotune(dmrg_sb* sb, int prec, int reps, cudaStream_t st, double* out);

}  // namespace dmrg
