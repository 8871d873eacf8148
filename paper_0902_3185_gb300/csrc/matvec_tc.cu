// Tensor-core path: not built yet.
#include "internal.h"
#include "tc.h"

namespace dmrg {
void tc_build(dmrg_sb*) {}
void tc_free(dmrg_sb*) {}
bool tc_available(const dmrg_sb*) { return false; }
void tc_set_coeffs(dmrg_sb*) {}
double tc_operand_bytes(const dmrg_sb*) { return 0.0; }
int tc_launches(const dmrg_sb*, int) { return 0; }
void tc_matvec(dmrg_sb*, int, const double*, double*, int, const int32_t*, cudaStream_t) {}
void tc_matvec_T(dmrg_sb*, int, const double*, double*, cudaStream_t) {}
}  // namespace dmrg
