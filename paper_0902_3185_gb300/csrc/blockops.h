// Launchers of the block kernels of the DMRG step around the product:
// Kronecker growth of block operators, batched float64 GEMMs (density
// matrices, basis changes), batched symmetric eigensolves and the global
// top-m selection of density-matrix eigenvalues.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

namespace dmrg {

// dst[i][j] += scale * S(i, j) for a rows x cols destination rectangle;
// S(i, j) = src[i*ld_src + j] (trans 0), src[j*ld_src + i] (trans 1), or
// the identity (src == nullptr).  Destinations of one launch must not overlap.
struct ScatJob {
  const double* src;
  double* dst;
  int32_t rows, cols, ld_src, ld_dst, trans, pad;
  double scale;
};
void launch_scatter(const std::vector<ScatJob>& jobs, cudaStream_t st);

// C = alpha op(A) op(B) + beta C for every job (op = transpose when t* = 1):
// op(A) is M x K (A row-major with leading dimension lda), op(B) K x N.
// beta = 0 does not read C.  Outputs of one launch must not overlap.
struct GemmJob {
  const double* A;
  const double* B;
  double* C;
  int32_t M, N, K, lda, ldb, ldc, ta, tb;
  double alpha, beta;
};
void launch_gemm(const std::vector<GemmJob>& jobs, cudaStream_t st);

// Eigen-decomposition of symmetric n x n matrices by cyclic Jacobi rotations
// (one block per matrix): w (n) in decreasing order, V (n x n row-major, column
// j the eigenvector of w[j]).  A is not modified.  work: 2 n (n + 1) doubles of
// device memory per job whose n exceeds the shared-memory limit (else unused).
struct EigJob {
  const double* A;
  double* V;
  double* w;
  double* work;
  int32_t n, pad;
};
constexpr int EIG_SMEM_MAX_N = 110;  // A and V in shared memory up to this size
void launch_eig(const std::vector<EigJob>& jobs, cudaStream_t st);

// Global selection of the m largest density-matrix eigenvalues over n
// candidates (lam, sector, index within the sector in decreasing order):
// values within tie_tol of their neighbour in decreasing order form one
// cluster, and the order is (cluster, sector, index); the first m are kept.
// keep[i] = 1 for kept candidates; out[0] = sum of the discarded eigenvalues,
// out[1] = the m-th value minus the (m+1)-th (the gap at the cut; 0 if
// n <= m).  scratch: 4 n int32 + n double of device memory.
void launch_select(const double* lam, const int32_t* sec, const int32_t* idx, int32_t n, int32_t m,
                   double tie_tol, int32_t* keep, double* out, int32_t* scratch_i, double* scratch_d,
                   cudaStream_t st);

// x[i] = uniform(-1, 1) from splitmix64 of (seed, i): the Lanczos start
// vector of a DMRG step (any vector with a component along the ground state)
void launch_start_vector(double* x, int64_t n, uint64_t seed, cudaStream_t st);

}  // namespace dmrg
