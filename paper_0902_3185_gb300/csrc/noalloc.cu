// dmrg_apply_H_static_scratch: the float64 superblock product with its
// intermediate workspace in a fixed, statically allocated device buffer.
//
// Why it exists: some callers cannot call cudaMalloc when they apply H --
// processes whose device memory is owned by another framework's pool (a
// cudaMalloc behind the pool's back can fail or fragment it), or
// latency-critical loops that must not allocate (cudaMalloc can synchronise
// the device and take milliseconds).  dmrg_apply_H itself does
// not allocate either, but it relies on the workspace that the superblock
// reserved for itself; this entry point uses instead one buffer of fixed
// size that is part of the loaded library, so the product needs no memory
// beyond the caller's input and output and the superblock's operator data.
//
// The buffer: DMRG_STATIC_SCRATCH_DOUBLES float64 values (32 MiB) per GPU,
// held by every GPU that loads the library until the process exits.
// Host code cannot use the array's name as a device address, so the first
// call on each device looks the address up with cudaGetSymbolAddress (with
// that device current) and caches it; make that first call before any stream
// capture begins.  The cache lives as long as the process: destroying and
// re-creating a device's primary context (cudaDeviceReset) while the library
// is loaded is not supported by this entry point.  All calls on a device share the buffer and it keeps the
// previous call's contents, so calls whose kernels overlap on the GPU (for
// example on two streams) race and must be serialised by the caller.  Nothing
// in it needs to start at zero: the first phase of the product writes every
// intermediate element before the second phase reads it.
//
// The paper has no counterpart to this entry point.

#include <mutex>

#include "internal.h"

#define DMRG_STATIC_SCRATCH_DOUBLES (4ll * 1024 * 1024)

static __device__ __align__(256) double g_static_scratch[DMRG_STATIC_SCRATCH_DOUBLES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_addr[kMaxDevices] = {};

// Address of the static buffer on the current device (set up once per device).
cudaError_t scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = static_cast<double*>(p);
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" dmrg_status dmrg_apply_H_static_scratch(dmrg_sb* sb, const double* psi, double* y, int32_t accumulate,
                                                   void* stream) {
  if (!sb) return DMRG_EINVAL;
  if (!psi || !y || psi == y) {
    sb->err = "apply_H_static_scratch: null or aliased psi / y";
    return DMRG_EINVAL;
  }
  if (sb->T_fwd_elems > DMRG_STATIC_SCRATCH_DOUBLES) {
    sb->err = "apply_H_static_scratch: this superblock needs " + std::to_string(sb->T_fwd_elems) +
              " float64 values of intermediate workspace; the static buffer holds " +
              std::to_string((long long)DMRG_STATIC_SCRATCH_DOUBLES);
    return DMRG_EINVAL;
  }
  double* scratch = nullptr;
  cudaError_t e = scratch_address(&scratch);
  if (e != cudaSuccess) {
    sb->err = std::string("apply_H_static_scratch: cudaGetSymbolAddress: ") + cudaGetErrorString(e);
    return DMRG_ECUDA;
  }
  cudaStream_t st = (cudaStream_t)stream;
  dmrg::Bufs bufs{{const_cast<double*>(psi), y, scratch, sb->d_ops, nullptr}};
  const int acc = accumulate ? 1 : 0;
  dmrg::launch_seg_gemm_f64(sb->f64_fwd1, bufs, sb->d_coeffs, sb->n_terms, 0, nullptr, nullptr, st);
  dmrg::launch_seg_gemm_f64(sb->f64_fwd2, bufs, sb->d_coeffs, sb->n_terms, acc, nullptr, nullptr, st);
  dmrg::launch_seg_gemm_f64(sb->f64_fwd3, bufs, sb->d_coeffs, sb->n_terms, acc, nullptr, nullptr, st);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    sb->err = std::string("apply_H_static_scratch: launch: ") + cudaGetErrorString(e);
    return DMRG_ECUDA;
  }
  return DMRG_OK;
}
