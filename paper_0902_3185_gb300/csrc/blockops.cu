// Block kernels of the DMRG step around the superblock product (paper
// Sec. 3.1 and Sec. 3.3: growth S' = S (x) site with the operators
// re-expressed in the product basis, the reduced density matrices
// rho_S = Psi Psi^T and rho_E = Psi^T Psi of Eqs. rhoSystem / rhoEnviron,
// their eigenvectors, the choice of the m most probable states, and the
// change of basis W^T O W of Eq. transformation).
//
// All of it is float64: the density-matrix eigenvectors decide the basis of
// every later step, and the paper's method keeps it exact to rounding.
// Sizes are small (sector blocks of a few hundred at most), so the kernels
// favour simple, bounded loops over peak throughput; the step's cost stays in
// the Lanczos solve.

#include <algorithm>
#include <cmath>
#include <stdexcept>
#include <string>

#include <cooperative_groups.h>

#include "blockops.h"

namespace dmrg {

namespace {

template <class T>
T* upload_async(const std::vector<T>& h, cudaStream_t st) {
  void* p = nullptr;
  cudaError_t e = cudaMallocAsync(&p, std::max<size_t>(1, h.size()) * sizeof(T), st);
  if (e != cudaSuccess) throw std::runtime_error(std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
  if (!h.empty()) {
    e = cudaMemcpyAsync(p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) throw std::runtime_error(std::string("cudaMemcpyAsync: ") + cudaGetErrorString(e));
  }
  return static_cast<T*>(p);
}

void check_launch(const char* what) {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) throw std::runtime_error(std::string(what) + ": " + cudaGetErrorString(e));
}

struct Tile {
  int32_t job, i0, j0, pad;
};

}  // namespace

// ------------------------------------------------------------------ scatter
// One 32 x 32 destination tile per block (32 x 8 threads); a transposed
// source goes through shared memory so that both the read and the write run
// along rows.
__global__ void __launch_bounds__(256) k_scatter(const ScatJob* __restrict__ jobs, const Tile* __restrict__ tiles) {
  __shared__ double t[32][33];
  const Tile tl = tiles[blockIdx.x];
  const ScatJob jb = jobs[tl.job];
  const int tx = threadIdx.x, ty = threadIdx.y;
  if (jb.src && jb.trans) {
    for (int r = ty; r < 32; r += 8) {
      const int j = tl.j0 + r, i = tl.i0 + tx;
      t[r][tx] = (j < jb.cols && i < jb.rows) ? jb.src[(int64_t)j * jb.ld_src + i] : 0.0;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
      const int i = tl.i0 + r, j = tl.j0 + tx;
      if (i < jb.rows && j < jb.cols) jb.dst[(int64_t)i * jb.ld_dst + j] += jb.scale * t[tx][r];
    }
  } else {
    for (int r = ty; r < 32; r += 8) {
      const int i = tl.i0 + r, j = tl.j0 + tx;
      if (i < jb.rows && j < jb.cols) {
        const double v = jb.src ? jb.src[(int64_t)i * jb.ld_src + j] : (i == j ? 1.0 : 0.0);
        jb.dst[(int64_t)i * jb.ld_dst + j] += jb.scale * v;
      }
    }
  }
}

void launch_scatter(const std::vector<ScatJob>& jobs, cudaStream_t st) {
  std::vector<Tile> tiles;
  for (size_t q = 0; q < jobs.size(); ++q)
    for (int i0 = 0; i0 < jobs[q].rows; i0 += 32)
      for (int j0 = 0; j0 < jobs[q].cols; j0 += 32) tiles.push_back({(int32_t)q, i0, j0, 0});
  if (tiles.empty()) return;
  ScatJob* dj = upload_async(jobs, st);
  Tile* dt = upload_async(tiles, st);
  k_scatter<<<(unsigned)tiles.size(), dim3(32, 8), 0, st>>>(dj, dt);
  check_launch("k_scatter");
  cudaFreeAsync(dj, st);
  cudaFreeAsync(dt, st);
}

// ------------------------------------------------------------------- gemm
// 64 x 64 output tile per block, 256 threads of 4 x 4 outputs each, K in
// chunks of 16 through shared memory (operands loaded along their
// contiguous index whatever the transpose).
__global__ void __launch_bounds__(256) k_gemm(const GemmJob* __restrict__ jobs, const Tile* __restrict__ tiles) {
  __shared__ double As[16][65];
  __shared__ double Bs[16][65];
  const Tile tl = tiles[blockIdx.x];
  const GemmJob jb = jobs[tl.job];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int m0 = tl.i0, n0 = tl.j0;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  for (int k0 = 0; k0 < jb.K; k0 += 16) {
    for (int e = tid; e < 1024; e += 256) {
      int mm, kk;
      if (jb.ta) { kk = e >> 6; mm = e & 63; } else { mm = e >> 4; kk = e & 15; }
      const int m = m0 + mm, k = k0 + kk;
      double v = 0.0;
      if (m < jb.M && k < jb.K) v = jb.ta ? jb.A[(int64_t)k * jb.lda + m] : jb.A[(int64_t)m * jb.lda + k];
      As[kk][mm] = v;
    }
    for (int e = tid; e < 1024; e += 256) {
      int nn, kk;
      if (jb.tb) { nn = e >> 4; kk = e & 15; } else { kk = e >> 6; nn = e & 63; }
      const int n = n0 + nn, k = k0 + kk;
      double v = 0.0;
      if (n < jb.N && k < jb.K) v = jb.tb ? jb.B[(int64_t)n * jb.ldb + k] : jb.B[(int64_t)k * jb.ldb + n];
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty + 16 * i;
    if (m >= jb.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx + 16 * j;
      if (n >= jb.N) continue;
      double* c = jb.C + (int64_t)m * jb.ldc + n;
      *c = jb.beta != 0.0 ? fma(jb.alpha, acc[i][j], jb.beta * *c) : jb.alpha * acc[i][j];
    }
  }
}

void launch_gemm(const std::vector<GemmJob>& jobs, cudaStream_t st) {
  std::vector<Tile> tiles;
  for (size_t q = 0; q < jobs.size(); ++q) {
    const GemmJob& j = jobs[q];
    if (j.M <= 0 || j.N <= 0) continue;
    for (int m0 = 0; m0 < j.M; m0 += 64)
      for (int n0 = 0; n0 < j.N; n0 += 64) tiles.push_back({(int32_t)q, m0, n0, 0});
  }
  if (tiles.empty()) return;
  GemmJob* dj = upload_async(jobs, st);
  Tile* dt = upload_async(tiles, st);
  k_gemm<<<(unsigned)tiles.size(), 256, 0, st>>>(dj, dt);
  check_launch("k_gemm");
  cudaFreeAsync(dj, st);
  cudaFreeAsync(dt, st);
}

// ---------------------------------------------------------------- eigen
// Cyclic Jacobi (Golub & Van Loan, Sec. 8.5) with the round-robin ordering:
// in each of the N2 - 1 rounds of a sweep the N2 / 2 rotations are disjoint,
// so all of them are applied at once -- rows p, q of A for every pair, then
// columns p, q of A and of V -- as A <- J^T A J, V <- V J.  The rotation that
// zeroes a_pq: tau = (a_qq - a_pp) / (2 a_pq), t = sign(tau) / (|tau| +
// sqrt(1 + tau^2)), c = 1 / sqrt(1 + t^2), s = t c.  A rotation is skipped
// when |a_pq| <= 4 eps |A|_F (threshold Jacobi: rounding leaves off-diagonal
// elements near eps |A|, so a tighter test would never pass), and the sweeps
// stop after one without a rotation (at most 40).  The eigenvalues are then
// accurate to a few eps |A| in absolute terms, as a LAPACK solver's.
constexpr int EIG_THREADS = 256;
constexpr int EIG_MAX_N = 4096;

__device__ __forceinline__ double eig_block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < EIG_THREADS / 32; ++w) t += red[w];
  return t;
}

__device__ __forceinline__ int rr_player(int slot, int r, int n2) {
  return slot == 0 ? 0 : 1 + (slot - 1 + r) % (n2 - 1);
}

__global__ void __launch_bounds__(EIG_THREADS) k_eig(const EigJob* __restrict__ jobs) {
  extern __shared__ double sm[];
  __shared__ double red[EIG_THREADS / 32];
  const EigJob jb = jobs[blockIdx.x];
  const int n = jb.n;
  if (n <= 0) return;
  const int ld = n + 1;
  const int n2 = (n + 1) & ~1;
  const int np = n2 / 2;
  const bool in_smem = n <= EIG_SMEM_MAX_N;
  double* a = in_smem ? sm : jb.work;
  double* v = in_smem ? sm + (size_t)n * ld : jb.work + (size_t)n * ld;
  double* base = in_smem ? sm + (size_t)2 * n * ld : sm;
  double* cs = base;           // [np]
  double* sn = base + np;      // [np]
  int* pp = reinterpret_cast<int*>(base + 2 * np);  // [np]
  int* qq = pp + np;                                 // [np]
  int* rank = qq + np;                               // [n]
  const int tid = threadIdx.x;
  for (int e = tid; e < n * n; e += EIG_THREADS) {
    const int i = e / n, j = e % n;
    a[i * ld + j] = jb.A[(int64_t)i * n + j];
    v[i * ld + j] = i == j ? 1.0 : 0.0;
  }
  __syncthreads();
  if (n > 1) {
    double fro = 0.0;
    for (int e = tid; e < n * n; e += EIG_THREADS) {
      const double x = a[(e / n) * ld + e % n];
      fro = fma(x, x, fro);
    }
    const double thr = 4.0 * 2.220446049250313e-16 * sqrt(eig_block_sum(fro, red));
    for (int sweep = 0; sweep < 40; ++sweep) {
      double rot = 0.0;  // rotations applied by this thread in the sweep
      for (int r = 0; r < n2 - 1; ++r) {
        for (int k = tid; k < np; k += EIG_THREADS) {
          int p = rr_player(k, r, n2), q = rr_player(n2 - 1 - k, r, n2);
          if (p > q) { const int t = p; p = q; q = t; }
          double c = 1.0, s = 0.0;
          if (q < n) {
            const double apq = a[p * ld + q];
            if (fabs(apq) > thr) {
              const double tau = (a[q * ld + q] - a[p * ld + p]) / (2.0 * apq);
              double t;
              if (fabs(tau) > 1e150) t = 0.5 / tau;
              else t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
              c = 1.0 / sqrt(1.0 + t * t);
              s = t * c;
              rot += 1.0;
            }
          }
          pp[k] = p;
          qq[k] = q;
          cs[k] = c;
          sn[k] = s;
        }
        __syncthreads();
        for (int e = tid; e < np * n; e += EIG_THREADS) {  // rows p, q
          const int k = e / n, j = e % n;
          const double s = sn[k];
          if (s == 0.0) continue;
          const double c = cs[k];
          const int p = pp[k], q = qq[k];
          const double x = a[p * ld + j], y = a[q * ld + j];
          a[p * ld + j] = c * x - s * y;
          a[q * ld + j] = s * x + c * y;
        }
        __syncthreads();
        for (int e = tid; e < np * n; e += EIG_THREADS) {  // columns p, q of A and V
          const int k = e / n, i = e % n;
          const double s = sn[k];
          if (s == 0.0) continue;
          const double c = cs[k];
          const int p = pp[k], q = qq[k];
          const double x = a[i * ld + p], y = a[i * ld + q];
          a[i * ld + p] = c * x - s * y;
          a[i * ld + q] = s * x + c * y;
          const double xv = v[i * ld + p], yv = v[i * ld + q];
          v[i * ld + p] = c * xv - s * yv;
          v[i * ld + q] = s * xv + c * yv;
        }
        __syncthreads();
      }
      if (eig_block_sum(rot, red) == 0.0) break;  // the same sum in every thread
    }
  }
  // decreasing order (ties by index)
  for (int i = tid; i < n; i += EIG_THREADS) {
    const double wi = a[i * ld + i];
    int rk = 0;
    for (int j = 0; j < n; ++j) {
      const double wj = a[j * ld + j];
      rk += (wj > wi) || (wj == wi && j < i);
    }
    rank[i] = rk;
  }
  __syncthreads();
  for (int i = tid; i < n; i += EIG_THREADS) jb.w[rank[i]] = a[i * ld + i];
  for (int e = tid; e < n * n; e += EIG_THREADS) {
    const int row = e / n, i = e % n;
    jb.V[(int64_t)row * n + rank[i]] = v[row * ld + i];
  }
}

// The same cyclic Jacobi for a matrix too large for one block's shared
// memory, on a cluster of EIG_CLUSTER blocks whose shared memories together
// hold A and V (thread-block clusters with distributed shared memory).  Row i
// of A and of V lives in block i % C (local row i / C).  A round of disjoint
// rotations: (1) the owner of row p = min(p, q) of each pair computes (c, s)
// from a_pp, a_pq (local) and a_qq (remote); (2) every block gathers all
// rotations, and the owner of p rotates rows p (local) and q (remote, read
// and written through distributed shared memory) -- no other block touches
// them; (3) every block rotates columns p, q of its own rows of A and V.
// Cluster barriers separate the phases.  All blocks sum the convergence test
// in the same order, so they leave the sweep loop together.
constexpr int EIG_CLUSTER = 16;

__global__ void __launch_bounds__(EIG_THREADS) k_eig_cluster(const EigJob* __restrict__ jobs) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ double sm[];
  __shared__ double red[EIG_THREADS / 32];
  __shared__ double sums[1];
  __shared__ int n_own;
  const int C = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const EigJob jb = jobs[blockIdx.x / C];
  const int n = jb.n;
  const int n2 = (n + 1) & ~1;
  const int np = n2 / 2;
  const int R = (n + C - 1) / C;
  const int rows = rank < n ? (n - 1 - rank) / C + 1 : 0;  // own rows: rank, rank + C, ...
  double* a = sm;                       // [R][n]
  double* v = sm + (size_t)R * n;       // [R][n]
  double* par = v + (size_t)R * n;      // [np][2] rotations of the pairs this block owns
  double* allp = par + 2 * np;          // [np][2] all rotations of the round
  double* dg = allp + 2 * np;           // [n] diagonal (final ordering)
  int* own = reinterpret_cast<int*>(dg + n);  // [np] pairs this block owns
  int* rk = own + np;                         // [n]
  const int tid = threadIdx.x;
  for (int e = tid; e < rows * n; e += EIG_THREADS) {
    const int li = e / n, j = e % n, i = rank + C * li;
    a[li * n + j] = jb.A[(int64_t)i * n + j];
    v[li * n + j] = i == j ? 1.0 : 0.0;
  }
  // sum over the cluster of one value per block, in the same order in every block
  auto cluster_sum = [&](double v) -> double {
    v = eig_block_sum(v, red);
    if (tid == 0) sums[0] = v;
    cl.sync();
    double t = 0.0;
    for (int b = 0; b < C; ++b) t += cl.map_shared_rank(sums, b)[0];
    cl.sync();  // read before any block writes the next one
    return t;
  };
  double fro = 0.0;
  for (int e = tid; e < rows * n; e += EIG_THREADS) {
    const double x = a[(e / n) * n + e % n];
    fro = fma(x, x, fro);
  }
  const double thr = 4.0 * 2.220446049250313e-16 * sqrt(cluster_sum(fro));
  for (int sweep = 0; sweep < 40; ++sweep) {
    double rot = 0.0;  // rotations this block computed in the sweep
    for (int r = 0; r < n2 - 1; ++r) {
      if (tid == 0) n_own = 0;
      __syncthreads();
      for (int k = tid; k < np; k += EIG_THREADS) {
        int p = rr_player(k, r, n2), q = rr_player(n2 - 1 - k, r, n2);
        if (p > q) { const int t = p; p = q; q = t; }
        if (p % C != rank) continue;
        double c = 1.0, s = 0.0;
        if (q < n) {
          const double apq = a[(p / C) * n + q];
          if (fabs(apq) > thr) {
            const double* ra = cl.map_shared_rank(a, q % C);
            const double aqq = ra[(q / C) * n + q];
            const double tau = (aqq - a[(p / C) * n + p]) / (2.0 * apq);
            double t;
            if (fabs(tau) > 1e150) t = 0.5 / tau;
            else t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + t * t);
            s = t * c;
            rot += 1.0;
          }
        }
        par[2 * k] = c;
        par[2 * k + 1] = s;
        if (s != 0.0) own[atomicAdd(&n_own, 1)] = k;
      }
      cl.sync();
      for (int k = tid; k < np; k += EIG_THREADS) {  // gather every pair's rotation
        int p = rr_player(k, r, n2), q = rr_player(n2 - 1 - k, r, n2);
        if (p > q) { const int t = p; p = q; q = t; }
        const double* rp = cl.map_shared_rank(par, p % C);
        allp[2 * k] = rp[2 * k];
        allp[2 * k + 1] = rp[2 * k + 1];
      }
      const int no = n_own;
      for (int e = tid; e < no * n; e += EIG_THREADS) {  // rows p (local) and q (remote) of owned pairs
        const int k = own[e / n], j = e % n;
        int p = rr_player(k, r, n2), q = rr_player(n2 - 1 - k, r, n2);
        if (p > q) { const int t = p; p = q; q = t; }
        const double c = par[2 * k], s = par[2 * k + 1];
        double* rq = cl.map_shared_rank(a, q % C) + (size_t)(q / C) * n;
        double* rowp = a + (size_t)(p / C) * n;
        const double x = rowp[j], y = rq[j];
        rowp[j] = c * x - s * y;
        rq[j] = s * x + c * y;
      }
      cl.sync();
      for (int e = tid; e < rows * np; e += EIG_THREADS) {  // columns p, q of own rows of A and V
        const int li = e / np, k = e % np;
        const double s = allp[2 * k + 1];
        if (s == 0.0) continue;
        const double c = allp[2 * k];
        int p = rr_player(k, r, n2), q = rr_player(n2 - 1 - k, r, n2);
        if (p > q) { const int t = p; p = q; q = t; }
        double* ra = a + (size_t)li * n;
        double* rv = v + (size_t)li * n;
        const double x = ra[p], y = ra[q];
        ra[p] = c * x - s * y;
        ra[q] = s * x + c * y;
        const double xv = rv[p], yv = rv[q];
        rv[p] = c * xv - s * yv;
        rv[q] = s * xv + c * yv;
      }
      cl.sync();
    }
    if (cluster_sum(rot) == 0.0) break;  // every block leaves together
  }
  // decreasing order: every block gathers the diagonal, ranks it, and writes its own rows of V
  for (int i = tid; i < n; i += EIG_THREADS) {
    const double* ra = cl.map_shared_rank(a, i % C);
    dg[i] = ra[(i / C) * n + i];
  }
  __syncthreads();
  for (int i = tid; i < n; i += EIG_THREADS) {
    const double wi = dg[i];
    int r2 = 0;
    for (int j = 0; j < n; ++j) r2 += (dg[j] > wi) || (dg[j] == wi && j < i);
    rk[i] = r2;
  }
  __syncthreads();
  if (rank == 0)
    for (int i = tid; i < n; i += EIG_THREADS) jb.w[rk[i]] = dg[i];
  for (int e = tid; e < rows * n; e += EIG_THREADS) {
    const int li = e / n, j = e % n, i = rank + C * li;
    jb.V[(int64_t)i * n + rk[j]] = v[li * n + j];
  }
  cl.sync();  // no block leaves while others may still read its shared memory
}

size_t eig_cluster_smem(int n) {
  const size_t R = (size_t)(n + EIG_CLUSTER - 1) / EIG_CLUSTER, np = (size_t)(n + 1) / 2;
  return 2 * R * n * sizeof(double) + 4 * np * sizeof(double) + n * sizeof(double) + (np + n) * sizeof(int);
}

// largest n the cluster kernel takes (A and V in the cluster's shared memory)
constexpr int EIG_CLUSTER_MAX_N = 448;

// -1: not tried, 0: unavailable on this device, 1: available
int g_cluster_ok = -1;

bool launch_eig_cluster(const std::vector<EigJob>& jobs, cudaStream_t st) {
  if (jobs.empty()) return true;
  size_t smem = 0;
  for (const EigJob& j : jobs) smem = std::max(smem, eig_cluster_smem(j.n));
  smem = (smem + 15) & ~(size_t)15;
  if (g_cluster_ok == 0) return false;
  if (cudaFuncSetAttribute(k_eig_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess ||
      cudaFuncSetAttribute(k_eig_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
    cudaGetLastError();
    g_cluster_ok = 0;
    return false;
  }
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)(EIG_CLUSTER * jobs.size()));
  cfg.blockDim = dim3(EIG_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = EIG_CLUSTER;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int clusters = 0;
  if (cudaOccupancyMaxActiveClusters(&clusters, k_eig_cluster, &cfg) != cudaSuccess || clusters < 1) {
    cudaGetLastError();
    g_cluster_ok = 0;
    return false;
  }
  g_cluster_ok = 1;
  EigJob* dj = upload_async(jobs, st);
  const cudaError_t e = cudaLaunchKernelEx(&cfg, k_eig_cluster, (const EigJob*)dj);
  if (e != cudaSuccess) throw std::runtime_error(std::string("k_eig_cluster: ") + cudaGetErrorString(e));
  cudaFreeAsync(dj, st);
  return true;
}

void launch_eig(const std::vector<EigJob>& all, cudaStream_t st) {
  if (all.empty()) return;
  // sizes between the one-block shared-memory limit and the cluster limit go to
  // the cluster kernel when the device runs it; the rest to the one-block kernel
  std::vector<EigJob> mid, jobs;
  for (const EigJob& j : all) (j.n > EIG_SMEM_MAX_N && j.n <= EIG_CLUSTER_MAX_N ? mid : jobs).push_back(j);
  if (!launch_eig_cluster(mid, st))
    for (const EigJob& j : mid) {
      if (!j.work) throw std::logic_error("eigensolve: missing workspace");
      jobs.push_back(j);
    }
  if (jobs.empty()) return;
  size_t smem = 0;
  for (const EigJob& j : jobs) {
    if (j.n > EIG_MAX_N) throw std::logic_error("eigensolve: block larger than 4096");
    if (j.n > EIG_SMEM_MAX_N && !j.work) throw std::logic_error("eigensolve: missing workspace");
    const size_t n = (size_t)std::max(j.n, 1), np = (n + 1) / 2;
    size_t b = (np * 2) * sizeof(double) + (np * 2 + n) * sizeof(int);
    if (j.n <= EIG_SMEM_MAX_N) b += 2 * n * (n + 1) * sizeof(double);
    smem = std::max(smem, b);
  }
  smem = (smem + 15) & ~(size_t)15;
  cudaError_t e = cudaFuncSetAttribute(k_eig, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) throw std::runtime_error(std::string("k_eig smem: ") + cudaGetErrorString(e));
  EigJob* dj = upload_async(jobs, st);
  k_eig<<<(unsigned)jobs.size(), EIG_THREADS, smem, st>>>(dj);
  check_launch("k_eig");
  cudaFreeAsync(dj, st);
}

// -------------------------------------------------------------- selection
__device__ __forceinline__ bool key_less(double la, int sa, int ia, double lb, int sb, int ib) {
  // decreasing eigenvalue, then sector, then index
  if (la != lb) return la > lb;
  if (sa != sb) return sa < sb;
  return ia < ib;
}

// rank[i] by (-lam, sec, idx); order[rank[i]] = i
__global__ void k_sel_rank(const double* __restrict__ lam, const int32_t* __restrict__ sec,
                           const int32_t* __restrict__ idx, int n, int32_t* __restrict__ rank,
                           int32_t* __restrict__ order) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double li = lam[i];
  const int si = sec[i], ii = idx[i];
  int r = 0;
  for (int j = 0; j < n; ++j) r += key_less(lam[j], sec[j], idx[j], li, si, ii);
  rank[i] = r;
  order[r] = i;
}

// cluster id (1-based) of every candidate: in decreasing order, a new cluster
// starts where the value drops by more than tie_tol from its predecessor
__global__ void __launch_bounds__(1024) k_sel_cluster(const double* __restrict__ lam, const int32_t* __restrict__ order,
                                                      const int32_t* __restrict__ rank, int n, double tie_tol,
                                                      int32_t* __restrict__ cl_sorted, int32_t* __restrict__ cl) {
  __shared__ int32_t cnt[1024];
  const int tid = threadIdx.x;
  const int per = (n + 1023) / 1024;
  const int b = min(n, tid * per), e = min(n, b + per);
  auto flag = [&](int r) { return r == 0 || (lam[order[r - 1]] - lam[order[r]] > tie_tol); };
  int c = 0;
  for (int r = b; r < e; ++r) c += flag(r);
  cnt[tid] = c;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {  // inclusive scan
    const int add = tid >= o ? cnt[tid - o] : 0;
    __syncthreads();
    cnt[tid] += add;
    __syncthreads();
  }
  int id = cnt[tid] - c;
  for (int r = b; r < e; ++r) {
    id += flag(r);
    cl_sorted[r] = id;
  }
  __syncthreads();
  for (int i = tid; i < n; i += 1024) cl[i] = cl_sorted[rank[i]];
}

// final rank by (cluster, sec, idx); keep the first m
__global__ void k_sel_keep(const int32_t* __restrict__ cl, const int32_t* __restrict__ sec,
                           const int32_t* __restrict__ idx, int n, int m, int32_t* __restrict__ keep,
                           int32_t* __restrict__ order2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int ci = cl[i], si = sec[i], ii = idx[i];
  int r = 0;
  for (int j = 0; j < n; ++j) {
    const int cj = cl[j], sj = sec[j];
    r += cj < ci || (cj == ci && (sj < si || (sj == si && idx[j] < ii)));
  }
  keep[i] = r < m;
  order2[r] = i;
}

// discarded weight (fixed-order block sum) and the gap at the cut
__global__ void __launch_bounds__(256) k_sel_stats(const double* __restrict__ lam, const int32_t* __restrict__ keep,
                                                   const int32_t* __restrict__ order2, int n, int m,
                                                   double* __restrict__ out) {
  __shared__ double red[8];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += 256)
    if (!keep[i]) s += lam[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    out[0] = t;
    out[1] = (m >= 1 && m < n) ? lam[order2[m - 1]] - lam[order2[m]] : 0.0;
  }
}

void launch_select(const double* lam, const int32_t* sec, const int32_t* idx, int32_t n, int32_t m, double tie_tol,
                   int32_t* keep, double* out, int32_t* scratch_i, double* scratch_d, cudaStream_t st) {
  (void)scratch_d;
  if (n <= 0) {
    cudaMemsetAsync(out, 0, 2 * sizeof(double), st);
    return;
  }
  int32_t* rank = scratch_i;
  int32_t* order = scratch_i + n;
  int32_t* cl_sorted = scratch_i + 2 * (size_t)n;
  int32_t* cl = scratch_i + 3 * (size_t)n;
  const unsigned g = (unsigned)((n + 255) / 256);
  k_sel_rank<<<g, 256, 0, st>>>(lam, sec, idx, n, rank, order);
  k_sel_cluster<<<1, 1024, 0, st>>>(lam, order, rank, n, tie_tol, cl_sorted, cl);
  // order is free again: it receives the final order
  k_sel_keep<<<g, 256, 0, st>>>(cl, sec, idx, n, m, keep, order);
  k_sel_stats<<<1, 256, 0, st>>>(lam, keep, order, n, m, out);
  check_launch("select");
}

// ----------------------------------------------------------- start vector
// splitmix64 (Steele, Lea and Flood, 2014): the state advances by the golden
// ratio increment and is finalised by two xor-shift-multiply rounds
__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void k_start(double* __restrict__ x, int64_t n, uint64_t seed) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t z = splitmix64(seed * 0xD1B54A32D192ED03ull + (uint64_t)i);
    x[i] = 2.0 * ((double)(z >> 11) * 0x1.0p-53) - 1.0;
  }
}

void launch_start_vector(double* x, int64_t n, uint64_t seed, cudaStream_t st) {
  if (n <= 0) return;
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, 152 * 8);
  k_start<<<(unsigned)blocks, 256, 0, st>>>(x, n, seed);
  check_launch("k_start");
}

}  // namespace dmrg
