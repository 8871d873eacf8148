// C ABI of the superblock library: descriptor validation, device arenas,
// the (term, sector pair) task lists, the product, its reverse mode, the
// Hellmann-Feynman gradient and the graph-captured Lanczos driver.
//
// Paper Sec. 3.2 (symmetry blocks, partition), Sec. 3.3 (the on-the-fly
// superblock product x += H y as system, environment and connection tasks;
// Lanczos needs only that product).

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <stdexcept>
#include <numeric>

#include "internal.h"
#include "lanczos.h"
#include "refine.h"
#include "tc.h"

using namespace dmrg;

namespace {

struct CudaError {
  cudaError_t e;
  const char* what;
};

#define CK(x)                                   \
  do {                                          \
    cudaError_t e_ = (x);                       \
    if (e_ != cudaSuccess) throw CudaError{e_, #x}; \
  } while (0)

struct Invalid {
  std::string msg;
};
struct Timeout {
  std::string msg;
};

// Testing hook: DMRG_TEST_FAIL_ALLOC=n makes the n-th device allocation of
// the process report out-of-memory (host-side fault injection).
long g_alloc_count = 0;
long fail_alloc_at() {
  static const long at = [] {
    const char* e = getenv("DMRG_TEST_FAIL_ALLOC");
    return e ? atol(e) : 0L;
  }();
  return at;
}

template <class T>
T* dalloc(size_t n) {
  if (n == 0) n = 1;
  void* p = nullptr;
  if (fail_alloc_at() > 0 && ++g_alloc_count == fail_alloc_at()) throw CudaError{cudaErrorMemoryAllocation, "cudaMalloc (injected)"};
  CK(cudaMalloc(&p, n * sizeof(T)));
  return static_cast<T*>(p);
}

template <class T>
void upload(T*& d, const std::vector<T>& h) {
  if (d) cudaFree(d);
  d = dalloc<T>(h.size());
  if (!h.empty()) CK(cudaMemcpy(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
}

template <class F>
dmrg_status guard(dmrg_sb* sb, F&& fn) {
  try {
    return fn();
  } catch (const CudaError& ce) {
    if (sb) sb->err = std::string(ce.what) + ": " + cudaGetErrorString(ce.e);
    return ce.e == cudaErrorMemoryAllocation ? DMRG_ENOMEM : DMRG_ECUDA;
  } catch (const Invalid& iv) {
    if (sb) sb->err = iv.msg;
    return DMRG_EINVAL;
  } catch (const Timeout& to) {
    if (sb) sb->err = to.msg;
    return DMRG_ETIMEOUT;
  } catch (const std::logic_error& le) {
    if (sb) sb->err = le.what();
    return DMRG_EINVAL;
  } catch (const std::runtime_error& re) {
    if (sb) sb->err = re.what();
    return DMRG_ECUDA;
  } catch (const std::bad_alloc&) {
    if (sb) sb->err = "host allocation failed";
    return DMRG_ENOMEM;
  }
}

// ----------------------------------------------------------- task building
// An operator block as seen by one product: element (i, j) lives at
// ops[off + (trans ? j*ld + i : i*ld + j)] (trans = 1 reads A^T / B^T).
struct OpAcc {
  int64_t off;
  int32_t ld, trans;
};

// A (term, sector pair) in the direction of one product: forward pairs, or
// the transposed pairs of H^T.  A is r[s_out] x r[s_in], B is c[s_out] x c[s_in].
struct GPair {
  int32_t term, s_out, s_in, flags, order;
  OpAcc A, B;
};

SegF64 seg_base() {
  SegF64 g{};
  g.coef = -1;
  return g;
}

// L = a block operand (no members)
void set_L_op(SegF64& g, const OpAcc& o) {
  g.l_buf = BUF_OPS;
  g.l_off = o.off;
  g.ldl = o.ld;
  g.l_trans = o.trans;
}
// R(k, n) = B(n, k): the transposed block as the right operand
void set_R_opT(SegF64& g, const OpAcc& o) {
  g.r_buf = BUF_OPS;
  g.r_off = o.off;
  g.ldr = o.ld;
  g.r_trans = o.trans ? 0 : 1;
}

// Tile shape of an M x N output: the 16*ni x 16*nj tiling (ni, nj in 1..4)
// with the least padded area; among equals the largest tile (fewer operand
// reloads).  Returns ni | nj << 8.
int32_t f64_shape(int32_t M, int32_t N) {
  int64_t best = -1;
  int32_t shape = 4 | (4 << 8);
  for (int32_t ni = 1; ni <= 4; ++ni)
    for (int32_t nj = 1; nj <= 4; ++nj) {
      const int64_t bm = 16 * ni, bn = 16 * nj;
      const int64_t area = ((M + bm - 1) / bm * bm) * ((N + bn - 1) / bn * bn);
      const int64_t bs = (int64_t)(shape & 0xff) * (shape >> 8);
      if (best < 0 || area < best || (area == best && ni * nj > bs)) {
        best = area;
        shape = ni | (nj << 8);
      }
    }
  return shape;
}

// Append the tiles of one M x N output and its segment list; returns the
// positions (before sorting) of the new tiles in *ids.
void add_output(TaskListF64& tl, const TileF64& proto, const std::vector<SegF64>& segs, std::vector<int64_t>* ids) {
  if (proto.M <= 0 || proto.N <= 0) return;
  const int32_t sb = (int32_t)tl.h_segs.size();
  tl.h_segs.insert(tl.h_segs.end(), segs.begin(), segs.end());
  const int32_t se = (int32_t)tl.h_segs.size();
  const int32_t shape = f64_shape(proto.M, proto.N);
  const int32_t bm = 16 * (shape & 0xff), bn = 16 * (shape >> 8);
  for (int32_t m0 = 0; m0 < proto.M; m0 += bm)
    for (int32_t n0 = 0; n0 < proto.N; n0 += bn) {
      TileF64 t = proto;
      t.m0 = m0;
      t.n0 = n0;
      t.seg_begin = sb;
      t.seg_end = se;
      t.shape = shape;
      if (ids) ids->push_back((int64_t)tl.h_tiles.size());
      tl.h_tiles.push_back(t);
    }
}

TileF64 out_tile(int32_t buf, int64_t off, int32_t ldc, int32_t M, int32_t N, int32_t mode) {
  TileF64 t{};
  t.c_buf = buf;
  t.c_off = off;
  t.ldc = ldc;
  t.M = M;
  t.N = N;
  t.mode = mode;
  return t;
}

// Heaviest tiles first (one CTA per tile); returns new position of each old tile.
std::vector<int64_t> sort_tiles(TaskListF64& tl) {
  const size_t n = tl.h_tiles.size();
  std::vector<int64_t> w(n), perm(n), where(n);
  for (size_t i = 0; i < n; ++i) {
    int64_t k = 0;
    for (int32_t s = tl.h_tiles[i].seg_begin; s < tl.h_tiles[i].seg_end; ++s) k += tl.h_segs[s].K;
    w[i] = k * (tl.h_tiles[i].shape & 0xff) * (tl.h_tiles[i].shape >> 8);  // FMAs per thread
  }
  std::iota(perm.begin(), perm.end(), 0);
  std::stable_sort(perm.begin(), perm.end(), [&](int64_t a, int64_t b) { return w[a] > w[b]; });
  std::vector<TileF64> nt(n);
  for (size_t i = 0; i < n; ++i) {
    nt[i] = tl.h_tiles[perm[i]];
    where[perm[i]] = (int64_t)i;
  }
  tl.h_tiles.swap(nt);
  return where;
}

void finish(TaskListF64& tl) {
  tl.n_tiles = (int64_t)tl.h_tiles.size();
  upload(tl.d_tiles, tl.h_tiles);
  upload(tl.d_segs, tl.h_segs);
}

void free_tl(TaskListF64& tl) {
  if (tl.d_tiles) cudaFree(tl.d_tiles);
  if (tl.d_segs) cudaFree(tl.d_segs);
  tl.d_tiles = nullptr;
  tl.d_segs = nullptr;
}

bool is_gemm_pair(int flags) { return (flags & (DMRG_ID_A | DMRG_ID_B)) == 0; }

// One product over a pair set with the batch members stacked:
//   phase 1 (two-GEMM pairs): order 1  X_b = c Psi_b B^T  (members along M)
//                              order 0  T_b = c A Psi_b    (members along N)
//   group M (members along M): Y_b += c Psi_b B^T (A = 1), Y_b += T_b B^T
//   group N (members along N): Y_b += c A Psi_b (B = 1),   Y_b += A X_b
// Intermediates: member b, pair i at T + b*Tm + toff[i], row-major (order 1:
// r_in x c_out, order 0: r_out x c_in).  scaled = false drops every
// coefficient (for the per-term dot products).
// dots = true (with scaled = false): the output tiles are TM_STORE_DOTS and
// each segment carries its term (coef) for the tile to apply per member.
void build_stacked(const dmrg_sb* sb, const std::vector<GPair>& P, const std::vector<int64_t>& toff, int64_t Tm,
                   bool scaled, TaskListF64& ph1, TaskListF64* gM, TaskListF64* gN, bool dots = false) {
  const int nb = sb->batch;
  const int64_t D = sb->D;
  const auto& r = sb->r;
  const auto& c = sb->c;
  for (size_t i = 0; i < P.size(); ++i) {
    const GPair& p = P[i];
    if (!is_gemm_pair(p.flags)) continue;
    const int32_t ro = r[p.s_out], ri = r[p.s_in], co = c[p.s_out], ci = c[p.s_in];
    SegF64 g = seg_base();
    g.K = p.order == 1 ? ci : ri;
    if (scaled) { g.coef = p.term; g.coef_mode = p.order == 1 ? 1 : 2; }
    if (p.order == 1) {  // X_b = Psi_b B^T : M = (b, a'), N = beta, K = c_in
      g.l_buf = BUF_X; g.l_off = sb->off[p.s_in]; g.ldl = ci; g.l_rm = ri; g.l_bs = D;
      set_R_opT(g, p.B);
      TileF64 t = out_tile(BUF_T, toff[i], co, nb * ri, co, TM_STORE);
      t.c_rm = ri; t.c_axis = 0; t.c_bs = Tm;
      add_output(ph1, t, {g}, nullptr);
    } else {  // T_b = A Psi_b : M = alpha, N = (b, beta'), K = r_in
      set_L_op(g, p.A);
      g.r_buf = BUF_X; g.r_off = sb->off[p.s_in]; g.ldr = ci; g.r_trans = 0; g.r_rm = ci; g.r_bs = D;
      TileF64 t = out_tile(BUF_T, toff[i], ci, ro, nb * ci, TM_STORE);
      t.c_rm = ci; t.c_axis = 1; t.c_bs = Tm;
      add_output(ph1, t, {g}, nullptr);
    }
  }
  if (!gM) return;
  std::vector<std::vector<size_t>> by_out(sb->S);
  for (size_t i = 0; i < P.size(); ++i) by_out[P[i].s_out].push_back(i);
  for (int s = 0; s < sb->S; ++s) {
    if ((int64_t)r[s] * c[s] == 0) continue;
    std::vector<SegF64> sM, sN;
    for (size_t i : by_out[s]) {
      const GPair& p = P[i];
      const int32_t ri = r[p.s_in], ci = c[p.s_in], co = c[p.s_out];
      SegF64 g = seg_base();
      if (dots) {
        g.coef = p.term;
        g.coef_mode = -1;  // no scaling while loading: the tile scales the segment's sum
      }
      if (p.flags & DMRG_ID_A) {  // Y_b += c Psi_b B^T
        g.K = ci;
        g.l_buf = BUF_X; g.l_off = sb->off[p.s_in]; g.ldl = ci; g.l_rm = ri; g.l_bs = D;
        set_R_opT(g, p.B);
        if (scaled) { g.coef = p.term; g.coef_mode = 1; }
        sM.push_back(g);
      } else if (p.flags & DMRG_ID_B) {  // Y_b += c A Psi_b
        g.K = ri;
        set_L_op(g, p.A);
        g.r_buf = BUF_X; g.r_off = sb->off[p.s_in]; g.ldr = ci; g.r_trans = 0; g.r_rm = ci; g.r_bs = D;
        if (scaled) { g.coef = p.term; g.coef_mode = 2; }
        sN.push_back(g);
      } else if (p.order == 0) {  // Y_b += T_b B^T
        g.K = ci;
        g.l_buf = BUF_T; g.l_off = toff[i]; g.ldl = ci; g.l_rm = r[p.s_out]; g.l_bs = Tm;
        set_R_opT(g, p.B);
        sM.push_back(g);
      } else {  // Y_b += A X_b
        g.K = ri;
        set_L_op(g, p.A);
        g.r_buf = BUF_T; g.r_off = toff[i]; g.ldr = co; g.r_trans = 0; g.r_rm = co; g.r_bs = Tm;
        sN.push_back(g);
      }
    }
    const bool hasM = !sM.empty(), hasN = !sN.empty();
    const int32_t mode = dots ? TM_STORE_DOTS : TM_STORE;
    if (hasM || !hasN) {
      TileF64 t = out_tile(BUF_Y, sb->off[s], c[s], nb * r[s], c[s], mode);
      t.c_rm = r[s]; t.c_axis = 0; t.c_bs = D;
      add_output(*gM, t, sM, nullptr);
    }
    if (hasN) {
      TileF64 t = out_tile(BUF_Y, sb->off[s], c[s], r[s], nb * c[s], mode);
      t.c_rm = c[s]; t.c_axis = 1; t.c_bs = D; t.add = hasM ? 1 : 0;
      add_output(*gN, t, sN, nullptr);
    }
  }
}

// intermediate layout of a pair set: offsets per pair inside one member's T
int64_t layout_T(const dmrg_sb* sb, const std::vector<GPair>& P, std::vector<int64_t>& toff) {
  toff.assign(P.size(), -1);
  int64_t T = 0;
  for (size_t i = 0; i < P.size(); ++i) {
    const GPair& p = P[i];
    if (!is_gemm_pair(p.flags)) continue;
    const int64_t ro = sb->r[p.s_out], ri = sb->r[p.s_in], co = sb->c[p.s_out], ci = sb->c[p.s_in];
    toff[i] = T;
    T += p.order == 0 ? ro * ci : ri * co;
  }
  return T;
}

void build_f64_tasks(dmrg_sb* sb) {
  const int nt = sb->n_terms;
  const auto& r = sb->r;
  const auto& c = sb->c;
  std::vector<GPair> fw, bw;
  for (const PairH& p : sb->pairs) {
    const int32_t ro = r[p.s_out], ri = r[p.s_in], co = c[p.s_out], ci = c[p.s_in];
    GPair f{p.term, p.s_out, p.s_in, p.flags, p.order, {p.a_off, ri, 0}, {p.b_off, ci, 0}};
    fw.push_back(f);
    // transposed pair: s_in <- s_out, A^T (r_in x r_out), B^T (c_in x c_out)
    GPair t{p.term, p.s_in, p.s_out, p.flags, 0, {p.a_off, ri, 1}, {p.b_off, ci, 1}};
    if (is_gemm_pair(p.flags)) {
      const double c0 = 2.0 * ri * ro * co + 2.0 * ri * co * ci;  // (A^T G) B first
      const double c1 = 2.0 * ro * co * ci + 2.0 * ri * ro * ci;  // A^T (G B) first
      t.order = c0 <= c1 ? 0 : 1;
    }
    bw.push_back(t);
  }
  std::vector<int64_t> toff_f, toff_b;
  const int64_t Tf = layout_T(sb, fw, toff_f), Tb = layout_T(sb, bw, toff_b);
  const int64_t Tm = std::max(Tf, Tb);
  sb->T_elems = Tm * sb->batch;
  sb->T_fwd_elems = Tf > 0 ? Tm * (sb->batch - 1) + Tf : 0;  // member b's forward intermediates at b Tm + [0, Tf)
  if (sb->d_T) cudaFree(sb->d_T);
  sb->d_T = dalloc<double>((size_t)sb->T_elems);

  build_stacked(sb, fw, toff_f, Tm, true, sb->f64_fwd1, &sb->f64_fwd2, &sb->f64_fwd3);
  build_stacked(sb, bw, toff_b, Tm, true, sb->f64_bwd1, &sb->f64_bwd2, &sb->f64_bwd3);
  build_stacked(sb, fw, toff_f, Tm, false, sb->f64_dot1, nullptr, nullptr);

  // per-term dots: one unstacked output per (member, pair), dotted with G
  std::vector<std::vector<int64_t>> dot_list((size_t)sb->batch * nt);
  for (int b = 0; b < sb->batch; ++b) {
    const int64_t xb = (int64_t)b * sb->D, tb = (int64_t)b * Tm;
    for (size_t i = 0; i < fw.size(); ++i) {
      const GPair& p = fw[i];
      const int32_t ri = r[p.s_in], ci = c[p.s_in], co = c[p.s_out];
      SegF64 g = seg_base();
      if (p.flags & DMRG_ID_B) {
        g.K = ri; set_L_op(g, p.A);
        g.r_buf = BUF_X; g.r_off = xb + sb->off[p.s_in]; g.ldr = ci; g.r_trans = 0;
      } else if (p.flags & DMRG_ID_A) {
        g.K = ci; g.l_buf = BUF_X; g.l_off = xb + sb->off[p.s_in]; g.ldl = ci; set_R_opT(g, p.B);
      } else if (p.order == 0) {
        g.K = ci; g.l_buf = BUF_T; g.l_off = tb + toff_f[i]; g.ldl = ci; set_R_opT(g, p.B);
      } else {
        g.K = ri; set_L_op(g, p.A);
        g.r_buf = BUF_T; g.r_off = tb + toff_f[i]; g.ldr = co; g.r_trans = 0;
      }
      std::vector<int64_t> ids;
      add_output(sb->f64_dot2, out_tile(BUF_G, xb + sb->off[p.s_out], c[p.s_out], r[p.s_out], c[p.s_out], TM_DOT),
                 {g}, &ids);
      for (int64_t id : ids) dot_list[(size_t)b * nt + p.term].push_back(id);
    }
  }
  // H psi with the per-term dots <psi, (A_k x B_k) psi> in one pass: the
  // output launches of the product with unscaled segments (after f64_dot1's
  // unscaled intermediates); the tiles apply c(member, term) themselves
  {
    TaskListF64 unused;
    build_stacked(sb, fw, toff_f, Tm, false, unused, &sb->f64_pdot2, &sb->f64_pdot3, true);
  }
  for (TaskListF64* tl : {&sb->f64_fwd1, &sb->f64_fwd2, &sb->f64_fwd3, &sb->f64_bwd1, &sb->f64_bwd2, &sb->f64_bwd3,
                          &sb->f64_dot1, &sb->f64_pdot2, &sb->f64_pdot3})
    sort_tiles(*tl);
  {  // partials of f64_pdot2/3: 64 per (tile, segment) in tile order, then the (member, term) lists
    std::vector<std::vector<int32_t>> lists((size_t)sb->batch * nt);
    int32_t base = 0;
    for (TaskListF64* tl : {&sb->f64_pdot2, &sb->f64_pdot3})
      for (TileF64& t : tl->h_tiles) {
        t.dot_base = base;
        const bool by_col = t.c_rm && t.c_axis == 1;
        const int32_t bm = 16 * (t.shape & 0xff), bn = 16 * (t.shape >> 8);
        for (int32_t q = t.seg_begin; q < t.seg_end; ++q) {
          const int32_t term = tl->h_segs[q].coef;
          const int64_t slot = (int64_t)(base + (q - t.seg_begin)) * 64;
          for (int32_t e = 0; e < (by_col ? bn : bm); ++e) {
            const int32_t g = (by_col ? t.n0 : t.m0) + e;
            if (g >= (by_col ? t.N : t.M)) break;
            const int32_t member = t.c_rm ? g / t.c_rm : t.member;
            lists[(size_t)member * nt + term].push_back((int32_t)(slot + e));
          }
        }
        base += t.seg_end - t.seg_begin;
      }
    if ((int64_t)base * 64 > INT32_MAX) throw Invalid{"too many product segments for the per-term dots"};
    std::vector<int32_t> ptr(1, 0), idx;
    for (auto& l : lists) {
      idx.insert(idx.end(), l.begin(), l.end());
      ptr.push_back((int32_t)idx.size());
    }
    upload(sb->d_pdot_ptr, ptr);
    upload(sb->d_pdot_idx, idx);
    if (sb->d_pdot_partial) cudaFree(sb->d_pdot_partial);
    sb->d_pdot_partial = dalloc<double>((size_t)std::max<int64_t>(1, (int64_t)base * 64));
  }
  const std::vector<int64_t> where = sort_tiles(sb->f64_dot2);
  std::vector<int32_t> ptr(1, 0), idx;
  for (auto& lst : dot_list) {
    for (int64_t id : lst) idx.push_back((int32_t)where[id]);
    ptr.push_back((int32_t)idx.size());
  }
  upload(sb->d_dot_red_ptr, ptr);
  upload(sb->d_dot_red_idx, idx);
  if (sb->d_dot_partial) cudaFree(sb->d_dot_partial);
  sb->d_dot_partial = dalloc<double>((size_t)std::max<int64_t>(1, (int64_t)sb->f64_dot2.h_tiles.size()));
  for (TaskListF64* tl : {&sb->f64_fwd1, &sb->f64_fwd2, &sb->f64_fwd3, &sb->f64_dot1, &sb->f64_dot2, &sb->f64_bwd1,
                          &sb->f64_bwd2, &sb->f64_bwd3, &sb->f64_pdot2, &sb->f64_pdot3})
    finish(*tl);
}

// ------------------------------------------------------------- products
// Double-float products read pre-split pairs: the operator arena (split at
// the first such product) and the input, split into a buffer of its own each
// time; the intermediates are written and read as pairs.  Returns the
// buffers and their pair mask.
uint32_t df_bufs(dmrg_sb* sb, const double* x, double* y, Bufs& bufs, cudaStream_t st) {
  if (!sb->d_ops_df) {
    sb->d_ops_df = dalloc<double>((size_t)std::max<int64_t>(sb->ops_elems, 1));
    launch_split_pairs(sb->d_ops, sb->d_ops_df, sb->ops_elems, st);
  }
  if (!sb->d_x_df) sb->d_x_df = dalloc<double>((size_t)(sb->batch * sb->D));
  launch_split_pairs(x, sb->d_x_df, sb->batch * sb->D, st);
  bufs = Bufs{{sb->d_x_df, y, sb->d_T, sb->d_ops_df, nullptr}};
  return (1u << BUF_X) | (1u << BUF_T) | (1u << BUF_OPS);
}

// member_done (tensor-core precisions only, may be null): device [batch]
// flags; members whose flag is nonzero are skipped (their rows of y are left
// as they are)
void matvec(dmrg_sb* sb, int prec, const double* x, double* y, int accumulate, const int32_t* skip,
            cudaStream_t st, const int32_t* member_done = nullptr) {
  if (prec == DMRG_FP64) {
    Bufs bufs{{const_cast<double*>(x), y, sb->d_T, sb->d_ops, nullptr}};
    launch_seg_gemm_f64(sb->f64_fwd1, bufs, sb->d_coeffs, sb->n_terms, 0, nullptr, skip, st);
    launch_seg_gemm_f64(sb->f64_fwd2, bufs, sb->d_coeffs, sb->n_terms, accumulate, nullptr, skip, st);
    launch_seg_gemm_f64(sb->f64_fwd3, bufs, sb->d_coeffs, sb->n_terms, accumulate, nullptr, skip, st);
  } else if (prec == DMRG_DF64) {  // the same task lists in double-float arithmetic
    Bufs bufs;
    const uint32_t pm = df_bufs(sb, x, y, bufs, st);
    launch_seg_gemm_df(sb->f64_fwd1, bufs, sb->d_coeffs, sb->n_terms, 0, nullptr, skip, st, pm);
    launch_seg_gemm_df(sb->f64_fwd2, bufs, sb->d_coeffs, sb->n_terms, accumulate, nullptr, skip, st, pm);
    launch_seg_gemm_df(sb->f64_fwd3, bufs, sb->d_coeffs, sb->n_terms, accumulate, nullptr, skip, st, pm);
  } else {
    tc_matvec(sb, prec, x, y, accumulate, skip, st, member_done);
  }
  CK(cudaGetLastError());
}

// y = H psi and dc[b][k] = <psi_b, (A_k x B_k) psi_b> in one pass, in float64
// or (df) double-float arithmetic
void matvec_f64_dots(dmrg_sb* sb, const double* psi, double* y, double* dc, cudaStream_t st, bool df = false) {
  Bufs bufs{{const_cast<double*>(psi), y, sb->d_T, sb->d_ops, nullptr}};
  if (df) {
    const uint32_t pm = df_bufs(sb, psi, y, bufs, st);
    launch_seg_gemm_df(sb->f64_dot1, bufs, sb->d_coeffs, sb->n_terms, 0, nullptr, nullptr, st, pm);
    launch_seg_gemm_df_dots(sb->f64_pdot2, bufs, sb->d_coeffs, sb->n_terms, 0, sb->d_pdot_partial, nullptr, st, pm);
    launch_seg_gemm_df_dots(sb->f64_pdot3, bufs, sb->d_coeffs, sb->n_terms, 0, sb->d_pdot_partial, nullptr, st, pm);
  } else {
    launch_seg_gemm_f64(sb->f64_dot1, bufs, sb->d_coeffs, sb->n_terms, 0, nullptr, nullptr, st);
    launch_seg_gemm_f64_dots(sb->f64_pdot2, bufs, sb->d_coeffs, sb->n_terms, 0, sb->d_pdot_partial, nullptr, st);
    launch_seg_gemm_f64_dots(sb->f64_pdot3, bufs, sb->d_coeffs, sb->n_terms, 0, sb->d_pdot_partial, nullptr, st);
  }
  lz_launch_reduce_terms(sb->d_pdot_partial, sb->d_pdot_ptr, sb->d_pdot_idx, dc, sb->batch * sb->n_terms, st);
  CK(cudaGetLastError());
}

void term_dots(dmrg_sb* sb, const double* psi, const double* g, double* dc, cudaStream_t st) {
  Bufs bufs{{const_cast<double*>(psi), nullptr, sb->d_T, sb->d_ops, const_cast<double*>(g)}};
  launch_seg_gemm_f64(sb->f64_dot1, bufs, sb->d_coeffs, sb->n_terms, 0, nullptr, nullptr, st);
  launch_seg_gemm_f64(sb->f64_dot2, bufs, sb->d_coeffs, sb->n_terms, 0, sb->d_dot_partial, nullptr, st);
  lz_launch_reduce_terms(sb->d_dot_partial, sb->d_dot_red_ptr, sb->d_dot_red_idx, dc, sb->batch * sb->n_terms, st);
  CK(cudaGetLastError());
}

// --------------------------------------------------------------- Lanczos
void lz_free(dmrg_sb* sb) {
  for (int i = 0; i < 8; ++i)
    if (sb->lz_graphs[i]) {
      cudaGraphExecDestroy((cudaGraphExec_t)sb->lz_graphs[i]);
      sb->lz_graphs[i] = nullptr;
      sb->lz_graph_key[i] = 0;
    }
  for (double* p : {sb->lz_V, sb->lz_w, sb->lz_vcur, sb->lz_partial, sb->lz_h, sb->lz_npart, sb->lz_ab, sb->lz_s,
                    sb->lz_out, sb->rf_q, sb->rf_sc, sb->rf_diag, sb->rf_part})
    if (p) cudaFree(p);
  for (float* p : {sb->rf_res, sb->rf_p, sb->rf_hp, sb->rf_t, sb->rf_psi32, sb->rf_minv})
    if (p) cudaFree(p);
  if (sb->lz_ctl) cudaFree(sb->lz_ctl);
  if (sb->lz_gate) cudaFree(sb->lz_gate);
  if (sb->rf_ctl) cudaFree(sb->rf_ctl);
  sb->rf_q = sb->rf_sc = sb->rf_diag = sb->rf_part = nullptr;
  sb->rf_res = sb->rf_p = sb->rf_hp = sb->rf_t = sb->rf_psi32 = sb->rf_minv = nullptr;
  sb->rf_ctl = nullptr;
  if (sb->h_ctl) cudaFreeHost(sb->h_ctl);
  sb->lz_V = sb->lz_w = sb->lz_vcur = sb->lz_partial = sb->lz_h = sb->lz_npart = sb->lz_ab = sb->lz_s =
      sb->lz_out = nullptr;
  sb->lz_ctl = sb->lz_gate = nullptr;
  sb->h_ctl = nullptr;
  sb->lz_cap = 0;
}

void lz_alloc(dmrg_sb* sb, int cap) {
  if (cap <= sb->lz_cap) return;
  lz_free(sb);
  const int64_t D = sb->D, B = sb->batch;
  sb->lz_nchunk = lz_nchunk(D);
  sb->lz_V = dalloc<double>((size_t)(cap * B * D));
  sb->lz_w = dalloc<double>((size_t)(B * D));
  sb->lz_vcur = dalloc<double>((size_t)(B * D));
  // per-chunk partials of the vector kernels, or per-warp dot partials of every Krylov row
  sb->lz_partial = dalloc<double>((size_t)B * std::max(sb->lz_nchunk, lz_dot_nparts(sb->D)) * cap);
  sb->lz_h = dalloc<double>((size_t)(3 * B * cap));
  sb->lz_npart = dalloc<double>((size_t)(3 * B * sb->lz_nchunk));
  sb->lz_gate = dalloc<int32_t>((size_t)B);
  sb->lz_ab = dalloc<double>((size_t)(2 * B * cap));
  sb->lz_s = dalloc<double>((size_t)(B * cap));
  sb->lz_out = dalloc<double>((size_t)(4 * B + 1));
  sb->lz_ctl = dalloc<int32_t>((size_t)(LZ_CTL_MEMBER + 2 * B));
  void* hp = nullptr;
  CK(cudaMallocHost(&hp, sizeof(int32_t) * (LZ_CTL_MEMBER + 2 * B)));
  sb->h_ctl = static_cast<int32_t*>(hp);
  CK(cudaMemset(sb->lz_ab, 0, sizeof(double) * 2 * B * cap));
  sb->rf_res = dalloc<float>((size_t)(B * D));
  sb->rf_p = dalloc<float>((size_t)(B * D));
  sb->rf_q = dalloc<double>((size_t)(B * D));
  sb->rf_hp = dalloc<float>((size_t)(B * D));
  sb->rf_t = dalloc<float>((size_t)(B * D));
  sb->rf_psi32 = dalloc<float>((size_t)(B * D));
  sb->rf_sc = dalloc<double>((size_t)(RF_NSC * B + 2));
  sb->rf_ctl = dalloc<int32_t>((size_t)(2 * B + 2));
  sb->rf_diag = dalloc<double>((size_t)(B * D));
  sb->rf_minv = dalloc<float>((size_t)(B * D));
  sb->rf_part = dalloc<double>((size_t)(4 * B * sb->lz_nchunk));
  sb->lz_cap = cap;
}

// Krylov basis storage: float64 for float64 solves, double-float pairs (and
// double-float Gram-Schmidt passes) for the mixed-precision solves
bool lz_pair(int prec) { return prec != DMRG_FP64; }

// one Lanczos iteration for every running member (all on stream st)
void lz_enqueue_iteration(dmrg_sb* sb, int prec, cudaStream_t st) {
  const int64_t D = sb->D;
  const int B = sb->batch, cap = sb->lz_cap, nch = sb->lz_nchunk;
  int32_t* ctl = sb->lz_ctl;
  // members that have stopped (converged, pending, or held from an earlier run) get no product
  matvec(sb, prec, sb->lz_vcur, sb->lz_w, 0, ctl + LZ_CTL_ALLDONE, st, ctl + LZ_CTL_MEMBER);
  // reorthogonalisation: (A) three-term step, (B) full pass, (C) second full
  // pass where the DGKS test asks for it (see lanczos.cu)
  double* hA = sb->lz_h;
  double* hB = sb->lz_h + (size_t)B * cap;
  double* hC = sb->lz_h + (size_t)2 * B * cap;
  double* nA = sb->lz_npart;
  double* nB = sb->lz_npart + (size_t)B * nch;
  double* nC = sb->lz_npart + (size_t)2 * B * nch;
  const int ndot = lz_dot_nchunk(D);
  const bool pair = lz_pair(prec);  // the Krylov basis as double-float pairs (mixed-precision solves)
  lz_launch_dots_local(sb->lz_V, sb->lz_w, sb->lz_partial, ctl, D, B, cap, st, pair);
  lz_launch_reduce_rows(sb->lz_partial, hA, ctl, lz_dot_nparts(D), cap, B, 2, nullptr, st);
  // pass A's update runs inside pass B's dot sweep (norm partials per dot chunk)
  lz_launch_multidot(sb->lz_V, sb->lz_w, sb->lz_partial, ctl, D, B, cap, 0, nullptr, st, hA, nA, pair);
  lz_launch_reduce_rows(sb->lz_partial, hB, ctl, lz_dot_nparts(D), cap, B, 0, nullptr, st);
  lz_launch_multiaxpy(sb->lz_V, sb->lz_w, hB, nB, ctl, D, B, cap, nch, 0, nullptr, st, pair);
  lz_launch_dgks(nA, nB, sb->lz_gate, ctl, B, ndot, nch, st);
  lz_launch_multidot(sb->lz_V, sb->lz_w, sb->lz_partial, ctl, D, B, cap, 0, sb->lz_gate, st, nullptr, nullptr, pair);
  lz_launch_reduce_rows(sb->lz_partial, hC, ctl, lz_dot_nparts(D), cap, B, 0, sb->lz_gate, st);
  lz_launch_multiaxpy(sb->lz_V, sb->lz_w, hC, nC, ctl, D, B, cap, nch, 0, sb->lz_gate, st, pair);
  lz_launch_finalize_ab(sb->lz_h, nB, nC, sb->lz_gate, sb->lz_ab, ctl, B, cap, nch, st);
  lz_launch_tridiag(sb->lz_ab, sb->lz_s, sb->lz_out, ctl, sb->lz_out + 4 * B, B, cap, D, st);  // tol at out[4B]
  lz_launch_next_vector(sb->lz_w, sb->lz_ab, sb->lz_V, sb->lz_vcur, ctl, D, B, cap, st, pair);
  lz_launch_advance(ctl, B, st);
  CK(cudaGetLastError());
}

cudaGraphExec_t lz_graph(dmrg_sb* sb, int prec, int K) {
  const int key = 1 + prec * 1024 + K;
  for (int i = 0; i < 8; ++i)
    if (sb->lz_graphs[i] && sb->lz_graph_key[i] == key) return (cudaGraphExec_t)sb->lz_graphs[i];
  // the products' panels must exist before the capture (building them allocates)
  if (prec == DMRG_TF32 || prec == DMRG_BF16X3) tc_prepare(sb, prec);
  cudaStream_t cs;
  CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  try {
    for (int k = 0; k < K; ++k) lz_enqueue_iteration(sb, prec, cs);
  } catch (...) {
    cudaStreamEndCapture(cs, &g);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    throw;
  }
  CK(cudaStreamEndCapture(cs, &g));
  cudaGraphExec_t ge = nullptr;
  cudaError_t e = cudaGraphInstantiate(&ge, g, 0);
  cudaGraphDestroy(g);
  cudaStreamDestroy(cs);
  CK(e);
  int slot = 0;
  for (int i = 0; i < 8; ++i)
    if (!sb->lz_graphs[i]) { slot = i; break; }
  if (sb->lz_graphs[slot]) cudaGraphExecDestroy((cudaGraphExec_t)sb->lz_graphs[slot]);
  sb->lz_graphs[slot] = ge;
  sb->lz_graph_key[slot] = key;
  return ge;
}

struct LzRun {
  std::vector<int32_t> code, iters, restarts;
  std::vector<double> theta, resid;
  int64_t launches = 0;
};

int matvec_launches(const dmrg_sb* sb, int prec) {
  if (prec == DMRG_FP64 || prec == DMRG_DF64)
    return (sb->f64_fwd1.n_tiles > 0) + (sb->f64_fwd2.n_tiles > 0) + (sb->f64_fwd3.n_tiles > 0);
  return tc_launches(sb, prec);
}
constexpr int LZ_KERNELS_PER_ITER = 13;  // everything in lz_enqueue_iteration besides the product

// One Lanczos run from psi0 (device [batch][D]) to psi_out for the members
// whose initial control code is LZ_RUNNING (the others are LZ_HOLD: skipped,
// their psi_out untouched).  Returns the per-member codes, Krylov lengths,
// theta and residual (from lz_out; unchanged for held members).
LzRun lz_run(dmrg_sb* sb, const double* psi0, double* psi_out, int prec, double tol, int max_iter,
             int check_every, int graph_iters, const std::vector<int32_t>& init, int force, cudaStream_t st) {
  const int64_t D = sb->D;
  const int B = sb->batch;
  const int cap = sb->lz_cap, nch = sb->lz_nchunk;
  // v_0 = psi0 / |psi0|
  double* part = sb->lz_partial;
  double* nrm2 = sb->d_scratch;
  lz_launch_sumsq(psi0, part, D, B, nch, st);
  lz_launch_sum_chunks(part, nrm2, nch, B, st);
  lz_launch_scale_unit(psi0, nrm2, sb->lz_V, sb->lz_vcur, D, B, st, lz_pair(prec));
  std::vector<int32_t> hc(LZ_CTL_MEMBER + 2 * B, 0);
  hc[LZ_CTL_MAXIT] = max_iter;
  hc[LZ_CTL_CHECK] = std::max(1, check_every);
  hc[LZ_CTL_FORCE] = force;
  for (int b = 0; b < B; ++b) hc[LZ_CTL_MEMBER + b] = init[b];
  CK(cudaMemcpyAsync(sb->lz_ctl, hc.data(), hc.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(sb->lz_out + 4 * B, &tol, sizeof(double), cudaMemcpyHostToDevice, st));
  CK(cudaStreamSynchronize(st));  // host vectors above are stack memory
  const int K = std::max(1, std::min(graph_iters, max_iter));
  cudaGraphExec_t ge = lz_graph(sb, prec, K);
  int launched = 0;
  for (;;) {
    CK(cudaGraphLaunch(ge, st));
    launched += K;
    CK(cudaMemcpyAsync(sb->h_ctl, sb->lz_ctl, sizeof(int32_t) * (LZ_CTL_MEMBER + 2 * B), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (sb->h_ctl[LZ_CTL_ALLDONE]) break;
    if (launched > max_iter + K) throw Invalid{"Lanczos control did not terminate"};
  }
  // float64 eigenpairs of the members that stopped on the float32 test, side by side
  lz_launch_tridiag(sb->lz_ab, sb->lz_s, sb->lz_out, sb->lz_ctl, sb->lz_out + 4 * B, B, cap, D, st, 1);
  CK(cudaMemcpyAsync(sb->h_ctl, sb->lz_ctl, sizeof(int32_t) * (LZ_CTL_MEMBER + 2 * B), cudaMemcpyDeviceToHost, st));
  lz_launch_ritz(sb->lz_V, sb->lz_s, sb->lz_ctl, psi_out, D, B, cap, st, lz_pair(prec));
  lz_launch_sumsq(psi_out, part, D, B, nch, st);
  lz_launch_sum_chunks(part, nrm2, nch, B, st);
  lz_launch_scale_unit(psi_out, nrm2, psi_out, nullptr, D, B, st);
  std::vector<double> out(4 * B);
  int32_t tc_err = 0;
  CK(cudaMemcpyAsync(out.data(), sb->lz_out, sizeof(double) * 4 * B, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&tc_err, sb->d_tc_err, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  CK(cudaGetLastError());
  if (tc_err) throw Timeout{"a tensor-core kernel gave up a bounded wait"};
  LzRun r;
  r.launches = 3 + (int64_t)launched * (LZ_KERNELS_PER_ITER + matvec_launches(sb, prec)) + 5;
  for (int b = 0; b < B; ++b) {
    r.code.push_back(sb->h_ctl[LZ_CTL_MEMBER + b]);
    r.iters.push_back(sb->h_ctl[LZ_CTL_MEMBER + B + b]);
    r.theta.push_back(out[4 * b]);
    r.resid.push_back(out[4 * b + 1]);
  }
  r.restarts.assign(B, 0);
  return r;
}

// Lanczos from psi0 (device [batch][D]) to psi_out; returns per-member results.
// A member that stopped on the float32 test but failed the float64 test after
// the loop (LZ_RESUME) is restarted from its Ritz vector with the iterations
// it has left, the others held, at most LZ_MAX_RESTARTS times.
constexpr int LZ_MAX_RESTARTS = 3;
LzRun lz_solve(dmrg_sb* sb, const double* psi0, double* psi_out, int prec, double tol, int max_iter,
               int check_every, int graph_iters, cudaStream_t st) {
  const int64_t D = sb->D;
  const int B = sb->batch;
  max_iter = (int)std::min<int64_t>(std::min(std::max(1, max_iter), 768), D);  // tridiagonal kernel keeps 60 B per Krylov vector in shared memory (48 KB)
  lz_alloc(sb, max_iter + 1);
  const int force = sb->test_force_pending;
  sb->test_force_pending = 0;
  LzRun r = lz_run(sb, psi0, psi_out, prec, tol, max_iter, check_every, graph_iters,
                   std::vector<int32_t>(B, LZ_RUNNING), force, st);
  for (int k = 0; k < LZ_MAX_RESTARTS; ++k) {
    std::vector<int32_t> init(B, LZ_HOLD);
    int used = 0;
    bool any = false;
    for (int b = 0; b < B; ++b)
      if (r.code[b] == LZ_RESUME) {
        init[b] = LZ_RUNNING;
        used = std::max(used, r.iters[b]);
        any = true;
      }
    if (!any || max_iter - used < 2) break;
    LzRun q = lz_run(sb, psi_out, psi_out, prec, tol, max_iter - used, check_every, graph_iters, init, 0, st);
    r.launches += q.launches;
    for (int b = 0; b < B; ++b)
      if (init[b] == LZ_RUNNING) {
        r.code[b] = q.code[b];
        r.iters[b] += q.iters[b];
        r.theta[b] = q.theta[b];
        r.resid[b] = q.resid[b];
        r.restarts[b] += 1;
      }
  }
  for (int b = 0; b < B; ++b)
    if (r.code[b] == LZ_RESUME) r.code[b] = LZ_CAP;
  return r;
}

// ------------------------------------------------------------ refinement
void rf_enqueue_inner(dmrg_sb* sb, int prec, cudaStream_t st) {
  const int64_t D = sb->D;
  const int B = sb->batch;
  int32_t* ctl = sb->rf_ctl;
  int32_t* stop = ctl + 2 * B;
  double* sc = sb->rf_sc;
  const float* psi = sb->rf_psi32;  // the current iterate, rounded for the inner solve
  tc_matvec_f32in(sb, prec, sb->rf_p, sb->rf_q, 0, stop, st, ctl);  // q = H p (mixed); done members skipped
  rf_launch_dots4(sb->rf_q, sb->rf_p, psi, sb->rf_hp, sc, ctl, sb->rf_part, D, B, stop, st);
  rf_launch_alpha4(sb->rf_part, sc, ctl, D, B, stop, st);
  rf_launch_update(sb->rf_t, sb->rf_res, sb->rf_p, sb->rf_hp, psi, sb->rf_minv, sc, ctl, sb->rf_part, D, B, stop,
                   st);
  rf_launch_sum4(sb->rf_part, sc, D, B, 0, ctl, stop, st);
  rf_launch_beta(sc, ctl, sc + RF_NSC * B, B, stop, st);
  rf_launch_dir(sb->rf_p, sb->rf_res, psi, sb->rf_minv, sc, ctl, D, B, 0, stop, st);
  CK(cudaGetLastError());
}
constexpr int RF_KERNELS_PER_ITER = 6;

cudaGraphExec_t rf_graph(dmrg_sb* sb, int prec, int K) {
  const int key = (1 << 20) + 1 + prec * 1024 + K;
  for (int i = 0; i < 8; ++i)
    if (sb->lz_graphs[i] && sb->lz_graph_key[i] == key) return (cudaGraphExec_t)sb->lz_graphs[i];
  // the products' panels must exist before the capture (building them allocates)
  if (prec == DMRG_TF32 || prec == DMRG_BF16X3) tc_prepare(sb, prec);
  cudaStream_t cs;
  CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  try {
    for (int k = 0; k < K; ++k) rf_enqueue_inner(sb, prec, cs);
  } catch (...) {
    cudaStreamEndCapture(cs, &g);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    throw;
  }
  CK(cudaStreamEndCapture(cs, &g));
  cudaGraphExec_t ge = nullptr;
  cudaError_t e = cudaGraphInstantiate(&ge, g, 0);
  cudaGraphDestroy(g);
  cudaStreamDestroy(cs);
  CK(e);
  int slot = -1;
  for (int i = 0; i < 8; ++i)
    if (!sb->lz_graphs[i]) { slot = i; break; }
  if (slot < 0) {
    slot = 7;
    cudaGraphExecDestroy((cudaGraphExec_t)sb->lz_graphs[slot]);
  }
  sb->lz_graphs[slot] = ge;
  sb->lz_graph_key[slot] = key;
  return ge;
}

// the smallest residual reduction factor one Newton step is counted on when
// predicting the last residual product (the mixed products' error bounds it)
constexpr double RF_STEP_FLOOR = 1.0 / 4000.0;

struct RfRun {
  std::vector<int32_t> code;  // LZ_CONVERGED or LZ_CAP
  std::vector<double> theta, resid;
  int outer = 0;              // float64 products spent
  std::vector<int32_t> inner; // mixed CG iterations per member (all outer steps)
  int64_t launches = 0;
  bool dots_final = false;    // dc holds the per-term dots of the returned psi
};

// Newton refinement of psi (device [batch][D], normalised) in place.  With
// dc != NULL the float64 residual products after the first also give the
// per-term dots <psi, (A_k x B_k) psi> (one pass, f64_pdot2/3); the last one is
// of the returned psi.
RfRun rf_solve(dmrg_sb* sb, double* psi, int prec, int rprec, double tol, int max_outer, int max_inner,
               double eps_in, int K, cudaStream_t st, double* dc = nullptr) {
  const int64_t D = sb->D;
  const int B = sb->batch, nch = sb->lz_nchunk;
  double* part = sb->lz_partial;
  double* tmp = sb->d_scratch;
  double* cur = sb->lz_vcur;
  CK(cudaMemcpyAsync(cur, psi, sizeof(double) * B * D, cudaMemcpyDeviceToDevice, st));
  RfRun r;
  r.code.assign(B, LZ_CAP);
  r.theta.assign(B, 0.0);
  r.resid.assign(B, 0.0);
  r.inner.assign(B, 0);
  std::vector<double> hsc(RF_NSC * B);
  std::vector<int32_t> hctl(2 * B + 2, 0), mask(B, 0);
  std::vector<uint8_t> conv(B, 0);
  const int Kg = std::max(1, K);
  rf_launch_diag(sb->d_dg, sb->d_dg_terms, (int)sb->dg_terms.size(), sb->d_coeffs, sb->n_terms, sb->rf_diag, D, B,
                 st);
  ++r.launches;
  // whether the next residual product is expected to be the last one (its
  // per-term dots are then the gradient of the returned psi); the first is
  // never the last in practice: the mixed solve stops far above the tolerance
  bool expect_last = false;
  for (int o = 0; o < max_outer; ++o) {
    const bool with_dots = dc && o >= 1 && (expect_last || o + 1 == max_outer);
    if (with_dots) matvec_f64_dots(sb, cur, sb->lz_w, dc, st, rprec == DMRG_DF64);
    else matvec(sb, rprec, cur, sb->lz_w, 0, nullptr, st);
    r.dots_final = with_dots;
    lz_launch_dot(cur, sb->lz_w, part, D, B, nch, st);
    lz_launch_sum_chunks(part, tmp, nch, B, st);
    rf_launch_set(sb->rf_sc, tmp, RF_THETA, B, 0, st);
    // preconditioner, right-hand side -r, first direction p = K (-r)
    rf_launch_minv(sb->rf_diag, sb->rf_sc, sb->rf_minv, D, B, st);
    rf_launch_start(sb->lz_w, cur, sb->rf_minv, sb->rf_res, sb->rf_t, sb->rf_psi32, sb->rf_sc, sb->rf_part, D, B,
                    st);
    rf_launch_sum4(sb->rf_part, sb->rf_sc, D, B, 1, nullptr, nullptr, st);
    rf_launch_rho0(sb->rf_sc, B, st);
    rf_launch_dir(sb->rf_p, sb->rf_res, sb->rf_psi32, sb->rf_minv, sb->rf_sc, nullptr, D, B, 1, nullptr, st);
    CK(cudaMemcpyAsync(hsc.data(), sb->rf_sc, sizeof(double) * RF_NSC * B, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    r.launches += 9 + (with_dots ? 4 : matvec_launches(sb, rprec));
    ++r.outer;
    bool all = true;
    for (int b = 0; b < B; ++b) {
      const double th = hsc[b * RF_NSC + RF_THETA], rn = hsc[b * RF_NSC + RF_BNORM];
      r.theta[b] = th;
      r.resid[b] = rn;
      conv[b] = rn <= tol * std::max(1.0, std::fabs(th));
      if (!std::isfinite(th) || !std::isfinite(rn)) throw Invalid{"refinement met a non-finite residual"};
      r.code[b] = conv[b] ? LZ_CONVERGED : LZ_CAP;
      all = all && conv[b];
    }
    if (all || o + 1 == max_outer) break;
    // mixed-precision CG on the correction equation
    for (int b = 0; b < B; ++b) {
      hctl[b] = conv[b] ? 1 : 0;
      hctl[B + b] = 0;
      mask[b] = conv[b] ? 0 : 1;
    }
    hctl[2 * B] = 0;
    hctl[2 * B + 1] = max_inner;
    // inner accuracy, within [1e-5, eps_in]: each outer step shrinks the
    // residual by about the inner solve's relative accuracy (until the mixed
    // product's own error bounds it), so from the mixed solve's result the
    // reduction still needed (tolerance / residual, with a factor 4 margin) is
    // split evenly over two outer steps (its square root), and a later step
    // asks for all of what remains
    double eps = eps_in;
    for (int b = 0; b < B; ++b) {
      if (conv[b]) continue;
      const double need = 0.25 * tol * std::max(1.0, std::fabs(r.theta[b])) / std::max(r.resid[b], 1e-300);
      eps = std::min(eps, std::max(o == 0 ? std::sqrt(need) : need, 1e-5));
    }
    // the step shrinks a residual by about eps, but by no more than the mixed
    // product's own error allows (about 1/4000 per step on the ladder): the
    // next residual is expected to be the last when that meets the tolerance
    // for every member still refining
    expect_last = true;
    for (int b = 0; b < B; ++b)
      if (!conv[b] && r.resid[b] * std::max(eps, RF_STEP_FLOOR) > tol * std::max(1.0, std::fabs(r.theta[b])))
        expect_last = false;
    CK(cudaMemcpyAsync(sb->rf_ctl, hctl.data(), sizeof(int32_t) * (2 * B + 2), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(sb->rf_sc + RF_NSC * B, &eps, sizeof(double), cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
    cudaGraphExec_t ge = rf_graph(sb, prec, Kg);
    int launched = 0;
    for (;;) {
      CK(cudaGraphLaunch(ge, st));
      launched += Kg;
      r.launches += (int64_t)Kg * (RF_KERNELS_PER_ITER + matvec_launches(sb, prec));
      int32_t stop = 0;
      CK(cudaMemcpyAsync(&stop, sb->rf_ctl + 2 * B, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      if (stop) break;
      if (launched > max_inner + Kg) throw Invalid{"refinement control did not terminate"};
    }
    CK(cudaMemcpyAsync(hctl.data(), sb->rf_ctl, sizeof(int32_t) * (2 * B + 2), cudaMemcpyDeviceToHost, st));
    int32_t* dmask = reinterpret_cast<int32_t*>(sb->rf_ctl);  // reuse: done flags no longer needed
    CK(cudaMemcpyAsync(dmask, mask.data(), sizeof(int32_t) * B, cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
    for (int b = 0; b < B; ++b) r.inner[b] += hctl[B + b];
    // psi <- (psi + t) / |psi + t|
    rf_launch_apply(cur, sb->rf_t, dmask, D, B, st);
    lz_launch_sumsq(cur, part, D, B, nch, st);
    lz_launch_sum_chunks(part, tmp, nch, B, st);
    lz_launch_scale_unit(cur, tmp, cur, nullptr, D, B, st);
    r.launches += 4;
  }
  CK(cudaMemcpyAsync(psi, cur, sizeof(double) * B * D, cudaMemcpyDeviceToDevice, st));
  CK(cudaStreamSynchronize(st));
  CK(cudaGetLastError());
  return r;
}

dmrg_status code_to_status(int code) {
  switch (code) {
    case LZ_CONVERGED: return DMRG_OK;
    case LZ_BREAKDOWN: return DMRG_EBREAKDOWN;
    case LZ_NAN: return DMRG_ENAN;
    case LZ_CAP: return DMRG_ENOCONV;
    default: return DMRG_ENOCONV;
  }
}

void validate_and_copy(dmrg_sb* sb, const dmrg_sb_desc* d, int32_t batch) {
  if (!d) throw Invalid{"null descriptor"};
  if (batch < 1) throw Invalid{"batch must be >= 1"};
  if (d->n_sectors < 0 || d->n_terms < 1 || d->n_pairs < 0) throw Invalid{"bad counts"};
  if (d->n_sectors > 0 && (!d->r || !d->c)) throw Invalid{"null sector dims"};
  if (!d->coeffs) throw Invalid{"null coeffs"};
  if (d->n_pairs > 0 && !d->pairs) throw Invalid{"null pair list"};
  sb->S = d->n_sectors;
  sb->n_terms = d->n_terms;
  sb->batch = batch;
  sb->r.assign(d->r, d->r + sb->S);
  sb->c.assign(d->c, d->c + sb->S);
  sb->off.assign(sb->S + 1, 0);
  for (int s = 0; s < sb->S; ++s) {
    if (sb->r[s] < 0 || sb->c[s] < 0) throw Invalid{"negative sector dimension"};
    sb->off[s + 1] = sb->off[s] + (int64_t)sb->r[s] * sb->c[s];
  }
  sb->D = sb->off[sb->S];
  if (sb->D == 0) throw Invalid{"empty target space (D = 0)"};
  sb->coeffs.assign(d->coeffs, d->coeffs + (size_t)batch * sb->n_terms);
  // pairs: validate, lay out the float64 arena (ld = number of columns)
  std::vector<const dmrg_pair*> keep;
  int64_t ops = 0;
  for (int i = 0; i < d->n_pairs; ++i) {
    const dmrg_pair& p = d->pairs[i];
    char buf[160];
    if (p.term < 0 || p.term >= sb->n_terms || p.s_out < 0 || p.s_out >= sb->S || p.s_in < 0 || p.s_in >= sb->S) {
      snprintf(buf, sizeof buf, "pair %d: term or sector out of range", i);
      throw Invalid{buf};
    }
    if ((p.flags & DMRG_ID_A) && (p.flags & DMRG_ID_B)) {
      snprintf(buf, sizeof buf, "pair %d: both sides identity", i);
      throw Invalid{buf};
    }
    const int64_t ro = sb->r[p.s_out], ri = sb->r[p.s_in], co = sb->c[p.s_out], ci = sb->c[p.s_in];
    if ((p.flags & DMRG_ID_A) && ro != ri) {
      snprintf(buf, sizeof buf, "pair %d: identity A needs r[s_out] == r[s_in]", i);
      throw Invalid{buf};
    }
    if ((p.flags & DMRG_ID_B) && co != ci) {
      snprintf(buf, sizeof buf, "pair %d: identity B needs c[s_out] == c[s_in]", i);
      throw Invalid{buf};
    }
    if (!(p.flags & DMRG_ID_A) && ro * ri > 0 && (!p.A || p.lda < ri)) {
      snprintf(buf, sizeof buf, "pair %d: A missing or lda < r[s_in]", i);
      throw Invalid{buf};
    }
    if (!(p.flags & DMRG_ID_B) && co * ci > 0 && (!p.B || p.ldb < ci)) {
      snprintf(buf, sizeof buf, "pair %d: B missing or ldb < c[s_in]", i);
      throw Invalid{buf};
    }
    if (ro * co == 0 || ri * ci == 0) continue;  // touches an empty sector: contributes nothing
    keep.push_back(&p);
    if (!(p.flags & DMRG_ID_A)) ops += ro * ri;
    if (!(p.flags & DMRG_ID_B)) ops += co * ci;
  }
  sb->ops_elems = ops;
  std::vector<double> host((size_t)std::max<int64_t>(ops, 1));
  int64_t pos = 0;
  sb->flops = 0;
  for (const dmrg_pair* pp : keep) {
    const dmrg_pair& p = *pp;
    PairH h{};
    h.term = p.term;
    h.s_out = p.s_out;
    h.s_in = p.s_in;
    h.flags = p.flags & (DMRG_ID_A | DMRG_ID_B);
    const int64_t ro = sb->r[p.s_out], ri = sb->r[p.s_in], co = sb->c[p.s_out], ci = sb->c[p.s_in];
    h.a_off = h.b_off = -1;
    auto copy_block = [&](const double* src, int64_t ld, int64_t rows, int64_t cols) {
      const int64_t at = pos;
      if (d->blocks_on_device) {
        CK(cudaMemcpy2D(host.data() + pos, cols * sizeof(double), src, ld * sizeof(double), cols * sizeof(double),
                        rows, cudaMemcpyDeviceToHost));
      } else {
        for (int64_t i = 0; i < rows; ++i) memcpy(host.data() + pos + i * cols, src + i * ld, cols * sizeof(double));
      }
      pos += rows * cols;
      return at;
    };
    if (!(h.flags & DMRG_ID_A)) h.a_off = copy_block(p.A, p.lda, ro, ri);
    if (!(h.flags & DMRG_ID_B)) h.b_off = copy_block(p.B, p.ldb, co, ci);
    if (h.flags & DMRG_ID_A) sb->flops += 2.0 * ro * ci * co;
    else if (h.flags & DMRG_ID_B) sb->flops += 2.0 * ro * ri * co;
    else {
      const double c0 = 2.0 * ro * ri * ci + 2.0 * ro * ci * co;  // (A Psi) B^T
      const double c1 = 2.0 * ri * ci * co + 2.0 * ro * ri * co;  // A (Psi B^T)
      h.order = c0 <= c1 ? 0 : 1;
      sb->flops += std::min(c0, c1);
    }
    sb->pairs.push_back(h);
  }
  sb->d_ops = dalloc<double>((size_t)std::max<int64_t>(ops, 1));
  if (ops) CK(cudaMemcpy(sb->d_ops, host.data(), ops * sizeof(double), cudaMemcpyHostToDevice));
  // diagonal of every term with diagonal blocks (s_out == s_in): the
  // refinement's preconditioner sums them with the member's coefficients
  {
    std::vector<int32_t> slot(sb->n_terms, -1);
    std::vector<double> dg;
    for (const PairH& h : sb->pairs) {
      if (h.s_out != h.s_in) continue;
      if (slot[h.term] < 0) {
        slot[h.term] = (int32_t)sb->dg_terms.size();
        sb->dg_terms.push_back(h.term);
        dg.resize(dg.size() + (size_t)sb->D, 0.0);
      }
      const int64_t r = sb->r[h.s_in], c = sb->c[h.s_in];
      double* out = dg.data() + (size_t)slot[h.term] * sb->D + sb->off[h.s_in];
      for (int64_t a = 0; a < r; ++a) {
        const double aa = (h.flags & DMRG_ID_A) ? 1.0 : host[h.a_off + a * r + a];
        for (int64_t bb = 0; bb < c; ++bb) {
          const double bv = (h.flags & DMRG_ID_B) ? 1.0 : host[h.b_off + bb * c + bb];
          out[a * c + bb] += aa * bv;
        }
      }
    }
    if (!sb->dg_terms.empty()) {
      upload(sb->d_dg, dg);
      upload(sb->d_dg_terms, sb->dg_terms);
    }
  }
  sb->h_ops = std::move(host);
  sb->d_tc_err = dalloc<int32_t>(1);
  CK(cudaMemset(sb->d_tc_err, 0, sizeof(int32_t)));
  upload(sb->d_coeffs, sb->coeffs);
  sb->d_scratch = dalloc<double>((size_t)(4 * batch + 16));
  sb->d_red = dalloc<double>((size_t)batch * lz_nchunk(sb->D));
}

void destroy(dmrg_sb* sb) {
  if (!sb) return;
  lz_free(sb);
  tc_free(sb);
  for (TaskListF64* tl : {&sb->f64_fwd1, &sb->f64_fwd2, &sb->f64_fwd3, &sb->f64_dot1, &sb->f64_dot2, &sb->f64_bwd1,
                          &sb->f64_bwd2, &sb->f64_bwd3, &sb->f64_pdot2, &sb->f64_pdot3})
    free_tl(*tl);
  for (double* p : {sb->d_coeffs, sb->d_ops, sb->d_T, sb->d_dot_partial, sb->d_scratch, sb->d_red, sb->d_dg,
                    sb->d_pdot_partial, sb->d_ops_df, sb->d_x_df})
    if (p) cudaFree(p);
  for (int32_t* p : {sb->d_pdot_ptr, sb->d_pdot_idx})
    if (p) cudaFree(p);
  if (sb->d_dg_terms) cudaFree(sb->d_dg_terms);
  if (sb->d_tc_err) cudaFree(sb->d_tc_err);
  if (sb->h_coeffs_pinned) cudaFreeHost(sb->h_coeffs_pinned);
  if (sb->d_dot_red_ptr) cudaFree(sb->d_dot_red_ptr);
  if (sb->d_dot_red_idx) cudaFree(sb->d_dot_red_idx);
  delete sb;
}

}  // namespace

// ================================================================ C ABI
extern "C" {

dmrg_status dmrg_create_superblock(const dmrg_sb_desc* d, int32_t batch, dmrg_sb** out) {
  if (!out) return DMRG_EINVAL;
  *out = nullptr;
  dmrg_sb* sb = new (std::nothrow) dmrg_sb();
  if (!sb) return DMRG_ENOMEM;
  const dmrg_status st = guard(sb, [&] {
    validate_and_copy(sb, d, batch);
    build_f64_tasks(sb);
    tc_build(sb);
    sb->h_ops.clear();
    sb->h_ops.shrink_to_fit();
    CK(cudaDeviceSynchronize());
    return DMRG_OK;
  });
  if (st != DMRG_OK) {
    static thread_local std::string last;
    last = sb->err;
    destroy(sb);
    fprintf(stderr, "dmrg_create_superblock: %s\n", last.c_str());
    return st;
  }
  *out = sb;
  return DMRG_OK;
}

void dmrg_destroy_superblock(dmrg_sb* sb) { destroy(sb); }

const char* dmrg_last_error(const dmrg_sb* sb) { return sb ? sb->err.c_str() : "null superblock"; }

dmrg_status dmrg_query(const dmrg_sb* sb, dmrg_sb_info* info) {
  if (!sb || !info) return DMRG_EINVAL;
  info->dim = sb->D;
  info->batch = sb->batch;
  info->n_sectors = sb->S;
  info->n_terms = sb->n_terms;
  info->n_pairs = (int32_t)sb->pairs.size();
  info->flops_per_matvec = sb->flops * sb->batch;
  info->op_bytes_f64 = (double)sb->ops_elems * 8.0;
  info->op_bytes_mixed = tc_operand_bytes(sb);
  return DMRG_OK;
}

dmrg_status dmrg_set_coeffs(dmrg_sb* sb, const double* coeffs, void* stream) {
  if (!sb || !coeffs) return DMRG_EINVAL;
  return guard(sb, [&] {
    cudaStream_t st = (cudaStream_t)stream;
    const size_t n = (size_t)sb->batch * sb->n_terms;
    sb->coeffs.assign(coeffs, coeffs + n);
    // through a pinned staging copy, ordered on the caller's stream after the
    // products already queued there (which read the old table); the stream is
    // synchronised so that the staging copy is free for the next call
    if (!sb->h_coeffs_pinned) {
      void* hp = nullptr;
      CK(cudaMallocHost(&hp, n * sizeof(double)));
      sb->h_coeffs_pinned = static_cast<double*>(hp);
    }
    memcpy(sb->h_coeffs_pinned, coeffs, n * sizeof(double));
    CK(cudaMemcpyAsync(sb->d_coeffs, sb->h_coeffs_pinned, n * sizeof(double), cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
    if (tc_set_coeffs(sb))  // tensor-core panels with folded coefficients were rebuilt
      for (int i = 0; i < 8; ++i)
        if (sb->lz_graphs[i]) {
          cudaGraphExecDestroy((cudaGraphExec_t)sb->lz_graphs[i]);
          sb->lz_graphs[i] = nullptr;
          sb->lz_graph_key[i] = 0;
        }
    return DMRG_OK;
  });
}

dmrg_status dmrg_apply_H(dmrg_sb* sb, const double* psi, double* y, int32_t accumulate, int32_t prec,
                         void* stream) {
  if (!sb) return DMRG_EINVAL;
  if (!psi || !y || psi == y) {
    sb->err = "apply_H: null or aliased psi / y";
    return DMRG_EINVAL;
  }
  if (prec < DMRG_FP64 || prec > DMRG_DF64) {
    sb->err = "apply_H: unknown precision";
    return DMRG_EINVAL;
  }
  if ((prec == DMRG_TF32 || prec == DMRG_BF16X3) && !tc_available(sb)) {
    sb->err = "apply_H: tensor-core path not available on this device";
    return DMRG_EUNSUPPORTED;
  }
  return guard(sb, [&] {
    matvec(sb, prec, psi, y, accumulate ? 1 : 0, nullptr, (cudaStream_t)stream);
    return DMRG_OK;
  });
}

dmrg_status dmrg_apply_H_backward(dmrg_sb* sb, const double* psi, const double* g, double* dpsi, double* dc,
                                  int32_t prec, void* stream) {
  if (!sb) return DMRG_EINVAL;
  if (!g || (dc && !psi) || (dpsi && dpsi == g)) {
    sb->err = "apply_H_backward: bad pointers";
    return DMRG_EINVAL;
  }
  if (prec < DMRG_FP64 || prec > DMRG_BF16X3) return DMRG_EINVAL;
  return guard(sb, [&] {
    cudaStream_t st = (cudaStream_t)stream;
    if (dpsi) {
      if (prec == DMRG_FP64 || !tc_available(sb)) {
        Bufs bufs{{const_cast<double*>(g), dpsi, sb->d_T, sb->d_ops, nullptr}};
        launch_seg_gemm_f64(sb->f64_bwd1, bufs, sb->d_coeffs, sb->n_terms, 0, nullptr, nullptr, st);
        launch_seg_gemm_f64(sb->f64_bwd2, bufs, sb->d_coeffs, sb->n_terms, 0, nullptr, nullptr, st);
        launch_seg_gemm_f64(sb->f64_bwd3, bufs, sb->d_coeffs, sb->n_terms, 0, nullptr, nullptr, st);
      } else {
        tc_matvec_T(sb, prec, g, dpsi, st);
      }
    }
    if (dc) term_dots(sb, psi, g, dc, st);
    CK(cudaGetLastError());
    return DMRG_OK;
  });
}

dmrg_status dmrg_autotune(dmrg_sb* sb, int32_t prec, int32_t reps, void* stream, dmrg_tune_info* info) {
  if (!sb || (prec != DMRG_TF32 && prec != DMRG_BF16X3)) return DMRG_EINVAL;
  if (!tc_available(sb)) {
    sb->err = "autotune: tensor-core path not available on this device";
    return DMRG_EUNSUPPORTED;
  }
  return guard(sb, [&] {
    double out[7] = {};
    tc_autotune(sb, prec, reps, (cudaStream_t)stream, out);
    // captured graphs hold the old task lists
    for (int i = 0; i < 8; ++i)
      if (sb->lz_graphs[i]) {
        cudaGraphExecDestroy((cudaGraphExec_t)sb->lz_graphs[i]);
        sb->lz_graphs[i] = nullptr;
        sb->lz_graph_key[i] = 0;
      }
    if (info) {
      info->best_ms = out[0];
      info->default_ms = out[1];
      info->per_block_ms = out[2];
      info->best_tile_n = (int32_t)out[3];
      info->heavy_first = (int32_t)out[4];
      info->candidates = (int32_t)out[5];
      info->pieces = (int32_t)out[6];
    }
    return DMRG_OK;
  });
}

dmrg_status dmrg_sync_status(dmrg_sb* sb, void* stream) {
  if (!sb) return DMRG_EINVAL;
  return guard(sb, [&] {
    cudaStream_t st = (cudaStream_t)stream;
    int32_t flag = 0;
    CK(cudaMemcpyAsync(&flag, sb->d_tc_err, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (flag) {
      CK(cudaMemsetAsync(sb->d_tc_err, 0, sizeof(int32_t), st));
      CK(cudaStreamSynchronize(st));
      sb->err = "a tensor-core kernel gave up a bounded wait; its output was not written";
      return DMRG_ETIMEOUT;
    }
    return DMRG_OK;
  });
}

dmrg_status dmrg_test_inject(dmrg_sb* sb, int32_t what) {
  if (!sb || what < 0 || what > 2) return DMRG_EINVAL;
  if (what == 2) {
    sb->test_force_pending = 1;
    return DMRG_OK;
  }
  sb->test_stall = what;
  sb->test_force_pending = 0;
  return DMRG_OK;
}

dmrg_status dmrg_energy_grad(dmrg_sb* sb, const double* psi, double* dE_dc, int32_t prec, void* stream) {
  if (!sb || !psi || !dE_dc) return DMRG_EINVAL;
  (void)prec;
  return guard(sb, [&] {
    cudaStream_t st = (cudaStream_t)stream;
    term_dots(sb, psi, psi, dE_dc, st);
    const int nch = lz_nchunk(sb->D);
    lz_launch_sumsq(psi, sb->d_red, sb->D, sb->batch, nch, st);
    lz_launch_sum_chunks(sb->d_red, sb->d_scratch, nch, sb->batch, st);
    lz_launch_div_rows(dE_dc, sb->d_scratch, sb->n_terms, sb->batch, st);
    CK(cudaGetLastError());
    return DMRG_OK;
  });
}

static dmrg_status lanczos_impl(dmrg_sb* sb, const double* psi0, double* psi_out, double* e0, double* dE_dc,
                                const dmrg_lanczos_opts* opts, dmrg_lanczos_info* info, void* stream) {
  if (!sb || !psi0 || !psi_out || !e0 || !opts) return DMRG_EINVAL;
  if (opts->prec < DMRG_FP64 || opts->prec > DMRG_BF16X3 || !(opts->tol > 0) || opts->max_iter < 1 ||
      opts->refine < 0 || opts->refine > 3) {
    sb->err = "lanczos: bad options";
    return DMRG_EINVAL;
  }
  if (opts->prec != DMRG_FP64 && !tc_available(sb)) {
    sb->err = "lanczos: tensor-core path not available on this device";
    return DMRG_EUNSUPPORTED;
  }
  return guard(sb, [&] {
    cudaStream_t st = (cudaStream_t)stream;
    const int B = sb->batch;
    const int ge = std::max(1, opts->graph_iters);
    LzRun r = lz_solve(sb, psi0, psi_out, opts->prec, opts->tol, opts->max_iter, opts->check_every, ge, st);
    const double rtol = opts->refine_tol > 0 ? opts->refine_tol : 1e-10;
    const int mode = opts->prec == DMRG_FP64 ? 0 : opts->refine;
    LzRun rr;   // mode 1: float64 Lanczos restarted from the mixed result
    RfRun rn;   // mode 2: Newton steps, float64 residual + mixed CG correction
    if (mode == 1)
      rr = lz_solve(sb, psi_out, psi_out, DMRG_FP64, rtol, opts->max_iter, opts->check_every, ge, st);
    else if (mode >= 2)
      rn = rf_solve(sb, psi_out, opts->prec, mode == 3 ? DMRG_DF64 : DMRG_FP64, rtol, 8, 400, 1e-2, ge, st, dE_dc);
    int64_t grad_launches = 0;
    if (dE_dc) {
      // Hellmann-Feynman: dots of the returned psi / <psi, psi>, from the
      // refinement's last float64 product when it carried them
      if (!(mode >= 2 && rn.dots_final)) {
        term_dots(sb, psi_out, psi_out, dE_dc, st);
        grad_launches += 3;
      }
      const int nch = lz_nchunk(sb->D);
      lz_launch_sumsq(psi_out, sb->d_red, sb->D, B, nch, st);
      lz_launch_sum_chunks(sb->d_red, sb->d_scratch, nch, B, st);
      lz_launch_div_rows(dE_dc, sb->d_scratch, sb->n_terms, B, st);
      CK(cudaGetLastError());
      grad_launches += 3;
    }
    dmrg_status worst = DMRG_OK;
    for (int b = 0; b < B; ++b) {
      int code = r.code[b];
      double th = r.theta[b], res = r.resid[b];
      if (mode == 1) { code = rr.code[b]; th = rr.theta[b]; res = rr.resid[b]; }
      if (mode >= 2) { code = rn.code[b]; th = rn.theta[b]; res = rn.resid[b]; }
      dmrg_status s = code_to_status(code);
      const dmrg_status report = s == DMRG_EBREAKDOWN ? DMRG_OK : s;
      if (report != DMRG_OK && worst == DMRG_OK) worst = report;
      e0[b] = th;
      if (info) {
        info[b].e0 = th;
        info[b].residual = res;
        info[b].iters = r.iters[b];
        info[b].refine_iters = mode == 1 ? rr.iters[b] : (mode >= 2 ? rn.outer : 0);
        const int mixed_lz = opts->prec != DMRG_FP64 ? r.iters[b] : 0;
        info[b].mixed_matvecs = mixed_lz + (mode >= 2 ? rn.inner[b] : 0);
        info[b].fp64_matvecs = opts->prec == DMRG_FP64 ? r.iters[b] : (mode == 1 ? rr.iters[b] : (mode >= 2 ? rn.outer : 0));
        info[b].status = s;
        info[b].breakdown = code == LZ_BREAKDOWN;
        info[b].kernel_launches = (int32_t)(r.launches + (mode == 1 ? rr.launches : 0) + (mode >= 2 ? rn.launches : 0) +
                                            grad_launches);
        info[b].restarts = r.restarts[b] + (mode == 1 ? rr.restarts[b] : 0);
      }
    }
    return worst;
  });
}

dmrg_status dmrg_lanczos_ground(dmrg_sb* sb, const double* psi0, double* psi_out, double* e0,
                                const dmrg_lanczos_opts* opts, dmrg_lanczos_info* info, void* stream) {
  return lanczos_impl(sb, psi0, psi_out, e0, nullptr, opts, info, stream);
}

dmrg_status dmrg_lanczos_ground_grad(dmrg_sb* sb, const double* psi0, double* psi_out, double* e0, double* dE_dc,
                                     const dmrg_lanczos_opts* opts, dmrg_lanczos_info* info, void* stream) {
  if (!dE_dc) return DMRG_EINVAL;
  return lanczos_impl(sb, psi0, psi_out, e0, dE_dc, opts, info, stream);
}

dmrg_status dmrg_apply_H_term_dots(dmrg_sb* sb, const double* psi, double* y, double* dots, int32_t prec,
                                   void* stream) {
  if (!sb) return DMRG_EINVAL;
  if (!psi || !y || !dots || psi == y) {
    sb->err = "apply_H_term_dots: null or aliased psi / y / dots";
    return DMRG_EINVAL;
  }
  if (prec != DMRG_FP64 && prec != DMRG_DF64) {
    sb->err = "apply_H_term_dots: precision must be DMRG_FP64 or DMRG_DF64";
    return DMRG_EINVAL;
  }
  return guard(sb, [&] {
    matvec_f64_dots(sb, psi, y, dots, (cudaStream_t)stream, prec == DMRG_DF64);
    return DMRG_OK;
  });
}

dmrg_status dmrg_lanczos_coeffs(dmrg_sb* sb, const double* phi0, int32_t n_max, int32_t prec, double* alpha,
                                double* beta, double* norm2, int32_t* n_out, void* stream) {
  if (!sb) return DMRG_EINVAL;
  if (!phi0 || !alpha || !beta || !norm2 || !n_out || n_max < 1 || prec < DMRG_FP64 || prec > DMRG_BF16X3) {
    sb->err = "lanczos_coeffs: bad pointers, n_max or precision";
    return DMRG_EINVAL;
  }
  if (prec != DMRG_FP64 && !tc_available(sb)) {
    sb->err = "lanczos_coeffs: tensor-core path not available on this device";
    return DMRG_EUNSUPPORTED;
  }
  return guard(sb, [&] {
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t D = sb->D;
    const int B = sb->batch;
    const int nmax = (int)std::min<int64_t>(std::min(n_max, 768), D);
    lz_alloc(sb, nmax + 1);
    lz_launch_sumsq(phi0, sb->lz_partial, D, B, sb->lz_nchunk, st);  // |phi0|^2 before it is normalised
    lz_launch_sum_chunks(sb->lz_partial, norm2, sb->lz_nchunk, B, st);
    // no convergence test (tolerance 0, tridiagonal check only at the cap or an
    // invariant subspace); the Ritz vector goes to scratch
    LzRun r = lz_solve(sb, phi0, sb->rf_q, prec, 0.0, nmax, nmax + 1, 8, st);
    const int cap = sb->lz_cap;
    CK(cudaMemcpy2DAsync(alpha, sizeof(double) * (size_t)n_max, sb->lz_ab, sizeof(double) * (size_t)cap,
                         sizeof(double) * (size_t)nmax, (size_t)B, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpy2DAsync(beta, sizeof(double) * (size_t)n_max, sb->lz_ab + (size_t)B * cap,
                         sizeof(double) * (size_t)cap, sizeof(double) * (size_t)nmax, (size_t)B,
                         cudaMemcpyDeviceToDevice, st));
    std::vector<double> hn2((size_t)B);
    CK(cudaMemcpyAsync(hn2.data(), norm2, sizeof(double) * B, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    dmrg_status s = DMRG_OK;
    for (int b = 0; b < B; ++b) {
      n_out[b] = r.iters[b];
      if (hn2[b] == 0.0) n_out[b] = 0;  // phi0 = 0 (e.g. c on an empty site): no coefficients, G = 0
      else if (r.code[b] == LZ_NAN) s = DMRG_ENAN;
    }
    return s;
  });
}

dmrg_status dmrg_time_reorth(dmrg_sb* sb, int32_t prec, int32_t j, int32_t reps, double* ms, double* bytes,
                             void* stream) {
  if (!sb || !ms || !bytes || prec < DMRG_FP64 || prec > DMRG_BF16X3 || j < 0 || j > 767 || reps < 1) {
    if (sb) sb->err = "time_reorth: bad arguments";
    return DMRG_EINVAL;
  }
  return guard(sb, [&] {
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t D = sb->D;
    const int B = sb->batch;
    lz_alloc(sb, j + 1);
    const int cap = sb->lz_cap, nch = sb->lz_nchunk;
    const bool pair = lz_pair(prec);
    // every member running at Krylov index j; the basis rows and w hold whatever
    // the last solve left (the timing does not depend on the values)
    std::vector<int32_t> hc(LZ_CTL_MEMBER + 2 * B, 0);
    hc[LZ_CTL_J] = j;
    hc[LZ_CTL_MAXIT] = cap;
    hc[LZ_CTL_CHECK] = 1;
    CK(cudaMemcpyAsync(sb->lz_ctl, hc.data(), hc.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(sb->lz_w, 0, sizeof(double) * (size_t)B * D, st));
    double* hB = sb->lz_h + (size_t)B * cap;
    double* nB = sb->lz_npart + (size_t)B * nch;
    auto pass = [&] {
      lz_launch_multidot(sb->lz_V, sb->lz_w, sb->lz_partial, sb->lz_ctl, D, B, cap, 0, nullptr, st, nullptr, nullptr,
                         pair);
      lz_launch_reduce_rows(sb->lz_partial, hB, sb->lz_ctl, lz_dot_nparts(D), cap, B, 0, nullptr, st);
      lz_launch_multiaxpy(sb->lz_V, sb->lz_w, hB, nB, sb->lz_ctl, D, B, cap, nch, 0, nullptr, st, pair);
    };
    pass();
    cudaEvent_t a, b;
    CK(cudaEventCreate(&a));
    CK(cudaEventCreate(&b));
    CK(cudaEventRecord(a, st));
    for (int r = 0; r < reps; ++r) pass();
    CK(cudaEventRecord(b, st));
    CK(cudaEventSynchronize(b));
    float t = 0.0f;
    CK(cudaEventElapsedTime(&t, a, b));
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    CK(cudaGetLastError());
    *ms = (double)t / reps;
    // the dots read rows 0..j and w; the update reads rows 0..j, reads and writes w
    *bytes = (2.0 * (j + 1) + 3.0) * (double)D * B * 8.0;
    return DMRG_OK;
  });
}

dmrg_status dmrg_continued_fraction(const double* norm2, const double* alpha, const double* beta, const int32_t* n,
                                    int32_t batch, int32_t ld, const double* z_re, const double* z_im, int32_t n_z,
                                    double* g_re, double* g_im, void* stream) {
  if (!norm2 || !alpha || !beta || !n || !z_re || !z_im || !g_re || !g_im || batch < 0 || ld < 1 || n_z < 0)
    return DMRG_EINVAL;
  lz_launch_cfrac(norm2, alpha, beta, n, ld, z_re, z_im, n_z, g_re, g_im, batch, (cudaStream_t)stream);
  return cudaGetLastError() == cudaSuccess ? DMRG_OK : DMRG_ECUDA;
}

}  // extern "C"
