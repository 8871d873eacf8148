// The DMRG driver around the superblock product (paper Sec. 3.1, Fig.
// infiniteloop; Sec. 3.2-3.3 for the bases and the block operators): block
// growth, superblock assembly, the Lanczos ground state, the reduced density
// matrices, truncation and the change of basis, all on the device; the host
// keeps only the sector bookkeeping (quantum numbers, dimensions, which block
// goes where).
//
// Blocks are sector-blocked: a block basis is a list of symmetry sectors
// (effective quantum number q, fermion parity, dimension) in increasing q,
// and an operator is a list of dense row-major blocks (out sector, in sector)
// in one device arena per block.  Growth re-expresses every operator in the
// product basis block (x) site (left block) or site (x) block (right block):
// a product sector is the concatenation of components (block sector z, site
// state t) -- for the left block in the order of z, then t; for the right
// block in the order of t, then z; each order is that of the Kronecker
// index sorted stably by q, as in the paper's outer product followed by the
// symmetry ordering.  Every block of a Kronecker product of a block operator
// and a site matrix is then a scaled (possibly transposed) copy of a block
// operator's block into a sub-rectangle of a product block: one scatter job.

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <memory>
#include <new>
#include <stdexcept>
#include <string>
#include <tuple>
#include <vector>

#include "blockops.h"
#include "dmrg_sys.h"
#include "internal.h"

namespace {

using namespace dmrg;

#define SYS_CK(x)                                                                                 \
  do {                                                                                            \
    cudaError_t e_ = (x);                                                                         \
    if (e_ != cudaSuccess) throw std::runtime_error(std::string(#x) + ": " + cudaGetErrorString(e_)); \
  } while (0)

struct Bad {
  std::string msg;
};

// owned device array of doubles
struct DBuf {
  double* p = nullptr;
  size_t n = 0;
  explicit DBuf(size_t n_) {
    n = std::max<size_t>(n_, 1);
    SYS_CK(cudaMalloc(&p, n * sizeof(double)));
  }
  ~DBuf() {
    if (p) cudaFree(p);
  }
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
};
using DBufP = std::shared_ptr<DBuf>;

template <class T>
struct DArr {  // owned device array of a plain type
  T* p = nullptr;
  explicit DArr(size_t n) { SYS_CK(cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T))); }
  ~DArr() {
    if (p) cudaFree(p);
  }
  DArr(const DArr&) = delete;
  DArr& operator=(const DArr&) = delete;
};

struct Basis {
  std::vector<int64_t> q;
  std::vector<int32_t> par, dim;
  int size() const { return (int)q.size(); }
  int find(int64_t qq) const {
    auto it = std::lower_bound(q.begin(), q.end(), qq);
    return (it != q.end() && *it == qq) ? (int)(it - q.begin()) : -1;
  }
};

struct OpB {
  int32_t so, si;
  int64_t off;
};
struct Op {
  std::vector<OpB> b;
};

struct Comp {
  int32_t z, t, off;  // parent sector, site state, row offset inside the product sector
};

// how a truncated block came from its grown parent: the grown basis, its
// components, and the kept eigenvectors W[z] = V_z[:, 0:k[z]] (row-major
// n_z x n_z at V + voff[z])
struct Trunc {
  Basis grown;
  std::vector<std::vector<Comp>> comps;
  bool left = true;
  DBufP V;
  std::vector<int64_t> voff;
  std::vector<int32_t> k, newsec;
};

struct Blk {
  int n = 0;
  Basis bs;
  std::vector<Op> H;                      // per coupling class (unit coupling)
  std::map<std::pair<int, int>, Op> ops;  // (end distance, site operator) -> operator
  DBufP arena;
  // grown blocks: components of each sector and where (z, t) went
  std::vector<std::vector<Comp>> comps;
  std::map<std::pair<int, int>, std::pair<int, int>> where;
  bool left = true;
  std::shared_ptr<Trunc> trunc;  // truncated blocks: how they were made
  const double* ptr(const OpB& x) const { return arena->p + x.off; }
};
using BlkP = std::shared_ptr<Blk>;

// ------------------------------------------------------------------ model
struct Model {
  int d = 0;
  std::vector<int64_t> sq;
  std::vector<int32_t> spar;
  int n_ops = 0;
  std::vector<double> ops;
  std::vector<int32_t> ferm;
  int n_classes = 0;
  std::vector<double> g;
  std::vector<int32_t> on_cls;
  std::vector<double> on;
  struct Rule {
    int delta, cls, mod, rem;
  };
  std::vector<Rule> rules;
  std::vector<dmrg_bond_term> terms;
  double density = 1.0;
  int64_t Q = 0;
  int reach = 1;

  std::vector<double> mat(int o, int trans) const {
    std::vector<double> m((size_t)d * d);
    for (int a = 0; a < d; ++a)
      for (int b = 0; b < d; ++b) m[a * d + b] = trans ? ops[((size_t)o * d + b) * d + a] : ops[((size_t)o * d + a) * d + b];
    return m;
  }
  std::vector<double> eye() const {
    std::vector<double> m((size_t)d * d, 0.0);
    for (int a = 0; a < d; ++a) m[a * d + a] = 1.0;
    return m;
  }
  std::vector<double> F() const {
    std::vector<double> m((size_t)d * d, 0.0);
    for (int a = 0; a < d; ++a) m[a * d + a] = spar[a] ? -1.0 : 1.0;
    return m;
  }
  std::vector<double> times_F(std::vector<double> m) const {  // m F (columns scaled by parity)
    for (int a = 0; a < d; ++a)
      for (int b = 0; b < d; ++b)
        if (spar[b]) m[a * d + b] = -m[a * d + b];
    return m;
  }
  // bonds (p, p + delta, class) of a lattice of L sites
  std::vector<std::tuple<int, int, int>> bonds(int L) const {
    std::vector<std::tuple<int, int, int>> out;
    for (int p = 0; p < L; ++p)
      for (const Rule& r : rules)
        if (p % r.mod == r.rem && p + r.delta < L) out.emplace_back(p, p + r.delta, r.cls);
    return out;
  }
  int64_t target(int L) const {
    int64_t N = llround(density * L);
    N -= N % 2;
    return N / 2 + Q * (N / 2);
  }
  bool fermionic(const dmrg_bond_term& t) const { return ferm[t.op_a] != 0; }
};

Model make_model(const dmrg_model_desc* m) {
  if (!m) throw Bad{"null model"};
  Model M;
  if (m->d < 1 || !m->site_q || !m->site_parity) throw Bad{"model: bad site basis"};
  M.d = m->d;
  M.sq.assign(m->site_q, m->site_q + m->d);
  M.spar.assign(m->site_parity, m->site_parity + m->d);
  for (int a = 0; a < M.d; ++a)
    for (int b = a + 1; b < M.d; ++b)
      if (M.sq[a] == M.sq[b]) throw Bad{"model: site states must have distinct quantum numbers"};
  if (m->n_ops < 1 || !m->ops || !m->op_fermion) throw Bad{"model: no site operators"};
  M.n_ops = m->n_ops;
  M.ops.assign(m->ops, m->ops + (size_t)m->n_ops * m->d * m->d);
  M.ferm.assign(m->op_fermion, m->op_fermion + m->n_ops);
  if (m->n_classes < 1 || !m->couplings) throw Bad{"model: no coupling classes"};
  M.n_classes = m->n_classes;
  M.g.assign(m->couplings, m->couplings + m->n_classes);
  if (m->n_onsite < 0 || (m->n_onsite > 0 && (!m->onsite || !m->onsite_class))) throw Bad{"model: bad on-site terms"};
  M.on_cls.assign(m->onsite_class, m->onsite_class + m->n_onsite);
  M.on.assign(m->onsite, m->onsite + (size_t)m->n_onsite * m->d * m->d);
  for (int c : M.on_cls)
    if (c < 0 || c >= M.n_classes) throw Bad{"model: on-site class out of range"};
  if (m->n_bond_rules < 0 || (m->n_bond_rules > 0 && !m->bond_rules)) throw Bad{"model: bad bond rules"};
  M.reach = 1;
  for (int i = 0; i < m->n_bond_rules; ++i) {
    const int32_t* r = m->bond_rules + 4 * i;
    if (r[0] < 1 || r[1] < 0 || r[1] >= M.n_classes || r[2] < 1 || r[3] < 0 || r[3] >= r[2])
      throw Bad{"model: bond rule out of range"};
    M.rules.push_back({r[0], r[1], r[2], r[3]});
    M.reach = std::max(M.reach, (int)r[0]);
  }
  if (m->n_bond_terms < 0 || (m->n_bond_terms > 0 && !m->bond_terms)) throw Bad{"model: bad bond terms"};
  M.terms.assign(m->bond_terms, m->bond_terms + m->n_bond_terms);
  for (const dmrg_bond_term& t : M.terms) {
    if (t.op_a < 0 || t.op_a >= M.n_ops || t.op_b < 0 || t.op_b >= M.n_ops) throw Bad{"model: bond term operator"};
    if (M.ferm[t.op_a] != M.ferm[t.op_b]) throw Bad{"model: a bond term mixes fermionic and bosonic operators"};
  }
  if (!(m->density > 0)) throw Bad{"model: density must be positive"};
  M.density = m->density;
  M.Q = m->Q;
  return M;
}

// ------------------------------------------------------------ Kronecker jobs
// One term of a product-basis operator: (block part) (x) (site part).  The
// block part is the block operator X (transposed when tX, times the block
// parity F on the right when fcol), the identity, or F; the site part is a
// d x d matrix.
enum BlockPart { BP_OP = 0, BP_ID = 1, BP_F = 2 };
struct KTerm {
  int part = BP_OP;
  const Op* X = nullptr;
  int tX = 0;
  bool fcol = false;
  std::vector<double> y;
  double scale = 1.0;
};

struct PartBlock {  // one block of the block part: (zo, zi), its source and factor
  int zo, zi;
  const double* src;
  int ld_src, trans;
  double f;
};

std::vector<PartBlock> part_blocks(const Blk& S, const KTerm& k) {
  std::vector<PartBlock> out;
  const Basis& b = S.bs;
  if (k.part == BP_OP) {
    for (const OpB& x : k.X->b) {
      PartBlock p;
      if (k.tX) {
        p.zo = x.si;
        p.zi = x.so;
      } else {
        p.zo = x.so;
        p.zi = x.si;
      }
      p.src = S.ptr(x);
      p.ld_src = b.dim[x.si];
      p.trans = k.tX;
      p.f = (k.fcol && b.par[p.zi]) ? -1.0 : 1.0;
      out.push_back(p);
    }
  } else {
    for (int z = 0; z < b.size(); ++z)
      out.push_back({z, z, nullptr, 0, 0, (k.part == BP_F && b.par[z]) ? -1.0 : 1.0});
  }
  return out;
}

// ------------------------------------------------------------------ growth
// S' = S (x) site (left) or E' = site (x) S (right), n + 1 sites.
BlkP grow(const Model& M, const Blk& S, bool left, cudaStream_t st) {
  auto G = std::make_shared<Blk>();
  G->n = S.n + 1;
  G->left = left;
  const int d = M.d;
  // product basis
  std::vector<std::tuple<int64_t, int, int>> cand;  // (q, z, t) in Kronecker order
  if (left) {
    for (int z = 0; z < S.bs.size(); ++z)
      for (int t = 0; t < d; ++t) cand.emplace_back(S.bs.q[z] + M.sq[t], z, t);
  } else {
    for (int t = 0; t < d; ++t)
      for (int z = 0; z < S.bs.size(); ++z) cand.emplace_back(S.bs.q[z] + M.sq[t], z, t);
  }
  std::vector<int64_t> qs;
  for (auto& c : cand) qs.push_back(std::get<0>(c));
  std::sort(qs.begin(), qs.end());
  qs.erase(std::unique(qs.begin(), qs.end()), qs.end());
  G->bs.q = qs;
  G->bs.dim.assign(qs.size(), 0);
  G->bs.par.assign(qs.size(), -1);
  G->comps.resize(qs.size());
  for (auto& c : cand) {
    const int s = G->bs.find(std::get<0>(c));
    const int z = std::get<1>(c), t = std::get<2>(c);
    const int par = S.bs.par[z] ^ M.spar[t];
    if (G->bs.par[s] < 0) G->bs.par[s] = par;
    else if (G->bs.par[s] != par) throw Bad{"a symmetry sector mixes fermion parities: q must fix the parity"};
    G->comps[s].push_back({z, t, G->bs.dim[s]});
    G->where[{z, t}] = {s, G->bs.dim[s]};
    G->bs.dim[s] += S.bs.dim[z];
  }

  // the operators of the grown block as sums of Kronecker terms
  struct OutOp {
    int kind;  // 0: H class, 1: site operator
    int cls;
    std::pair<int, int> key;
    std::vector<KTerm> terms;
  };
  std::vector<OutOp> outs;
  const std::vector<double> I = M.eye(), Fs = M.F();
  const int nw = S.n;  // end distance of the new site
  for (int c = 0; c < M.n_classes; ++c) {
    OutOp o{0, c, {0, 0}, {}};
    KTerm kt;
    kt.part = BP_OP;
    kt.X = &S.H[c];
    kt.y = I;
    o.terms.push_back(kt);
    for (size_t k = 0; k < M.on_cls.size(); ++k)
      if (M.on_cls[k] == c) {
        KTerm ko;
        ko.part = BP_ID;
        ko.y.assign(M.on.begin() + k * d * d, M.on.begin() + (k + 1) * d * d);
        o.terms.push_back(ko);
      }
    // bonds between the new site and the block's sites (left-anchored lattice
    // of n + 1 sites; the geometry is mirror symmetric, so it also serves the
    // right block in end-distance labels)
    for (auto& bd : M.bonds(G->n)) {
      const int i = std::get<0>(bd), j = std::get<1>(bd), cls = std::get<2>(bd);
      if (j != nw || cls != c) continue;
      for (const dmrg_bond_term& tm : M.terms) {
        const bool fer = M.fermionic(tm);
        KTerm kb;
        kb.part = BP_OP;
        kb.scale = tm.coef;
        if (left) {  // old site i < new site: kron(X_i(a)^{ta} F_S, y_b^{tb})
          auto it = S.ops.find({i, tm.op_a});
          if (it == S.ops.end()) throw Bad{"growth: a bonded site's operator was not kept"};
          kb.X = &it->second;
          kb.tX = tm.trans_a;
          kb.fcol = fer;
          kb.y = M.mat(tm.op_b, tm.trans_b);
        } else {  // new site (lowest label) < old site: kron(y_a^{ta} F_s, X_i(b)^{tb})
          auto it = S.ops.find({i, tm.op_b});
          if (it == S.ops.end()) throw Bad{"growth: a bonded site's operator was not kept"};
          kb.X = &it->second;
          kb.tX = tm.trans_b;
          kb.y = M.mat(tm.op_a, tm.trans_a);
          if (fer) kb.y = M.times_F(kb.y);
        }
        o.terms.push_back(kb);
      }
    }
    outs.push_back(std::move(o));
  }
  for (auto& kv : S.ops) {  // old site operators in the product basis
    OutOp o{1, 0, kv.first, {}};
    KTerm kt;
    kt.part = BP_OP;
    kt.X = &kv.second;
    kt.y = (!left && M.ferm[kv.first.second]) ? Fs : I;  // right: the new site precedes them
    o.terms.push_back(kt);
    outs.push_back(std::move(o));
  }
  for (int op = 0; op < M.n_ops; ++op) {  // the new site's operators
    OutOp o{1, 0, {nw, op}, {}};
    KTerm kt;
    kt.part = (left && M.ferm[op]) ? BP_F : BP_ID;  // left: the block precedes the new site
    kt.y = M.mat(op, 0);
    o.terms.push_back(kt);
    outs.push_back(std::move(o));
  }

  // layout: the destination blocks of every output operator
  std::vector<std::map<std::pair<int, int>, int64_t>> lay(outs.size());
  int64_t total = 0;
  for (size_t oi = 0; oi < outs.size(); ++oi) {
    for (const KTerm& kt : outs[oi].terms)
      for (const PartBlock& pb : part_blocks(S, kt))
        for (int to = 0; to < d; ++to)
          for (int ti = 0; ti < d; ++ti) {
            if (kt.y[to * d + ti] == 0.0) continue;
            const int so = G->where.at({pb.zo, to}).first, si = G->where.at({pb.zi, ti}).first;
            lay[oi].emplace(std::make_pair(so, si), -1);
          }
    for (auto& kv : lay[oi]) {
      kv.second = total;
      total += (int64_t)G->bs.dim[kv.first.first] * G->bs.dim[kv.first.second];
    }
  }
  G->arena = std::make_shared<DBuf>((size_t)total);
  SYS_CK(cudaMemsetAsync(G->arena->p, 0, std::max<int64_t>(total, 1) * sizeof(double), st));
  for (size_t oi = 0; oi < outs.size(); ++oi) {
    Op op;
    for (auto& kv : lay[oi]) op.b.push_back({kv.first.first, kv.first.second, kv.second});
    for (const KTerm& kt : outs[oi].terms) {
      std::vector<ScatJob> jobs;
      for (const PartBlock& pb : part_blocks(S, kt))
        for (int to = 0; to < d; ++to)
          for (int ti = 0; ti < d; ++ti) {
            const double yv = kt.y[to * d + ti];
            if (yv == 0.0) continue;
            const auto wo = G->where.at({pb.zo, to}), wi = G->where.at({pb.zi, ti});
            const int64_t boff = lay[oi].at({wo.first, wi.first});
            const int ldd = G->bs.dim[wi.first];
            ScatJob j{};
            j.src = pb.src;
            j.dst = G->arena->p + boff + (int64_t)wo.second * ldd + wi.second;
            j.rows = S.bs.dim[pb.zo];
            j.cols = S.bs.dim[pb.zi];
            j.ld_src = pb.ld_src;
            j.ld_dst = ldd;
            j.trans = pb.trans;
            j.scale = kt.scale * yv * pb.f;
            jobs.push_back(j);
          }
      launch_scatter(jobs, st);
    }
    if (outs[oi].kind == 0) {
      if ((int)G->H.size() <= outs[oi].cls) G->H.resize(outs[oi].cls + 1);
      G->H[outs[oi].cls] = std::move(op);
    } else {
      G->ops[outs[oi].key] = std::move(op);
    }
  }
  return G;
}

// the single-site block: sectors are the site states in increasing q
BlkP site_block(const Model& M, cudaStream_t st) {
  auto B = std::make_shared<Blk>();
  B->n = 1;
  const int d = M.d;
  std::vector<int> order(d);
  for (int t = 0; t < d; ++t) order[t] = t;
  std::sort(order.begin(), order.end(), [&](int a, int b) { return M.sq[a] < M.sq[b]; });
  std::vector<int> sec_of(d);
  for (int s = 0; s < d; ++s) {
    B->bs.q.push_back(M.sq[order[s]]);
    B->bs.par.push_back(M.spar[order[s]]);
    B->bs.dim.push_back(1);
    sec_of[order[s]] = s;
  }
  // H classes: on-site terms (diagonal in q: blocks (s, s)); operators: one
  // 1 x 1 block per nonzero element
  std::vector<double> host;
  auto add_block = [&](Op& op, int so, int si, double v) {
    op.b.push_back({so, si, (int64_t)host.size()});
    host.push_back(v);
  };
  B->H.resize(M.n_classes);
  for (int c = 0; c < M.n_classes; ++c)
    for (int s = 0; s < d; ++s) {
      double v = 0.0;
      for (size_t k = 0; k < M.on_cls.size(); ++k)
        if (M.on_cls[k] == c) v += M.on[k * d * d + order[s] * d + order[s]];
      add_block(B->H[c], s, s, v);
    }
  for (size_t k = 0; k < M.on_cls.size(); ++k)
    for (int a = 0; a < d; ++a)
      for (int b = 0; b < d; ++b)
        if (a != b && M.on[k * d * d + a * d + b] != 0.0) throw Bad{"model: an on-site term must conserve q"};
  for (int op = 0; op < M.n_ops; ++op) {
    Op& o = B->ops[{0, op}];
    for (int a = 0; a < d; ++a)
      for (int b = 0; b < d; ++b) {
        const double v = M.ops[((size_t)op * d + a) * d + b];
        if (v != 0.0) add_block(o, sec_of[a], sec_of[b], v);
      }
    std::sort(o.b.begin(), o.b.end(), [](const OpB& x, const OpB& y) { return std::tie(x.so, x.si) < std::tie(y.so, y.si); });
  }
  B->arena = std::make_shared<DBuf>(host.size());
  SYS_CK(cudaMemcpyAsync(B->arena->p, host.data(), host.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  SYS_CK(cudaStreamSynchronize(st));
  return B;
}

// ---------------------------------------------------------------- superblock
struct SbView {  // a superblock of S' (x) E' and its host copies
  std::vector<int32_t> r, c;
  std::vector<int64_t> qS, off;
  std::vector<int32_t> zS, zE;          // per target sector: S' and E' sectors
  std::vector<int32_t> tsecS, tsecE;    // S' / E' sector -> target sector or -1
  std::vector<double> coeffs, mult;
  std::vector<int32_t> cls;
  std::vector<dmrg_pair> pairs;
  std::vector<double> hS, hE, hC;       // host copies of the arenas the pairs point into
  int64_t D = 0;
  int n_terms = 0;
};

void build_superblock(const Model& M, const Blk& Sp, const Blk& Ep, int L, SbView& V, cudaStream_t st) {
  const int64_t Qt = M.target(L);
  V = SbView{};
  V.tsecS.assign(Sp.bs.size(), -1);
  V.tsecE.assign(Ep.bs.size(), -1);
  int64_t off = 0;
  V.off.push_back(0);
  for (int z = 0; z < Sp.bs.size(); ++z) {
    const int e = Ep.bs.find(Qt - Sp.bs.q[z]);
    if (e < 0 || Sp.bs.dim[z] == 0 || Ep.bs.dim[e] == 0) continue;
    V.tsecS[z] = (int)V.r.size();
    V.tsecE[e] = (int)V.r.size();
    V.r.push_back(Sp.bs.dim[z]);
    V.c.push_back(Ep.bs.dim[e]);
    V.qS.push_back(Sp.bs.q[z]);
    V.zS.push_back(z);
    V.zE.push_back(e);
    off += (int64_t)Sp.bs.dim[z] * Ep.bs.dim[e];
    V.off.push_back(off);
  }
  V.D = off;
  if (V.D == 0) throw Bad{"the superblock's target sector is empty"};
  // host copies of both blocks' arenas
  V.hS.resize(Sp.arena->n);
  V.hE.resize(Ep.arena->n);
  SYS_CK(cudaMemcpyAsync(V.hS.data(), Sp.arena->p, Sp.arena->n * sizeof(double), cudaMemcpyDeviceToHost, st));
  SYS_CK(cudaMemcpyAsync(V.hE.data(), Ep.arena->p, Ep.arena->n * sizeof(double), cudaMemcpyDeviceToHost, st));
  int term = 0;
  // H_S' (x) 1 and 1 (x) H_E', per class
  for (int c = 0; c < M.n_classes; ++c, ++term) {
    V.cls.push_back(c);
    V.mult.push_back(1.0);
    for (const OpB& x : Sp.H[c].b) {
      if (x.so != x.si) throw Bad{"block Hamiltonian not diagonal in q"};
      const int s = V.tsecS[x.so];
      if (s < 0) continue;
      dmrg_pair p{};
      p.term = term;
      p.s_out = p.s_in = s;
      p.flags = DMRG_ID_B;
      p.A = V.hS.data() + x.off;
      p.lda = Sp.bs.dim[x.si];
      V.pairs.push_back(p);
    }
  }
  for (int c = 0; c < M.n_classes; ++c, ++term) {
    V.cls.push_back(c);
    V.mult.push_back(1.0);
    for (const OpB& x : Ep.H[c].b) {
      if (x.so != x.si) throw Bad{"block Hamiltonian not diagonal in q"};
      const int s = V.tsecE[x.so];
      if (s < 0) continue;
      dmrg_pair p{};
      p.term = term;
      p.s_out = p.s_in = s;
      p.flags = DMRG_ID_A;
      p.B = V.hE.data() + x.off;
      p.ldb = Ep.bs.dim[x.si];
      V.pairs.push_back(p);
    }
  }
  // connection terms: for each bond crossing the cut and each bond-term
  // template, A = op(X_i)^{ta} (times F_S' when fermionic), B = op(Y_j)^{tb},
  // materialised as dense blocks (transposes and signs applied) in one arena
  struct CB {
    int term, zo, zi;  // A: S' sectors, B: E' sectors
    int64_t off;
    int rows, cols;
  };
  std::vector<CB> ablk, bblk;
  std::vector<ScatJob> jobs;
  int64_t ctot = 0;
  std::vector<std::pair<int, int>> conn;  // (term, dummy)
  const int nS = Sp.n;
  for (auto& bd : M.bonds(L)) {
    const int i = std::get<0>(bd), j = std::get<1>(bd), cls = std::get<2>(bd);
    if (!(i < nS && nS <= j)) continue;
    const int jd = L - 1 - j;
    for (const dmrg_bond_term& tm : M.terms) {
      const bool fer = M.fermionic(tm);
      auto ia = Sp.ops.find({i, tm.op_a});
      auto jb = Ep.ops.find({jd, tm.op_b});
      if (ia == Sp.ops.end() || jb == Ep.ops.end()) throw Bad{"superblock: a bonded site's operator was not kept"};
      V.cls.push_back(cls);
      V.mult.push_back(tm.coef);
      for (const OpB& x : ia->second.b) {
        const int zo = tm.trans_a ? x.si : x.so, zi = tm.trans_a ? x.so : x.si;
        if (V.tsecS[zo] < 0 || V.tsecS[zi] < 0) continue;
        const int rows = Sp.bs.dim[zo], cols = Sp.bs.dim[zi];
        ablk.push_back({term, zo, zi, ctot, rows, cols});
        ScatJob sj{};
        sj.src = Sp.ptr(x);
        sj.ld_src = Sp.bs.dim[x.si];
        sj.trans = tm.trans_a;
        sj.rows = rows;
        sj.cols = cols;
        sj.ld_dst = cols;
        sj.scale = (fer && Sp.bs.par[zi]) ? -1.0 : 1.0;
        sj.dst = reinterpret_cast<double*>(ctot);  // offset; rebased below
        jobs.push_back(sj);
        ctot += (int64_t)rows * cols;
      }
      for (const OpB& x : jb->second.b) {
        const int eo = tm.trans_b ? x.si : x.so, ei = tm.trans_b ? x.so : x.si;
        if (V.tsecE[eo] < 0 || V.tsecE[ei] < 0) continue;
        const int rows = Ep.bs.dim[eo], cols = Ep.bs.dim[ei];
        bblk.push_back({term, eo, ei, ctot, rows, cols});
        ScatJob sj{};
        sj.src = Ep.ptr(x);
        sj.ld_src = Ep.bs.dim[x.si];
        sj.trans = tm.trans_b;
        sj.rows = rows;
        sj.cols = cols;
        sj.ld_dst = cols;
        sj.scale = 1.0;
        sj.dst = reinterpret_cast<double*>(ctot);
        jobs.push_back(sj);
        ctot += (int64_t)rows * cols;
      }
      ++term;
    }
  }
  V.n_terms = term;
  if (ctot > 0) {
    DBuf carena((size_t)ctot);
    SYS_CK(cudaMemsetAsync(carena.p, 0, ctot * sizeof(double), st));
    for (ScatJob& sj : jobs) sj.dst = carena.p + reinterpret_cast<int64_t>(sj.dst);
    launch_scatter(jobs, st);
    V.hC.resize((size_t)ctot);
    SYS_CK(cudaMemcpyAsync(V.hC.data(), carena.p, ctot * sizeof(double), cudaMemcpyDeviceToHost, st));
    SYS_CK(cudaStreamSynchronize(st));
  }
  SYS_CK(cudaStreamSynchronize(st));
  // pairs of the connection terms: A block (zo, zi) with B block (eo, ei) where
  // (zo, eo) and (zi, ei) are target sectors
  std::map<std::pair<int, int>, std::vector<const CB*>> b_by;  // (term, eo) -> B blocks
  for (const CB& b : bblk) b_by[{b.term, b.zo}].push_back(&b);
  for (const CB& a : ablk) {
    const int so = V.tsecS[a.zo], si = V.tsecS[a.zi];
    auto it = b_by.find({a.term, V.zE[so]});
    if (it == b_by.end()) continue;
    for (const CB* b : it->second) {
      if (b->zi != V.zE[si]) continue;
      dmrg_pair p{};
      p.term = a.term;
      p.s_out = so;
      p.s_in = si;
      p.flags = 0;
      p.A = V.hC.data() + a.off;
      p.lda = a.cols;
      p.B = V.hC.data() + b->off;
      p.ldb = b->cols;
      V.pairs.push_back(p);
    }
  }
  V.coeffs.resize(V.n_terms);
  for (int k = 0; k < V.n_terms; ++k) V.coeffs[k] = V.mult[k] * M.g[V.cls[k]];
}

// ---------------------------------------------------------------- truncation
struct TruncOut {
  BlkP blk;
  double eps = 0.0, gap = 0.0;
  int kept = 0;
  double ms_eig = 0.0, ms_select = 0.0, ms_transform = 0.0;  // density matrices and eigensolves; choice; W^T O W
};

double host_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Keep the m most probable states of the grown block G (side S: rows of the
// target blocks, rho = Psi Psi^T; side E: columns, rho = Psi^T Psi) and carry
// H and the operators of end distance >= keep_from to the new basis.
TruncOut truncate(const Model& M, const Blk& G, bool sideS, const SbView& V, const double* psi, int m,
                  double tie_tol, int keep_from, cudaStream_t st) {
  const Basis& b = G.bs;
  const int nz = b.size();
  std::vector<int64_t> roff(nz + 1, 0), coff(nz + 1, 0), woff(nz + 1, 0);
  for (int z = 0; z < nz; ++z) {
    const int64_t n = b.dim[z];
    roff[z + 1] = roff[z] + n * n;
    coff[z + 1] = coff[z] + n;
    woff[z + 1] = woff[z] + (n > EIG_SMEM_MAX_N ? 2 * n * (n + 1) : 0);
  }
  const int64_t ncand = coff[nz];
  const double t0 = host_ms();
  DBuf rho((size_t)roff[nz]);
  auto Vv = std::make_shared<DBuf>((size_t)roff[nz]);
  DBuf lam((size_t)ncand), work((size_t)std::max<int64_t>(woff[nz], 1));
  SYS_CK(cudaMemsetAsync(rho.p, 0, roff[nz] * sizeof(double), st));
  std::vector<GemmJob> gj;
  for (int z = 0; z < nz; ++z) {
    const int s = sideS ? V.tsecS[z] : V.tsecE[z];
    if (s < 0) continue;
    const int r = V.r[s], c = V.c[s];
    GemmJob j{};
    j.A = j.B = psi + V.off[s];
    j.C = rho.p + roff[z];
    j.alpha = 1.0;
    j.beta = 0.0;
    j.lda = j.ldb = c;
    if (sideS) {  // Psi Psi^T
      j.M = j.N = r;
      j.K = c;
      j.ta = 0;
      j.tb = 1;
      j.ldc = r;
    } else {  // Psi^T Psi
      j.M = j.N = c;
      j.K = r;
      j.ta = 1;
      j.tb = 0;
      j.ldc = c;
    }
    gj.push_back(j);
  }
  launch_gemm(gj, st);
  std::vector<EigJob> ej;
  for (int z = 0; z < nz; ++z) {
    EigJob j{};
    j.A = rho.p + roff[z];
    j.V = Vv->p + roff[z];
    j.w = lam.p + coff[z];
    j.work = b.dim[z] > EIG_SMEM_MAX_N ? work.p + woff[z] : nullptr;
    j.n = b.dim[z];
    ej.push_back(j);
  }
  launch_eig(ej, st);
  SYS_CK(cudaStreamSynchronize(st));
  const double t1 = host_ms();
  // global selection
  std::vector<int32_t> hsec((size_t)ncand), hidx((size_t)ncand);
  for (int z = 0; z < nz; ++z)
    for (int i = 0; i < b.dim[z]; ++i) {
      hsec[coff[z] + i] = z;
      hidx[coff[z] + i] = i;
    }
  DArr<int32_t> dsec((size_t)ncand), didx((size_t)ncand), dkeep((size_t)ncand), scr((size_t)4 * ncand);
  DBuf stats(2);
  SYS_CK(cudaMemcpyAsync(dsec.p, hsec.data(), ncand * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  SYS_CK(cudaMemcpyAsync(didx.p, hidx.data(), ncand * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  const int meff = (int)std::min<int64_t>(m, ncand);
  launch_select(lam.p, dsec.p, didx.p, (int32_t)ncand, meff, tie_tol, dkeep.p, stats.p, scr.p, nullptr, st);
  std::vector<int32_t> keep((size_t)ncand);
  double hst[2] = {0.0, 0.0};
  SYS_CK(cudaMemcpyAsync(keep.data(), dkeep.p, ncand * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  SYS_CK(cudaMemcpyAsync(hst, stats.p, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
  SYS_CK(cudaStreamSynchronize(st));
  const double t2 = host_ms();
  auto tr = std::make_shared<Trunc>();
  tr->grown = b;
  tr->comps = G.comps;
  tr->left = G.left;
  tr->V = Vv;
  tr->voff.assign(roff.begin(), roff.end() - 1);
  tr->k.assign(nz, 0);
  tr->newsec.assign(nz, -1);
  for (int z = 0; z < nz; ++z) {
    int k = 0;
    for (int i = 0; i < b.dim[z]; ++i) k += keep[coff[z] + i];
    for (int i = 0; i < k; ++i)
      if (!keep[coff[z] + i]) throw std::logic_error("truncation: kept states of a sector are not a prefix");
    tr->k[z] = k;
  }
  auto N = std::make_shared<Blk>();
  N->n = G.n;
  N->left = G.left;
  for (int z = 0; z < nz; ++z)
    if (tr->k[z] > 0) {
      tr->newsec[z] = N->bs.size();
      N->bs.q.push_back(b.q[z]);
      N->bs.par.push_back(b.par[z]);
      N->bs.dim.push_back(tr->k[z]);
    }
  // W^T O W for H and the operators still needed
  std::vector<std::pair<const Op*, Op*>> todo;
  N->H.resize(G.H.size());
  for (size_t c = 0; c < G.H.size(); ++c) todo.push_back({&G.H[c], &N->H[c]});
  for (auto& kv : G.ops)
    if (kv.first.first >= keep_from) todo.push_back({&kv.second, &N->ops[kv.first]});
  int64_t total = 0, ttot = 0;
  std::vector<std::tuple<const OpB*, Op*, int64_t, int64_t>> blocks;  // (source block, dest op, dest off, T off)
  for (auto& td : todo)
    for (const OpB& x : td.first->b) {
      const int ko = tr->k[x.so], ki = tr->k[x.si];
      if (ko == 0 || ki == 0) continue;
      blocks.emplace_back(&x, td.second, total, ttot);
      td.second->b.push_back({tr->newsec[x.so], tr->newsec[x.si], total});
      total += (int64_t)ko * ki;
      ttot += (int64_t)b.dim[x.so] * ki;
    }
  N->arena = std::make_shared<DBuf>((size_t)total);
  DBuf T((size_t)std::max<int64_t>(ttot, 1));
  std::vector<GemmJob> j1, j2;
  for (auto& bk : blocks) {
    const OpB& x = *std::get<0>(bk);
    const int no = b.dim[x.so], ni = b.dim[x.si], ko = tr->k[x.so], ki = tr->k[x.si];
    GemmJob a{};  // T = O W_i : (no x ni) (ni x ki)
    a.A = G.ptr(x);
    a.lda = ni;
    a.B = Vv->p + roff[x.si];
    a.ldb = ni;
    a.C = T.p + std::get<3>(bk);
    a.ldc = ki;
    a.M = no;
    a.N = ki;
    a.K = ni;
    a.alpha = 1.0;
    j1.push_back(a);
    GemmJob c{};  // O' = W_o^T T : (ko x no) (no x ki)
    c.A = Vv->p + roff[x.so];
    c.lda = no;
    c.ta = 1;
    c.B = T.p + std::get<3>(bk);
    c.ldb = ki;
    c.C = N->arena->p + std::get<2>(bk);
    c.ldc = ki;
    c.M = ko;
    c.N = ki;
    c.K = no;
    c.alpha = 1.0;
    j2.push_back(c);
  }
  launch_gemm(j1, st);
  launch_gemm(j2, st);
  SYS_CK(cudaStreamSynchronize(st));
  N->trunc = tr;
  TruncOut out;
  out.ms_eig = t1 - t0;
  out.ms_select = t2 - t1;
  out.ms_transform = host_ms() - t2;
  out.blk = N;
  out.eps = std::max(0.0, hst[0]);
  out.gap = hst[1];
  out.kept = meff;
  return out;
}

// ------------------------------------------------- wavefunction transformation
// The previous step's ground state carried to the next step's basis (White's
// wavefunction transformation, named in the paper's closing notes as the
// initial guess that cuts the Lanczos iterations of the finite algorithm).
// Index structure of a superblock (no data):
struct SbIdx {
  std::vector<int32_t> r, c, zS, zE, tsecS, tsecE;
  std::vector<int64_t> off;
  int64_t D = 0;
};
SbIdx index_of(const SbView& V) {
  SbIdx x;
  x.r = V.r;
  x.c = V.c;
  x.zS = V.zS;
  x.zE = V.zE;
  x.tsecS = V.tsecS;
  x.tsecE = V.tsecE;
  x.off = V.off;
  x.D = V.D;
  return x;
}

struct Prev {
  bool valid = false;
  int l = 0, dir = 0;  // split (sites of S') and direction of the step
  SbIdx ix;
  BlkP Sp, Ep;         // its grown blocks (their product structure)
  DBufP psi;
};

std::vector<int> inverse_newsec(const Trunc& t) {
  int n = 0;
  for (int v : t.newsec) n = std::max(n, v + 1);
  std::vector<int> inv(n, -1);
  for (size_t z = 0; z < t.newsec.size(); ++z)
    if (t.newsec[z] >= 0) inv[t.newsec[z]] = (int)z;
  return inv;
}

bool same_basis(const Basis& a, const Basis& b) { return a.q == b.q && a.dim == b.dim; }

// Move to the right (split l -> l + 1).  Old state Psi(alpha', beta') with
// alpha' in S' (truncated to A = left[l] by W_S) and beta' in E' = site (x) B.
// New S'' = A (x) site, E'' = site (x) B'' with B = trunc(E'') by W_E:
//   X = W_S^T Psi;  beta' = (t, b) regrouped so that (a, t) = alpha'';
//   Psi''(alpha'', beta'') = sum_b X(alpha'', b) W_E(beta'', b).
bool guess_right(const Prev& P, const Blk& A, const Blk& Snew, const Blk& B, const Blk& Enew, const SbView& Vn,
                 double* out, cudaStream_t st) {
  if (!A.trunc || !B.trunc || !same_basis(B.trunc->grown, Enew.bs) || !same_basis(A.trunc->grown, P.Sp->bs))
    return false;
  const Trunc& TA = *A.trunc;
  const Trunc& TB = *B.trunc;
  const SbIdx& ix = P.ix;
  const int ns = (int)ix.r.size();
  std::vector<int64_t> xo(ns + 1, 0);
  std::vector<GemmJob> ga;
  for (int s = 0; s < ns; ++s) {
    const int z = ix.zS[s], k = TA.k[z];
    xo[s + 1] = xo[s] + (int64_t)k * ix.c[s];
  }
  DBuf X((size_t)std::max<int64_t>(xo[ns], 1));
  for (int s = 0; s < ns; ++s) {
    const int z = ix.zS[s], k = TA.k[z];
    if (k == 0) continue;
    GemmJob j{};
    j.A = TA.V->p + TA.voff[z];  // W_S^T: A(m, kk) = V[kk * n + m]
    j.lda = ix.r[s];
    j.ta = 1;
    j.M = k;
    j.K = ix.r[s];
    j.B = P.psi->p + ix.off[s];
    j.ldb = ix.c[s];
    j.N = ix.c[s];
    j.C = X.p + xo[s];
    j.ldc = ix.c[s];
    j.alpha = 1.0;
    ga.push_back(j);
  }
  launch_gemm(ga, st);
  const std::vector<int> invA = inverse_newsec(TA);
  const int nn = (int)Vn.r.size();
  std::vector<int64_t> po(nn + 1, 0);
  std::vector<int> ky(nn, 0);
  for (int s = 0; s < nn; ++s) {
    const int y = TB.newsec[Vn.zE[s]];
    ky[s] = y >= 0 ? B.bs.dim[y] : 0;
    po[s + 1] = po[s] + (int64_t)Vn.r[s] * ky[s];
  }
  DBuf P2((size_t)std::max<int64_t>(po[nn], 1));
  SYS_CK(cudaMemsetAsync(P2.p, 0, std::max<int64_t>(po[nn], 1) * sizeof(double), st));
  std::vector<ScatJob> jobs;
  for (int s2 = 0; s2 < nn; ++s2) {
    if (ky[s2] == 0) continue;
    const int y = TB.newsec[Vn.zE[s2]];
    for (const Comp& cp : Snew.comps[Vn.zS[s2]]) {
      const int zold = cp.z < (int)invA.size() ? invA[cp.z] : -1;
      if (zold < 0) continue;
      auto w = P.Ep->where.find({y, cp.t});
      if (w == P.Ep->where.end()) continue;
      const int s = ix.tsecS[zold];
      if (s < 0 || ix.zE[s] != w->second.first) continue;
      ScatJob j{};
      j.src = X.p + xo[s] + w->second.second;
      j.ld_src = ix.c[s];
      j.rows = A.bs.dim[cp.z];
      j.cols = ky[s2];
      j.dst = P2.p + po[s2] + (int64_t)cp.off * ky[s2];
      j.ld_dst = ky[s2];
      j.scale = 1.0;
      jobs.push_back(j);
    }
  }
  launch_scatter(jobs, st);
  SYS_CK(cudaMemsetAsync(out, 0, Vn.D * sizeof(double), st));
  std::vector<GemmJob> gc;
  for (int s2 = 0; s2 < nn; ++s2) {
    if (ky[s2] == 0) continue;
    const int e = Vn.zE[s2];
    GemmJob j{};
    j.A = P2.p + po[s2];
    j.lda = ky[s2];
    j.M = Vn.r[s2];
    j.K = ky[s2];
    j.B = TB.V->p + TB.voff[e];  // W_E^T: B(kk, n) = V[n * c + kk]
    j.ldb = Vn.c[s2];
    j.tb = 1;
    j.N = Vn.c[s2];
    j.C = out + Vn.off[s2];
    j.ldc = Vn.c[s2];
    j.alpha = 1.0;
    gc.push_back(j);
  }
  launch_gemm(gc, st);
  SYS_CK(cudaStreamSynchronize(st));
  return true;
}

// Move to the left (split l -> l - 1), the mirror image: X = Psi W_E (E'
// truncated to A = right[L - l]); alpha' = (a, t) regrouped so that (t, b) =
// beta''; Psi''(alpha'', beta'') = sum_a W_S(alpha'', a) X(a, beta'') with
// B = left[l - 1] = trunc(S'') by W_S.
bool guess_left(const Prev& P, const Blk& A, const Blk& Enew, const Blk& B, const Blk& Snew, const SbView& Vn,
                double* out, cudaStream_t st) {
  if (!A.trunc || !B.trunc || !same_basis(B.trunc->grown, Snew.bs) || !same_basis(A.trunc->grown, P.Ep->bs))
    return false;
  const Trunc& TA = *A.trunc;
  const Trunc& TB = *B.trunc;
  const SbIdx& ix = P.ix;
  const int ns = (int)ix.r.size();
  std::vector<int64_t> xo(ns + 1, 0);
  for (int s = 0; s < ns; ++s) xo[s + 1] = xo[s] + (int64_t)ix.r[s] * TA.k[ix.zE[s]];
  DBuf X((size_t)std::max<int64_t>(xo[ns], 1));
  std::vector<GemmJob> ga;
  for (int s = 0; s < ns; ++s) {
    const int e = ix.zE[s], k = TA.k[e];
    if (k == 0) continue;
    GemmJob j{};
    j.A = P.psi->p + ix.off[s];
    j.lda = ix.c[s];
    j.M = ix.r[s];
    j.K = ix.c[s];
    j.B = TA.V->p + TA.voff[e];  // W_E: B(kk, n) = V[kk * c + n]
    j.ldb = ix.c[s];
    j.N = k;
    j.C = X.p + xo[s];
    j.ldc = k;
    j.alpha = 1.0;
    ga.push_back(j);
  }
  launch_gemm(ga, st);
  const std::vector<int> invA = inverse_newsec(TA);
  const int nn = (int)Vn.r.size();
  std::vector<int64_t> po(nn + 1, 0);
  std::vector<int> kx(nn, 0);
  for (int s = 0; s < nn; ++s) {
    const int x = TB.newsec[Vn.zS[s]];
    kx[s] = x >= 0 ? B.bs.dim[x] : 0;
    po[s + 1] = po[s] + (int64_t)kx[s] * Vn.c[s];
  }
  DBuf P2((size_t)std::max<int64_t>(po[nn], 1));
  SYS_CK(cudaMemsetAsync(P2.p, 0, std::max<int64_t>(po[nn], 1) * sizeof(double), st));
  std::vector<ScatJob> jobs;
  for (int s2 = 0; s2 < nn; ++s2) {
    if (kx[s2] == 0) continue;
    const int x = TB.newsec[Vn.zS[s2]];
    for (const Comp& cp : Enew.comps[Vn.zE[s2]]) {
      const int eold = cp.z < (int)invA.size() ? invA[cp.z] : -1;
      if (eold < 0) continue;
      auto w = P.Sp->where.find({x, cp.t});
      if (w == P.Sp->where.end()) continue;
      const int s = ix.tsecS[w->second.first];
      if (s < 0 || ix.zE[s] != eold) continue;
      const int kE = TA.k[eold];
      ScatJob j{};
      j.src = X.p + xo[s] + (int64_t)w->second.second * kE;
      j.ld_src = kE;
      j.rows = kx[s2];
      j.cols = kE;
      j.dst = P2.p + po[s2] + cp.off;
      j.ld_dst = Vn.c[s2];
      j.scale = 1.0;
      jobs.push_back(j);
    }
  }
  launch_scatter(jobs, st);
  SYS_CK(cudaMemsetAsync(out, 0, Vn.D * sizeof(double), st));
  std::vector<GemmJob> gc;
  for (int s2 = 0; s2 < nn; ++s2) {
    if (kx[s2] == 0) continue;
    const int z = Vn.zS[s2];
    GemmJob j{};
    j.A = TB.V->p + TB.voff[z];  // W_S: A(m, kk) = V[m * r + kk]
    j.lda = Vn.r[s2];
    j.M = Vn.r[s2];
    j.K = kx[s2];
    j.B = P2.p + po[s2];
    j.ldb = Vn.c[s2];
    j.N = Vn.c[s2];
    j.C = out + Vn.off[s2];
    j.ldc = Vn.c[s2];
    j.alpha = 1.0;
    gc.push_back(j);
  }
  launch_gemm(gc, st);
  SYS_CK(cudaStreamSynchronize(st));
  return true;
}

}  // namespace

// ------------------------------------------------------------------ system
struct dmrg_sys {
  Model M;
  int L = 0, m = 0;
  dmrg_sys_opts opts{};
  std::map<int, BlkP> left, right;  // truncated blocks by number of sites
  bool infinite_done = false;
  int64_t step_count = 0;
  // the last step
  SbView view;
  std::vector<double> psi_host;
  int last_nS = 0, last_L = 0;
  Prev prev;  // the previous step, for the wavefunction transformation
  std::string err;
};

namespace {

double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// guess(V, out): writes a start vector for the superblock V into out and
// returns true, or returns false (random start)
using GuessFn = std::function<bool(const SbView&, double*)>;

void solve_step(dmrg_sys* sys, const BlkP& SpP, const BlkP& EpP, int L, int dir, dmrg_step_info& info,
                const GuessFn& guess, cudaStream_t st) {
  const Blk& Sp = *SpP;
  const Blk& Ep = *EpP;
  const double t0 = now_ms();
  build_superblock(sys->M, Sp, Ep, L, sys->view, st);
  SbView& V = sys->view;
  dmrg_sb_desc desc{};
  desc.n_sectors = (int32_t)V.r.size();
  desc.r = V.r.data();
  desc.c = V.c.data();
  desc.n_terms = V.n_terms;
  desc.coeffs = V.coeffs.data();
  desc.n_pairs = (int32_t)V.pairs.size();
  desc.pairs = V.pairs.data();
  desc.blocks_on_device = 0;
  dmrg_sb* sb = nullptr;
  dmrg_status s = dmrg_create_superblock(&desc, 1, &sb);
  if (s != DMRG_OK) throw std::runtime_error("dmrg_create_superblock failed in a DMRG step (status " + std::to_string(s) + ")");
  struct SbGuard {
    dmrg_sb* p;
    ~SbGuard() { dmrg_destroy_superblock(p); }
  } guard{sb};
  const double t1 = now_ms();
  info.ms_superblock = t1 - t0;
  DBuf psi0((size_t)V.D);
  const bool guessed = sys->opts.guess && guess && guess(V, psi0.p);
  if (!guessed) launch_start_vector(psi0.p, V.D, sys->opts.seed * 1000003ull + (uint64_t)sys->step_count, st);
  info.guessed = guessed ? 1 : 0;
  DBufP psi_out = std::make_shared<DBuf>((size_t)V.D);
  dmrg_lanczos_opts o{};
  const bool mixed = sys->opts.prec != DMRG_FP64;
  o.tol = mixed ? sys->opts.mixed_tol : sys->opts.tol;
  o.max_iter = sys->opts.max_iter;
  o.prec = sys->opts.prec;
  o.refine = mixed ? sys->opts.refine : 0;
  o.refine_tol = sys->opts.tol;
  o.check_every = 1;
  o.graph_iters = 8;
  double e0 = 0.0;
  dmrg_lanczos_info li{};
  s = dmrg_lanczos_ground(sb, psi0.p, psi_out->p, &e0, &o, &li, st);
  if (s != DMRG_OK && s != DMRG_ENOCONV)
    throw std::runtime_error(std::string("Lanczos failed in a DMRG step: ") + dmrg_last_error(sb));
  info.status = s;
  info.energy = e0;
  info.iters = li.iters + li.refine_iters;
  info.dim = V.D;
  info.n_terms = V.n_terms;
  info.L = L;
  info.n_sys = Sp.n;
  sys->psi_host.resize((size_t)V.D);
  SYS_CK(cudaMemcpyAsync(sys->psi_host.data(), psi_out->p, V.D * sizeof(double), cudaMemcpyDeviceToHost, st));
  SYS_CK(cudaStreamSynchronize(st));
  sys->last_nS = Sp.n;
  sys->last_L = L;
  ++sys->step_count;
  info.ms_solve = now_ms() - t1;
  Prev& P = sys->prev;
  P.valid = true;
  P.l = Sp.n;
  P.dir = dir;
  P.ix = index_of(V);
  P.Sp = SpP;
  P.Ep = EpP;
  P.psi = psi_out;
}

int max_dim(const Blk& b) {
  int m = 0;
  for (int d : b.bs.dim) m = std::max(m, d);
  return m;
}

template <class F>
dmrg_status sys_guard(dmrg_sys* sys, F&& fn) {
  try {
    return fn();
  } catch (const Bad& b) {
    if (sys) sys->err = b.msg;
    return DMRG_EINVAL;
  } catch (const std::logic_error& e) {
    if (sys) sys->err = e.what();
    return DMRG_EINVAL;
  } catch (const std::bad_alloc&) {
    if (sys) sys->err = "host allocation failed";
    return DMRG_ENOMEM;
  } catch (const std::runtime_error& e) {
    if (sys) sys->err = e.what();
    const cudaError_t ce = cudaGetLastError();
    return ce == cudaErrorMemoryAllocation ? DMRG_ENOMEM : DMRG_ECUDA;
  }
}

}  // namespace

extern "C" {

dmrg_status dmrg_sys_create(const dmrg_model_desc* model, int32_t L, int32_t m, const dmrg_sys_opts* opts,
                            dmrg_sys** out) {
  if (!out) return DMRG_EINVAL;
  *out = nullptr;
  dmrg_sys* sys = new (std::nothrow) dmrg_sys();
  if (!sys) return DMRG_ENOMEM;
  const dmrg_status s = sys_guard(sys, [&] {
    if (L < 4 || L % 2) throw Bad{"L must be even and >= 4"};
    if (m < 1) throw Bad{"m must be >= 1"};
    if (!opts || !(opts->tol > 0) || opts->max_iter < 1 || opts->prec < DMRG_FP64 || opts->prec > DMRG_BF16X3 ||
        !(opts->tie_tol >= 0) || opts->guess < 0 || opts->guess > 1 ||
        (opts->prec != DMRG_FP64 && !(opts->mixed_tol > 0)))
      throw Bad{"bad options"};
    sys->M = make_model(model);
    sys->L = L;
    sys->m = m;
    sys->opts = *opts;
    return DMRG_OK;
  });
  if (s != DMRG_OK) {
    fprintf(stderr, "dmrg_sys_create: %s\n", sys->err.c_str());
    delete sys;
    return s;
  }
  *out = sys;
  return DMRG_OK;
}

void dmrg_sys_destroy(dmrg_sys* sys) { delete sys; }

const char* dmrg_sys_last_error(const dmrg_sys* sys) { return sys ? sys->err.c_str() : "null system"; }

dmrg_status dmrg_sys_infinite(dmrg_sys* sys, dmrg_step_info* steps, int32_t* n_steps) {
  if (!sys || !steps || !n_steps) return DMRG_EINVAL;
  *n_steps = 0;
  return sys_guard(sys, [&] {
    if (sys->infinite_done) throw Bad{"the infinite phase has already run"};
    cudaStream_t st = nullptr;
    const Model& M = sys->M;
    BlkP S = site_block(M, st), E = site_block(M, st);
    sys->left[1] = S;
    sys->right[1] = E;
    dmrg_status worst = DMRG_OK;
    for (int k = 0; k < sys->L / 2 - 1; ++k) {
      const double t0 = now_ms();
      BlkP Sp = grow(M, *S, true, st), Ep = grow(M, *E, false, st);
      SYS_CK(cudaStreamSynchronize(st));
      const int Lk = Sp->n + Ep->n;
      dmrg_step_info info{};
      info.ms_grow = now_ms() - t0;
      solve_step(sys, Sp, Ep, Lk, 0, info, nullptr, st);
      const double* psi = sys->prev.psi->p;
      const double t2 = now_ms();
      TruncOut ts = truncate(M, *Sp, true, sys->view, psi, sys->m, sys->opts.tie_tol, Sp->n - M.reach, st);
      TruncOut te = truncate(M, *Ep, false, sys->view, psi, sys->m, sys->opts.tie_tol, Ep->n - M.reach, st);
      info.ms_truncate = now_ms() - t2;
      info.ms_eig = ts.ms_eig + te.ms_eig;
      info.ms_select = ts.ms_select + te.ms_select;
      info.ms_transform = ts.ms_transform + te.ms_transform;
      info.max_sector = std::max(max_dim(*Sp), max_dim(*Ep));
      S = ts.blk;
      E = te.blk;
      sys->left[S->n] = S;
      sys->right[E->n] = E;
      info.direction = 0;
      info.eps_S = ts.eps;
      info.eps_E = te.eps;
      info.gap_S = ts.gap;
      info.gap_E = te.gap;
      info.kept_S = ts.kept;
      info.kept_E = te.kept;
      info.ms = now_ms() - t0;
      steps[k] = info;
      *n_steps = k + 1;
      if (info.status != DMRG_OK && worst == DMRG_OK) worst = (dmrg_status)info.status;
    }
    sys->infinite_done = true;
    return worst;
  });
}

dmrg_status dmrg_sys_sweeps(dmrg_sys* sys, int32_t n_sweeps, dmrg_step_info* steps, int32_t* n_steps) {
  if (!sys || !steps || !n_steps || n_sweeps < 0) return DMRG_EINVAL;
  *n_steps = 0;
  return sys_guard(sys, [&] {
    if (!sys->infinite_done) throw Bad{"run the infinite phase first"};
    cudaStream_t st = nullptr;
    const Model& M = sys->M;
    const int L = sys->L, half = L / 2;
    std::vector<std::pair<int, int>> path;  // (split l, direction)
    for (int s = 0; s < n_sweeps; ++s) {
      for (int l = half + 1; l < L - 1; ++l) path.push_back({l, 1});
      for (int l = L - 2; l > 1; --l) path.push_back({l, -1});
      for (int l = 2; l <= half; ++l) path.push_back({l, 1});
    }
    dmrg_status worst = DMRG_OK;
    int k = 0;
    for (auto& pl : path) {
      const int l = pl.first, dir = pl.second;
      const double t0 = now_ms();
      auto il = sys->left.find(l - 1);
      auto ir = sys->right.find(L - l - 1);
      if (il == sys->left.end() || ir == sys->right.end()) throw std::logic_error("sweep: missing block on the stack");
      BlkP Sp = grow(M, *il->second, true, st), Ep = grow(M, *ir->second, false, st);
      SYS_CK(cudaStreamSynchronize(st));
      dmrg_step_info info{};
      info.ms_grow = now_ms() - t0;
      const BlkP Sold = il->second, Eold = ir->second;
      GuessFn guess = [&](const SbView& Vn, double* out) -> bool {
        const Prev& P = sys->prev;
        if (!P.valid) return false;
        if (P.l == l && P.ix.D == Vn.D && P.ix.r == Vn.r && P.ix.c == Vn.c) {  // same superblock (turning point)
          SYS_CK(cudaMemcpyAsync(out, P.psi->p, Vn.D * sizeof(double), cudaMemcpyDeviceToDevice, st));
          return true;
        }
        if (l == P.l + 1 && P.dir >= 0) {  // moved right: S' of the last step was truncated into left[l - 1]
          auto a = sys->left.find(P.l);
          auto b = sys->right.find(L - l);
          if (a == sys->left.end() || b == sys->right.end() || a->second != Sold) return false;
          return guess_right(P, *a->second, *Sp, *b->second, *Ep, Vn, out, st);
        }
        if (l == P.l - 1 && P.dir < 0) {  // moved left: E' of the last step was truncated into right[L - l - 1]
          auto a = sys->right.find(L - P.l);
          auto b = sys->left.find(l);
          if (a == sys->right.end() || b == sys->left.end() || a->second != Eold) return false;
          return guess_left(P, *a->second, *Ep, *b->second, *Sp, Vn, out, st);
        }
        return false;
      };
      solve_step(sys, Sp, Ep, L, dir, info, guess, st);
      const double* psi = sys->prev.psi->p;
      const double t2 = now_ms();
      info.max_sector = dir > 0 ? max_dim(*Sp) : max_dim(*Ep);
      if (dir > 0) {
        TruncOut ts = truncate(M, *Sp, true, sys->view, psi, sys->m, sys->opts.tie_tol, Sp->n - M.reach, st);
        sys->left[Sp->n] = ts.blk;
        info.ms_eig = ts.ms_eig;
        info.ms_select = ts.ms_select;
        info.ms_transform = ts.ms_transform;
        info.eps_S = ts.eps;
        info.gap_S = ts.gap;
        info.kept_S = ts.kept;
      } else {
        TruncOut te = truncate(M, *Ep, false, sys->view, psi, sys->m, sys->opts.tie_tol, Ep->n - M.reach, st);
        sys->right[Ep->n] = te.blk;
        info.ms_eig = te.ms_eig;
        info.ms_select = te.ms_select;
        info.ms_transform = te.ms_transform;
        info.eps_E = te.eps;
        info.gap_E = te.gap;
        info.kept_E = te.kept;
      }
      info.direction = dir;
      info.ms_truncate = now_ms() - t2;
      info.ms = now_ms() - t0;
      steps[k] = info;
      *n_steps = ++k;
      if (info.status != DMRG_OK && worst == DMRG_OK) worst = (dmrg_status)info.status;
    }
    return worst;
  });
}

dmrg_status dmrg_sys_last_superblock(dmrg_sys* sys, dmrg_sys_superblock_view* out, double* psi) {
  if (!sys || !out) return DMRG_EINVAL;
  if (sys->view.D == 0) {
    sys->err = "no step has run";
    return DMRG_EINVAL;
  }
  SbView& V = sys->view;
  out->desc.n_sectors = (int32_t)V.r.size();
  out->desc.r = V.r.data();
  out->desc.c = V.c.data();
  out->desc.n_terms = V.n_terms;
  out->desc.coeffs = V.coeffs.data();
  out->desc.n_pairs = (int32_t)V.pairs.size();
  out->desc.pairs = V.pairs.data();
  out->desc.blocks_on_device = 0;
  out->term_class = V.cls.data();
  out->term_mult = V.mult.data();
  out->sector_q = V.qS.data();
  out->n_sys = sys->last_nS;
  out->L = sys->last_L;
  if (psi) memcpy(psi, sys->psi_host.data(), sys->psi_host.size() * sizeof(double));
  return DMRG_OK;
}

dmrg_status dmrg_sym_eig_batched(int32_t count, const int32_t* n, const double* const* A, double* const* V,
                                 double* const* w, void* stream) {
  if (count < 0 || (count > 0 && (!n || !A || !V || !w))) return DMRG_EINVAL;
  try {
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<EigJob> jobs;
    int64_t work = 0;
    for (int i = 0; i < count; ++i) {
      if (n[i] < 0 || n[i] > 4096 || (n[i] > 0 && (!A[i] || !V[i] || !w[i]))) return DMRG_EINVAL;
      if (n[i] > EIG_SMEM_MAX_N) work += 2 * (int64_t)n[i] * (n[i] + 1);
    }
    double* ws = nullptr;
    if (work > 0) SYS_CK(cudaMallocAsync(reinterpret_cast<void**>(&ws), work * sizeof(double), st));
    int64_t off = 0;
    for (int i = 0; i < count; ++i) {
      if (n[i] == 0) continue;
      EigJob j{};
      j.A = A[i];
      j.V = V[i];
      j.w = w[i];
      j.n = n[i];
      if (n[i] > EIG_SMEM_MAX_N) {
        j.work = ws + off;
        off += 2 * (int64_t)n[i] * (n[i] + 1);
      }
      jobs.push_back(j);
    }
    launch_eig(jobs, st);
    if (ws) SYS_CK(cudaFreeAsync(ws, st));
    return DMRG_OK;
  } catch (const std::logic_error&) {
    return DMRG_EINVAL;
  } catch (const std::exception&) {
    return DMRG_ECUDA;
  }
}

}  // extern "C"
