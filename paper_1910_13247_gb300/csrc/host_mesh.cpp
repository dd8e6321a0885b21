// Octree meshes on the host: validation, cell order, DoF numbering and
// hanging-node / Dirichlet constraints (Sec. 3.1 local refinement with
// hanging nodes, Fig. 2; Sec. 3.3).
//
// Rules (shared with the mesh description in include/mfx.h):
//  * leaves tile the coarse box and are 2:1 balanced across faces and edges;
//  * cell order: coarse cell lexicographic, then Morton order of the
//    leaf's lower corner at the finest level (x bit lowest);
//  * a node is identified per dimension by its exact position: a rational
//    position for GLL nodes 0, 1/2 (even k) and 1, otherwise the triple
//    (level, cell index, local node); DoFs are numbered on first encounter;
//  * hanging nodes: nodes of a finer leaf lying on a face or an edge of a
//    coarser leaf without being one of its nodes get the coarse face (edge)
//    Lagrange interpolation weights; Dirichlet (box boundary) wins; zero
//    weights and Dirichlet masters are dropped; masters sorted by DoF.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <unordered_map>
#include <utility>

#include "mfx_internal.h"

namespace mfx {

namespace {

inline uint64_t leaf_key(int L, int64_t i, int64_t j, int64_t l) {
  return ((uint64_t)L << 60) | ((uint64_t)i << 40) | ((uint64_t)j << 20) | (uint64_t)l;
}

struct Octree {
  int nx, ny, nz, Lmax;
  std::vector<std::array<int32_t, 4>> leaves;
  std::unordered_map<uint64_t, int32_t> index;

  int64_t extent(int d, int L) const { return (int64_t)(d == 0 ? nx : d == 1 ? ny : nz) << L; }

  // Leaf of level <= L covering the level-L cell p, or -1 if p is inside the box and refined
  // deeper, or -2 if p is outside the box.
  int32_t covering(int L, const int64_t p[3]) const {
    for (int d = 0; d < 3; ++d)
      if (p[d] < 0 || p[d] >= extent(d, L)) return -2;
    for (int Lc = L; Lc >= 0; --Lc) {
      const int sh = L - Lc;
      auto it = index.find(leaf_key(Lc, p[0] >> sh, p[1] >> sh, p[2] >> sh));
      if (it != index.end()) return it->second;
    }
    return -1;
  }
};

uint64_t morton(uint64_t x, uint64_t y, uint64_t z, int bits) {
  uint64_t m = 0;
  for (int b = 0; b < bits; ++b) {
    m |= ((x >> b) & 1) << (3 * b);
    m |= ((y >> b) & 1) << (3 * b + 1);
    m |= ((z >> b) & 1) << (3 * b + 2);
  }
  return m;
}

mfx_status build(const Mesh& m, Octree* t) {
  t->nx = m.nx;
  t->ny = m.ny;
  t->nz = m.nz;
  const size_t nl = m.leaves.size() / 4;
  t->leaves.resize(nl);
  t->Lmax = 0;
  for (size_t q = 0; q < nl; ++q) {
    for (int c = 0; c < 4; ++c) t->leaves[q][c] = m.leaves[4 * q + c];
    t->Lmax = std::max(t->Lmax, t->leaves[q][0]);
  }
  t->index.reserve(nl * 2);
  for (size_t q = 0; q < nl; ++q) t->index[leaf_key(t->leaves[q][0], t->leaves[q][1], t->leaves[q][2], t->leaves[q][3])] = (int32_t)q;
  return MFX_OK;
}

}  // namespace

mfx_status octree_sort_and_check(Mesh* m) {
  const size_t nl = m->leaves.size() / 4;
  int Lmax = 0;
  for (size_t q = 0; q < nl; ++q) {
    const int L = m->leaves[4 * q];
    if (L < 0 || L > 8) return set_error(MFX_EMESH, "leaf level out of range 0..8");
    const int64_t e[3] = {(int64_t)m->nx << L, (int64_t)m->ny << L, (int64_t)m->nz << L};
    for (int d = 0; d < 3; ++d) {
      const int64_t v = m->leaves[4 * q + 1 + d];
      if (v < 0 || v >= e[d]) return set_error(MFX_EMESH, "leaf index out of range");
    }
    Lmax = std::max(Lmax, L);
  }
  Octree t;
  build(*m, &t);
  if (t.index.size() != nl) return set_error(MFX_EMESH, "duplicate leaves");
  // disjoint: no leaf has a leaf ancestor; complete: volumes add up
  unsigned __int128 vol = 0;
  for (size_t q = 0; q < nl; ++q) {
    const auto& lf = t.leaves[q];
    for (int La = lf[0] - 1; La >= 0; --La) {
      const int sh = lf[0] - La;
      if (t.index.count(leaf_key(La, lf[1] >> sh, lf[2] >> sh, lf[3] >> sh)))
        return set_error(MFX_EMESH, "overlapping leaves");
    }
    vol += (unsigned __int128)1 << (3 * (Lmax - lf[0]));
  }
  if (vol != ((unsigned __int128)m->nx * m->ny * m->nz) << (3 * Lmax))
    return set_error(MFX_EMESH, "leaves do not cover the coarse box");
  // 2:1 balance: the same-size face and edge neighbours of every leaf are covered by
  // leaves at most one level coarser (finer neighbours are checked from their side)
  for (size_t q = 0; q < nl; ++q) {
    const auto& lf = t.leaves[q];
    const int L = lf[0];
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          const int nnz = (dx != 0) + (dy != 0) + (dz != 0);
          if (nnz == 0 || nnz == 3) continue;
          const int64_t p[3] = {lf[1] + dx, lf[2] + dy, lf[3] + dz};
          const int32_t c = t.covering(L, p);
          if (c >= 0 && t.leaves[c][0] < L - 1) return set_error(MFX_EMESH, "mesh is not 2:1 balanced across faces and edges");
        }
  }
  // cell order
  std::vector<std::pair<std::pair<int64_t, uint64_t>, size_t>> order(nl);
  for (size_t q = 0; q < nl; ++q) {
    const auto& lf = t.leaves[q];
    const int L = lf[0], sh = Lmax - L;
    const int64_t ci = lf[1] >> L, cj = lf[2] >> L, cl = lf[3] >> L;
    const uint64_t mo = morton((uint64_t)(lf[1] - (ci << L)) << sh, (uint64_t)(lf[2] - (cj << L)) << sh,
                               (uint64_t)(lf[3] - (cl << L)) << sh, Lmax);
    order[q] = {{ci + (int64_t)m->nx * (cj + (int64_t)m->ny * cl), mo}, q};
  }
  std::sort(order.begin(), order.end());
  std::vector<int32_t> sorted(4 * nl);
  for (size_t q = 0; q < nl; ++q)
    for (int c = 0; c < 4; ++c) sorted[4 * q + c] = t.leaves[order[q].second][c];
  m->leaves.swap(sorted);
  m->max_level = Lmax;
  return MFX_OK;
}

namespace {

// Per-dimension node identity packed in 32 bits: bit 31 clear -> rational position in units of
// 2^-(Lmax+1) coarse cells (GLL nodes 0, 1/2 and 1 of a cell); bit 31 set -> interior GLL node a of
// the level-L cell row I: (L << 27) | (I << 4) | a (I < 2^23, a < 16).
struct NodeKey {
  uint32_t d[3];
  bool operator==(const NodeKey& o) const { return d[0] == o.d[0] && d[1] == o.d[1] && d[2] == o.d[2]; }
};

inline bool irrational(uint32_t dk) { return (dk >> 31) != 0; }

// Flat open-addressing table NodeKey -> DoF (linear probing, power-of-two capacity); key and DoF share
// one 16-byte slot, so a probe touches one cache line.
class NodeTable {
 public:
  explicit NodeTable(size_t expected) {
    size_t cap = 16;
    while (cap < 2 * expected + 16) cap <<= 1;
    slots_.assign(cap, Slot{{~0u, ~0u, ~0u}, -1});
    mask_ = cap - 1;
  }
  size_t slot(const NodeKey& k) const { return hash(k) & mask_; }
  void prefetch(size_t h) const { __builtin_prefetch(&slots_[h]); }
  // DoF of the key (whose home slot is h), inserting `next` if absent; returns (dof, inserted).
  std::pair<int32_t, bool> find_or_insert(const NodeKey& k, size_t h, int32_t next) {
    for (;;) {
      Slot& s = slots_[h];
      if (s.dof < 0) {
        s.key = k;
        s.dof = next;
        return {next, true};
      }
      if (s.key == k) return {s.dof, false};
      h = (h + 1) & mask_;
    }
  }

 private:
  static size_t hash(const NodeKey& k) {
    uint64_t x = ((uint64_t)k.d[0] << 32) ^ ((uint64_t)k.d[1] * 0x9E3779B97F4A7C15ull) ^ (uint64_t)k.d[2];
    x ^= x >> 30;
    x *= 0xbf58476d1ce4e5b9ull;
    x ^= x >> 27;
    x *= 0x94d049bb133111ebull;
    x ^= x >> 31;
    return (size_t)x;
  }
  struct Slot {
    NodeKey key;
    int32_t dof;
  };
  std::vector<Slot> slots_;
  size_t mask_ = 0;
};

}  // namespace

mfx_status octree_tables(const Mesh& m, int k, OctreeTables* out) {
  Octree t;
  build(m, &t);
  const int Lmax = m.max_level;
  const int n = k + 1, n3 = n * n * n;
  const int64_t C = (int64_t)t.leaves.size();
  double g[kMaxN];
  gauss_lobatto(k, g);
  out->n_cells = C;
  out->cell_vertices.assign(C * 24, 0.0);
  // vertices: trilinear map of the coarse cell at the leaf's reference corners
  for (int64_t c = 0; c < C; ++c) {
    const auto& lf = t.leaves[c];
    const int L = lf[0];
    const int64_t ci = lf[1] >> L, cj = lf[2] >> L, cl = lf[3] >> L;
    double X[8][3];
    for (int w = 0; w < 8; ++w) {
      const int a = w & 1, b = (w >> 1) & 1, e = (w >> 2) & 1;
      const size_t vi = (ci + a) + (size_t)(m.nx + 1) * ((cj + b) + (size_t)(m.ny + 1) * (cl + e));
      for (int d = 0; d < 3; ++d) X[w][d] = m.vertices[3 * vi + d];
    }
    for (int v = 0; v < 8; ++v) {
      const int a = v & 1, b = (v >> 1) & 1, e = (v >> 2) & 1;
      const double s = (double)((lf[1] - (ci << L)) + a) / (double)(1 << L);
      const double tt = (double)((lf[2] - (cj << L)) + b) / (double)(1 << L);
      const double u = (double)((lf[3] - (cl << L)) + e) / (double)(1 << L);
      double p[3] = {0, 0, 0};
      for (int w = 0; w < 8; ++w) {
        const int wa = w & 1, wb = (w >> 1) & 1, we = (w >> 2) & 1;
        const double f = (wa ? s : 1 - s) * (wb ? tt : 1 - tt) * (we ? u : 1 - u);
        for (int d = 0; d < 3; ++d) p[d] = p[d] + f * X[w][d];
      }
      for (int d = 0; d < 3; ++d) out->cell_vertices[c * 24 + 3 * v + d] = p[d];
    }
  }
  const uint32_t R2 = 1u << (Lmax + 1);
  if ((uint64_t)std::max(m.nx, std::max(m.ny, m.nz)) * R2 >= (1ull << 31) ||
      ((uint64_t)std::max(m.nx, std::max(m.ny, m.nz)) << Lmax) >= (1ull << 23))
    return set_error(MFX_EUNSUPPORTED, "octree too large for the node keys");
  auto dim_key = [&](int L, int64_t I, int a) -> uint32_t {
    if (a == 0) return (uint32_t)(I * (R2 >> L));
    if (a == k) return (uint32_t)((I + 1) * (R2 >> L));
    if (2 * a == k) return (uint32_t)((2 * I + 1) * (R2 >> (L + 1)));
    return (1u << 31) | ((uint32_t)L << 27) | ((uint32_t)I << 4) | (uint32_t)a;
  };
  auto node_key = [&](int64_t c, int a1, int a2, int a3) {
    const auto& lf = t.leaves[c];
    NodeKey key;
    key.d[0] = dim_key(lf[0], lf[1], a1);
    key.d[1] = dim_key(lf[0], lf[2], a2);
    key.d[2] = dim_key(lf[0], lf[3], a3);
    return key;
  };
  // nodes whose three per-dimension keys are all interior GLL nodes belong to one cell only
  int interior_1d = 0;
  for (int a = 0; a <= k; ++a)
    if (a != 0 && a != k && 2 * a != k) ++interior_1d;
  // shared (non-interior) node visits; each distinct shared node is visited about twice or more
  const size_t shared_visits = (size_t)C * (size_t)(n3 - interior_1d * interior_1d * interior_1d);
  NodeTable dof_of(shared_visits / 2 + 64);
  out->cell_dofs.assign(C * n3, 0);
  std::vector<NodeKey> keys_by_dof;
  keys_by_dof.reserve((size_t)C * n3 / 2 + 16);
  // keys of one cell, with their home slots prefetched before the (sequential) first-encounter pass
  std::vector<NodeKey> ck(n3);
  std::vector<size_t> cs(n3);
  for (int64_t c = 0; c < C; ++c) {
    for (int a3 = 0; a3 < n; ++a3)
      for (int a2 = 0; a2 < n; ++a2)
        for (int a1 = 0; a1 < n; ++a1) {
          const int li = a1 + n * (a2 + n * a3);
          ck[li] = node_key(c, a1, a2, a3);
          cs[li] = dof_of.slot(ck[li]);
          dof_of.prefetch(cs[li]);
        }
    for (int li = 0; li < n3; ++li) {
      const NodeKey& key = ck[li];
      if (keys_by_dof.size() >= (size_t)INT32_MAX) return set_error(MFX_EUNSUPPORTED, "more than 2^31 - 1 DoFs");
      const int32_t next = (int32_t)keys_by_dof.size();
      int32_t dof = next;
      if (!(irrational(key.d[0]) && irrational(key.d[1]) && irrational(key.d[2]))) {
        auto r = dof_of.find_or_insert(key, cs[li], next);
        dof = r.first;
        if (r.second) keys_by_dof.push_back(key);
      } else {
        keys_by_dof.push_back(key);
      }
      out->cell_dofs[c * n3 + li] = dof;
    }
  }
  const int64_t N = (int64_t)keys_by_dof.size();
  out->n_dofs = N;
  const uint32_t ext[3] = {(uint32_t)m.nx * R2, (uint32_t)m.ny * R2, (uint32_t)m.nz * R2};
  std::vector<uint8_t> dirichlet(N, 0);
  for (int64_t d = 0; d < N; ++d)
    for (int e = 0; e < 3; ++e) {
      const uint32_t dk = keys_by_dof[d].d[e];
      if (!irrational(dk) && ((dk == 0 && (m.dirichlet >> (2 * e) & 1u)) || (dk == ext[e] && (m.dirichlet >> (2 * e + 1) & 1u))))
        dirichlet[d] = 1;
    }
  // hanging constraints
  std::unordered_map<int32_t, std::vector<std::pair<int32_t, double>>> hanging;
  hanging.reserve((size_t)C / 8 + 1024);  // hanging nodes lie on coarse-fine interfaces only
  // a hanging node is reached once per fine cell around it; the 2:1 balance makes every visit give the
  // same constraint, so the first one is kept and the others are skipped before their masters are formed
  std::vector<uint8_t> is_hanging(N, 0);
  auto known = [&](int32_t dof) { return dirichlet[dof] != 0 || is_hanging[dof] != 0; };
  // 1D weights of the constraints: W1[c][b][m] = l_m((c + x_b) / 2), the coarse basis at node b of half c
  std::vector<double> W1((size_t)2 * n * n);
  for (int c2 = 0; c2 < 2; ++c2)
    for (int b = 0; b < n; ++b)
      for (int mm = 0; mm < n; ++mm)
        W1[((size_t)c2 * n + b) * n + mm] = lagrange_value(n, g, mm, ((double)c2 + g[b]) * 0.5);
  auto add = [&](int32_t dof, std::vector<std::pair<int32_t, double>>& raw) -> mfx_status {
    if (dirichlet[dof]) return MFX_OK;
    std::vector<std::pair<int32_t, double>> clean;
    for (auto& mw : raw)
      if (mw.second != 0.0 && !dirichlet[mw.first]) clean.push_back(mw);
    std::sort(clean.begin(), clean.end());
    auto it = hanging.find(dof);
    if (it == hanging.end()) {
      hanging.emplace(dof, std::move(clean));
      is_hanging[dof] = 1;
      return MFX_OK;
    }
    const auto& old = it->second;
    bool same = old.size() == clean.size();
    for (size_t i = 0; same && i < old.size(); ++i)
      same = old[i].first == clean[i].first && std::fabs(old[i].second - clean[i].second) <= 1e-12;
    if (!same) return set_error(MFX_EMESH, "inconsistent hanging-node constraints");
    return MFX_OK;
  };
  // is the key a node of leaf c: every per-dimension key is one of c's per-dimension keys
  auto is_node_of = [&](int64_t c, const NodeKey& key) {
    const auto& lf = t.leaves[c];
    for (int e = 0; e < 3; ++e) {
      bool found = false;
      for (int a = 0; a < n && !found; ++a) found = dim_key(lf[0], lf[1 + e], a) == key.d[e];
      if (!found) return false;
    }
    return true;
  };
  std::vector<std::pair<int32_t, double>> raw;
  // tensor-product form: per fine cell, its hanging faces (with the coarse face's DoFs) and edges
  out->hface.assign(C, 0u);
  out->hedge.assign(C, 0u);
  std::unordered_map<int64_t, std::vector<int32_t>> face_dofs, edge_dofs;  // key: cell * 16 + face / edge
  for (int64_t c = 0; c < C; ++c) {
    const auto& lf = t.leaves[c];
    const int L = lf[0];
    // a leaf of the finest level has no finer neighbour: none of its faces or edges is refined across
    if (L == Lmax) continue;
    const int64_t idx[3] = {lf[1], lf[2], lf[3]};
    // faces
    for (int d = 0; d < 3; ++d) {
      const int u = d == 0 ? 1 : 0, v = d == 2 ? 1 : 2;
      for (int sd = 0; sd < 2; ++sd) {
        int64_t p[3] = {idx[0], idx[1], idx[2]};
        p[d] += sd ? 1 : -1;
        if (t.covering(L, p) != -1) continue;  // not refined across this face
        for (int cv = 0; cv < 2; ++cv)
          for (int cu = 0; cu < 2; ++cu) {
            int64_t f[3];
            f[d] = 2 * p[d] + (sd ? 0 : 1);
            f[u] = 2 * idx[u] + cu;
            f[v] = 2 * idx[v] + cv;
            auto it = t.index.find(leaf_key(L + 1, f[0], f[1], f[2]));
            if (it == t.index.end()) return set_error(MFX_EMESH, "mesh is not 2:1 balanced");
            const int64_t e = it->second;
            const int ae_d = sd ? 0 : k, ac_d = sd ? k : 0;
            {
              const int fe = 2 * d + (sd ? 0 : 1);  // the fine cell's face on the coarse face
              out->hface[e] |= (1u << fe) | ((uint32_t)cu << (6 + 2 * fe)) | ((uint32_t)cv << (7 + 2 * fe));
              std::vector<int32_t>& fd = face_dofs[e * 16 + fe];
              if (fd.empty()) {
                fd.resize((size_t)n * n);
                for (int mv = 0; mv < n; ++mv)
                  for (int mu = 0; mu < n; ++mu) {
                    int ac[3];
                    ac[d] = ac_d;
                    ac[u] = mu;
                    ac[v] = mv;
                    fd[mu + n * mv] = out->cell_dofs[c * n3 + ac[0] + n * (ac[1] + n * ac[2])];
                  }
              }
            }
            for (int bv = 0; bv < n; ++bv)
              for (int bu = 0; bu < n; ++bu) {
                int ae[3];
                ae[d] = ae_d;
                ae[u] = bu;
                ae[v] = bv;
                const int li = ae[0] + n * (ae[1] + n * ae[2]);
                if (known(out->cell_dofs[e * n3 + li])) continue;
                if (is_node_of(c, node_key(e, ae[0], ae[1], ae[2]))) continue;
                const double* Wu = &W1[((size_t)cu * n + bu) * n];
                const double* Wv = &W1[((size_t)cv * n + bv) * n];
                raw.clear();
                for (int mv = 0; mv < n; ++mv)
                  for (int mu = 0; mu < n; ++mu) {
                    int ac[3];
                    ac[d] = ac_d;
                    ac[u] = mu;
                    ac[v] = mv;
                    const double w = Wu[mu] * Wv[mv];
                    raw.push_back({out->cell_dofs[c * n3 + ac[0] + n * (ac[1] + n * ac[2])], w});
                  }
                mfx_status st = add(out->cell_dofs[e * n3 + li], raw);
                if (st != MFX_OK) return st;
              }
          }
      }
    }
    // edges along d at sides (su, sv) of the two other dimensions
    for (int d = 0; d < 3; ++d) {
      const int u = d == 0 ? 1 : 0, v = d == 2 ? 1 : 2;
      for (int sv = 0; sv < 2; ++sv)
        for (int su = 0; su < 2; ++su) {
          // the three other cells around the edge
          const int64_t du = su ? 1 : -1, dv = sv ? 1 : -1;
          const int64_t offs[3][2] = {{du, 0}, {0, dv}, {du, dv}};
          for (auto& o : offs) {
            int64_t p[3] = {idx[0], idx[1], idx[2]};
            p[u] += o[0];
            p[v] += o[1];
            if (t.covering(L, p) != -1) continue;
            // the two children of p along d that touch our edge
            for (int cd = 0; cd < 2; ++cd) {
              int64_t f[3];
              f[d] = 2 * idx[d] + cd;
              f[u] = 2 * p[u] + (o[0] == 0 ? su : (su ? 0 : 1));
              f[v] = 2 * p[v] + (o[1] == 0 ? sv : (sv ? 0 : 1));
              auto it = t.index.find(leaf_key(L + 1, f[0], f[1], f[2]));
              if (it == t.index.end()) return set_error(MFX_EMESH, "mesh is not 2:1 balanced");
              const int64_t e = it->second;
              // position of the edge line in the fine leaf
              const int64_t edge_u = 2 * (idx[u] + su), edge_v = 2 * (idx[v] + sv);
              const int au = edge_u == f[u] ? 0 : k, av = edge_v == f[v] ? 0 : k;
              {
                const int ee = 4 * d + 2 * (av == k ? 1 : 0) + (au == k ? 1 : 0);
                if (!(out->hedge[e] >> ee & 1u)) {
                  out->hedge[e] |= (1u << ee) | ((uint32_t)cd << (12 + ee));
                  std::vector<int32_t>& ed = edge_dofs[e * 16 + ee];
                  ed.resize(n);
                  for (int md = 0; md < n; ++md) {
                    int ac[3];
                    ac[d] = md;
                    ac[u] = su * k;
                    ac[v] = sv * k;
                    ed[md] = out->cell_dofs[c * n3 + ac[0] + n * (ac[1] + n * ac[2])];
                  }
                }
              }
              for (int bd = 0; bd < n; ++bd) {
                int ae[3];
                ae[d] = bd;
                ae[u] = au;
                ae[v] = av;
                const int li = ae[0] + n * (ae[1] + n * ae[2]);
                if (known(out->cell_dofs[e * n3 + li])) continue;
                if (is_node_of(c, node_key(e, ae[0], ae[1], ae[2]))) continue;
                const double* Wd = &W1[((size_t)cd * n + bd) * n];
                raw.clear();
                for (int md = 0; md < n; ++md) {
                  int ac[3];
                  ac[d] = md;
                  ac[u] = su * k;
                  ac[v] = sv * k;
                  raw.push_back({out->cell_dofs[c * n3 + ac[0] + n * (ac[1] + n * ac[2])], Wd[md]});
                }
                mfx_status st = add(out->cell_dofs[e * n3 + li], raw);
                if (st != MFX_OK) return st;
              }
            }
          }
        }
    }
  }
  // compact per-cell lists; an edge on a hanging face of the same cell is left to the face
  out->hoff.assign(C, 0);
  out->hdofs.clear();
  auto coarse = [&](int32_t dof) { return (dirichlet[dof] || is_hanging[dof]) ? -1 : dof; };
  for (int64_t c = 0; c < C; ++c) {
    out->hoff[c] = (int64_t)out->hdofs.size();
    const uint32_t hf = out->hface[c] & 0x3Fu;
    uint32_t keep = 0u;
    for (int ee = 0; ee < 12; ++ee) {
      if (!(out->hedge[c] >> ee & 1u)) continue;
      const int d = ee >> 2, u = d == 0 ? 1 : 0, v = d == 2 ? 1 : 2;
      const int su = ee & 1, sv = (ee >> 1) & 1;
      if ((hf >> (2 * u + su) & 1u) || (hf >> (2 * v + sv) & 1u)) continue;
      keep |= 1u << ee;
    }
    out->hedge[c] = keep | (out->hedge[c] & (keep << 12));
    for (int f = 0; f < 6; ++f)
      if (hf >> f & 1u)
        for (int32_t dof : face_dofs[c * 16 + f]) out->hdofs.push_back(coarse(dof));
    for (int ee = 0; ee < 12; ++ee)
      if (keep >> ee & 1u)
        for (int32_t dof : edge_dofs[c * 16 + ee]) out->hdofs.push_back(coarse(dof));
  }
  out->constrained.clear();
  size_t n_masters = 0;
  for (int64_t d = 0; d < N; ++d)
    if (dirichlet[d] || is_hanging[d]) out->constrained.push_back((int32_t)d);
  for (auto& h : hanging) n_masters += h.second.size();
  out->cptr.assign(1, 0);
  out->cptr.reserve(out->constrained.size() + 1);
  out->cmaster.clear();
  out->cweight.clear();
  out->cmaster.reserve(n_masters);
  out->cweight.reserve(n_masters);
  for (int32_t d : out->constrained) {
    auto it = is_hanging[d] ? hanging.find(d) : hanging.end();
    if (it != hanging.end())
      for (auto& mw : it->second) {
        if (is_hanging[mw.first]) return set_error(MFX_EMESH, "constraint master is itself constrained");
        out->cmaster.push_back(mw.first);
        out->cweight.push_back(mw.second);
      }
    out->cptr.push_back((int64_t)out->cmaster.size());
  }
  return MFX_OK;
}

}  // namespace mfx
