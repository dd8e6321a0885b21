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
#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <utility>

#include "mfx_internal.h"

namespace mfx {

namespace {

uint64_t morton(uint64_t x, uint64_t y, uint64_t z, int bits) {
  uint64_t m = 0;
  for (int b = 0; b < bits; ++b) {
    m |= ((x >> b) & 1) << (3 * b);
    m |= ((y >> b) & 1) << (3 * b + 1);
    m |= ((z >> b) & 1) << (3 * b + 2);
  }
  return m;
}

// f(lo, hi) on contiguous chunks of [0, n), on up to 16 threads for large n
template <typename F>
void parallel_chunks(int64_t n, const F& f) {
  const int64_t grain = 1 << 16;
  const int hw = (int)std::max(1u, std::thread::hardware_concurrency());
  const int nt = (int)std::min<int64_t>(std::min(hw, 16), (n + grain - 1) / grain);
  if (nt <= 1) {
    if (n > 0) f((int64_t)0, n);
    return;
  }
  std::vector<std::thread> th;
  th.reserve(nt);
  for (int i = 0; i < nt; ++i) th.emplace_back([&f, i, nt, n] { f(n * i / nt, n * (i + 1) / nt); });
  for (auto& x : th) x.join();
}

// f(i) for i in [0, n) on up to 16 threads, each taking the next index when done (uneven work per index)
template <typename F>
void parallel_dynamic(int64_t n, const F& f) {
  const int hw = (int)std::max(1u, std::thread::hardware_concurrency());
  const int nt = (int)std::min<int64_t>(std::min(hw, 16), n);
  std::atomic<int64_t> next{0};
  auto work = [&] {
    for (int64_t i; (i = next.fetch_add(1)) < n;) f(i);
  };
  if (nt <= 1) {
    work();
    return;
  }
  std::vector<std::thread> th;
  th.reserve(nt);
  for (int i = 0; i < nt; ++i) th.emplace_back(work);
  for (auto& x : th) x.join();
}

// Sorted leaves with a point locator: leaves ordered by (coarse cell, Morton code of the lower corner at
// the finest level Lmax); the leaves of one coarse cell tile its Morton range [0, 8^Lmax), so the leaf
// containing a point is found by one binary search among the leaves of its coarse cell.
struct Octree {
  int nx, ny, nz, Lmax;
  std::vector<std::array<int32_t, 4>> leaves;
  std::vector<uint64_t> code;   // per leaf: Morton code of its lower corner at level Lmax
  std::vector<int64_t> first;   // per coarse cell: its first leaf (n_coarse + 1 entries)

  int64_t extent(int d, int L) const { return (int64_t)(d == 0 ? nx : d == 1 ? ny : nz) << L; }

  // coarse cell and Morton code at level Lmax of the lower corner of the level-L cell p (inside the box)
  void key_of(int L, const int64_t p[3], int64_t* cc, uint64_t* mo) const {
    const int64_t c0 = p[0] >> L, c1 = p[1] >> L, c2 = p[2] >> L;
    const int sh = Lmax - L;
    *cc = c0 + (int64_t)nx * (c1 + (int64_t)ny * c2);
    *mo = morton((uint64_t)(p[0] - (c0 << L)) << sh, (uint64_t)(p[1] - (c1 << L)) << sh,
                 (uint64_t)(p[2] - (c2 << L)) << sh, Lmax);
  }
  // the leaf containing the lower corner of the level-L cell p (L <= Lmax), or -2 if p is outside the box
  int32_t locate(int L, const int64_t p[3]) const {
    for (int d = 0; d < 3; ++d)
      if (p[d] < 0 || p[d] >= extent(d, L)) return -2;
    int64_t cc;
    uint64_t mo;
    key_of(L, p, &cc, &mo);
    const uint64_t* b = code.data() + first[cc];
    const uint64_t* e = code.data() + first[cc + 1];
    return (int32_t)(std::upper_bound(b, e, mo) - code.data() - 1);
  }
  // Leaf of level <= L covering the level-L cell p, or -1 if p is inside the box and refined
  // deeper, or -2 if p is outside the box.
  int32_t covering(int L, const int64_t p[3]) const {
    const int32_t q = locate(L, p);
    if (q < 0) return q;
    return leaves[q][0] <= L ? q : -1;
  }
  // some coarse cell across a face or an edge of the coarse cell c holds more than one leaf
  bool refined_near(const int64_t c[3]) const {
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          const int nnz = (dx != 0) + (dy != 0) + (dz != 0);
          if (nnz == 0 || nnz == 3) continue;
          const int64_t p[3] = {c[0] + dx, c[1] + dy, c[2] + dz};
          if (p[0] < 0 || p[0] >= nx || p[1] < 0 || p[1] >= ny || p[2] < 0 || p[2] >= nz) continue;
          const int64_t cc = p[0] + (int64_t)nx * (p[1] + (int64_t)ny * p[2]);
          if (first[cc + 1] - first[cc] > 1) return true;
        }
    return false;
  }
  // the leaf that is the level-L cell p, or -1
  int32_t exact(int L, const int64_t p[3]) const {
    const int32_t q = locate(L, p);
    return q >= 0 && leaves[q][0] == L ? q : -1;
  }
};

// the locator of leaves already sorted (octree_sort_and_check)
void build(const Mesh& m, Octree* t) {
  t->nx = m.nx;
  t->ny = m.ny;
  t->nz = m.nz;
  t->Lmax = m.max_level;
  const int64_t nl = (int64_t)m.leaves.size() / 4;
  t->leaves.resize(nl);
  t->code.resize(nl);
  const int64_t ncoarse = (int64_t)m.nx * m.ny * m.nz;
  t->first.assign(ncoarse + 1, nl);
  parallel_chunks(nl, [&](int64_t lo, int64_t hi) {
    for (int64_t q = lo; q < hi; ++q) {
      for (int c = 0; c < 4; ++c) t->leaves[q][c] = m.leaves[4 * q + c];
      const int64_t p[3] = {t->leaves[q][1], t->leaves[q][2], t->leaves[q][3]};
      int64_t cc;
      t->key_of(t->leaves[q][0], p, &cc, &t->code[q]);
    }
  });
  // first[cc]: the first leaf of coarse cell cc (leaves are grouped by coarse cell in increasing order)
  for (int64_t q = nl - 1; q >= 0; --q) {
    const auto& lf = t->leaves[q];
    const int L = lf[0];
    t->first[(lf[1] >> L) + (int64_t)m.nx * ((lf[2] >> L) + (int64_t)m.ny * (lf[3] >> L))] = q;
  }
  for (int64_t cc = ncoarse - 1; cc >= 0; --cc) t->first[cc] = std::min(t->first[cc], t->first[cc + 1]);
}

}  // namespace

mfx_status octree_sort_and_check(Mesh* m) {
  const int64_t nl = (int64_t)m->leaves.size() / 4;
  if (nl >= (int64_t)INT32_MAX) return set_error(MFX_EUNSUPPORTED, "more than 2^31 - 2 leaves");
  int Lmax = 0;
  for (int64_t q = 0; q < nl; ++q) {
    const int L = m->leaves[4 * q];
    if (L < 0 || L > 8) return set_error(MFX_EMESH, "leaf level out of range 0..8");
    const int64_t e[3] = {(int64_t)m->nx << L, (int64_t)m->ny << L, (int64_t)m->nz << L};
    for (int d = 0; d < 3; ++d) {
      const int64_t v = m->leaves[4 * q + 1 + d];
      if (v < 0 || v >= e[d]) return set_error(MFX_EMESH, "leaf index out of range");
    }
    Lmax = std::max(Lmax, L);
  }
  // cell order: coarse cell lexicographic, then Morton order of the lower corner at level Lmax
  // (every coarse cell holds a leaf, so n_coarse <= n_leaves < 2^31 and the key (coarse cell, Morton code)
  // fits in 31 + 24 bits)
  const int64_t ncoarse = (int64_t)m->nx * m->ny * m->nz;
  if (ncoarse > nl) return set_error(MFX_EMESH, "leaves do not cover the coarse box");
  const int mbits = 3 * Lmax;
  std::vector<uint64_t> key(nl);
  parallel_chunks(nl, [&](int64_t lo, int64_t hi) {
    for (int64_t q = lo; q < hi; ++q) {
      const int32_t* lf = &m->leaves[4 * q];
      const int L = lf[0], sh = Lmax - L;
      const int64_t ci = lf[1] >> L, cj = lf[2] >> L, cl = lf[3] >> L;
      const uint64_t mo = morton((uint64_t)(lf[1] - (ci << L)) << sh, (uint64_t)(lf[2] - (cj << L)) << sh,
                                 (uint64_t)(lf[3] - (cl << L)) << sh, Lmax);
      key[q] = ((uint64_t)(ci + (int64_t)m->nx * (cj + (int64_t)m->ny * cl)) << mbits) | mo;
    }
  });
  // stable LSD radix sort of (key, leaf) by key, 11 bits per pass (equal keys keep input order)
  std::vector<int32_t> order(nl);
  for (int64_t q = 0; q < nl; ++q) order[q] = (int32_t)q;
  {
    int bits = mbits;
    while (bits < 64 && ((uint64_t)(ncoarse - 1) >> (bits - mbits)) != 0) ++bits;
    std::vector<uint64_t> key2(nl);
    std::vector<int32_t> order2(nl);
    std::vector<int64_t> cnt(2049);
    for (int shift = 0; shift < bits; shift += 11) {
      std::fill(cnt.begin(), cnt.end(), 0);
      for (int64_t q = 0; q < nl; ++q) ++cnt[((key[q] >> shift) & 2047) + 1];
      for (int i = 0; i < 2048; ++i) cnt[i + 1] += cnt[i];
      for (int64_t q = 0; q < nl; ++q) {
        const int64_t dst = cnt[(key[q] >> shift) & 2047]++;
        key2[dst] = key[q];
        order2[dst] = order[q];
      }
      key.swap(key2);
      order.swap(order2);
    }
  }
  // the leaves of every coarse cell tile its Morton range: each starts where the previous one ends
  // (a leaf of level L spans 8^(Lmax - L) codes), the first at 0 and the last ending at 8^Lmax
  const uint64_t full = 1ull << mbits;
  {
    int64_t q = 0;
    for (int64_t cc = 0; cc < ncoarse; ++cc) {
      uint64_t next = 0;
      for (; q < nl && (int64_t)(key[q] >> mbits) == cc; ++q) {
        const uint64_t mo = key[q] & (full - 1);
        const int L = m->leaves[4 * (int64_t)order[q]];
        if (mo > next) return set_error(MFX_EMESH, "leaves do not cover the coarse box");
        if (mo < next) {
          const bool dup = q > 0 && key[q - 1] == key[q] && m->leaves[4 * (int64_t)order[q - 1]] == L;
          return set_error(MFX_EMESH, dup ? "duplicate leaves" : "overlapping leaves");
        }
        next = mo + (1ull << (3 * (Lmax - L)));
      }
      if (next != full) return set_error(MFX_EMESH, "leaves do not cover the coarse box");
    }
  }
  key.clear();
  key.shrink_to_fit();
  std::vector<int32_t> sorted(4 * nl);
  parallel_chunks(nl, [&](int64_t lo, int64_t hi) {
    for (int64_t q = lo; q < hi; ++q)
      for (int c = 0; c < 4; ++c) sorted[4 * q + c] = m->leaves[4 * (int64_t)order[q] + c];
  });
  order.clear();
  order.shrink_to_fit();
  m->leaves.swap(sorted);
  m->max_level = Lmax;
  // 2:1 balance: the same-size face and edge neighbours of every leaf are covered by
  // leaves at most one level coarser (finer neighbours are checked from their side)
  Octree t;
  build(*m, &t);
  bool balanced = true;
  std::mutex mu;
  parallel_chunks(nl, [&](int64_t lo, int64_t hi) {
    for (int64_t q = lo; q < hi; ++q) {
      const auto& lf = t.leaves[q];
      const int L = lf[0];
      if (L < 2) continue;  // no leaf is coarser than level 0
      for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx) {
            const int nnz = (dx != 0) + (dy != 0) + (dz != 0);
            if (nnz == 0 || nnz == 3) continue;
            const int64_t p[3] = {lf[1] + dx, lf[2] + dy, lf[3] + dz};
            const int32_t c = t.covering(L, p);
            if (c >= 0 && t.leaves[c][0] < L - 1) {
              std::lock_guard<std::mutex> g(mu);
              balanced = false;
              return;
            }
          }
    }
  });
  if (!balanced) return set_error(MFX_EMESH, "mesh is not 2:1 balanced across faces and edges");
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

// Open-addressing table NodeKey -> (smallest visit, DoF) filled by several threads at once (linear
// probing, power-of-two capacity).  A slot is claimed by one compare-and-swap of its visit word (empty ->
// busy), its key written and the visit published; a thread that meets its key lowers the visit word to
// its own visit if that is smaller.  Readers compare keys only after seeing a published visit.
class VisitTable {
 public:
  static constexpr int64_t kEmpty = -1, kBusy = -2;
  explicit VisitTable(size_t cap) : slots_(cap), mask_(cap - 1) {
    for (auto& s : slots_) s.visit.store(kEmpty, std::memory_order_relaxed);
  }
  size_t capacity() const { return slots_.size(); }
  // slot of the key (whose home slot is h), inserted with `visit` if absent (*added: whether this call
  // inserted it); SIZE_MAX when every slot was probed (the table is full)
  size_t home(const NodeKey& k) const { return hash(k) & mask_; }
  void prefetch(size_t h) const { __builtin_prefetch(&slots_[h], 1); }
  size_t insert(const NodeKey& k, size_t h, int64_t visit, bool* added) {
    *added = false;
    for (size_t probes = 0; probes <= mask_;) {
      Slot& s = slots_[h];
      int64_t v = s.visit.load(std::memory_order_acquire);
      if (v == kEmpty) {
        if (s.visit.compare_exchange_strong(v, kBusy, std::memory_order_acq_rel)) {
          s.key = k;
          s.visit.store(visit, std::memory_order_release);
          *added = true;
          return h;
        }
        continue;  // claimed meanwhile: look at this slot again
      }
      if (v == kBusy) continue;  // its key is being written
      if (s.key == k) {
        while (visit < v && !s.visit.compare_exchange_weak(v, visit, std::memory_order_acq_rel)) {
        }
        return h;
      }
      h = (h + 1) & mask_;
      ++probes;
    }
    return SIZE_MAX;
  }
  int64_t visit(size_t h) const { return slots_[h].visit.load(std::memory_order_relaxed); }
  int32_t& dof(size_t h) { return slots_[h].dof; }

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
    std::atomic<int64_t> visit;
  };
  std::vector<Slot> slots_;
  size_t mask_;
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
  // DoF numbering in first-encounter order (the order of the visits c n^3 + li of the cells' local
  // nodes), on threads: (1) every visit of a shared node enters the table, which keeps the smallest
  // visit of each key; (2) per chunk of cells the first visits are counted (interior nodes belong to one
  // cell: each of their visits is a first one); (3) they are numbered in visit order, each chunk from the
  // sum of the counts before it; (4) the other visits read the number of their key.
  const int64_t nv = C * n3;
  out->cell_dofs.assign(nv, 0);
  constexpr uint32_t kNoSlot = 0xFFFFFFFFu;
  std::vector<uint32_t> vslot(nv);  // table slot of each visit, kNoSlot for interior nodes
  std::vector<uint8_t> first(nv);   // the visit is the first of its node
  auto interior_key = [](const NodeKey& key) {
    return irrational(key.d[0]) && irrational(key.d[1]) && irrational(key.d[2]);
  };
  // distinct shared nodes: about k^3 - interior_1d^3 per cell away from refinement interfaces; a table
  // that passes 70 % load is dropped and the pass repeated with twice the capacity
  size_t expect = (size_t)C * (size_t)std::max(1, k * k * k - interior_1d * interior_1d * interior_1d) + 1024;
  std::unique_ptr<VisitTable> table;
  for (;;) {
    size_t cap = 16;
    while (2 * cap < 3 * expect) cap <<= 1;
    if (cap > (size_t)kNoSlot) return set_error(MFX_EUNSUPPORTED, "octree too large for the node table");
    table.reset(new VisitTable(cap));
    std::atomic<size_t> inserted{0};
    std::atomic<bool> full{false};
    const size_t limit = cap / 10 * 7;
    parallel_chunks(C, [&](int64_t lo, int64_t hi) {
      // keys and home slots of the next D cells formed and prefetched ahead (a ring of D cells)
      const int D = std::max(2, 64 / n3);
      std::vector<NodeKey> ck((size_t)D * n3);
      std::vector<size_t> cs((size_t)D * n3);
      auto stage = [&](int64_t c) {
        const size_t o = (size_t)(c % D) * n3;
        for (int a3 = 0; a3 < n; ++a3)
          for (int a2 = 0; a2 < n; ++a2)
            for (int a1 = 0; a1 < n; ++a1) {
              const size_t li = o + a1 + n * (a2 + n * a3);
              ck[li] = node_key(c, a1, a2, a3);
              if (!interior_key(ck[li])) {
                cs[li] = table->home(ck[li]);
                table->prefetch(cs[li]);
              }
            }
      };
      for (int64_t c = lo; c < std::min<int64_t>(lo + D, hi); ++c) stage(c);
      size_t mine = 0;
      for (int64_t c = lo; c < hi; ++c) {
        const size_t o = (size_t)(c % D) * n3;
        for (int li = 0; li < n3; ++li) {
          const int64_t v = c * n3 + li;
          if (interior_key(ck[o + li])) {
            vslot[v] = kNoSlot;
            first[v] = 1;
            continue;
          }
          bool added;
          const size_t h = table->insert(ck[o + li], cs[o + li], v, &added);
          if (h == SIZE_MAX) {
            full.store(true);
            return;
          }
          vslot[v] = (uint32_t)h;
          mine += added ? 1 : 0;
        }
        if (c + D < hi) stage(c + D);
        // the shared count, at most every 64k node visits of this thread
        if (mine >= 65536 || (c + 1) % std::max<int64_t>(1, 65536 / n3) == 0 || c + 1 == hi) {
          if (inserted.fetch_add(mine) + mine > limit) full.store(true);
          mine = 0;
          if (full.load(std::memory_order_relaxed)) return;
        }
      }
    });
    if (!full.load()) break;
    expect *= 2;
  }
  // first visits of shared nodes: the smallest visit each slot of the table holds
  parallel_chunks((int64_t)table->capacity(), [&](int64_t lo, int64_t hi) {
    for (int64_t h = lo; h < hi; ++h) {
      const int64_t v = table->visit((size_t)h);
      if (v >= 0) first[v] = 1;
    }
  });
  auto is_first = [&](int64_t v) { return first[v] != 0; };
  const int64_t csz = std::max<int64_t>(4096, (C + 255) / 256);  // cells per chunk
  const int64_t nch = (C + csz - 1) / csz;
  std::vector<int64_t> base(nch + 1, 0);
  parallel_chunks(nch, [&](int64_t lo, int64_t hi) {
    for (int64_t ch = lo; ch < hi; ++ch) {
      int64_t cnt = 0;
      for (int64_t v = ch * csz * n3; v < std::min(C, (ch + 1) * csz) * n3; ++v) cnt += is_first(v) ? 1 : 0;
      base[ch + 1] = cnt;
    }
  });
  for (int64_t ch = 0; ch < nch; ++ch) base[ch + 1] += base[ch];
  if (base[nch] >= (int64_t)INT32_MAX) return set_error(MFX_EUNSUPPORTED, "more than 2^31 - 1 DoFs");
  std::vector<NodeKey> keys_by_dof(base[nch]);
  parallel_chunks(nch, [&](int64_t lo, int64_t hi) {
    for (int64_t ch = lo; ch < hi; ++ch) {
      int32_t next = (int32_t)base[ch];
      for (int64_t v = ch * csz * n3; v < std::min(C, (ch + 1) * csz) * n3; ++v) {
        if (!is_first(v)) continue;
        const int64_t c = v / n3;
        const int li = (int)(v - c * n3);
        keys_by_dof[next] = node_key(c, li % n, (li / n) % n, li / (n * n));
        if (vslot[v] != kNoSlot) table->dof(vslot[v]) = next;
        out->cell_dofs[v] = next++;
      }
    }
  });
  parallel_chunks(nv, [&](int64_t lo, int64_t hi) {
    for (int64_t v = lo; v < hi; ++v) {
      if (v + 32 < hi && !first[v + 32]) table->prefetch(vslot[v + 32]);
      if (!is_first(v)) out->cell_dofs[v] = table->dof(vslot[v]);
    }
  });
  table.reset();
  vslot.clear();
  vslot.shrink_to_fit();
  first.clear();
  first.shrink_to_fit();
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
  // hanging constraints, on threads: each part of the leaf range records the constraints of the hanging
  // nodes it reaches (every visit of a hanging node gives the same constraint under the 2:1 balance; a part
  // keeps its first visit, the merge keeps the first in leaf order and checks the others against it), and
  // the coarse DoFs of its fine cells' hanging faces and edges; the cells' face and edge words are set
  // with atomic ORs (an edge word's bits once, by the first visitor)
  // 1D weights of the constraints: W1[c][b][m] = l_m((c + x_b) / 2), the coarse basis at node b of half c
  std::vector<double> W1((size_t)2 * n * n);
  for (int c2 = 0; c2 < 2; ++c2)
    for (int b = 0; b < n; ++b)
      for (int mm = 0; mm < n; ++mm)
        W1[((size_t)c2 * n + b) * n + mm] = lagrange_value(n, g, mm, ((double)c2 + g[b]) * 0.5);
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
  out->hface.assign(C, 0u);
  out->hedge.assign(C, 0u);
  struct HangRec {
    int32_t dof;
    int64_t order;  // visit order: leaf * 4096 + visit within the leaf
    std::vector<std::pair<int32_t, double>> masters;
  };
  struct DofsRec {
    int64_t key;  // cell * 16 + face / edge
    std::vector<int32_t> dofs;
  };
  struct Scan {
    std::vector<HangRec> hang;
    std::vector<DofsRec> faces, edges;
    mfx_status st = MFX_OK;
    const char* msg = nullptr;
  };
  const int64_t nparts = std::max<int64_t>(1, std::min<int64_t>(256, C / 4096));
  std::vector<Scan> scans((size_t)nparts);
  parallel_dynamic(nparts, [&](int64_t part) {
    {
      Scan& sc = scans[part];
      std::unordered_set<int32_t> seen;  // hanging nodes this part has recorded
      std::vector<std::pair<int32_t, double>> raw;
      int64_t order = 0;
      auto known = [&](int32_t dof) { return dirichlet[dof] != 0 || seen.count(dof) != 0; };
      auto add = [&](int32_t dof, std::vector<std::pair<int32_t, double>>& masters) {
        std::vector<std::pair<int32_t, double>> clean;
        for (auto& mw : masters)
          if (mw.second != 0.0 && !dirichlet[mw.first]) clean.push_back(mw);
        std::sort(clean.begin(), clean.end());
        sc.hang.push_back({dof, order++, std::move(clean)});
        seen.insert(dof);
      };
      auto fail = [&](const char* m) {
        sc.st = MFX_EMESH;
        sc.msg = m;
      };
      for (int64_t c = C * part / nparts; c < C * (part + 1) / nparts && sc.st == MFX_OK; ++c) {
        order = c * 4096;
        const auto& lf = t.leaves[c];
        const int L = lf[0];
        // a leaf of the finest level has no finer neighbour: none of its faces or edges is refined across
        if (L == Lmax) continue;
        const int64_t idx[3] = {lf[1], lf[2], lf[3]};
        // a level-0 leaf is a whole coarse cell: it has a finer face or edge neighbour only if one of the
        // coarse cells across its faces and edges holds more than one leaf
        if (L == 0 && !t.refined_near(idx)) continue;
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
                const int32_t fe_leaf = t.exact(L + 1, f);
                if (fe_leaf < 0) {
                  fail("mesh is not 2:1 balanced");
                  break;
                }
                const int64_t e = fe_leaf;
                const int ae_d = sd ? 0 : k, ac_d = sd ? k : 0;
                {
                  const int fe = 2 * d + (sd ? 0 : 1);  // the fine cell's face on the coarse face
                  __atomic_fetch_or(&out->hface[e], (1u << fe) | ((uint32_t)cu << (6 + 2 * fe)) | ((uint32_t)cv << (7 + 2 * fe)),
                                    __ATOMIC_RELAXED);
                  {
                    sc.faces.push_back({e * 16 + fe, std::vector<int32_t>((size_t)n * n)});
                    std::vector<int32_t>& fd = sc.faces.back().dofs;
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
                    add(out->cell_dofs[e * n3 + li], raw);
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
                  const int32_t fe_leaf = t.exact(L + 1, f);
                  if (fe_leaf < 0) {
                  fail("mesh is not 2:1 balanced");
                  break;
                }
                  const int64_t e = fe_leaf;
                  // position of the edge line in the fine leaf
                  const int64_t edge_u = 2 * (idx[u] + su), edge_v = 2 * (idx[v] + sv);
                  const int au = edge_u == f[u] ? 0 : k, av = edge_v == f[v] ? 0 : k;
                  {
                    const int ee = 4 * d + 2 * (av == k ? 1 : 0) + (au == k ? 1 : 0);
                    const uint32_t bits = (1u << ee) | ((uint32_t)cd << (12 + ee));
                    uint32_t old = __atomic_load_n(&out->hedge[e], __ATOMIC_RELAXED);
                    bool mine = false;
                    while (!(old >> ee & 1u) &&
                           !(mine = __atomic_compare_exchange_n(&out->hedge[e], &old, old | bits, false, __ATOMIC_RELAXED,
                                                                __ATOMIC_RELAXED))) {
                    }
                    if (mine) {
                      sc.edges.push_back({e * 16 + ee, std::vector<int32_t>((size_t)n)});
                      std::vector<int32_t>& ed = sc.edges.back().dofs;
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
                    add(out->cell_dofs[e * n3 + li], raw);
                  }
                }
              }
            }
        }
  
      }
    }
  });
  for (const Scan& sc : scans)
    if (sc.st != MFX_OK) return set_error(sc.st, sc.msg);
  // merge: the first visit of each hanging node in leaf order, the others checked against it
  std::vector<HangRec> recs;
  for (Scan& sc : scans)
    for (HangRec& r : sc.hang) recs.push_back(std::move(r));
  std::sort(recs.begin(), recs.end(), [](const HangRec& x, const HangRec& y) {
    return x.dof != y.dof ? x.dof < y.dof : x.order < y.order;
  });
  std::unordered_map<int32_t, std::vector<std::pair<int32_t, double>>> hanging;
  hanging.reserve(recs.size());
  std::vector<uint8_t> is_hanging(N, 0);
  for (size_t i = 0; i < recs.size();) {
    size_t j = i + 1;
    for (; j < recs.size() && recs[j].dof == recs[i].dof; ++j) {
      const auto& x = recs[i].masters;
      const auto& y = recs[j].masters;
      bool same = x.size() == y.size();
      for (size_t q = 0; same && q < x.size(); ++q)
        same = x[q].first == y[q].first && std::fabs(x[q].second - y[q].second) <= 1e-12;
      if (!same) return set_error(MFX_EMESH, "inconsistent hanging-node constraints");
    }
    is_hanging[recs[i].dof] = 1;
    hanging.emplace(recs[i].dof, std::move(recs[i].masters));
    i = j;
  }
  recs.clear();
  // the coarse DoFs of the hanging faces and edges, sorted by (cell, face / edge)
  std::vector<DofsRec> face_dofs, edge_dofs;
  for (Scan& sc : scans) {
    for (DofsRec& r : sc.faces) face_dofs.push_back(std::move(r));
    for (DofsRec& r : sc.edges) edge_dofs.push_back(std::move(r));
  }
  scans.clear();
  auto by_key = [](const DofsRec& x, const DofsRec& y) { return x.key < y.key; };
  std::sort(face_dofs.begin(), face_dofs.end(), by_key);
  std::sort(edge_dofs.begin(), edge_dofs.end(), by_key);
  auto first_at = [](const std::vector<DofsRec>& v, int64_t key) {
    return (size_t)(std::lower_bound(v.begin(), v.end(), key,
                                     [](const DofsRec& r, int64_t k2) { return r.key < k2; }) -
                    v.begin());
  };
  // compact per-cell lists; an edge on a hanging face of the same cell is left to the face.  Per chunk of
  // cells: the kept edges and the list lengths, then (after the prefix over the cells) the lists
  auto coarse = [&](int32_t dof) { return (dirichlet[dof] || is_hanging[dof]) ? -1 : dof; };
  out->hoff.assign(C, 0);
  const int64_t nn = (int64_t)n * n;
  parallel_chunks(C, [&](int64_t lo, int64_t hi) {
    for (int64_t c = lo; c < hi; ++c) {
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
      out->hoff[c] = nn * __builtin_popcount(hf) + (int64_t)n * __builtin_popcount(keep);
    }
  });
  int64_t total = 0;
  for (int64_t c = 0; c < C; ++c) {  // exclusive prefix
    const int64_t len = out->hoff[c];
    out->hoff[c] = total;
    total += len;
  }
  out->hdofs.assign((size_t)total, 0);
  parallel_chunks(C, [&](int64_t lo, int64_t hi) {
    size_t fi = first_at(face_dofs, lo * 16), ei = first_at(edge_dofs, lo * 16);
    for (int64_t c = lo; c < hi; ++c) {
      int64_t o = out->hoff[c];
      for (; fi < face_dofs.size() && face_dofs[fi].key < (c + 1) * 16; ++fi)
        if (out->hface[c] >> (face_dofs[fi].key - c * 16) & 1u)
          for (int32_t dof : face_dofs[fi].dofs) out->hdofs[o++] = coarse(dof);
      for (; ei < edge_dofs.size() && edge_dofs[ei].key < (c + 1) * 16; ++ei)
        if (out->hedge[c] >> (edge_dofs[ei].key - c * 16) & 1u)
          for (int32_t dof : edge_dofs[ei].dofs) out->hdofs[o++] = coarse(dof);
    }
  });
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
