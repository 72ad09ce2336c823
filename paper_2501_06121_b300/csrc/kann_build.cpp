// kann_build.cpp -- multi-threaded host construction of the HNSW graph that
// the device search consumes (the paper's indexing pipeline, Sec. 2 / Fig. 1,
// with HNSW per Malkov & Yashunin).  Search treats the graph as a fixed
// input; this builder exists so that a user (and the benchmark) can make one.
//
// Insertion follows Malkov & Yashunin Alg. 1 with the neighbour-selection
// heuristic of Alg. 4: greedy descent to the node's top layer, then per layer
// an efConstruction-wide beam, heuristic selection of M neighbours, links in
// both directions, and heuristic shrinking of a neighbour's overfull list
// (caps M on upper layers, 2M on layer 0).  Nodes are inserted by `nthreads`
// workers under per-node locks, so with more than one thread the edge set
// depends on scheduling (the levels never do: they are a pure function of
// (seed, id)).  Distances are FP32.
#include <atomic>
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/kann.h"

namespace {

struct DC {
  float d;
  int32_t id;
};
inline bool dc_less(const DC& a, const DC& b) {
  float da = std::isnan(a.d) ? INFINITY : a.d, db = std::isnan(b.d) ? INFINITY : b.d;
  return da < db || (da == db && a.id < b.id);
}
struct DCLess {
  bool operator()(const DC& a, const DC& b) const { return dc_less(a, b); }
};
struct DCGreater {
  bool operator()(const DC& a, const DC& b) const { return dc_less(b, a); }
};

// ---- levels: floor(-ln U / ln M), U = (u53 + 1) / 2^53 from one SplitMix64
// step (Steele, Lea & Flood) out of state seed ^ id * golden-gamma.
uint64_t mix_step(uint64_t state) {
  uint64_t z = state + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

int node_level(uint64_t seed, uint64_t id, int M) {
  const uint64_t u = mix_step(seed ^ (id * 0x9E3779B97F4A7C15ULL)) >> 11;
  const double U = ((double)u + 1.0) / 9007199254740992.0;
  double l = std::floor(-std::log(U) / std::log((double)M));
  return l > 60 ? 60 : (int)l;
}

// ---- distance spaces --------------------------------------------------------
__attribute__((target_clones("avx512f", "avx2", "default")))
float l2_f32(const float* a, const float* b, int d) {
  float s = 0.f;
  for (int i = 0; i < d; ++i) {
    float t = a[i] - b[i];
    s += t * t;
  }
  return s;
}

__attribute__((target_clones("avx512f", "avx2", "default")))
float dot_f32(const float* a, const float* b, int d) {
  float s = 0.f;
  for (int i = 0; i < d; ++i) s += a[i] * b[i];
  return s;
}

struct DenseSpace {
  const float* x;
  int d, metric;
  float dist(const float* q, int32_t j) const {
    const float* r = x + (size_t)j * d;
    return metric == KANN_L2 ? l2_f32(q, r, d) : -dot_f32(q, r, d);
  }
  float ndist(int32_t a, int32_t b) const { return dist(x + (size_t)a * d, b); }
  const float* item(int32_t a) const { return x + (size_t)a * d; }
};

struct SparseSpace {
  const int64_t* ip;
  const uint16_t* t;
  const float* w;
  struct Item {
    int64_t b, e;
  };
  float dot(int64_t ab, int64_t ae, int64_t bb, int64_t be) const {
    float s = 0.f;
    while (ab < ae && bb < be) {
      if (t[ab] < t[bb]) ++ab;
      else if (t[ab] > t[bb]) ++bb;
      else s += w[ab++] * w[bb++];
    }
    return s;
  }
  float dist(const Item& q, int32_t j) const { return -dot(q.b, q.e, ip[j], ip[j + 1]); }
  float ndist(int32_t a, int32_t b) const { return -dot(ip[a], ip[a + 1], ip[b], ip[b + 1]); }
  Item item(int32_t a) const { return Item{ip[a], ip[a + 1]}; }
};

// ---- the graph under construction -----------------------------------------
struct Builder {
  int64_t n;
  int M, M0, L, efc;
  const int8_t* level;
  int32_t* l0;
  int32_t* upper_slot;
  int32_t* upper;
  std::vector<int32_t> cnt0;                 // layer-0 list lengths
  std::vector<int32_t> cntu;                 // [n_upper][L] upper list lengths
  std::vector<std::mutex> locks;
  std::mutex entry_lock;
  std::atomic<int32_t> entry{-1};
  std::atomic<int> top{-1};

  int32_t* list(int32_t v, int l) {
    return l == 0 ? l0 + (size_t)v * M0 : upper + ((size_t)upper_slot[v] * L + (l - 1)) * M;
  }
  int32_t& count(int32_t v, int l) { return l == 0 ? cnt0[v] : cntu[(size_t)upper_slot[v] * L + (l - 1)]; }
  int cap(int l) const { return l == 0 ? M0 : M; }

  void copy_list(int32_t v, int l, std::vector<int32_t>& out) {
    std::lock_guard<std::mutex> g(locks[v]);
    const int c = count(v, l);
    out.assign(list(v, l), list(v, l) + c);
  }
};

struct Visited {
  std::vector<uint32_t> tag;
  uint32_t epoch = 0;
  explicit Visited(int64_t n) : tag(n, 0) {}
  void next() {
    if (++epoch == 0) {
      std::fill(tag.begin(), tag.end(), 0);
      epoch = 1;
    }
  }
  bool test_set(int32_t v) {
    if (tag[v] == epoch) return true;
    tag[v] = epoch;
    return false;
  }
};

template <class S, class Q>
std::vector<DC> search_layer(Builder& B, const S& sp, const Q& q, int32_t self, const std::vector<DC>& eps, int ef,
                             int l, Visited& vis, std::vector<int32_t>& buf) {
  vis.next();
  // the node being inserted is never its own candidate: a concurrent insertion
  // may already have linked to it on this layer
  vis.test_set(self);
  std::vector<DC> C, W;  // C: min-heap, W: max-heap
  for (const DC& e : eps) {
    if (vis.test_set(e.id)) continue;
    C.push_back(e);
    std::push_heap(C.begin(), C.end(), DCGreater());
    W.push_back(e);
    std::push_heap(W.begin(), W.end(), DCLess());
  }
  while ((int)W.size() > ef) {
    std::pop_heap(W.begin(), W.end(), DCLess());
    W.pop_back();
  }
  while (!C.empty()) {
    DC c = C.front();
    std::pop_heap(C.begin(), C.end(), DCGreater());
    C.pop_back();
    if (dc_less(W.front(), c)) break;
    B.copy_list(c.id, l, buf);
    for (int32_t e : buf) {
      if (vis.test_set(e)) continue;
      DC ce{sp.dist(q, e), e};
      if ((int)W.size() < ef || dc_less(ce, W.front())) {
        C.push_back(ce);
        std::push_heap(C.begin(), C.end(), DCGreater());
        W.push_back(ce);
        std::push_heap(W.begin(), W.end(), DCLess());
        if ((int)W.size() > ef) {
          std::pop_heap(W.begin(), W.end(), DCLess());
          W.pop_back();
        }
      }
    }
  }
  std::sort(W.begin(), W.end(), DCLess());
  return W;
}

template <class S>
std::vector<DC> heuristic(const S& sp, std::vector<DC> cands, int cap) {
  std::sort(cands.begin(), cands.end(), DCLess());
  std::vector<DC> R;
  for (const DC& e : cands) {
    if ((int)R.size() >= cap) break;
    bool good = true;
    for (const DC& r : R)
      if (!(e.d < sp.ndist(e.id, r.id))) {
        good = false;
        break;
      }
    if (good) R.push_back(e);
  }
  return R;
}

template <class S>
void insert(Builder& B, const S& sp, int32_t i, Visited& vis, std::vector<int32_t>& buf) {
  const int li = B.level[i];
  const auto q = sp.item(i);
  // A node whose level is above the current top keeps the entry lock for its
  // whole insertion: a second such node inserted meanwhile would otherwise
  // link only up to the old top and be left without edges on the new layers.
  std::unique_lock<std::mutex> glock(B.entry_lock);
  const int32_t ep = B.entry.load();
  const int top = B.top.load();
  if (ep < 0) {
    B.entry = i;
    B.top = li;
    return;
  }
  if (li <= top) glock.unlock();
  DC cur{sp.dist(q, ep), ep};
  for (int l = top; l > li; --l) {
    bool moved = true;
    while (moved) {
      moved = false;
      B.copy_list(cur.id, l, buf);
      for (int32_t e : buf) {
        DC ce{sp.dist(q, e), e};
        if (dc_less(ce, cur)) {
          cur = ce;
          moved = true;
        }
      }
    }
  }
  std::vector<DC> eps{cur};
  for (int l = std::min(top, li); l >= 0; --l) {
    std::vector<DC> W = search_layer(B, sp, q, i, eps, B.efc, l, vis, buf);
    std::vector<DC> nb = heuristic(sp, W, B.M);
    {
      std::lock_guard<std::mutex> g(B.locks[i]);
      int32_t* lst = B.list(i, l);
      int c = 0;
      for (const DC& e : nb) lst[c++] = e.id;
      B.count(i, l) = c;
    }
    for (const DC& e : nb) {
      std::lock_guard<std::mutex> g(B.locks[e.id]);
      int32_t* lst = B.list(e.id, l);
      int32_t& c = B.count(e.id, l);
      bool present = false;
      for (int j = 0; j < c; ++j) present |= lst[j] == i;
      if (present) continue;
      if (c < B.cap(l)) {
        lst[c++] = i;
        continue;
      }
      std::vector<DC> cs;
      cs.reserve(c + 1);
      for (int j = 0; j < c; ++j) cs.push_back(DC{sp.ndist(e.id, lst[j]), lst[j]});
      cs.push_back(DC{e.d, i});
      std::vector<DC> keep = heuristic(sp, cs, B.cap(l));
      c = 0;
      for (const DC& k : keep) lst[c++] = k.id;
      for (int j = c; j < B.cap(l); ++j) lst[j] = -1;
    }
    eps = W;
  }
  if (li > top) {  // still under the entry lock
    B.top = li;
    B.entry = i;
  }
}

}  // namespace

extern "C" int kann_hnsw_levels(int64_t n, int M, uint64_t seed, int8_t* h_level, int32_t* h_max_level,
                                int64_t* h_n_upper) {
  if (n < 0 || M < 2 || !h_level || !h_max_level || !h_n_upper) return KANN_EINVAL;
  int mx = 0;
  int64_t nu = 0;
  for (int64_t i = 0; i < n; ++i) {
    const int l = node_level(seed, (uint64_t)i, M);
    h_level[i] = (int8_t)l;
    mx = std::max(mx, l);
    nu += l >= 1;
  }
  *h_max_level = mx;
  *h_n_upper = nu;
  return KANN_OK;
}

namespace {
template <class S>
int build_any(const S& sp, int64_t n, int M, int efc, int nthreads, const int8_t* level, int32_t* l0,
              int32_t* upper_slot, int32_t* upper, int32_t* entry) {
  Builder B;
  B.n = n;
  B.M = M;
  B.M0 = 2 * M;
  B.efc = efc;
  B.level = level;
  B.l0 = l0;
  B.upper_slot = upper_slot;
  B.upper = upper;
  int L = 0;
  int64_t nu = 0;
  for (int64_t i = 0; i < n; ++i) {
    L = std::max(L, (int)level[i]);
    upper_slot[i] = level[i] >= 1 ? (int32_t)nu++ : -1;
  }
  B.L = L;
  B.cnt0.assign(n, 0);
  B.cntu.assign((size_t)nu * (L > 0 ? L : 1), 0);
  std::vector<std::mutex> locks(n);
  B.locks.swap(locks);
  std::fill(l0, l0 + (size_t)n * B.M0, -1);
  if (upper && L > 0) std::fill(upper, upper + (size_t)nu * L * M, -1);
  if (n == 0) {
    *entry = -1;
    return KANN_OK;
  }
  int T = nthreads > 0 ? nthreads : (int)std::thread::hardware_concurrency();
  if (T < 1) T = 1;
  {
    Visited vis(n);
    std::vector<int32_t> buf;
    insert(B, sp, 0, vis, buf);
  }
  std::atomic<int64_t> next{1};
  auto work = [&]() {
    Visited vis(n);
    std::vector<int32_t> buf;
    for (;;) {
      const int64_t i = next.fetch_add(1);
      if (i >= n) break;
      insert(B, sp, (int32_t)i, vis, buf);
    }
  };
  std::vector<std::thread> th;
  for (int t = 1; t < T; ++t) th.emplace_back(work);
  work();
  for (auto& t : th) t.join();
  *entry = B.entry.load();
  return KANN_OK;
}
}  // namespace

extern "C" int kann_hnsw_build_dense(const float* h_x, int64_t n, int d, int metric, int M, int ef_construction,
                                     uint64_t seed, int nthreads, const int8_t* h_level, int32_t* h_l0,
                                     int32_t* h_upper_slot, int32_t* h_upper, int32_t* h_entry) {
  (void)seed;
  if (!h_x || n < 1 || n >= ((int64_t)1 << 31) || d < 1 || M < 2 || M > 32 || ef_construction < 1) return KANN_EINVAL;
  if (metric != KANN_L2 && metric != KANN_IP) return KANN_EINVAL;
  if (!h_level || !h_l0 || !h_upper_slot || !h_entry) return KANN_EINVAL;
  DenseSpace sp{h_x, d, metric};
  return build_any(sp, n, M, ef_construction, nthreads, h_level, h_l0, h_upper_slot, h_upper, h_entry);
}

extern "C" int kann_hnsw_build_sparse(const int64_t* h_indptr, const uint16_t* h_terms, const float* h_weights,
                                      int64_t n, int M, int ef_construction, uint64_t seed, int nthreads,
                                      const int8_t* h_level, int32_t* h_l0, int32_t* h_upper_slot,
                                      int32_t* h_upper, int32_t* h_entry) {
  (void)seed;
  if (!h_indptr || !h_terms || !h_weights || n < 1 || n >= ((int64_t)1 << 31) || M < 2 || M > 32 ||
      ef_construction < 1)
    return KANN_EINVAL;
  if (!h_level || !h_l0 || !h_upper_slot || !h_entry) return KANN_EINVAL;
  SparseSpace sp{h_indptr, h_terms, h_weights};
  return build_any(sp, n, M, ef_construction, nthreads, h_level, h_l0, h_upper_slot, h_upper, h_entry);
}
