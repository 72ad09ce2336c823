// kann_oracle.cpp -- the plain FP64 CPU oracle for batched HNSW search.
//
// TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
// reference that the CUDA search path is checked against.  Only the test
// suite, the smoke check and the CPU-baseline leg of the benchmark may load
// it.  It shares no code, header, table or helper with the CUDA library.
//
// What it follows (the paper, kANNolo, cites but does not restate these):
//   * HNSW (the paper's only index, Sec. 2 "Design of kANNolo", citing
//     Malkov & Yashunin): layer assignment, insertion with the neighbour
//     selection heuristic, greedy descent through the upper layers and the
//     ef-bounded beam search on layer 0 (Malkov & Yashunin, Algorithms 1-4).
//   * Product Quantization (Sec. 2, citing Jegou et al.): per-subspace
//     k-means codebooks, nearest-centroid encoding, asymmetric distance via a
//     per-query lookup table.
//   * The three measures of the experiments (Sec. 3, Table 1): dense L2,
//     dense inner product, sparse inner product.  Distances are "smaller is
//     better": L2 = sum (q-x)^2, IP = -sum q*x.
//
// Readings taken where the paper is silent are listed in the design notes;
// each one is named again at the function that takes it.
//
// Arithmetic: every distance is accumulated in FP64, sequentially, in the
// direct form (never ||q||^2 - 2 q.x + ||x||^2).  All orderings use the total
// order on (distance, id): distance first, NaN counted as +inf, then id.
//
// Parity status per function:
//   pinned    levels (SplitMix64 published vector + level law), graph
//             invariants, both layer-0 search forms (brute force at ef >= n,
//             hand-worked golden case, mutual equality), forgetful visited
//             set, PQ identities, sparse = densified, precision encoders
//             (library casts, format definitions).
//   parity unpinned: the construction heuristic's exact edge choice and the
//             PQ training choices (k-means++ seeding, 25 Lloyd iterations,
//             empty-cluster reseeding); only internal consistency checks
//             (invariants, monotone objective) hold them.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <queue>
#include <unordered_set>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// ---------------------------------------------------------------------------
// Total order on (distance, id).  NaN compares as +inf.
// ---------------------------------------------------------------------------
struct Cand {
  double d;
  int64_t id;
};

inline double nan_as_inf(double d) { return std::isnan(d) ? INFINITY : d; }

inline bool cand_less(const Cand& a, const Cand& b) {
  double da = nan_as_inf(a.d), db = nan_as_inf(b.d);
  if (da < db) return true;
  if (da > db) return false;
  return a.id < b.id;
}

struct CandLess {
  bool operator()(const Cand& a, const Cand& b) const { return cand_less(a, b); }
};
struct CandGreater {
  bool operator()(const Cand& a, const Cand& b) const { return cand_less(b, a); }
};

// ---------------------------------------------------------------------------
// Number formats, written from their definitions (IEEE 754 binary16, the
// bfloat16 truncation of binary32, OCP FP8 E4M3 "fn": 4 exponent bits with
// bias 7, 3 mantissa bits, no infinities, max finite 448).
// ---------------------------------------------------------------------------
double decode_f16(uint16_t h) {
  int s = h >> 15, e = (h >> 10) & 31, m = h & 1023;
  double v;
  if (e == 0) v = std::ldexp((double)m, -24);
  else if (e == 31) v = m ? NAN : INFINITY;
  else v = std::ldexp(1024.0 + m, e - 25);
  return s ? -v : v;
}

double decode_bf16(uint16_t b) {
  uint32_t u = (uint32_t)b << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return (double)f;
}

double decode_e4m3(uint8_t c) {
  int s = c >> 7, e = (c >> 3) & 15, m = c & 7;
  double v;
  if (e == 15 && m == 7) v = NAN;
  else if (e == 0) v = std::ldexp((double)m, -9);
  else v = std::ldexp(8.0 + m, e - 10);
  return s ? -v : v;
}

// Round a value to a binary format with p significand bits (implicit bit
// included), minimum normal exponent emin, largest finite value maxval.
// Round-to-nearest, ties to even.  Overflow gives +-inf, or +-maxval when
// satfinite is set.
double round_to_format(double v, int p, int emin, double maxval, bool satfinite) {
  if (std::isnan(v) || v == 0.0) return v;
  double a = std::fabs(v);
  if (std::isinf(a)) return satfinite ? std::copysign(maxval, v) : v;
  int E;
  std::frexp(a, &E);             // a = f * 2^E, f in [0.5, 1)
  int lead = E - 1;              // exponent of the leading bit
  int ee = lead < emin ? emin : lead;
  double quantum = std::ldexp(1.0, ee - (p - 1));
  double r = std::nearbyint(a / quantum);  // default rounding mode: ties to even
  double res = r * quantum;
  if (res > maxval) res = satfinite ? maxval : INFINITY;
  return std::copysign(res, v);
}

uint16_t encode_f16(float x) {
  double v = round_to_format((double)x, 11, -14, 65504.0, false);
  uint16_t s = std::signbit(v) ? 0x8000 : 0;
  double a = std::fabs(v);
  if (std::isnan(v)) return 0x7e00;
  if (std::isinf(a)) return s | 0x7c00;
  if (a == 0.0) return s;
  int E;
  std::frexp(a, &E);
  int lead = E - 1;
  if (lead < -14) return s | (uint16_t)std::ldexp(a, 24);          // subnormal
  uint16_t m = (uint16_t)(std::ldexp(a, 10 - lead) - 1024.0);
  return s | (uint16_t)((lead + 15) << 10) | m;
}

uint16_t encode_bf16(float x) {
  double v = round_to_format((double)x, 8, -126, std::ldexp(255.0, 120), false);
  if (std::isnan(v)) return 0x7fc0;
  float f = (float)v;  // exact: v is representable in binary32
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return (uint16_t)(u >> 16);
}

uint8_t encode_e4m3(float x) {
  double v = round_to_format((double)x, 4, -6, 448.0, true);
  uint8_t s = std::signbit(v) ? 0x80 : 0;
  double a = std::fabs(v);
  if (std::isnan(v)) return 0x7f;
  if (a == 0.0) return s;
  int E;
  std::frexp(a, &E);
  int lead = E - 1;
  if (lead < -6) return s | (uint8_t)std::ldexp(a, 9);             // subnormal
  uint8_t m = (uint8_t)(std::ldexp(a, 3 - lead) - 8.0);
  return s | (uint8_t)((lead + 7) << 3) | m;
}

// ---------------------------------------------------------------------------
// Spaces: how a distance between the query and item j (or two items) is
// computed.  The index only ever asks "how far is j".
// ---------------------------------------------------------------------------
enum { DT_F32 = 0, DT_F16 = 1, DT_BF16 = 2, DT_E4M3 = 3 };
enum { MET_L2 = 0, MET_IP = 1 };

struct Space {
  virtual ~Space() {}
  // distance from the current query to item j
  virtual double qdist(int64_t j) const = 0;
  // distance between items a and b (graph construction only)
  virtual double ndist(int64_t a, int64_t b) const = 0;
  // make item a the current "query" (graph construction)
  virtual void set_query_item(int64_t a) = 0;
};

// Dense vectors in one of the storage formats; the stored value is decoded
// exactly to FP64 (E4M3 times its per-vector FP32 scale is exact in FP64).
struct DenseSpace : Space {
  int dtype, d, metric;
  const void* data;
  const float* scale;
  std::vector<double> q;

  DenseSpace(int dtype_, const void* data_, const float* scale_, int d_, int metric_)
      : dtype(dtype_), d(d_), metric(metric_), data(data_), scale(scale_), q(d_) {}

  double x(int64_t j, int k) const {
    size_t o = (size_t)j * d + k;
    switch (dtype) {
      case DT_F32: return (double)((const float*)data)[o];
      case DT_F16: return decode_f16(((const uint16_t*)data)[o]);
      case DT_BF16: return decode_bf16(((const uint16_t*)data)[o]);
      default: return decode_e4m3(((const uint8_t*)data)[o]) * (double)scale[j];
    }
  }
  void set_query(const float* qv) {
    for (int k = 0; k < d; ++k) q[k] = (double)qv[k];
  }
  void set_query_item(int64_t a) override {
    for (int k = 0; k < d; ++k) q[k] = x(a, k);
  }
  double qdist(int64_t j) const override {
    double s = 0.0;
    if (metric == MET_L2) {
      for (int k = 0; k < d; ++k) { double t = q[k] - x(j, k); s += t * t; }
    } else {
      for (int k = 0; k < d; ++k) s -= q[k] * x(j, k);
    }
    return s;
  }
  double ndist(int64_t a, int64_t b) const override {
    double s = 0.0;
    if (metric == MET_L2) {
      for (int k = 0; k < d; ++k) { double t = x(a, k) - x(b, k); s += t * t; }
    } else {
      for (int k = 0; k < d; ++k) s -= x(a, k) * x(b, k);
    }
    return s;
  }
};

// Product-quantized vectors: asymmetric distance through a per-query table
// (Jegou et al.): LUT[j][c] = partial distance of query sub-vector j to
// centroid c of subspace j; d(q, x) = sum_j LUT[j][code_j(x)].
// With lut_f16 the table is held at reduced precision (a reading: the paper
// does not fix the table's precision): every entry is scaled by 2^-e, where
// 2^e is the power of two that brings the largest |entry| to at most 2^15,
// rounded to FP16 (nearest, ties to even), and scaled back; the scaling is
// exact, so only the FP16 rounding of each entry remains.
// lut mode 2, the uint8 reading (also a reading: the paper does not fix the
// table's precision): every entry is computed in FP32 -- over the
// sub-vector's dimensions in order, L2: u = q - c, s = fmaf(u, u, s); IP:
// s = fmaf(q, c, s), entry -s -- then per subspace j min_j and range_j =
// max_j - min_j (FP32), one scale = max_j range_j / 255 (FP32 division; 1
// when every range is 0), and the entry's code value
// v = rint(clamp((entry - min_j) / scale, 0, 255)) (FP32 subtraction and
// division, ties to even; NaN counts as 0).  The row distance is the integer
// sum of v over its codes -- exact, and ordered as (sum, id) -- and stands for
// sum_j min_j + scale * sum.  Both the oracle and the kernel take these
// FP32 decisions in the same operations, so the integer tables agree.
struct PQTableU8 {
  std::vector<uint8_t> v;  // [m][ksub]
  float scale = 1.f, summin = 0.f;
};

PQTableU8 pq_table_u8(const float* codebooks, int m, int ksub, int dsub, int metric, const float* qv) {
  PQTableU8 t;
  std::vector<float> e((size_t)m * ksub), mn(m), mx(m);
  for (int j = 0; j < m; ++j)
    for (int c = 0; c < ksub; ++c) {
      const float* C = codebooks + ((size_t)j * ksub + c) * dsub;
      float s = 0.f;
      for (int k = 0; k < dsub; ++k) {
        const float q = qv[j * dsub + k], cc = C[k];
        if (metric == MET_L2) {
          const float u = q - cc;
          s = std::fmaf(u, u, s);
        } else {
          s = std::fmaf(q, cc, s);
        }
      }
      e[(size_t)j * ksub + c] = metric == MET_L2 ? s : -s;
    }
  float rmax = 0.f;
  for (int j = 0; j < m; ++j) {
    float lo = INFINITY, hi = -INFINITY;
    for (int c = 0; c < ksub; ++c) {
      lo = std::fmin(lo, e[(size_t)j * ksub + c]);
      hi = std::fmax(hi, e[(size_t)j * ksub + c]);
    }
    mn[j] = lo;
    mx[j] = hi;
    rmax = std::fmax(rmax, hi - lo);
  }
  t.scale = rmax > 0.f ? rmax / 255.0f : 1.0f;
  t.v.resize((size_t)m * ksub);
  for (int j = 0; j < m; ++j)
    for (int c = 0; c < ksub; ++c) {
      const float r = std::fmin(std::fmax((e[(size_t)j * ksub + c] - mn[j]) / t.scale, 0.f), 255.f);
      t.v[(size_t)j * ksub + c] = (uint8_t)std::rint(r);
    }
  float sm = 0.f;
  for (int j = 0; j < m; ++j) sm += mn[j];
  t.summin = sm;
  return t;
}

struct PQSpace : Space {
  int m, ksub, dsub, metric;
  const uint8_t* codes;
  const float* codebooks;  // [m][ksub][dsub]
  std::vector<double> lut;
  bool lut_f16;
  bool lut_u8;

  // lut_mode: 0 exact (FP64 entries), 1 the FP16 reading, 2 the uint8 reading
  PQSpace(const uint8_t* codes_, const float* cb_, int m_, int ksub_, int dsub_, int metric_, int lut_mode = 0)
      : m(m_), ksub(ksub_), dsub(dsub_), metric(metric_), codes(codes_), codebooks(cb_),
        lut((size_t)m_ * ksub_), lut_f16(lut_mode == 1), lut_u8(lut_mode == 2) {}

  void set_query(const float* qv) {
    if (lut_u8) {
      const PQTableU8 t = pq_table_u8(codebooks, m, ksub, dsub, metric, qv);
      for (size_t i = 0; i < lut.size(); ++i) lut[i] = t.v[i];
      return;
    }
    for (int j = 0; j < m; ++j)
      for (int c = 0; c < ksub; ++c) {
        const float* C = codebooks + ((size_t)j * ksub + c) * dsub;
        double s = 0.0;
        for (int t = 0; t < dsub; ++t) {
          double qq = qv[j * dsub + t], cc = C[t];
          if (metric == MET_L2) s += (qq - cc) * (qq - cc);
          else s -= qq * cc;
        }
        lut[(size_t)j * ksub + c] = s;
      }
    if (lut_f16) {
      double mx = 0.0;
      for (double v : lut) mx = std::fmax(mx, std::fabs(v));
      int E = 0;
      if (mx > 0.0) std::frexp(mx, &E);  // mx = f * 2^E, f in [0.5, 1)
      const int e = E - 15;
      for (double& v : lut) v = std::ldexp(round_to_format(std::ldexp(v, -e), 11, -14, 65504.0, false), e);
    }
  }
  void set_query_item(int64_t) override {}
  double qdist(int64_t i) const override {
    double s = 0.0;
    const uint8_t* ci = codes + (size_t)i * m;
    for (int j = 0; j < m; ++j) s += lut[(size_t)j * ksub + ci[j]];
    return s;
  }
  double ndist(int64_t, int64_t) const override { return NAN; }
};

// Sparse vectors: sorted unique uint16 term ids with FP32 weights (CSR).
// IP by a merge-join of the two term lists, accumulated in FP64.
struct SparseSpace : Space {
  const int64_t* indptr;
  const uint16_t* terms;
  const float* w;
  std::vector<uint16_t> qt;
  std::vector<double> qw;

  SparseSpace(const int64_t* ip, const uint16_t* t, const float* w_) : indptr(ip), terms(t), w(w_) {}

  static double merge_ip(const uint16_t* ta, const float* wa, int64_t na,
                         const uint16_t* tb, const double* wb_d, const float* wb_f, int64_t nb) {
    double s = 0.0;
    int64_t i = 0, j = 0;
    while (i < na && j < nb) {
      if (ta[i] < tb[j]) ++i;
      else if (ta[i] > tb[j]) ++j;
      else {
        double wb = wb_d ? wb_d[j] : (double)wb_f[j];
        s += (double)wa[i] * wb;
        ++i; ++j;
      }
    }
    return s;
  }
  void set_query(const uint16_t* t, const float* wq, int64_t nnz) {
    qt.assign(t, t + nnz);
    qw.resize(nnz);
    for (int64_t i = 0; i < nnz; ++i) qw[i] = wq[i];
  }
  void set_query_item(int64_t a) override {
    int64_t b = indptr[a], e = indptr[a + 1];
    qt.assign(terms + b, terms + e);
    qw.resize(e - b);
    for (int64_t i = b; i < e; ++i) qw[i - b] = w[i];
  }
  double qdist(int64_t j) const override {
    int64_t b = indptr[j], e = indptr[j + 1];
    return -merge_ip(terms + b, w + b, e - b, qt.data(), qw.data(), nullptr, (int64_t)qt.size());
  }
  double ndist(int64_t a, int64_t b) const override {
    int64_t ba = indptr[a], ea = indptr[a + 1], bb = indptr[b], eb = indptr[b + 1];
    return -merge_ip(terms + ba, w + ba, ea - ba, terms + bb, nullptr, w + bb, eb - bb);
  }
};

// ---------------------------------------------------------------------------
// Levels (HNSW layer assignment, Malkov & Yashunin Sec. 4):
// level = floor(-ln U * mL) with mL = 1/ln M.  U comes from a counter-based
// generator keyed by (seed, i): one SplitMix64 step (Steele, Lea & Flood 2014;
// Vigna's public-domain reference) taken from state seed XOR i*gamma, so a
// node's level depends on nothing but its id.  U = (u53 + 1) / 2^53 in (0,1].
// ---------------------------------------------------------------------------
const uint64_t GAMMA = 0x9E3779B97F4A7C15ULL;

uint64_t splitmix64_next(uint64_t& state) {
  state += GAMMA;
  uint64_t z = state;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

double counter_uniform(uint64_t seed, uint64_t i) {
  uint64_t st = seed ^ (i * GAMMA);
  uint64_t u = splitmix64_next(st) >> 11;
  return ((double)u + 1.0) / 9007199254740992.0;  // 2^53
}

int level_of(uint64_t seed, uint64_t i, int M) {
  double U = counter_uniform(seed, i);
  double l = std::floor(-std::log(U) / std::log((double)M));
  if (l > 60) l = 60;
  return (int)l;
}

// ---------------------------------------------------------------------------
// The graph.  Layer 0 lists hold up to M0 = 2M ids, upper layers up to M.
// ---------------------------------------------------------------------------
struct Graph {
  int64_t n = 0;
  int M = 0, M0 = 0, max_level = 0;
  int64_t entry = -1;
  std::vector<int8_t> level;
  std::vector<std::vector<std::vector<int32_t>>> adj;  // adj[node][layer]

  const std::vector<int32_t>& nbrs(int64_t v, int layer) const { return adj[v][layer]; }
  int cap(int layer) const { return layer == 0 ? M0 : M; }
};

// Malkov & Yashunin Alg. 2, SEARCH-LAYER, in its literal two-heap form:
// C = candidates (nearest first), W = found (furthest on top).
std::vector<Cand> search_layer_two_heap(const Graph& g, const Space& sp, const std::vector<Cand>& eps,
                                        int ef, int layer, int64_t* n_dist, int64_t* n_exp) {
  std::unordered_set<int64_t> visited;
  std::priority_queue<Cand, std::vector<Cand>, CandGreater> C;  // min-heap
  std::priority_queue<Cand, std::vector<Cand>, CandLess> W;     // max-heap
  for (const Cand& e : eps) {
    visited.insert(e.id);
    C.push(e);
    W.push(e);
    if ((int)W.size() > ef) W.pop();
  }
  while (!C.empty()) {
    Cand c = C.top();
    C.pop();
    Cand f = W.top();
    if (cand_less(f, c)) break;  // c is further than the furthest kept
    if (n_exp) ++*n_exp;
    for (int32_t e : g.nbrs(c.id, layer)) {
      if (e < 0) continue;
      if (visited.count(e)) continue;
      visited.insert(e);
      Cand ce{sp.qdist(e), e};
      if (n_dist) ++*n_dist;
      f = W.top();
      if ((int)W.size() < ef || cand_less(ce, f)) {
        C.push(ce);
        W.push(ce);
        if ((int)W.size() > ef) W.pop();
      }
    }
  }
  std::vector<Cand> out;
  while (!W.empty()) { out.push_back(W.top()); W.pop(); }
  std::reverse(out.begin(), out.end());
  return out;
}

// Visited set that may forget but never lies.  cap == 0: exact set.
// cap > 0: a direct-mapped table of `cap` slots; a new id overwrites the
// slot's previous occupant, which is thereby forgotten.
struct VisitedSet {
  int64_t cap;
  std::unordered_set<int64_t> exact;
  std::vector<int64_t> slots;
  explicit VisitedSet(int64_t c) : cap(c), slots(c > 0 ? c : 0, -1) {}
  size_t slot(int64_t id) const { return (size_t)(((uint64_t)id * GAMMA) >> 32) % (size_t)cap; }
  bool contains(int64_t id) const { return cap == 0 ? exact.count(id) > 0 : slots[slot(id)] == id; }
  void insert(int64_t id) {
    if (cap == 0) exact.insert(id);
    else slots[slot(id)] = id;
  }
};

// Layer-0 search in the "ef buffer with expanded flags" form: W is kept
// sorted by (d, id); each step expands the best unexpanded entry; each
// neighbour not yet visited is evaluated and inserted if W has room or it
// beats worst(W); an id already present in W is never inserted twice.  It
// returns the same W as the two-heap form under the (d, id) total order: a
// candidate the two-heap form still holds in C after it fell out of W is
// worse than worst(W), which only improves, so it is never expanded there
// either.
std::vector<Cand> search_layer_flags(const Graph& g, const Space& sp, Cand ep, int ef, int layer,
                                     int64_t visited_cap, int64_t* n_dist, int64_t* n_exp) {
  std::vector<Cand> W{ep};
  std::vector<char> expanded{0};
  VisitedSet visited(visited_cap);
  visited.insert(ep.id);
  for (;;) {
    size_t c = 0;
    while (c < W.size() && expanded[c]) ++c;
    if (c == W.size()) break;
    expanded[c] = 1;
    int64_t cid = W[c].id;
    if (n_exp) ++*n_exp;
    for (int32_t e : g.nbrs(cid, layer)) {
      if (e < 0) continue;
      if (visited.contains(e)) continue;
      visited.insert(e);
      Cand ce{sp.qdist(e), e};
      if (n_dist) ++*n_dist;
      bool full = (int)W.size() >= ef;
      if (full && !cand_less(ce, W.back())) continue;
      size_t pos = std::lower_bound(W.begin(), W.end(), ce, CandLess()) - W.begin();
      if (pos < W.size() && W[pos].id == ce.id) continue;  // already in W
      W.insert(W.begin() + pos, ce);
      expanded.insert(expanded.begin() + pos, 0);
      if ((int)W.size() > ef) { W.pop_back(); expanded.pop_back(); }
    }
  }
  return W;
}

// Layer-0 search that expands the p best unexpanded entries of W per step
// (a batched variant of the flag-buffer search above; it is not the search
// of the HNSW paper, which expands one entry at a time, so for p > 1 its
// results are not those of search_layer_flags).  A step marks the first p
// unexpanded entries of W (in (d, id) order) expanded, evaluates every
// neighbour of theirs that was not visited before (the lists in the order
// of the chosen entries, each list in order), and inserts the new candidates
// into W with the same bounded rule; the W after a step is the ef best of W
// and the step's candidates, whatever the order within the step.  Stops when
// W has no unexpanded entry.  The visited set is exact.
std::vector<Cand> search_layer_multi(const Graph& g, const Space& sp, Cand ep, int ef, int p, int layer,
                                     int64_t* n_dist, int64_t* n_exp) {
  std::vector<Cand> W{ep};
  std::vector<char> expanded{0};
  std::unordered_set<int64_t> visited{ep.id};
  for (;;) {
    std::vector<int64_t> chosen;
    for (size_t c = 0; c < W.size() && (int)chosen.size() < p; ++c) {
      if (expanded[c]) continue;
      expanded[c] = 1;
      chosen.push_back(W[c].id);
    }
    if (chosen.empty()) break;
    if (n_exp) *n_exp += (int64_t)chosen.size();
    std::vector<Cand> fresh;
    for (int64_t cid : chosen) {
      for (int32_t e : g.nbrs(cid, layer)) {
        if (e < 0 || visited.count(e)) continue;
        visited.insert(e);
        fresh.push_back(Cand{sp.qdist(e), e});
        if (n_dist) ++*n_dist;
      }
    }
    for (const Cand& ce : fresh) {
      bool full = (int)W.size() >= ef;
      if (full && !cand_less(ce, W.back())) continue;
      size_t pos = std::lower_bound(W.begin(), W.end(), ce, CandLess()) - W.begin();
      if (pos < W.size() && W[pos].id == ce.id) continue;
      W.insert(W.begin() + pos, ce);
      expanded.insert(expanded.begin() + pos, 0);
      if ((int)W.size() > ef) { W.pop_back(); expanded.pop_back(); }
    }
  }
  return W;
}

// Upper-layer descent, plain greedy form: move to the (d, id)-best
// neighbour while it beats the current node; equals SEARCH-LAYER with ef=1.
Cand greedy_layer(const Graph& g, const Space& sp, Cand cur, int layer, int64_t* n_dist, int64_t* n_hops) {
  for (;;) {
    Cand best = cur;
    for (int32_t e : g.nbrs(cur.id, layer)) {
      if (e < 0) continue;
      Cand ce{sp.qdist(e), e};
      if (n_dist) ++*n_dist;
      if (cand_less(ce, best)) best = ce;
    }
    if (n_hops) ++*n_hops;
    if (best.id == cur.id) return cur;
    cur = best;
  }
}

// Malkov & Yashunin Alg. 4, SELECT-NEIGHBORS-HEURISTIC (no extendCandidates,
// no keepPrunedConnections): walk candidates nearest first; keep e when it is
// closer to the base than to every element kept so far.  `simple` selects
// Alg. 3 instead (the nearest `cap`).
std::vector<Cand> select_neighbors(const Space& sp, std::vector<Cand> cands, int cap, bool simple) {
  std::sort(cands.begin(), cands.end(), CandLess());
  std::vector<Cand> R;
  for (const Cand& e : cands) {
    if ((int)R.size() >= cap) break;
    if (simple) { R.push_back(e); continue; }
    bool good = true;
    for (const Cand& r : R) {
      if (!(e.d < sp.ndist(e.id, r.id))) { good = false; break; }
    }
    if (good) R.push_back(e);
  }
  return R;
}

// Malkov & Yashunin Alg. 1, INSERT, applied to ids 0..n-1 in order.  The
// first node is the entry point; a node with a strictly greater level takes
// over as entry point.  Links are made in both directions; an overfull list
// is shrunk with the same selection rule, seen from its owner.
void build_graph(Graph& g, Space& sp, int64_t n, int M, int efC, uint64_t seed, bool simple) {
  g.n = n;
  g.M = M;
  g.M0 = 2 * M;
  g.level.resize(n);
  g.adj.resize(n);
  g.max_level = 0;
  for (int64_t i = 0; i < n; ++i) {
    int l = level_of(seed, (uint64_t)i, M);
    g.level[i] = (int8_t)l;
    g.adj[i].resize(l + 1);
  }
  if (n == 0) return;
  g.entry = 0;
  g.max_level = g.level[0];
  for (int64_t i = 1; i < n; ++i) {
    int l = g.level[i];
    sp.set_query_item(i);
    Cand ep{sp.qdist(g.entry), g.entry};
    int L = g.max_level;
    for (int lc = L; lc > l; --lc) {
      std::vector<Cand> W = search_layer_two_heap(g, sp, {ep}, 1, lc, nullptr, nullptr);
      ep = W.front();
    }
    std::vector<Cand> eps{ep};
    for (int lc = std::min(L, l); lc >= 0; --lc) {
      std::vector<Cand> W = search_layer_two_heap(g, sp, eps, efC, lc, nullptr, nullptr);
      std::vector<Cand> nb = select_neighbors(sp, W, M, simple);
      for (const Cand& e : nb) g.adj[i][lc].push_back((int32_t)e.id);
      for (const Cand& e : nb) {
        std::vector<int32_t>& lst = g.adj[e.id][lc];
        lst.push_back((int32_t)i);
        if ((int)lst.size() > g.cap(lc)) {
          std::vector<Cand> cs;
          for (int32_t v : lst) cs.push_back(Cand{sp.ndist(e.id, v), v});
          std::vector<Cand> keep = select_neighbors(sp, cs, g.cap(lc), simple);
          lst.clear();
          for (const Cand& k : keep) lst.push_back((int32_t)k.id);
        }
      }
      eps = W;
    }
    if (l > g.max_level) {
      g.max_level = l;
      g.entry = i;
    }
  }
}

// HNSW K-NN-SEARCH (Malkov & Yashunin Alg. 5).  form 0: literal two-heap
// SEARCH-LAYER everywhere.  form 1: plain greedy upper descent and the
// flag-buffer layer-0 search (with an optionally forgetful visited set).
// counters: [dist evals on layer 0, expansions on layer 0, dist evals on the
// upper layers, upper-layer hops].
// expand >= 1: the layer-0 search is search_layer_multi with that many
// entries per step (upper layers as in form 1); 0: `form` decides.
std::vector<Cand> knn_search(const Graph& g, const Space& sp, int k, int ef, int form,
                             int64_t visited_cap, int64_t* counters, int expand = 0) {
  int64_t c0 = 0, c1 = 0, c2 = 0, c3 = 0;
  std::vector<Cand> out;
  if (g.n > 0) {
    int efe = std::max(ef, k);
    Cand ep{sp.qdist(g.entry), g.entry};
    ++c2;
    for (int lc = g.max_level; lc >= 1; --lc) {
      if (form == 0) {
        std::vector<Cand> W = search_layer_two_heap(g, sp, {ep}, 1, lc, &c2, &c3);
        ep = W.front();
      } else {
        ep = greedy_layer(g, sp, ep, lc, &c2, &c3);
      }
    }
    std::vector<Cand> W = expand >= 1 ? search_layer_multi(g, sp, ep, efe, expand, 0, &c0, &c1)
                          : form == 0 ? search_layer_two_heap(g, sp, {ep}, efe, 0, &c0, &c1)
                                      : search_layer_flags(g, sp, ep, efe, 0, visited_cap, &c0, &c1);
    for (int i = 0; i < k && i < (int)W.size(); ++i) out.push_back(W[i]);
  }
  if (counters) {
    counters[0] = c0; counters[1] = c1; counters[2] = c2; counters[3] = c3;
  }
  return out;
}

void write_results(const std::vector<Cand>& r, int k, int32_t* ids, double* dists) {
  for (int i = 0; i < k; ++i) {
    if (i < (int)r.size()) { ids[i] = (int32_t)r[i].id; dists[i] = r[i].d; }
    else { ids[i] = -1; dists[i] = INFINITY; }
  }
}

int threads_or_default(int nthreads) {
#ifdef _OPENMP
  return nthreads > 0 ? nthreads : omp_get_max_threads();
#else
  (void)nthreads;
  return 1;
#endif
}

}  // namespace

extern "C" {

// ----------------------------- formats -------------------------------------
void orc_encode_f16(const float* x, int64_t n, uint16_t* out) {
  for (int64_t i = 0; i < n; ++i) out[i] = encode_f16(x[i]);
}
void orc_encode_bf16(const float* x, int64_t n, uint16_t* out) {
  for (int64_t i = 0; i < n; ++i) out[i] = encode_bf16(x[i]);
}
void orc_decode_f16(const uint16_t* h, int64_t n, double* out) {
  for (int64_t i = 0; i < n; ++i) out[i] = decode_f16(h[i]);
}
void orc_decode_bf16(const uint16_t* h, int64_t n, double* out) {
  for (int64_t i = 0; i < n; ++i) out[i] = decode_bf16(h[i]);
}
void orc_decode_e4m3(const uint8_t* c, int64_t n, double* out) {
  for (int64_t i = 0; i < n; ++i) out[i] = decode_e4m3(c[i]);
}
// Per-vector scaled E4M3: s = max|x| / 448 (FP32 division), code =
// RNE_satfinite(x / s) with x / s an FP32 division.  An all-zero row gets
// s = 0 and zero codes.
void orc_encode_e4m3_rows(const float* x, int64_t n, int d, uint8_t* codes, float* scales) {
  for (int64_t i = 0; i < n; ++i) {
    const float* r = x + (size_t)i * d;
    float mx = 0.0f;
    for (int k = 0; k < d; ++k) mx = std::max(mx, std::fabs(r[k]));
    float s = mx / 448.0f;
    scales[i] = s;
    for (int k = 0; k < d; ++k) {
      if (s == 0.0f) { codes[(size_t)i * d + k] = 0; continue; }
      float t = r[k] / s;
      codes[(size_t)i * d + k] = encode_e4m3(t);
    }
  }
}

// ----------------------------- levels --------------------------------------
void orc_splitmix64_seq(uint64_t state, int64_t n, uint64_t* out) {
  for (int64_t i = 0; i < n; ++i) out[i] = splitmix64_next(state);
}
void orc_levels(int64_t n, int M, uint64_t seed, int8_t* out) {
  for (int64_t i = 0; i < n; ++i) out[i] = (int8_t)level_of(seed, (uint64_t)i, M);
}

// ----------------------------- graphs --------------------------------------
void* orc_graph_build_dense(int dtype, const void* data, const float* scale, int64_t n, int d, int metric,
                            int M, int efC, uint64_t seed, int simple) {
  Graph* g = new Graph();
  DenseSpace sp(dtype, data, scale, d, metric);
  build_graph(*g, sp, n, M, efC, seed, simple != 0);
  return g;
}

void* orc_graph_build_sparse(const int64_t* indptr, const uint16_t* terms, const float* w, int64_t n, int M,
                             int efC, uint64_t seed, int simple) {
  Graph* g = new Graph();
  SparseSpace sp(indptr, terms, w);
  build_graph(*g, sp, n, M, efC, seed, simple != 0);
  return g;
}

void orc_graph_free(void* gp) { delete (Graph*)gp; }

// n, M, M0, max_level, entry, n_upper (nodes with level >= 1)
void orc_graph_info(const void* gp, int64_t* info) {
  const Graph& g = *(const Graph*)gp;
  int64_t nu = 0;
  for (int64_t i = 0; i < g.n; ++i) nu += g.level[i] >= 1;
  info[0] = g.n; info[1] = g.M; info[2] = g.M0; info[3] = g.max_level; info[4] = g.entry; info[5] = nu;
}

// Fixed-width serialisation: level[n]; l0[n][M0] (-1 padded);
// upper_slot[n] (-1 for level-0-only nodes, else 0.. in id order);
// upper[n_upper][max_level][M] (-1 padded), layer l at index l-1.
void orc_graph_export(const void* gp, int8_t* level, int32_t* l0, int32_t* upper_slot, int32_t* upper) {
  const Graph& g = *(const Graph*)gp;
  int64_t slot = 0;
  int L = g.max_level;
  for (int64_t i = 0; i < g.n; ++i) {
    level[i] = g.level[i];
    const std::vector<int32_t>& a0 = g.adj[i][0];
    for (int j = 0; j < g.M0; ++j) l0[(size_t)i * g.M0 + j] = j < (int)a0.size() ? a0[j] : -1;
    if (g.level[i] >= 1) {
      upper_slot[i] = (int32_t)slot;
      for (int l = 1; l <= L; ++l)
        for (int j = 0; j < g.M; ++j) {
          int32_t v = -1;
          if (l <= g.level[i] && j < (int)g.adj[i][l].size()) v = g.adj[i][l][j];
          upper[((size_t)slot * L + (l - 1)) * g.M + j] = v;
        }
      ++slot;
    } else {
      upper_slot[i] = -1;
    }
  }
}

// Rebuild an oracle graph from the serialised arrays (for graphs made
// elsewhere, e.g. by the library's own builder).
void* orc_graph_import(int64_t n, int M, int M0, int max_level, int64_t entry, const int8_t* level,
                       const int32_t* l0, const int32_t* upper_slot, const int32_t* upper) {
  Graph* g = new Graph();
  g->n = n; g->M = M; g->M0 = M0; g->max_level = max_level; g->entry = entry;
  g->level.assign(level, level + n);
  g->adj.resize(n);
  for (int64_t i = 0; i < n; ++i) {
    g->adj[i].resize(level[i] + 1);
    for (int j = 0; j < M0; ++j) {
      int32_t v = l0[(size_t)i * M0 + j];
      if (v >= 0) g->adj[i][0].push_back(v);
    }
    for (int l = 1; l <= level[i]; ++l)
      for (int j = 0; j < M; ++j) {
        int32_t v = upper[((size_t)upper_slot[i] * max_level + (l - 1)) * M + j];
        if (v >= 0) g->adj[i][l].push_back(v);
      }
  }
  return g;
}

// ----------------------------- search --------------------------------------
// ids [nq][k], dists [nq][k] FP64, counters [nq][4] (nullable).
void orc_search_dense(const void* gp, int dtype, const void* data, const float* scale, int d, int metric,
                      const float* queries, int64_t nq, int k, int ef, int form, int64_t visited_cap,
                      int nthreads, int32_t* ids, double* dists, int64_t* counters) {
  const Graph& g = *(const Graph*)gp;
#pragma omp parallel num_threads(threads_or_default(nthreads))
  {
    DenseSpace sp(dtype, data, scale, d, metric);
#pragma omp for schedule(dynamic, 1)
    for (int64_t qi = 0; qi < nq; ++qi) {
      sp.set_query(queries + (size_t)qi * d);
      std::vector<Cand> r = knn_search(g, sp, k, ef, form, visited_cap, counters ? counters + qi * 4 : nullptr);
      write_results(r, k, ids + qi * k, dists + qi * k);
    }
  }
}

// Dense search whose layer-0 step expands `expand` entries at once
// (search_layer_multi); the upper layers descend greedily.
void orc_search_dense_multi(const void* gp, int dtype, const void* data, const float* scale, int d, int metric,
                            const float* queries, int64_t nq, int k, int ef, int expand, int nthreads, int32_t* ids,
                            double* dists, int64_t* counters) {
  const Graph& g = *(const Graph*)gp;
#pragma omp parallel num_threads(threads_or_default(nthreads))
  {
    DenseSpace sp(dtype, data, scale, d, metric);
#pragma omp for schedule(dynamic, 1)
    for (int64_t qi = 0; qi < nq; ++qi) {
      sp.set_query(queries + (size_t)qi * d);
      std::vector<Cand> r = knn_search(g, sp, k, ef, 1, 0, counters ? counters + qi * 4 : nullptr, expand);
      write_results(r, k, ids + qi * k, dists + qi * k);
    }
  }
}

void orc_search_pq(const void* gp, const uint8_t* codes, const float* codebooks, int m, int ksub, int dsub,
                   int metric, int lut_mode, const float* queries, int64_t nq, int k, int ef, int form,
                   int nthreads, int32_t* ids, double* dists, int64_t* counters) {
  const Graph& g = *(const Graph*)gp;
#pragma omp parallel num_threads(threads_or_default(nthreads))
  {
    PQSpace sp(codes, codebooks, m, ksub, dsub, metric, lut_mode);
#pragma omp for schedule(dynamic, 1)
    for (int64_t qi = 0; qi < nq; ++qi) {
      sp.set_query(queries + (size_t)qi * m * dsub);
      std::vector<Cand> r = knn_search(g, sp, k, ef, form, 0, counters ? counters + qi * 4 : nullptr);
      write_results(r, k, ids + qi * k, dists + qi * k);
    }
  }
}

void orc_search_sparse(const void* gp, const int64_t* indptr, const uint16_t* terms, const float* w,
                       const int64_t* q_indptr, const uint16_t* q_terms, const float* q_w, int64_t nq, int k,
                       int ef, int form, int nthreads, int32_t* ids, double* dists, int64_t* counters) {
  const Graph& g = *(const Graph*)gp;
#pragma omp parallel num_threads(threads_or_default(nthreads))
  {
    SparseSpace sp(indptr, terms, w);
#pragma omp for schedule(dynamic, 1)
    for (int64_t qi = 0; qi < nq; ++qi) {
      sp.set_query(q_terms + q_indptr[qi], q_w + q_indptr[qi], q_indptr[qi + 1] - q_indptr[qi]);
      std::vector<Cand> r = knn_search(g, sp, k, ef, form, 0, counters ? counters + qi * 4 : nullptr);
      write_results(r, k, ids + qi * k, dists + qi * k);
    }
  }
}

// Exact re-rank of given candidate ids (row qi holds R ids, -1 ignored)
// against dense vectors; keeps the k best by (d, id).
void orc_rerank_dense(int dtype, const void* data, const float* scale, int d, int metric, const float* queries,
                      int64_t nq, const int32_t* cand, int R, int k, int32_t* ids, double* dists) {
  DenseSpace sp(dtype, data, scale, d, metric);
  for (int64_t qi = 0; qi < nq; ++qi) {
    sp.set_query(queries + (size_t)qi * d);
    std::vector<Cand> cs;
    for (int r = 0; r < R; ++r) {
      int32_t id = cand[qi * R + r];
      if (id >= 0) cs.push_back(Cand{sp.qdist(id), id});
    }
    std::sort(cs.begin(), cs.end(), CandLess());
    if ((int)cs.size() > k) cs.resize(k);
    write_results(cs, k, ids + qi * k, dists + qi * k);
  }
}

// Distances from each query to given ids (one by one), FP64.
void orc_dist_dense(int dtype, const void* data, const float* scale, int d, int metric, const float* queries,
                    int64_t nq, const int32_t* ids, int per_q, double* out) {
  DenseSpace sp(dtype, data, scale, d, metric);
  for (int64_t qi = 0; qi < nq; ++qi) {
    sp.set_query(queries + (size_t)qi * d);
    for (int r = 0; r < per_q; ++r) {
      int32_t id = ids[qi * per_q + r];
      out[qi * per_q + r] = id >= 0 ? sp.qdist(id) : INFINITY;
    }
  }
}

// ----------------------------- brute force ---------------------------------
void orc_exact_dense(int dtype, const void* data, const float* scale, int64_t n, int d, int metric,
                     const float* queries, int64_t nq, int k, int nthreads, int32_t* ids, double* dists) {
#pragma omp parallel num_threads(threads_or_default(nthreads))
  {
    DenseSpace sp(dtype, data, scale, d, metric);
#pragma omp for schedule(dynamic, 1)
    for (int64_t qi = 0; qi < nq; ++qi) {
      sp.set_query(queries + (size_t)qi * d);
      std::vector<Cand> all((size_t)n);
      for (int64_t j = 0; j < n; ++j) all[j] = Cand{sp.qdist(j), j};
      int kk = (int)std::min<int64_t>(k, n);
      std::partial_sort(all.begin(), all.begin() + kk, all.end(), CandLess());
      all.resize(kk);
      write_results(all, k, ids + qi * k, dists + qi * k);
    }
  }
}

void orc_exact_sparse(const int64_t* indptr, const uint16_t* terms, const float* w, int64_t n,
                      const int64_t* q_indptr, const uint16_t* q_terms, const float* q_w, int64_t nq, int k,
                      int nthreads, int32_t* ids, double* dists) {
#pragma omp parallel num_threads(threads_or_default(nthreads))
  {
    SparseSpace sp(indptr, terms, w);
#pragma omp for schedule(dynamic, 1)
    for (int64_t qi = 0; qi < nq; ++qi) {
      sp.set_query(q_terms + q_indptr[qi], q_w + q_indptr[qi], q_indptr[qi + 1] - q_indptr[qi]);
      std::vector<Cand> all((size_t)n);
      for (int64_t j = 0; j < n; ++j) all[j] = Cand{sp.qdist(j), j};
      int kk = (int)std::min<int64_t>(k, n);
      std::partial_sort(all.begin(), all.begin() + kk, all.end(), CandLess());
      all.resize(kk);
      write_results(all, k, ids + qi * k, dists + qi * k);
    }
  }
}

void orc_exact_pq(const uint8_t* codes, const float* codebooks, int64_t n, int m, int ksub, int dsub, int metric,
                  const float* queries, int64_t nq, int k, int32_t* ids, double* dists) {
  PQSpace sp(codes, codebooks, m, ksub, dsub, metric);
  for (int64_t qi = 0; qi < nq; ++qi) {
    sp.set_query(queries + (size_t)qi * m * dsub);
    std::vector<Cand> all((size_t)n);
    for (int64_t j = 0; j < n; ++j) all[j] = Cand{sp.qdist(j), j};
    int kk = (int)std::min<int64_t>(k, n);
    std::partial_sort(all.begin(), all.begin() + kk, all.end(), CandLess());
    all.resize(kk);
    write_results(all, k, ids + qi * k, dists + qi * k);
  }
}

// ----------------------------- PQ ------------------------------------------
// Per-query ADC table, [m][ksub] FP64.
// The uint8 reading of a query's table (values [m][ksub], scale, and the
// FP32 sum of the per-subspace minima).
void orc_pq_lut_u8(const float* codebooks, int m, int ksub, int dsub, int metric, const float* q, uint8_t* v,
                   float* scale, float* summin) {
  const PQTableU8 t = pq_table_u8(codebooks, m, ksub, dsub, metric, q);
  std::copy(t.v.begin(), t.v.end(), v);
  *scale = t.scale;
  *summin = t.summin;
}

void orc_pq_lut(const float* codebooks, int m, int ksub, int dsub, int metric, int lut_mode, const float* q,
                double* lut) {
  PQSpace sp(nullptr, codebooks, m, ksub, dsub, metric, lut_mode);
  sp.set_query(q);
  std::memcpy(lut, sp.lut.data(), sizeof(double) * (size_t)m * ksub);
}

// Nearest centroid per subspace under L2, ties to the lowest index.
void orc_pq_encode(const float* X, int64_t n, int m, int ksub, int dsub, const float* codebooks, uint8_t* codes) {
  for (int64_t i = 0; i < n; ++i)
    for (int j = 0; j < m; ++j) {
      const float* x = X + (size_t)i * m * dsub + (size_t)j * dsub;
      double best = INFINITY;
      int bc = 0;
      for (int c = 0; c < ksub; ++c) {
        const float* C = codebooks + ((size_t)j * ksub + c) * dsub;
        double s = 0.0;
        for (int t = 0; t < dsub; ++t) { double u = (double)x[t] - (double)C[t]; s += u * u; }
        if (s < best) { best = s; bc = c; }
      }
      codes[(size_t)i * m + j] = (uint8_t)bc;
    }
}

void orc_pq_reconstruct(const uint8_t* codes, int64_t n, int m, int ksub, int dsub, const float* codebooks,
                        float* out) {
  for (int64_t i = 0; i < n; ++i)
    for (int j = 0; j < m; ++j) {
      const float* C = codebooks + ((size_t)j * ksub + codes[(size_t)i * m + j]) * dsub;
      for (int t = 0; t < dsub; ++t) out[(size_t)i * m * dsub + (size_t)j * dsub + t] = C[t];
    }
}

// Lloyd k-means per subspace in FP64 (Jegou et al. train each subspace
// quantizer independently).  Readings: k-means++ seeding with the
// counter-based uniform keyed by (seed, subspace, draw); `iters` Lloyd
// iterations; an empty cluster takes the point farthest from its current
// centroid.  codebooks_out [m][ksub][dsub] is rounded to FP32 (the stored
// format); objective [m][iters+1] records the mean squared quantisation
// error before the first and after every iteration.
void orc_pq_train(const float* X, int64_t n, int m, int ksub, int dsub, int iters, uint64_t seed,
                  float* codebooks_out, double* objective) {
  for (int j = 0; j < m; ++j) {
    std::vector<double> x((size_t)n * dsub);
    for (int64_t i = 0; i < n; ++i)
      for (int t = 0; t < dsub; ++t) x[(size_t)i * dsub + t] = X[(size_t)i * m * dsub + (size_t)j * dsub + t];
    std::vector<double> C((size_t)ksub * dsub);
    auto sq = [&](const double* a, const double* b) {
      double s = 0.0;
      for (int t = 0; t < dsub; ++t) { double u = a[t] - b[t]; s += u * u; }
      return s;
    };
    uint64_t sub_seed = seed ^ ((uint64_t)(j + 1) * 0xD1B54A32D192ED03ULL);
    uint64_t draw = 0;
    // k-means++: first centre uniform, then proportional to D^2.
    int64_t first = (int64_t)std::min<double>((double)n - 1, std::floor(counter_uniform(sub_seed, draw++) * n));
    std::copy(&x[(size_t)first * dsub], &x[(size_t)first * dsub] + dsub, &C[0]);
    std::vector<double> D2(n);
    for (int64_t i = 0; i < n; ++i) D2[i] = sq(&x[(size_t)i * dsub], &C[0]);
    for (int c = 1; c < ksub; ++c) {
      double tot = 0.0;
      for (int64_t i = 0; i < n; ++i) tot += D2[i];
      int64_t pick = n - 1;
      if (tot > 0.0) {
        double r = counter_uniform(sub_seed, draw++) * tot, acc = 0.0;
        for (int64_t i = 0; i < n; ++i) {
          acc += D2[i];
          if (acc >= r) { pick = i; break; }
        }
      } else {
        pick = (int64_t)std::min<double>((double)n - 1, std::floor(counter_uniform(sub_seed, draw++) * n));
      }
      std::copy(&x[(size_t)pick * dsub], &x[(size_t)pick * dsub] + dsub, &C[(size_t)c * dsub]);
      for (int64_t i = 0; i < n; ++i) D2[i] = std::min(D2[i], sq(&x[(size_t)i * dsub], &C[(size_t)c * dsub]));
    }
    std::vector<int> assign(n);
    auto assign_all = [&]() {
      double obj = 0.0;
      for (int64_t i = 0; i < n; ++i) {
        double best = INFINITY;
        int bc = 0;
        for (int c = 0; c < ksub; ++c) {
          double s = sq(&x[(size_t)i * dsub], &C[(size_t)c * dsub]);
          if (s < best) { best = s; bc = c; }
        }
        assign[i] = bc;
        D2[i] = best;
        obj += best;
      }
      return obj / (double)n;
    };
    objective[(size_t)j * (iters + 1)] = assign_all();
    for (int it = 0; it < iters; ++it) {
      std::vector<double> sum((size_t)ksub * dsub, 0.0);
      std::vector<int64_t> cnt(ksub, 0);
      for (int64_t i = 0; i < n; ++i) {
        ++cnt[assign[i]];
        for (int t = 0; t < dsub; ++t) sum[(size_t)assign[i] * dsub + t] += x[(size_t)i * dsub + t];
      }
      for (int c = 0; c < ksub; ++c) {
        if (cnt[c] > 0) {
          for (int t = 0; t < dsub; ++t) C[(size_t)c * dsub + t] = sum[(size_t)c * dsub + t] / (double)cnt[c];
        } else {
          int64_t far = 0;
          for (int64_t i = 1; i < n; ++i) if (D2[i] > D2[far]) far = i;
          std::copy(&x[(size_t)far * dsub], &x[(size_t)far * dsub] + dsub, &C[(size_t)c * dsub]);
          D2[far] = 0.0;
        }
      }
      objective[(size_t)j * (iters + 1) + it + 1] = assign_all();
    }
    for (int c = 0; c < ksub; ++c)
      for (int t = 0; t < dsub; ++t)
        codebooks_out[((size_t)j * ksub + c) * dsub + t] = (float)C[(size_t)c * dsub + t];
  }
}

}  // extern "C"
