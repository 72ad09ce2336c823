// kann_search_impl.cuh -- batched HNSW search kernels for sm_103a (device code,
// included by the per-format translation units kann_search_{f32,f16,bf16,e4m3}.cu
// and by kann_search.cu, which holds the PQ and sparse kernels and the launchers;
// the sparse back-end is kann_search_sparse.cuh).
//
// One warp searches one query (HNSW K-NN-SEARCH, Malkov & Yashunin Alg. 5,
// the index of kANNolo Sec. 2):
//   1. distance to the entry point;
//   2. greedy descent through layers max_level..1: move to the (d, id)-best
//      neighbour while it beats the current node (SEARCH-LAYER with ef = 1);
//   3. layer-0 beam: W, the ef best (d, id) keys found so far, sorted, each
//      with an "expanded" bit.  Each step expands the best unexpanded entry:
//      its adjacency row (M0 ids) is read with one coalesced load per lane,
//      ids already in the visited table are dropped, the surviving rows are
//      gathered with 16-byte loads (several rows in flight per warp) and their
//      distances reduced with shuffles; keys that beat worst(W) are sorted by a
//      warp bitonic network and merged into W in place (rank by binary search,
//      move right-to-left).  The search ends when W has no unexpanded entry.
//      This is the two-heap SEARCH-LAYER (Alg. 2) in its flag-buffer form; both
//      give the same W under the (d, id) total order;
//   4. optional exact FP32 re-rank of the best R entries of W;
//   5. the k best keys are written out (id -1 / +inf padding).
//
// The visited table is a per-warp hash in shared memory (a compact table of
// 16-bit slots when the ids allow it, else 32-bit id slots).  It may forget
// (it is cleared and refilled with W's ids when it fills up, and an id that
// finds no free slot is not stored) but it never reports an unvisited id as
// visited.  Forgetting is harmless because an id
// already in W is never inserted twice (equal keys are detected in the merge),
// and an id that left W or was rejected is worse than worst(W), which only
// improves once W is full; the search therefore returns the same W as with an
// exact visited set.  Forgotten ids cost only a repeated distance.
#pragma once
#include <type_traits>

#include "kann_device.cuh"
#include "kann_internal.h"

namespace kann {
namespace {

constexpr u64 FLAG = 0x80000000ull;  // "expanded" bit, kept in the id word
constexpr uint32_t HEMPTY = 0xffffffffu;
constexpr int HASH_MAX_PROBE = 32;

__device__ __forceinline__ u64 kmask(u64 k) { return k & ~FLAG; }
__device__ __forceinline__ uint32_t key_id(u64 k) { return (uint32_t)k & 0x7fffffffu; }

// Wide visited table: 2^hbits 32-bit slots holding ids, open addressing.
// Returns 0 if id is present, 1 if it was inserted now, 2 if it is absent but
// the probe window is full (treated as unvisited, not stored).
__device__ __forceinline__ int visit32(uint32_t* H, int hbits, uint32_t id) {
  const uint32_t mask = (1u << hbits) - 1u;
  uint32_t h = (id * 2654435761u) >> (32 - hbits);
  volatile uint32_t* vh = H;
  for (int p = 0; p < HASH_MAX_PROBE; ++p) {
    uint32_t v = vh[h];
    if (v == id) return 0;
    if (v == HEMPTY) {
      uint32_t old = atomicCAS(&H[h], HEMPTY, id);
      if (old == HEMPTY) return 1;
      if (old == id) return 0;
    }
    h = (h + 1u) & mask;
  }
  return 2;
}

__device__ __forceinline__ uint4 lds_volatile16(const uint32_t* p) {
  uint4 r;
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ld.volatile.shared.v4.u32 {%0,%1,%2,%3}, [%4];" : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w) : "r"(a));
  return r;
}

// Nonzero exactly when one of the two 16-bit halves of x is zero (the
// borrow-based zero-lane test: with no zero half nothing borrows and no mask
// bit survives; the lowest zero half always sets its mask bit).
__device__ __forceinline__ uint32_t zero_halves(uint32_t x) { return (x - 0x00010001u) & ~x & 0x80008000u; }

// Compact visited table: 2^hbits 16-bit slots in buckets of 8 (one 16-byte
// row).  An id maps to x = (id * VIS_MUL) mod 2^vk -- a bijection of the
// vk-bit ids, VIS_MUL being odd -- whose bucket is x >> vr and whose slot
// value is 1 + (x mod 2^vr); a (bucket, value) pair therefore belongs to one
// id only, so a match is never a false positive.  Empty slots hold 0.  Same
// returns as visit32 (2: the bucket is full, the id is not stored).
constexpr uint32_t VIS_MUL = 0x9E3779B1u;
__device__ __forceinline__ int visit16(uint32_t* H, int vk, int vr, uint32_t id) {
  const uint32_t x = (id * VIS_MUL) & (0xffffffffu >> (32 - vk));
  uint32_t* B = H + ((x >> vr) << 2);
  const uint32_t tag = (x & ((1u << vr) - 1u)) + 1u;
  const uint32_t tt = tag * 0x00010001u;
  // each failed CAS means another lane filled a slot of this bucket: at most
  // eight of them
  for (int tries = 0; tries < 9; ++tries) {
    const uint4 v = lds_volatile16(B);
    if (zero_halves(v.x ^ tt) | zero_halves(v.y ^ tt) | zero_halves(v.z ^ tt) | zero_halves(v.w ^ tt)) return 0;
    int i;
    uint32_t w;
    if (zero_halves(v.x)) {
      i = 0;
      w = v.x;
    } else if (zero_halves(v.y)) {
      i = 1;
      w = v.y;
    } else if (zero_halves(v.z)) {
      i = 2;
      w = v.z;
    } else if (zero_halves(v.w)) {
      i = 3;
      w = v.w;
    } else {
      return 2;
    }
    const uint32_t nw = (w & 0xffffu) == 0u ? (w | tag) : (w | (tag << 16));
    if (atomicCAS(B + i, w, nw) == w) return 1;
  }
  return 2;
}

// The visited table of one warp (layout chosen on the host: vr >= 0 compact,
// vr < 0 wide).
struct Visited {
  uint32_t* H;
  int hbits, vk, vr;
  __device__ __forceinline__ bool compact() const { return vr >= 0; }
  __device__ __forceinline__ int insert(uint32_t id) const {
    return compact() ? visit16(H, vk, vr, id) : visit32(H, hbits, id);
  }
  // stored ids above which the table is cleared: 3/4 of the compact slots
  // (buckets of 8 rarely overflow below that), 1/2 of the wide ones
  __device__ __forceinline__ int limit() const { return compact() ? (3 << hbits) >> 2 : (1 << hbits) >> 1; }
  __device__ __forceinline__ void clear(int lane) const {
    if (compact()) {
      uint4* q = reinterpret_cast<uint4*>(H);
      for (int i = lane; i < (1 << hbits) / 8; i += 32) q[i] = make_uint4(0u, 0u, 0u, 0u);
    } else {
      for (int i = lane; i < (1 << hbits); i += 32) H[i] = HEMPTY;
    }
  }
};

__device__ __forceinline__ int lower_bound_w(const u64* W, int len, u64 key) {
  int lo = 0, hi = len;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (kmask(W[mid]) < key) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// number of entries of the ascending array A[0..n) that are <= x
__device__ __forceinline__ int count_le(const int* A, int n, int x) {
  int lo = 0, hi = n;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (A[mid] <= x) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Shared memory of one warp: W[efcap] keys, candidate keys[64] (with
// multi-expansion 64 per expanded entry plus 64 for the ranked survivors),
// candidate ids[64 per expanded entry] (which also hold the survivors'
// W-ranks once the step's distances are done: the two are never live
// together), then the visited table
// (2^hbits slots of 2 bytes, compact, or 4 bytes, wide), then back-end scratch.
struct WarpSmem {
  u64* W;
  u64* ck;
  int* cid;
  int* clb;
  uint32_t* H;
  unsigned char* extra;
  __device__ __forceinline__ WarpSmem(unsigned char* ws, int efcap, int hbits, bool compact, int expand) {
    W = reinterpret_cast<u64*>(ws);
    ck = W + efcap;
    cid = reinterpret_cast<int*>(ck + cand_keys(expand));
    clb = cid;
    H = reinterpret_cast<uint32_t*>(cid + 64 * expand);
    extra = reinterpret_cast<unsigned char*>(H) + ((compact ? 2 : 4) << hbits);
  }
  // one-expansion kernels (MULTI false) lay the area out for one expansion
  // at compile time; a multi-expansion kernel reads a.expand
  template <bool MULTI = false>
  __device__ __forceinline__ static WarpSmem of(unsigned char* ws, const SearchArgs& a) {
    return WarpSmem(ws, a.efcap, a.hbits, a.vis_r >= 0, MULTI ? a.expand : 1);
  }
};

enum { TEAM_DIST = 1, TEAM_RERANK = 2, TEAM_DONE = 3 };

struct TeamCtl {
  int cmd, cnt, qi, pad;
  float wmax[8];
};

__device__ __forceinline__ void team_bar(int T) { asm volatile("bar.sync 1, %0;" ::"r"(T * 32) : "memory"); }

// Slice [s0, s0 + n) of cnt candidates for warp w of a team of T.
__device__ __forceinline__ void team_slice(int cnt, int w, int T, int& s0, int& n) {
  const int per = (cnt + T - 1) / T;
  s0 = w * per;
  n = cnt - s0 < per ? cnt - s0 : per;
  if (n < 0) n = 0;
}

// ---------------------------------------------------------------------------
// Dense back-end: rows of `DT` elements; lanes are split into groups of `lpr`
// lanes per row, lane `sub` of a group owning 16-byte chunks sub, sub + lpr,
// ...  (CPL chunks at most).  The query's matching chunks stay in registers.
// U row-batches are loaded before any is consumed, so U * 32 / lpr rows are
// in flight per warp.  The summation order of a row's distance depends only
// on the row, never on its slot in the batch.
//
// LPR > 0 is the exact-tiling form: a row is exactly LPR * CPL chunks and lpr
// = LPR, so the lane mapping, the chunk bounds and the butterfly are
// compile-time constants.  LPR = 0 takes lpr and the chunk count from the
// launch.  Both forms give bit-identical distances.
// ---------------------------------------------------------------------------

// t0 = x0 - q0 and t1 = x1 - q1 for the two 16-bit elements x0 (low half) and
// x1 (high half) of w, each widened to FP32 inside the subtraction
// (mixed-precision sub.f32.f16 / sub.f32.bf16).  The widening is exact, so
// this equals converting first and subtracting in FP32; the squares equal
// those of q - x.
template <int DT>
__device__ __forceinline__ void sub2_wide(uint32_t w, float q0, float q1, float& t0, float& t1) {
  if (DT == KANN_F16)
    asm("{.reg .f16 l, h;\n\tmov.b32 {l, h}, %2;\n\tsub.rn.f32.f16 %0, l, %3;\n\tsub.rn.f32.f16 %1, h, %4;}"
        : "=f"(t0), "=f"(t1)
        : "r"(w), "f"(q0), "f"(q1));
  else
    asm("{.reg .b16 l, h;\n\tmov.b32 {l, h}, %2;\n\tsub.rn.f32.bf16 %0, l, %3;\n\tsub.rn.f32.bf16 %1, h, %4;}"
        : "=f"(t0), "=f"(t1)
        : "r"(w), "f"(q0), "f"(q1));
}

template <int DT, int CPL, bool LEAN = false, int MET = KANN_L2, int LPR = 0>
struct DenseBackend {
  static constexpr int EPC = Fmt<DT>::EPC;
  // row batches in flight: 32 buffer registers per lane, 16 in the lean form
  static constexpr int U = ((LEAN ? 4 : 8) / CPL) > 0 ? ((LEAN ? 4 : 8) / CPL) : 1;
  static constexpr bool WIDE_SUB = (DT == KANN_F16 || DT == KANN_BF16) && MET == KANN_L2;
  float qr[CPL][EPC];

  __device__ __forceinline__ static int lanes(const SearchArgs& a) { return LPR > 0 ? LPR : a.lpr; }
  __device__ __forceinline__ static int log2_lanes(const SearchArgs& a) {
    if (LPR > 0) return LPR >= 32 ? 5 : LPR >= 16 ? 4 : LPR >= 8 ? 3 : LPR >= 4 ? 2 : LPR >= 2 ? 1 : 0;
    return 31 - __clz(a.lpr);
  }
  __device__ __forceinline__ static bool has_chunk(const SearchArgs& a, int ch) { return LPR > 0 || ch < a.nchunks; }

  __device__ __forceinline__ void init(const SearchArgs& a, int qi, int lane, unsigned char*) {
    const float* q = a.q + (size_t)qi * a.d;
    const int lpr = lanes(a);
    const int sub = lane & (lpr - 1);
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
      const int ch = sub + c * lpr;
#pragma unroll
      for (int e4 = 0; e4 < EPC / 4; ++e4) {
        float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
        if (has_chunk(a, ch)) t = __ldg(reinterpret_cast<const float4*>(q + ch * EPC) + e4);
        qr[c][4 * e4 + 0] = t.x;
        qr[c][4 * e4 + 1] = t.y;
        qr[c][4 * e4 + 2] = t.z;
        qr[c][4 * e4 + 3] = t.w;
      }
    }
  }

  // a search team: every warp keeps the query in its own registers
  __device__ __forceinline__ void init_team(const SearchArgs& a, int qi, int lane, int, int, unsigned char*,
                                            TeamCtl*) {
    init(a, qi, lane, nullptr);
  }

  __device__ __forceinline__ void dists(const SearchArgs& a, const int* cid, int cnt, u64* ck, int lane) {
    const int lpr = lanes(a), lg = log2_lanes(a), rpi = 32 >> lg;
    const int sub = lane & (lpr - 1), grp = lane >> lg;
    for (int base = 0; base < cnt; base += rpi * U) {
      uint4 buf[U][CPL];
      float sc[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int r = base + u * rpi + grp;
        const int id = r < cnt ? cid[r] : -1;
        const unsigned char* row = a.data + (int64_t)(id < 0 ? 0 : id) * a.stride;
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
          const int ch = sub + c * lpr;
          buf[u][c] = (id >= 0 && has_chunk(a, ch)) ? ldg_stream16(row + ch * 16) : make_uint4(0u, 0u, 0u, 0u);
        }
        sc[u] = 1.f;
        if (DT == KANN_E4M3) sc[u] = id >= 0 ? __ldg(a.scale + id) : 0.f;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (base + u * rpi >= cnt) break;  // this and later row groups are empty
        const int r = base + u * rpi + grp;
        // two partial sums per lane: a0 over the even, a1 over the odd
        // elements of its chunks (in chunk order), then a0 + a1
        float a0 = 0.f, a1 = 0.f;
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
          if constexpr (WIDE_SUB) {
            const uint32_t w[4] = {buf[u][c].x, buf[u][c].y, buf[u][c].z, buf[u][c].w};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              float t0, t1;
              sub2_wide<DT>(w[i], qr[c][2 * i], qr[c][2 * i + 1], t0, t1);
              acc_sq2(a0, a1, t0, t1);
            }
          } else {
            float x[EPC];
            Fmt<DT>::unpack(buf[u][c], x);
#pragma unroll
            for (int e = 0; e < EPC; e += 2) {
              if (MET == KANN_L2) {
                if (DT == KANN_E4M3) {
                  // q - s x in one rounding
                  acc_sq2(a0, a1, fmaf(-x[e], sc[u], qr[c][e]), fmaf(-x[e + 1], sc[u], qr[c][e + 1]));
                } else {
                  acc_diff_sq2(a0, a1, qr[c][e], qr[c][e + 1], x[e], x[e + 1]);
                }
              } else {
                acc_mul2(a0, a1, qr[c][e], qr[c][e + 1], x[e], x[e + 1]);  // E4M3: scale applied once below
              }
            }
          }
        }
        float acc = a0 + a1;
        if (DT == KANN_E4M3 && MET != KANN_L2) acc *= sc[u];
        for (int o = lpr >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
        if (sub == 0 && r < cnt) ck[r] = make_key(MET == KANN_L2 ? acc : -acc, (uint32_t)cid[r]);
      }
    }
  }
};

// ---------------------------------------------------------------------------
// PQ back-end (asymmetric distance computation, Jegou et al.): the query's
// table LUT[j][c] = partial distance of query sub-vector j to centroid c of
// subspace j (L2: ||q_j - C_j[c]||^2, IP: -<q_j, C_j[c]>) is built in FP32
// in shared memory, then d(q, x) = sum_j LUT[j][code_j(x)].  A row is the m
// code bytes of an item; lanes own 16-byte chunks of it exactly as in the
// dense back-end, summing their lookups in byte order.
//
// LF (table format) = PQ_LUT_F32, or
//  PQ_LUT_F16: the table is held in FP16 (half the shared memory, so twice
//   the queries per SM at m = 192): entries are scaled by 2^-e, with 2^e the
//   power of two that brings the largest |entry| to at most 2^15, rounded to
//   nearest, and the FP32 sum of a row's lookups is scaled back by 2^e;
//  PQ_LUT_U8: a quarter of the shared memory: each FP32 entry becomes
//   v = rint(clamp((entry - min_j) / scale, 0, 255)) with min_j the minimum
//   of subspace j and scale = (largest range max_j - min_j) / 255; a row's
//   distance is the integer sum of its values (exact, order-free), which
//   stands for sum_j min_j + scale * sum (the output's distance).
// ---------------------------------------------------------------------------
constexpr int PQ_LUT_F32 = 0, PQ_LUT_F16 = 1, PQ_LUT_U8 = 2;

template <int CPL, int LF>
struct PQBackend {
  static constexpr bool L16 = LF == PQ_LUT_F16;
  static constexpr bool U8 = LF == PQ_LUT_U8;
  static constexpr int U = (8 / CPL) > 0 ? (8 / CPL) : 1;
  typedef typename std::conditional<U8, uint8_t, typename std::conditional<L16, __half, float>::type>::type LutT;
  LutT* lut;
  float scale;   // 2^e for the FP16 table, the step of the uint8 table, 1 otherwise
  float summin;  // uint8 table: sum of the subspace minima (FP32, in subspace order)

  __device__ __forceinline__ static float entry(const SearchArgs& a, const float* q, int e) {
    const int j = e >> 8, dsub = a.pq_dsub;
    const float* C = a.codebooks + (size_t)e * dsub;
    const float* qq = q + j * dsub;
    float s = 0.f;
    for (int t = 0; t < dsub; ++t) {
      const float cv = __ldg(C + t), qv = __ldg(qq + t);
      if (a.metric == KANN_L2) {
        const float u = qv - cv;
        s = fmaf(u, u, s);
      } else {
        s = fmaf(qv, cv, s);
      }
    }
    return a.metric == KANN_L2 ? s : -s;
  }

  __device__ __forceinline__ void init(const SearchArgs& a, int qi, int lane, unsigned char* extra) {
    static_assert(!U8, "the uint8 table is built by a team");
    lut = reinterpret_cast<LutT*>(extra);
    const int m = a.pq_m;
    const float* q = a.q + (size_t)qi * m * a.pq_dsub;
    scale = 1.f;
    if (!L16) {
      for (int e = lane; e < m * 256; e += 32) lut[e] = entry(a, q, e);
    } else {
      float mx = 0.f;
      for (int e = lane; e < m * 256; e += 32) mx = fmaxf(mx, fabsf(entry(a, q, e)));
      for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(FULL, mx, o));
      int E = 0;
      if (mx > 0.f) frexpf(mx, &E);  // mx = f * 2^E, f in [0.5, 1)
      const int sh = E - 15;
      for (int e = lane; e < m * 256; e += 32) lut[e] = __float2half_rn(ldexpf(entry(a, q, e), -sh));
      scale = ldexpf(1.f, sh);
    }
    __syncwarp();
  }

  // The same table built by a team of T warps (thread t of the team takes
  // entries t, t + 32 T, ...); ends with the team at barrier 1.
  __device__ void init_team(const SearchArgs& a, int qi, int lane, int w, int T, unsigned char* ws, TeamCtl* tc) {
    const WarpSmem s = WarpSmem::of(ws, a);
    lut = reinterpret_cast<LutT*>(s.extra);
    const int m = a.pq_m;
    const float* q = a.q + (size_t)qi * m * a.pq_dsub;
    const int t0 = w * 32 + lane, step = T * 32;
    scale = 1.f;
    summin = 0.f;
    if constexpr (U8) {
      // per-subspace minima and ranges (warp w takes subspaces w, w + T, ...),
      // kept after the table
      float* mn = reinterpret_cast<float*>(s.extra + (size_t)m * 256);
      float* rg = mn + m;
      for (int j = w; j < m; j += T) {
        float lo = __int_as_float(0x7f800000), hi = __int_as_float(0xff800000);
        for (int c = lane; c < 256; c += 32) {
          const float e = entry(a, q, j * 256 + c);
          lo = fminf(lo, e);
          hi = fmaxf(hi, e);
        }
        for (int o = 16; o > 0; o >>= 1) {
          lo = fminf(lo, __shfl_xor_sync(FULL, lo, o));
          hi = fmaxf(hi, __shfl_xor_sync(FULL, hi, o));
        }
        if (lane == 0) {
          mn[j] = lo;
          rg[j] = __fsub_rn(hi, lo);
        }
      }
      team_bar(T);
      float rmax = 0.f;
      for (int j = lane; j < m; j += 32) rmax = fmaxf(rmax, rg[j]);
      for (int o = 16; o > 0; o >>= 1) rmax = fmaxf(rmax, __shfl_xor_sync(FULL, rmax, o));
      scale = rmax > 0.f ? __fdiv_rn(rmax, 255.0f) : 1.0f;
      for (int e = t0; e < m * 256; e += step) {
        const float r = fminf(fmaxf(__fdiv_rn(__fsub_rn(entry(a, q, e), mn[e >> 8]), scale), 0.f), 255.f);
        lut[e] = (uint8_t)__float2uint_rn(r);
      }
      if (w == 0) {
        float sm = 0.f;
        for (int j = 0; j < m; ++j) sm = __fadd_rn(sm, mn[j]);
        summin = sm;
      }
      team_bar(T);
      return;
    }
    if (!L16) {
      for (int e = t0; e < m * 256; e += step) lut[e] = entry(a, q, e);
    } else {
      float mx = 0.f;
      for (int e = t0; e < m * 256; e += step) mx = fmaxf(mx, fabsf(entry(a, q, e)));
      for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(FULL, mx, o));
      if (lane == 0) tc->wmax[w] = mx;
      team_bar(T);
      mx = 0.f;
      for (int i = 0; i < T; ++i) mx = fmaxf(mx, tc->wmax[i]);
      int E = 0;
      if (mx > 0.f) frexpf(mx, &E);  // mx = f * 2^E, f in [0.5, 1)
      const int sh = E - 15;
      for (int e = t0; e < m * 256; e += step) lut[e] = __float2half_rn(ldexpf(entry(a, q, e), -sh));
      scale = ldexpf(1.f, sh);
    }
    team_bar(T);
  }

  // the distance the output reports for a traversal key's value
  __device__ __forceinline__ float out_dist(float d) const {
    if constexpr (U8) return __fadd_rn(__fmul_rn(scale, d), summin);
    return d;
  }

  __device__ __forceinline__ void dists(const SearchArgs& a, const int* cid, int cnt, u64* ck, int lane) {
    const int lpr = a.lpr, rpi = 32 / lpr;
    const int sub = lane & (lpr - 1), grp = lane / lpr;
    for (int base = 0; base < cnt; base += rpi * U) {
      uint4 buf[U][CPL];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int r = base + u * rpi + grp;
        const int id = r < cnt ? cid[r] : -1;
        const unsigned char* row = a.codes + (int64_t)(id < 0 ? 0 : id) * a.stride;
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
          const int ch = sub + c * lpr;
          buf[u][c] = (id >= 0 && ch < a.nchunks) ? ldg_stream16(row + ch * 16) : make_uint4(0u, 0u, 0u, 0u);
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (base + u * rpi >= cnt) break;  // this and later row groups are empty
        const int r = base + u * rpi + grp;
        float acc = 0.f;
        uint32_t iacc = 0u;  // uint8 table: exact integer sum (at most 512 * 255)
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
          const int ch = sub + c * lpr;
          if (ch < a.nchunks) {
            const uint32_t w[4] = {buf[u][c].x, buf[u][c].y, buf[u][c].z, buf[u][c].w};
            const LutT* L = lut + (size_t)ch * 16 * 256;
#pragma unroll
            for (int b = 0; b < 16; ++b) {
              const LutT v = L[b * 256 + ((w[b >> 2] >> (8 * (b & 3))) & 0xffu)];
              if constexpr (U8) iacc += v;
              else if constexpr (L16) acc += __half2float(v);
              else acc += v;
            }
          }
        }
        if constexpr (U8) {
          for (int o = lpr >> 1; o > 0; o >>= 1) iacc += __shfl_xor_sync(FULL, iacc, o);
          acc = (float)iacc;
        } else {
          for (int o = lpr >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
        }
        if (L16) acc *= scale;
        if (sub == 0 && r < cnt) ck[r] = make_key(acc, (uint32_t)cid[r]);
      }
    }
  }
};

// Exact FP32 distances for the re-rank, from the index's FP32 copy.  Same
// lane/chunk mapping and summation order as the FP32 dense back-end (chunks
// in order, even and odd elements in two partial sums, their sum, then the
// butterfly), so a re-ranked distance is bit-identical to the FP32 traversal
// distance of the same row.
template <int RDT>
__device__ __forceinline__ void rerank_dists(const unsigned char* rr, int64_t stride, int nchunks, int lpr, int metric,
                                             const float* q, const int* cid, int cnt, u64* ck, int lane) {
  constexpr int U = 4;
  constexpr int EPC = Fmt<RDT>::EPC;
  const int rpi = 32 / lpr;
  const int sub = lane & (lpr - 1), grp = lane / lpr;
  const int cpl = (nchunks + lpr - 1) / lpr;
  for (int base = 0; base < cnt; base += rpi * U) {
    float acc[U], acc1[U];  // even / odd element partial sums, as in the traversal
    int ids[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int r = base + u * rpi + grp;
      ids[u] = r < cnt ? cid[r] : -1;
      acc[u] = 0.f;
      acc1[u] = 0.f;
    }
    for (int c = 0; c < cpl; ++c) {
      const int ch = sub + c * lpr;
      float qq[EPC];
#pragma unroll
      for (int e4 = 0; e4 < EPC / 4; ++e4) {
        const float4 qv = ch < nchunks ? __ldg(reinterpret_cast<const float4*>(q + ch * EPC) + e4)
                                       : make_float4(0.f, 0.f, 0.f, 0.f);
        qq[4 * e4] = qv.x;
        qq[4 * e4 + 1] = qv.y;
        qq[4 * e4 + 2] = qv.z;
        qq[4 * e4 + 3] = qv.w;
      }
      uint4 buf[U];
#pragma unroll
      for (int u = 0; u < U; ++u)
        buf[u] = (ids[u] >= 0 && ch < nchunks) ? ldg_stream16(rr + (int64_t)ids[u] * stride + ch * 16)
                                               : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        float x[EPC];
        Fmt<RDT>::unpack(buf[u], x);
#pragma unroll
        for (int e = 0; e < EPC; e += 2) {
          if (metric == KANN_L2) acc_diff_sq2(acc[u], acc1[u], qq[e], qq[e + 1], x[e], x[e + 1]);
          else acc_mul2(acc[u], acc1[u], qq[e], qq[e + 1], x[e], x[e + 1]);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      float v = acc[u] + acc1[u];
      for (int o = lpr >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
      const int r = base + u * rpi + grp;
      if (sub == 0 && r < cnt) ck[r] = make_key(metric == KANN_L2 ? v : -v, (uint32_t)ids[u]);
    }
  }
}

// ---------------------------------------------------------------------------
// Search teams (the PQ kernel): a CTA of T warps searches one query and shares
// its lookup table.  Warp 0 runs the search; at every distance evaluation and
// re-rank batch it posts a command and the candidate count in TeamCtl and the
// team meets at named barrier 1 twice (go, done), each warp computing the
// distances of one contiguous slice of the candidates.  Every row is still
// evaluated by one lane group exactly as in the one-warp search, so the
// results are the same bit for bit.  Warp 0 reaches every barrier the helpers
// wait at: the search core has no early exit, and DONE ends the query.
// ---------------------------------------------------------------------------
template <int T, class B>
__device__ __forceinline__ void team_dists(B& be, const SearchArgs& a, const int* cid, int cnt, u64* ck, int lane,
                                           TeamCtl* tc) {
  if constexpr (T == 1) {
    be.dists(a, cid, cnt, ck, lane);
  } else {
    if (lane == 0) {
      tc->cmd = TEAM_DIST;
      tc->cnt = cnt;
    }
    team_bar(T);
    int s0, n;
    team_slice(cnt, 0, T, s0, n);
    be.dists(a, cid + s0, n, ck + s0, lane);
    team_bar(T);
  }
}

// Re-rank the best R entries of W exactly and sort them (cold path, once per
// query).  Returns the number of re-ranked entries now at the front of W.
__device__ __noinline__ int rerank_phase(const unsigned char* rr, int rr_dtype, int64_t stride, int nchunks, int lpr,
                                         int metric, const float* q, int R, u64* W, u64* ck, int* cid, int lane,
                                         TeamCtl* tc, int T) {
  // ask L2 for every re-rank row at once, so that the chunk-by-chunk loads
  // below wait for L2 rather than for DRAM
  for (int j = lane; j < R; j += 32) {
    const unsigned char* row = rr + (int64_t)key_id(W[j]) * stride;
    for (int off = 0; off < nchunks * 16; off += 128) asm volatile("prefetch.global.L2 [%0];" ::"l"(row + off));
  }
  for (int b = 0; b < R; b += 64) {
    const int cb = min(64, R - b);
    for (int j = lane; j < cb; j += 32) cid[j] = (int)key_id(W[b + j]);
    __syncwarp();
    int s0 = 0, n = cb;
    if (T > 1) {
      if (lane == 0) {
        tc->cmd = TEAM_RERANK;
        tc->cnt = cb;
      }
      team_bar(T);
      team_slice(cb, 0, T, s0, n);
    }
    if (rr_dtype == KANN_BF16) rerank_dists<KANN_BF16>(rr, stride, nchunks, lpr, metric, q, cid + s0, n, ck + s0, lane);
    else rerank_dists<KANN_F32>(rr, stride, nchunks, lpr, metric, q, cid + s0, n, ck + s0, lane);
    if (T > 1) team_bar(T);
    __syncwarp();
    for (int j = lane; j < cb; j += 32) W[b + j] = ck[j];
    __syncwarp();
  }
  warp_smem_sort_n(W, R, lane);
  return R;
}

// Clear the visited table and put W's ids back (cold path); returns the
// number of ids stored.
__device__ __noinline__ int reset_visited(const Visited V, const u64* W, int len, int lane) {
  V.clear(lane);
  __syncwarp();
  int n = 0;
  for (int i = lane; i < len; i += 32) n += V.insert(key_id(W[i])) == 1;
  __syncwarp();
  return __reduce_add_sync(FULL, n);
}

// Survivors of a step (keys that beat worst(W) and are not in W) ordered by a
// bitonic network, repeats inside the batch dropped; writes the ordered keys
// and their W-ranks to ck/clb and returns their number.  Used when a step has
// many survivors or repeated keys (cold path).
__device__ __noinline__ int order_by_sort(u64 e0, u64 e1, bool k0, bool k1, const u64* W, int len, u64* ck, int* clb,
                                          int lane) {
  const unsigned lt = (1u << lane) - 1u;
  if (!k0) e0 = KEY_MAX;
  if (!k1) e1 = KEY_MAX;
  if (__ballot_sync(FULL, k1)) warp_sort64(e0, e1, lane);
  else e0 = warp_sort32(e0, lane);
  const u64 last0 = __shfl_sync(FULL, e0, 31);
  const u64 up0 = __shfl_up_sync(FULL, e0, 1);
  const u64 up1 = __shfl_up_sync(FULL, e1, 1);
  const bool ok0 = e0 != KEY_MAX && !(lane > 0 && e0 == up0);
  const bool ok1 = e1 != KEY_MAX && !(lane > 0 ? e1 == up1 : e1 == last0);
  const int lb0 = ok0 ? lower_bound_w(W, len, e0) : 0;
  const int lb1 = ok1 ? lower_bound_w(W, len, e1) : 0;
  const unsigned s0 = __ballot_sync(FULL, ok0), s1 = __ballot_sync(FULL, ok1);
  const int cs0 = __popc(s0);
  __syncwarp();
  if (ok0) {
    ck[__popc(s0 & lt)] = e0;
    clb[__popc(s0 & lt)] = lb0;
  }
  if (ok1) {
    ck[cs0 + __popc(s1 & lt)] = e1;
    clb[cs0 + __popc(s1 & lt)] = lb1;
  }
  return cs0 + __popc(s1);
}

// Merge a batch of up to 64 candidate keys (two per lane, KEY_MAX = none)
// into W: the survivors are the keys that beat worst(W) and are not in W
// already; they are ranked (by counting, or by a sorting network when there
// are many or some repeat), W[lo..len) is moved right by the number of
// survivors ranked before each entry, last chunk first, and the survivors are
// dropped in place.  ck_out / clb receive the ranked survivors and their
// W-ranks (64 entries each).  The result is the ef best of W and the batch.
__device__ __forceinline__ void merge_batch(u64 e0, u64 e1, u64* W, int& len, int ef, int& cursor, u64* ck_out,
                                            int* clb, int lane) {
  const u64 worst = len >= ef ? kmask(W[len - 1]) : KEY_MAX;
  bool k0 = e0 < worst, k1 = e1 < worst;
  int lb0 = 0, lb1 = 0;
  if (k0) {
    lb0 = lower_bound_w(W, len, e0);
    k0 = !(lb0 < len && kmask(W[lb0]) == e0);
  }
  if (k1) {
    lb1 = lower_bound_w(W, len, e1);
    k1 = !(lb1 < len && kmask(W[lb1]) == e1);
  }
  const unsigned s0 = __ballot_sync(FULL, k0), s1 = __ballot_sync(FULL, k1);
  const int c = __popc(s0) + __popc(s1);
  if (c == 0) return;
  int cnew = 0;
  bool sorted = false;
  if (c <= 16) {
    // rank of a survivor = number of survivors with a smaller key
    int r0 = 0, r1 = 0;
    bool d0 = false, d1 = false;
    for (unsigned m = s0; m; m &= m - 1) {
      const int src = __ffs(m) - 1;
      const u64 x = __shfl_sync(FULL, e0, src);
      r0 += x < e0;
      r1 += x < e1;
      d0 |= (x == e0) && (src < lane);
      d1 |= x == e1;
    }
    for (unsigned m = s1; m; m &= m - 1) {
      const int src = __ffs(m) - 1;
      const u64 x = __shfl_sync(FULL, e1, src);
      r0 += x < e0;
      r1 += x < e1;
      d1 |= (x == e1) && (src < lane);
    }
    // a key repeated inside the batch (possible only after the visited
    // table forgot, with a repeated edge) takes the sorting path
    if (__ballot_sync(FULL, (k0 && d0) || (k1 && d1)) == 0) {
      __syncwarp();
      if (k0) {
        ck_out[r0] = e0;
        clb[r0] = lb0;
      }
      if (k1) {
        ck_out[r1] = e1;
        clb[r1] = lb1;
      }
      cnew = c;
      sorted = true;
    }
  }
  if (!sorted) cnew = order_by_sort(e0, e1, k0, k1, W, len, ck_out, clb, lane);
  __syncwarp();
  const int lo = clb[0];
  for (int top = len; top > lo; top -= 32) {
    const int i = top - 32 + lane;
    const bool act = i >= lo;
    u64 val = 0;
    int dest = 0;
    if (act) {
      val = W[i];
      dest = i + count_le(clb, cnew, i);
    }
    __syncwarp();
    if (act && dest < ef) W[dest] = val;
    __syncwarp();
  }
  for (int j = lane; j < cnew; j += 32) {
    const int pos = j + clb[j];
    if (pos < ef) W[pos] = ck_out[j];
  }
  __syncwarp();
  len = min(len + cnew, ef);
  if (lo < cursor) cursor = lo;
}

// Per-query status bits a back-end reports (the sparse back-end's truncated
// query; found by argument-dependent lookup where a back-end defines one).
template <class B>
__device__ __forceinline__ uint32_t backend_status(const B&) { return 0u; }

// The distance the output reports for a traversal key (the PQ back-end's
// uint8 table keeps integer sums in W); identity for the others.
template <class B>
__device__ __forceinline__ float backend_out_dist(const B&, float d) { return d; }
template <int CPL, int LF>
__device__ __forceinline__ float backend_out_dist(const PQBackend<CPL, LF>& b, float d) { return b.out_dist(d); }

// One step of the multi-expansion layer-0 search (a batched variant of the
// HNSW step, under its own oracle form; not the parity search): the
// min(a.expand, remaining hop budget) best unexpanded entries of W are
// marked expanded together, their adjacency rows read at once, their
// unvisited neighbours evaluated in one batch of up to 64 * a.expand rows,
// and the batch merged into W 64 keys at a time (the bounded top-ef merge
// does not depend on order).  More rows are in flight per dependent step
// than with one expansion.  Returns false when W has no unexpanded entry or
// the hop cap is reached.
template <int T, class B>
__device__ __forceinline__ bool multi_step(const SearchArgs& a, B& be, u64* W, u64* ck, int* cid, int* clb,
                                           const Visited& V, int& len, int ef, int& cursor, int& hops, int& stored,
                                           uint32_t& st, int& c_l0d, int& c_l0e, int lane, TeamCtl* tc) {
  const unsigned lt = (1u << lane) - 1u;
  const int P = a.expand;
  int s0 = -1, s1 = -1, s2 = -1, s3 = -1, ns = 0;
  for (int b = cursor; b < len && ns < P; b += 32) {
    const int i = b + lane;
    const bool un = i < len && !(W[i] & FLAG);
    unsigned m = __ballot_sync(FULL, un);
    while (m != 0u && ns < P) {
      const int pos = b + __ffs(m) - 1;
      m &= m - 1;
      if (ns == 0) s0 = pos;
      else if (ns == 1) s1 = pos;
      else if (ns == 2) s2 = pos;
      else s3 = pos;
      ++ns;
    }
  }
  if (ns == 0) return false;
  if (hops >= a.max_hops) {
    st |= KANN_QSTAT_HOPCAP;
    return false;
  }
  if (ns > a.max_hops - hops) ns = a.max_hops - hops;
  hops += ns;
  c_l0e += ns;
  const int sel[4] = {s0, s1, s2, s3};
  int ids[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) ids[j] = j < ns ? (int)key_id(W[sel[j]]) : -1;
  __syncwarp();
  if (lane == 0) {
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (j < ns) W[sel[j]] |= FLAG;
  }
  cursor = (ns == 1 ? s0 : ns == 2 ? s1 : ns == 3 ? s2 : s3) + 1;
  int v[8];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int32_t* nb = a.l0 + (int64_t)(ids[j] < 0 ? 0 : ids[j]) * a.M0;
    v[2 * j] = (j < ns && lane < a.M0) ? __ldg(nb + lane) : -1;
    v[2 * j + 1] = (j < ns && lane + 32 < a.M0) ? __ldg(nb + 32 + lane) : -1;
  }
  int cnt = 0;
  bool forgot = false, bad = false;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    int vj = v[j];
    bad |= vj >= a.n;
    if (vj >= a.n) vj = -1;
    const int r = vj >= 0 ? V.insert((uint32_t)vj) : 0;
    forgot |= r == 2;
    stored += __popc(__ballot_sync(FULL, r == 1));
    const unsigned bm = __ballot_sync(FULL, r != 0);
    if (r) cid[cnt + __popc(bm & lt)] = vj;
    cnt += __popc(bm);
  }
  if (forgot) st |= KANN_QSTAT_FORGOT;
  if (bad) st |= KANN_QSTAT_BAD_ID;
  __syncwarp();
  if (cnt == 0) return true;
  team_dists<T>(be, a, cid, cnt, ck, lane, tc);
  __syncwarp();
  c_l0d += cnt;
  u64* ck_out = ck + 64 * a.expand;  // past every candidate key of the batch
  for (int off = 0; off < cnt; off += 64) {
    const u64 e0 = off + lane < cnt ? ck[off + lane] : KEY_MAX;
    const u64 e1 = off + lane + 32 < cnt ? ck[off + lane + 32] : KEY_MAX;
    __syncwarp();
    merge_batch(e0, e1, W, len, ef, cursor, ck_out, clb, lane);
  }
  return true;
}

template <class B, int T = 1, bool MULTI = false>
__device__ __forceinline__ void search_one(const SearchArgs& a, B& be, int qi, int lane, unsigned char* ws,
                                           TeamCtl* tc = nullptr) {
  const WarpSmem s = WarpSmem::of<MULTI>(ws, a);
  u64* W = s.W;
  u64* ck = s.ck;
  int* cid = s.cid;
  int* clb = s.clb;
  const Visited V{s.H, a.hbits, a.vis_k, a.vis_r};
  const unsigned lt = (1u << lane) - 1u;

  int k = a.k, ef = a.ef;
  if (a.k_arr) {
    k = min(max(a.k_arr[qi], 1), a.kmax);
    ef = a.ef_arr[qi];
  }
  ef = min(max(ef, k), a.efmax);
  uint32_t st = 0;
  int c_l0d = 0, c_l0e = 0, c_upd = 0, c_uph = 0;

  if constexpr (T == 1) be.init(a, qi, lane, s.extra);  // a team builds its table together beforehand
  st |= backend_status(be);

  // 1. entry point
  if (lane == 0) cid[0] = a.entry;
  __syncwarp();
  team_dists<T>(be, a, cid, 1, ck, lane, tc);
  __syncwarp();
  u64 cur = ck[0];
  c_upd = 1;
  __syncwarp();

  // 2. greedy descent through the upper layers
  for (int l = a.max_level; l >= 1; --l) {
    for (;;) {
      const int cur_id = (int)key_id(cur);
      const int slot = __ldg(a.upper_slot + cur_id);
      int v = -1;
      if (slot >= 0 && lane < a.M) v = __ldg(a.upper + ((int64_t)slot * a.max_level + (l - 1)) * a.M + lane);
      if (slot < 0 || v >= a.n) st |= KANN_QSTAT_BAD_ID;
      if (v >= a.n) v = -1;
      const bool ok = v >= 0;
      const unsigned bal = __ballot_sync(FULL, ok);
      const int cnt = __popc(bal);
      if (ok) cid[__popc(bal & lt)] = v;
      __syncwarp();
      team_dists<T>(be, a, cid, cnt, ck, lane, tc);
      __syncwarp();
      c_upd += cnt;
      ++c_uph;
      const u64 best = warp_min64(lane < cnt ? ck[lane] : KEY_MAX);
      __syncwarp();
      if (best < cur) cur = best;
      else break;
    }
  }

  // 3. layer-0 beam
  V.clear(lane);
  __syncwarp();
  if (lane == 0) {
    V.insert(key_id(cur));
    W[0] = cur;
  }
  __syncwarp();
  int len = 1, cursor = 0, hops = 0, stored = 1;
  for (;;) {
    if constexpr (MULTI) {
      if (!multi_step<T>(a, be, W, ck, cid, clb, V, len, ef, cursor, hops, stored, st, c_l0d, c_l0e, lane, tc))
        break;
      if (stored > V.limit()) {
        st |= KANN_QSTAT_FORGOT;
        stored = reset_visited(V, W, len, lane);
      }
      continue;
    }
    int p = -1;
    for (int b = cursor; b < len; b += 32) {
      const int i = b + lane;
      const bool un = i < len && !(W[i] & FLAG);
      const unsigned m = __ballot_sync(FULL, un);
      if (m) {
        p = b + __ffs(m) - 1;
        break;
      }
    }
    if (p < 0) break;
    if (hops >= a.max_hops) {
      st |= KANN_QSTAT_HOPCAP;
      break;
    }
    ++hops;
    const u64 ce = W[p];
    __syncwarp();
    if (lane == 0) W[p] = ce | FLAG;
    cursor = p + 1;
    const int c_id = (int)key_id(ce);
    const int32_t* nb = a.l0 + (int64_t)c_id * a.M0;
    int v0 = lane < a.M0 ? __ldg(nb + lane) : -1;
    int v1 = lane + 32 < a.M0 ? __ldg(nb + 32 + lane) : -1;
    if (v0 >= a.n || v1 >= a.n) st |= KANN_QSTAT_BAD_ID;
    if (v0 >= a.n) v0 = -1;
    if (v1 >= a.n) v1 = -1;
    const int r0 = v0 >= 0 ? V.insert((uint32_t)v0) : 0;
    const int r1 = v1 >= 0 ? V.insert((uint32_t)v1) : 0;
    if (r0 == 2 || r1 == 2) st |= KANN_QSTAT_FORGOT;
    stored += __popc(__ballot_sync(FULL, r0 == 1)) + __popc(__ballot_sync(FULL, r1 == 1));
    const unsigned b0 = __ballot_sync(FULL, r0 != 0), b1 = __ballot_sync(FULL, r1 != 0);
    const int c0 = __popc(b0), cnt = c0 + __popc(b1);
    if (r0) cid[__popc(b0 & lt)] = v0;
    if (r1) cid[c0 + __popc(b1 & lt)] = v1;
    __syncwarp();
    ++c_l0e;
    if (cnt > 0) {
      team_dists<T>(be, a, cid, cnt, ck, lane, tc);
      __syncwarp();
      c_l0d += cnt;
      // survivors: keys that beat worst(W) and are not in W already (the
      // merge of merge_batch, written out here for the one-expansion step,
      // whose register allocation it keeps)
      const u64 worst = len >= ef ? kmask(W[len - 1]) : KEY_MAX;
      const u64 e0 = lane < cnt ? ck[lane] : KEY_MAX;
      const u64 e1 = lane + 32 < cnt ? ck[lane + 32] : KEY_MAX;
      bool k0 = e0 < worst, k1 = e1 < worst;
      int lb0 = 0, lb1 = 0;
      if (k0) {
        lb0 = lower_bound_w(W, len, e0);
        k0 = !(lb0 < len && kmask(W[lb0]) == e0);
      }
      if (k1) {
        lb1 = lower_bound_w(W, len, e1);
        k1 = !(lb1 < len && kmask(W[lb1]) == e1);
      }
      const unsigned s0 = __ballot_sync(FULL, k0), s1 = __ballot_sync(FULL, k1);
      const int c = __popc(s0) + __popc(s1);
      int cnew = 0;
      if (c > 0) {
        bool sorted = false;
        if (c <= 16) {
          int r0 = 0, r1 = 0;
          bool d0 = false, d1 = false;
          for (unsigned m = s0; m; m &= m - 1) {
            const int src = __ffs(m) - 1;
            const u64 x = __shfl_sync(FULL, e0, src);
            r0 += x < e0;
            r1 += x < e1;
            d0 |= (x == e0) && (src < lane);
            d1 |= x == e1;
          }
          for (unsigned m = s1; m; m &= m - 1) {
            const int src = __ffs(m) - 1;
            const u64 x = __shfl_sync(FULL, e1, src);
            r0 += x < e0;
            r1 += x < e1;
            d1 |= (x == e1) && (src < lane);
          }
          if (__ballot_sync(FULL, (k0 && d0) || (k1 && d1)) == 0) {
            __syncwarp();
            if (k0) {
              ck[r0] = e0;
              clb[r0] = lb0;
            }
            if (k1) {
              ck[r1] = e1;
              clb[r1] = lb1;
            }
            cnew = c;
            sorted = true;
          }
        }
        if (!sorted) cnew = order_by_sort(e0, e1, k0, k1, W, len, ck, clb, lane);
        __syncwarp();
        const int lo = clb[0];
        for (int top = len; top > lo; top -= 32) {
          const int i = top - 32 + lane;
          const bool act = i >= lo;
          u64 val = 0;
          int dest = 0;
          if (act) {
            val = W[i];
            dest = i + count_le(clb, cnew, i);
          }
          __syncwarp();
          if (act && dest < ef) W[dest] = val;
          __syncwarp();
        }
        for (int j = lane; j < cnew; j += 32) {
          const int pos = j + clb[j];
          if (pos < ef) W[pos] = ck[j];
        }
        __syncwarp();
        len = min(len + cnew, ef);
        if (lo < cursor) cursor = lo;
      }
    }
    // visited-table upkeep: keep the load factor below the table's limit
    if (stored > V.limit()) {
      st |= KANN_QSTAT_FORGOT;
      stored = reset_visited(V, W, len, lane);
    }
  }

  // 4. exact re-rank of the best R entries
  int nout = len;
  const bool reranked = a.R != 0 && a.rr_data != nullptr;
  if (reranked) {
    const int R = min(a.R < 0 ? ef : a.R, len);
    nout = rerank_phase(a.rr_data, a.rr_dtype, a.rr_stride, a.rr_nchunks, a.rr_lpr, a.metric, a.q + (size_t)qi * a.d, R, W, ck,
                        cid, lane, tc, T);
  }

  // 5. output
  const int ld = a.k_arr ? a.kmax : a.k;
  for (int j = lane; j < ld; j += 32) {
    int32_t id = -1;
    float dd = __int_as_float(0x7f800000);
    if (j < k && j < nout) {
      const u64 key = kmask(W[j]);
      id = (int32_t)key_id(key);
      dd = key_dist(key);
      if (!reranked) dd = backend_out_dist(be, dd);
    }
    a.out_ids[(size_t)qi * ld + j] = id;
    a.out_d[(size_t)qi * ld + j] = dd;
  }
  st = __reduce_or_sync(FULL, st);
  if (lane == 0) {
    if (a.status) a.status[qi] = st;
    if (a.counters) {
      a.counters[(size_t)qi * 4 + 0] = c_l0d;
      a.counters[(size_t)qi * 4 + 1] = c_l0e;
      a.counters[(size_t)qi * 4 + 2] = c_upd;
      a.counters[(size_t)qi * 4 + 3] = c_uph;
    }
  }
}

// Register budget from the query registers a lane holds: <= 8 -> 64
// registers (32 warps per SM), <= 16 -> 80 (24 warps), wider -> 128.  The
// lean form (half the rows in flight) always asks for 64 when q <= 16.
template <int DT, int CPLT, bool LEAN>
struct MinBlocks {
  static constexpr int q = CPLT * Fmt<DT>::EPC;
  static constexpr int value = q <= 8 ? 8 : (q <= 16 ? (LEAN ? 8 : 6) : 4);
};

// Queries of one launch: a plain grid gives warp w of CTA b query
// b * warps + w; the persistent form has every warp take the next query index
// from a device counter until the batch is exhausted (work stealing: a warp
// that finishes a cheap query starts the next one at once).
template <class B, bool MULTI = false>
__device__ __forceinline__ void run_queries(const SearchArgs& a, B& be) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned char* ws = smem + (size_t)warp * a.warp_smem;
  if (a.work_counter == nullptr) {
    const int qi = blockIdx.x * (blockDim.x >> 5) + warp;
    if (qi < a.nq) search_one<B, 1, MULTI>(a, be, qi, lane, ws);
    return;
  }
  int nq = a.nq;
  if (a.d_n) nq = min(nq, max(0, *a.d_n));
  for (;;) {
    int qi = 0;
    if (lane == 0) qi = atomicAdd(a.work_counter, 1);
    qi = __shfl_sync(FULL, qi, 0);
    if (qi >= nq) break;
    search_one<B, 1, MULTI>(a, be, qi, lane, ws);
  }
}

// A helper warp of a team: serve warp 0's commands until the query is done.
template <int T, class B>
__device__ __forceinline__ void team_helper(const SearchArgs& a, B& be, int qi, int lane, int w, unsigned char* ws,
                                            TeamCtl* tc) {
  const WarpSmem s = WarpSmem::of(ws, a);  // warp 0's candidate ids and keys
  for (;;) {
    team_bar(T);
    const int cmd = tc->cmd, cnt = tc->cnt;
    if (cmd == TEAM_DONE) break;
    int s0, n;
    team_slice(cnt, w, T, s0, n);
    if (cmd == TEAM_DIST) {
      be.dists(a, s.cid + s0, n, s.ck + s0, lane);
    } else {
      const float* q = a.q + (size_t)qi * a.d;
      if (a.rr_dtype == KANN_BF16)
        rerank_dists<KANN_BF16>(a.rr_data, a.rr_stride, a.rr_nchunks, a.rr_lpr, a.metric, q, s.cid + s0, n,
                                s.ck + s0, lane);
      else
        rerank_dists<KANN_F32>(a.rr_data, a.rr_stride, a.rr_nchunks, a.rr_lpr, a.metric, q, s.cid + s0, n,
                               s.ck + s0, lane);
    }
    team_bar(T);
  }
}

// Queries of a team launch: one query per CTA of T warps at a time (plain:
// CTA b takes query b; persistent: thread 0 takes the next index from the
// device counter).  The team builds the query's table, warp 0 searches, the
// others serve it; TeamCtl sits after the query's shared memory.
template <int T, class B>
__device__ __forceinline__ void run_queries_team(const SearchArgs& a, B& be) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  TeamCtl* tc = reinterpret_cast<TeamCtl*>(smem + a.warp_smem);
  int nq = a.nq;
  if (a.work_counter && a.d_n) nq = min(nq, max(0, *a.d_n));
  for (int it = 0;; ++it) {
    int qi;
    if (a.work_counter == nullptr) {
      if (it > 0) break;
      qi = blockIdx.x;
    } else {
      if (threadIdx.x == 0) tc->qi = atomicAdd(a.work_counter, 1);
      team_bar(T);
      qi = tc->qi;
      team_bar(T);
    }
    if (qi >= nq) break;
    be.init_team(a, qi, lane, w, T, smem, tc);
    if (w == 0) {
      search_one<B, T>(a, be, qi, lane, smem, tc);
      if (lane == 0) tc->cmd = TEAM_DONE;
      team_bar(T);
    } else {
      team_helper<T>(a, be, qi, lane, w, smem, tc);
    }
  }
}

template <int DT, int CPLT, bool LEAN, int MET, int LPR, bool MULTI = false>
__global__ void __launch_bounds__(128, MinBlocks<DT, CPLT, LEAN>::value) search_dense_kernel(const SearchArgs a) {
  DenseBackend<DT, CPLT, LEAN, MET, LPR> be;
  run_queries<decltype(be), MULTI>(a, be);
}

// A team of T warps per query (one CTA): the same rows in flight per warp
// and the same registers per thread as the one-warp kernel.
template <int DT, int CPLT, int MET, int LPR, int T>
__global__ void __launch_bounds__(T * 32, MinBlocks<DT, CPLT, false>::value * 4 / T)
    search_dense_team_kernel(const SearchArgs a) {
  DenseBackend<DT, CPLT, false, MET, LPR> be;
  run_queries_team<T>(a, be);
}

constexpr int PQ_TEAM = 8;  // warps sharing one query's lookup table (TeamCtl::wmax holds 8)

// Teams per SM the kernel is compiled for: the uint8 table (48 KB at m = 192)
// lets four 8-warp teams share an SM (64 registers a thread; measured 11%
// faster than three teams at 80 registers on a 200k x 768 set, despite the
// spills).
template <int LF>
struct PQTeamsPerSM {
  static constexpr int value = LF == PQ_LUT_U8 ? 4 : 1;
};

template <int CPLT, int LF>
__global__ void __launch_bounds__(PQ_TEAM * 32, PQTeamsPerSM<LF>::value) search_pq_kernel(const SearchArgs a) {
  PQBackend<CPLT, LF> be;
  run_queries_team<PQ_TEAM>(a, be);
}

template <int DT, int MET, bool MULTI = false>
SearchKernelFn pick_general(int cplt, bool lean) {
  switch (cplt * 2 + (lean ? 1 : 0)) {
    case 2: return search_dense_kernel<DT, 1, false, MET, 0, MULTI>;
    case 4: return search_dense_kernel<DT, 2, false, MET, 0, MULTI>;
    case 5: return MULTI ? nullptr : search_dense_kernel<DT, 2, true, MET, 0>;
    case 8: return search_dense_kernel<DT, 4, false, MET, 0, MULTI>;
    case 16: return search_dense_kernel<DT, 8, false, MET, 0, MULTI>;
    default: return nullptr;
  }
}

template <int DT, int CPLT, bool LEAN, int MET, bool MULTI = false>
SearchKernelFn pick_exact(int lpr) {
  switch (lpr) {
    case 2: return search_dense_kernel<DT, CPLT, LEAN, MET, 2, MULTI>;
    case 4: return search_dense_kernel<DT, CPLT, LEAN, MET, 4, MULTI>;
    case 8: return search_dense_kernel<DT, CPLT, LEAN, MET, 8, MULTI>;
    case 16: return search_dense_kernel<DT, CPLT, LEAN, MET, 16, MULTI>;
    case 32: return search_dense_kernel<DT, CPLT, LEAN, MET, 32, MULTI>;
    default: return nullptr;
  }
}

// Dense kernel of one storage format: the exact-tiling form when the launch's
// rows are lpr_exact * cplt chunks with cplt the format's default chunks per
// lane (the lean form exists for two chunks per lane), else the general form.
// Multi-expansion kernel of one storage format (no lean variant): the
// exact-tiling form at the format's default chunks per lane, else the
// general form.  Instantiated in kann_search_{f32,f16,bf16,e4m3}_multi.cu.
template <int DT>
SearchKernelFn pick_dense_multi_t(int cplt, int metric, int lpr_exact) {
  constexpr int CX = default_chunks_per_lane(DT);
  SearchKernelFn f = nullptr;
  if (lpr_exact > 0 && cplt == CX)
    f = metric == KANN_L2 ? pick_exact<DT, CX, false, KANN_L2, true>(lpr_exact)
                          : pick_exact<DT, CX, false, KANN_IP, true>(lpr_exact);
  if (!f) f = metric == KANN_L2 ? pick_general<DT, KANN_L2, true>(cplt, false) : pick_general<DT, KANN_IP, true>(cplt, false);
  return f;
}

template <int DT, int MET, int T>
SearchKernelFn pick_team(int cplt, int lpr_exact) {
  constexpr int CX = default_chunks_per_lane(DT);
  if (lpr_exact > 0 && cplt == CX) {
    switch (lpr_exact) {
      case 2: return search_dense_team_kernel<DT, CX, MET, 2, T>;
      case 4: return search_dense_team_kernel<DT, CX, MET, 4, T>;
      case 8: return search_dense_team_kernel<DT, CX, MET, 8, T>;
      case 16: return search_dense_team_kernel<DT, CX, MET, 16, T>;
      case 32: return search_dense_team_kernel<DT, CX, MET, 32, T>;
      default: break;
    }
  }
  switch (cplt) {
    case 1: return search_dense_team_kernel<DT, 1, MET, 0, T>;
    case 2: return search_dense_team_kernel<DT, 2, MET, 0, T>;
    case 4: return search_dense_team_kernel<DT, 4, MET, 0, T>;
    case 8: return search_dense_team_kernel<DT, 8, MET, 0, T>;
    default: return nullptr;
  }
}

// Team kernel of one storage format (team = 2 or 4 warps per query):
// exact-tiling form at the format's default chunks per lane, else general.
template <int DT>
SearchKernelFn pick_dense_team_t(int cplt, int metric, int lpr_exact, int team) {
  if (team == 2) return metric == KANN_L2 ? pick_team<DT, KANN_L2, 2>(cplt, lpr_exact) : pick_team<DT, KANN_IP, 2>(cplt, lpr_exact);
  if (team == 4) return metric == KANN_L2 ? pick_team<DT, KANN_L2, 4>(cplt, lpr_exact) : pick_team<DT, KANN_IP, 4>(cplt, lpr_exact);
  return nullptr;
}

template <int DT>
SearchKernelFn pick_dense_t(int cplt, bool lean, int metric, int lpr_exact) {
  constexpr int CX = default_chunks_per_lane(DT);
  SearchKernelFn f = nullptr;
  if (lpr_exact > 0 && cplt == CX) {
    if constexpr (CX == 2) {
      if (lean)
        f = metric == KANN_L2 ? pick_exact<DT, CX, true, KANN_L2>(lpr_exact) : pick_exact<DT, CX, true, KANN_IP>(lpr_exact);
    }
    if (!lean)
      f = metric == KANN_L2 ? pick_exact<DT, CX, false, KANN_L2>(lpr_exact) : pick_exact<DT, CX, false, KANN_IP>(lpr_exact);
  }
  if (!f) f = metric == KANN_L2 ? pick_general<DT, KANN_L2>(cplt, lean) : pick_general<DT, KANN_IP>(cplt, lean);
  return f;
}

}  // namespace
}  // namespace kann
