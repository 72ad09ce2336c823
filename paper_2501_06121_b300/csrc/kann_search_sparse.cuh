// kann_search_sparse.cuh -- the sparse back-end of the batched HNSW search
// (device code; the search core is kann_search_impl.cuh, the kernels and
// their launchers kann_search.cu).
#pragma once
#include "kann_search_impl.cuh"

namespace kann {
namespace {

// ---------------------------------------------------------------------------
// Sparse back-end (inner product over term/weight lists).  The query is held
// as a presence bitmap over the vocabulary, per-word prefix counts of set
// bits, and its weights in term order: query terms are sorted and unique, so
// the rank of a present term t -- the number of query terms below it, i.e.
// prefix[t / 32] + popcount of word t / 32 below bit t % 32 -- is its index
// in the weight array.  Each candidate document's term list is walked by a
// group of 8 lanes, each lane summing w_q(t) * w_x(t) over its positions in
// order; distance = -sum.  A query keeps its first 512 terms (flagged
// otherwise); terms >= vocab never match.
// ---------------------------------------------------------------------------
constexpr int SP_QMAX = 512;  // query terms kept
constexpr int SP_LPD = 8;     // lanes per document
constexpr int SP_TPL = 8;     // terms per lane loaded before their lookups

__host__ __device__ constexpr int sparse_words(int vocab) { return (vocab + 31) / 32; }
// bytes of a query's tables: bitmap (4 per word), prefix counts (2 per word,
// rounded to 4), weights
__host__ __device__ constexpr int sparse_query_bytes(int vocab) {
  return sparse_words(vocab) * 4 + (sparse_words(vocab) * 2 + 3) / 4 * 4 + SP_QMAX * 4;
}

struct SparseBackend {
  const SparseArgs* sp;
  uint32_t* bm;       // [words] presence bits
  uint16_t* pre;      // [words] set bits in the words before
  float* qw;          // [<= SP_QMAX] weights in term order
  uint32_t trunc;

  __device__ __forceinline__ void place(unsigned char* extra) {
    bm = reinterpret_cast<uint32_t*>(extra);
    pre = reinterpret_cast<uint16_t*>(bm + sparse_words(sp->vocab));
    qw = reinterpret_cast<float*>(extra + sparse_query_bytes(sp->vocab) - SP_QMAX * 4);
    trunc = 0u;
  }

  // a search team: warp 0 builds the query's tables in the team's region,
  // every warp reads them; ends with the team at barrier 1
  __device__ __forceinline__ void init_team(const SearchArgs& a, int qi, int lane, int w, int T, unsigned char* ws,
                                            TeamCtl*) {
    unsigned char* extra = WarpSmem::of(ws, a).extra;
    if (w == 0) init(a, qi, lane, extra);
    else place(extra);
    team_bar(T);
  }

  __device__ __forceinline__ void init(const SearchArgs& a, int qi, int lane, unsigned char* extra) {
    const int words = sparse_words(sp->vocab);
    place(extra);
    for (int i = lane; i < words; i += 32) bm[i] = 0u;
    __syncwarp();
    const int64_t b = sp->q_indptr[qi], e = sp->q_indptr[qi + 1];
    const int nt = e - b < SP_QMAX ? (int)(e - b) : SP_QMAX;
    trunc = e - b > SP_QMAX ? 1u : 0u;
    for (int j = lane; j < nt; j += 32) {
      const uint32_t t = sp->q_terms[b + j];
      if (t < (uint32_t)sp->vocab) atomicOr(bm + (t >> 5), 1u << (t & 31));
    }
    __syncwarp();
    // prefix counts: each lane a contiguous block of words, then a warp scan
    const int per = (words + 31) / 32, w0 = lane * per, w1 = min(words, w0 + per);
    int c = 0;
    for (int i = w0; i < w1; ++i) c += __popc(bm[i]);
    int incl = c;
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(FULL, incl, o);
      if (lane >= o) incl += v;
    }
    int run = incl - c;
    for (int i = w0; i < w1; ++i) {
      pre[i] = (uint16_t)run;
      run += __popc(bm[i]);
    }
    // weights in term order (terms >= vocab, which never match, keep their
    // slots so that the ranks of the others stay their positions)
    for (int j = lane; j < nt; j += 32) qw[j] = sp->q_w[b + j];
    __syncwarp();
  }

  // Distances of cnt (<= 64) candidate documents.  The offsets of every
  // candidate are loaded first, two documents per lane, so the batch pays
  // one round trip for them; then for each group of DPI documents every
  // lane loads up to SP_TPL of its document's terms and weights before the
  // first lookup (a document of up to SP_TPL * SP_LPD terms costs one more
  // round trip).  Lane sub of a document's group sums the products of terms
  // sub, sub + SP_LPD, ... in that order (fmaf), then the group's butterfly:
  // the same order for a document wherever it sits in a batch.
  __device__ __forceinline__ void dists(const SearchArgs&, const int* cid, int cnt, u64* ck, int lane) {
    const int sub = lane & (SP_LPD - 1), grp = lane / SP_LPD;
    constexpr int DPI = 32 / SP_LPD;  // documents per warp iteration
    const uint32_t vocab = (uint32_t)sp->vocab;
    int64_t ob[2] = {0, 0};  // offsets of candidates lane and lane + 32
    int ol[2] = {0, 0};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int r = lane + 32 * h;
      const int id = r < cnt ? cid[r] : -1;
      if (id >= 0) {
        ob[h] = __ldg(sp->indptr + id);
        ol[h] = (int)(__ldg(sp->indptr + id + 1) - ob[h]);
      }
    }
    for (int base = 0; base < cnt; base += DPI) {
      const int r = base + grp;
      const int src = r & 31;
      const int64_t bA = __shfl_sync(FULL, ob[0], src), bB = __shfl_sync(FULL, ob[1], src);
      const int lA = __shfl_sync(FULL, ol[0], src), lB = __shfl_sync(FULL, ol[1], src);
      const int id = r < cnt ? cid[r] : -1;
      const int len = id >= 0 ? (r < 32 ? lA : lB) : 0;
      const int64_t b = r < 32 ? bA : bB;
      const uint16_t* tp = sp->terms + b;
      const float* wp = sp->w + b;
      float acc = 0.f;
      for (int t0 = sub; t0 < len; t0 += SP_TPL * SP_LPD) {
        uint32_t tm[SP_TPL];
        float wx[SP_TPL];
#pragma unroll
        for (int u = 0; u < SP_TPL; ++u) {
          const int t = t0 + u * SP_LPD;
          tm[u] = t < len ? (uint32_t)__ldg(tp + t) : 0xffffffffu;
          wx[u] = t < len ? __ldg(wp + t) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < SP_TPL; ++u) {
          const uint32_t t = tm[u];
          if (t < vocab) {
            const uint32_t wd = bm[t >> 5];
            if ((wd >> (t & 31)) & 1u) {
              const int rk = pre[t >> 5] + __popc(wd & ((1u << (t & 31)) - 1u));
              acc = fmaf(qw[rk], wx[u], acc);
            }
          }
        }
      }
      for (int o = SP_LPD >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
      if (sub == 0 && r < cnt) ck[r] = make_key(-acc, (uint32_t)id);
    }
  }
};

__device__ __forceinline__ uint32_t backend_status(const SparseBackend& b) {
  return b.trunc ? KANN_QSTAT_QUERY_TRUNCATED : 0u;
}

}  // namespace
}  // namespace kann
