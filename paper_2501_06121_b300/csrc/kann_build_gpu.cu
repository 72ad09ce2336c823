// kann_build_gpu.cu -- HNSW construction with the layer-0 insertions on the GPU
// (the indexing pipeline of the paper, Sec. 2 / Fig. 1, HNSW per Malkov &
// Yashunin Alg. 1 and the neighbour-selection heuristic of Alg. 4).
//
// 1. Levels are the counter-based ones of kann_hnsw_levels.  Every node of
//    level >= 1 (about n / M of them) is inserted on the host, in id order,
//    by the library's host builder (one thread per 4,096 such nodes at
//    most): this makes the upper layers complete and gives layer 0 its first
//    nodes.
// 2. The remaining nodes (level 0) are inserted on the GPU in id order, in
//    batches of at most 1/32 of the nodes already in the graph (a node then
//    receives about M / 32 reverse links per batch on average; on the
//    1M x 128 set the graph searches as well as the sequentially built one:
//    recall@10 0.9541 against 0.9537 at ef 56, and 1/8 gave 0.9503).  For a
//    batch:
//      a. the library's search (greedy descent, then the layer-0 beam with
//         ef = efConstruction) returns each node's efConstruction best
//         candidates among the nodes inserted so far;
//      b. one warp per node keeps up to M of them by the heuristic (a
//         candidate is kept when it is closer to the node than to every
//         candidate kept before it) and writes the node's list;
//      c. each kept link also goes to the neighbour's inbox (INBOX slots per
//         node and batch; a link beyond them keeps only its forward edge);
//      d. one warp per neighbour that received links appends them, or, when
//         its list would exceed 2M, shrinks list + inbox to 2M by the same
//         heuristic seen from the neighbour.
//    Nodes of one batch do not see each other (they join the graph together);
//    that is the only difference from sequential insertion in this order.
// Distances are FP32 in the direct form.  The result is the serialised graph
// of include/kann.h in caller-owned device arrays.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <thread>
#include <vector>

#include "kann_device.cuh"
#include "kann_internal.h"

namespace kann {
namespace {

constexpr int INBOX = 16;  // reverse links a node can receive per batch
constexpr int CMAX = KANN_MAX_M0 + INBOX;  // candidates of a list merge
// shared memory of one merging warp, in 8-byte words: the candidates' keys
// [CMAX], the kept ids [KANN_MAX_M0 ints], the candidates' ids [CMAX ints]
constexpr int MRG_WORDS = CMAX + KANN_MAX_M0 / 2 + (CMAX + 1) / 2;

// FP32 distance between two rows of d floats (d a multiple of 4) computed by
// one thread: L2 = sum (a - b)^2, IP = -sum a b.
__device__ __forceinline__ float row_dist(const float* a, const float* b, int d, int metric);

// The items a build links: dense FP32 rows, or sparse term lists (distance
// -IP by a merge-join of the two sorted lists, FP32, one thread).
struct DenseItems {
  const float* X;
  int d, metric;
  __device__ __forceinline__ float dist(int a, int b) const {
    return row_dist(X + (size_t)a * d, X + (size_t)b * d, d, metric);
  }
};

struct SparseItems {
  const int64_t* ip;
  const uint16_t* t;
  const float* w;
  __device__ __forceinline__ float dist(int a, int b) const {
    int64_t i = __ldg(ip + a), ie = __ldg(ip + a + 1), j = __ldg(ip + b), je = __ldg(ip + b + 1);
    float s = 0.f;
    while (i < ie && j < je) {
      const uint16_t ti = __ldg(t + i), tj = __ldg(t + j);
      if (ti == tj) s = fmaf(__ldg(w + i++), __ldg(w + j++), s);
      else if (ti < tj) ++i;
      else ++j;
    }
    return -s;
  }
};

__device__ __forceinline__ float row_dist(const float* a, const float* b, int d, int metric) {
  float s0 = 0.f, s1 = 0.f;
  for (int t = 0; t < d; t += 4) {
    const float4 x = __ldg(reinterpret_cast<const float4*>(a + t));
    const float4 y = __ldg(reinterpret_cast<const float4*>(b + t));
    if (metric == KANN_L2) {
      acc_diff_sq2(s0, s1, x.x, x.y, y.x, y.y);
      acc_diff_sq2(s0, s1, x.z, x.w, y.z, y.w);
    } else {
      acc_mul2(s0, s1, x.x, x.y, y.x, y.y);
      acc_mul2(s0, s1, x.z, x.w, y.z, y.w);
    }
  }
  return metric == KANN_L2 ? s0 + s1 : -(s0 + s1);
}

// The heuristic by one warp: candidates (ids, their distances to the base
// node, ascending by (distance, id)), keep up to `cap`; kept ids go to
// out[0..cap) (-1 padded), out in global memory, `kept` in shared memory
// (cap ints).  Lane j checks the distance of the candidate to kept[j] (and
// kept[j + 32]).
template <class S>
__device__ void select_heuristic(const S& sp, const int* cid, const float* cdist, int ncand, int cap, int* kept,
                                 int32_t* out, int lane) {
  int nk = 0;
  for (int c = 0; c < ncand && nk < cap; ++c) {
    const int e = cid[c];
    if (e < 0) break;
    const float de = cdist[c];
    bool bad = false;
    for (int j = lane; j < nk; j += 32) bad |= !(de < sp.dist(e, kept[j]));
    if (__ballot_sync(FULL, bad) == 0u) {
      if (lane == 0) kept[nk] = e;
      __syncwarp();
      ++nk;
    }
  }
  __syncwarp();
  for (int j = lane; j < cap; j += 32) out[j] = j < nk ? kept[j] : -1;
}

// b. one warp per batch node: select up to M of its candidates, write its
// layer-0 list (M0 slots, -1 after the kept ones), post the reverse links.
template <class S>
__global__ void select_new_kernel(const S sp, const int32_t* batch, int nb, const int32_t* cids, const float* cdists,
                                  int efc, int M, int M0, int32_t* l0, int32_t* cnt_in, int32_t* inbox,
                                  int32_t* touched, int32_t* ntouched) {
  extern __shared__ int sm_kept[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int b = blockIdx.x * (blockDim.x >> 5) + w;
  if (b >= nb) return;
  int* kept = sm_kept + w * 64;
  const int node = batch[b];
  int32_t* row = l0 + (int64_t)node * M0;
  select_heuristic(sp, cids + (size_t)b * efc, cdists + (size_t)b * efc, efc, M, kept, row, lane);
  for (int j = M + lane; j < M0; j += 32) row[j] = -1;
  __syncwarp();
  for (int j = lane; j < M; j += 32) {
    const int e = row[j];
    if (e < 0) continue;
    const int slot = atomicAdd(cnt_in + e, 1);
    if (slot == 0) touched[atomicAdd(ntouched, 1)] = e;
    if (slot < INBOX) inbox[(size_t)e * INBOX + slot] = node;
  }
}

// d. one warp per node that received reverse links this batch.
template <class S>
__global__ void merge_inbox_kernel(const S sp, const int32_t* touched, const int32_t* ntouched, int M0, int32_t* l0,
                                   int32_t* cnt_in, const int32_t* inbox) {
  extern __shared__ unsigned char sm_raw[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int t = blockIdx.x * (blockDim.x >> 5) + w;
  if (t >= *ntouched) return;
  u64* keys = reinterpret_cast<u64*>(sm_raw) + (size_t)w * MRG_WORDS;
  int* cid = reinterpret_cast<int*>(keys + CMAX);              // kept ids
  int* ids = reinterpret_cast<int*>(keys + CMAX + KANN_MAX_M0 / 2);  // candidates' ids
  const int e = touched[t];
  int32_t* row = l0 + (int64_t)e * M0;
  const int nin = min(cnt_in[e], INBOX);
  int cur = 0;
  while (cur < M0 && row[cur] >= 0) ++cur;  // lists are packed, -1 after the last id
  if (cur + nin <= M0) {
    for (int j = lane; j < nin; j += 32) row[cur + j] = inbox[(size_t)e * INBOX + j];
    __syncwarp();
    if (lane == 0) cnt_in[e] = 0;
    return;
  }
  // shrink: candidates = list + inbox, by (distance to e, id), then the heuristic
  const int nc = cur + nin;
  for (int j = lane; j < CMAX; j += 32) {
    u64 k = KEY_MAX;
    if (j < nc) {
      const int v = j < cur ? row[j] : inbox[(size_t)e * INBOX + (j - cur)];
      k = make_key(sp.dist(e, v), (uint32_t)v);
    }
    keys[j] = k;
  }
  __syncwarp();
  warp_smem_sort_n(keys, nc, lane);
  // unpack: ids into ids[], distances over the first half of keys[]
  float* dists = reinterpret_cast<float*>(keys);
  for (int j = lane; j < nc; j += 32) ids[j] = (int)(uint32_t)keys[j];
  __syncwarp();
  float dv[3];
  for (int r = 0; r < 3; ++r) {
    const int j = lane + 32 * r;
    dv[r] = j < nc ? key_dist(keys[j]) : 0.f;
  }
  __syncwarp();
  for (int r = 0; r < 3; ++r) {
    const int j = lane + 32 * r;
    if (j < nc) dists[j] = dv[r];
  }
  __syncwarp();
  select_heuristic(sp, ids, dists, nc, M0, cid, row, lane);
  if (lane == 0) cnt_in[e] = 0;
}

// The batch's term lists gathered into a query CSR (one warp per node; the
// offsets come from the host).
__global__ void gather_terms_kernel(const int64_t* ip, const uint16_t* t, const float* w, const int32_t* ids, int n,
                                    const int64_t* q_ip, uint16_t* qt, float* qw) {
  const int lane = threadIdx.x & 31;
  const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r >= n) return;
  const int64_t b = ip[ids[r]], len = ip[ids[r] + 1] - b, o = q_ip[r];
  for (int64_t j = lane; j < len; j += 32) {
    qt[o + j] = t[b + j];
    qw[o + j] = w[b + j];
  }
}

__global__ void gather_rows_kernel(const float* X, int d, const int32_t* ids, int n, float* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t tot = (int64_t)n * (d / 4);
  if (i >= tot) return;
  const int r = (int)(i / (d / 4)), c = (int)(i % (d / 4));
  reinterpret_cast<float4*>(out)[i] = __ldg(reinterpret_cast<const float4*>(X + (size_t)ids[r] * d) + c);
}

__global__ void scatter_lists_kernel(const int32_t* src, const int32_t* ids, int n, int M0, int32_t* l0) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)n * M0) return;
  const int r = (int)(i / M0), c = (int)(i % M0);
  l0[(int64_t)ids[r] * M0 + c] = src[i];
}

struct BuildPlan {
  int batch_max;
  size_t q_off, cid_off, cd_off, cnt_off, inbox_off, touched_off, nt_off, ids_off, lvl_off, qip_off, qt_off, qw_off,
      total;
};

// Scratch of a build: batch queries (dense rows, or a gathered CSR of up to
// `nnz` terms for sparse items), candidates, reverse-link inboxes, touched
// lists, the insertion order and a device copy of the levels.
BuildPlan plan(int64_t n, int d, int M, int efc, int batch, int64_t nnz) {
  BuildPlan p;
  p.batch_max = batch > 0 ? batch : 65536;
  const size_t B = (size_t)p.batch_max;
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  size_t o = 0;
  p.q_off = o;
  o = al(o + B * (size_t)d * 4);
  p.cid_off = o;
  o = al(o + B * efc * 4);
  p.cd_off = o;
  o = al(o + B * efc * 4);
  p.cnt_off = o;
  o = al(o + (size_t)n * 4);
  p.inbox_off = o;
  o = al(o + (size_t)n * INBOX * 4);
  p.touched_off = o;
  o = al(o + B * M * 4);
  p.nt_off = o;
  o = al(o + 16);
  p.ids_off = o;
  o = al(o + (size_t)n * 4);
  p.lvl_off = o;
  o = al(o + (size_t)n);
  p.qip_off = o;
  o = al(o + (nnz > 0 ? (B + 1) * 8 : 0));
  p.qt_off = o;
  o = al(o + (size_t)nnz * 2);
  p.qw_off = o;
  o = al(o + (size_t)nnz * 4);
  p.total = o;
  return p;
}

int cuda_fail(cudaError_t e) {
  set_cuda_error((int)e);
  return KANN_ECUDA;
}

// The two kinds of items: how the upper nodes reach the host builder, how a
// batch is searched, and the device distance.
struct DenseBuild {
  const float* d_x;
  int d, metric;
  DenseItems items() const { return DenseItems{d_x, d, metric}; }
  // host rows of the given nodes, then the host builder over them
  int host_build(const std::vector<int32_t>& up, unsigned char* ws, const BuildPlan& p, cudaStream_t s, int M, int efc,
                 uint64_t seed, int th, const int8_t* lvl, int32_t* l0, int32_t* us, int32_t* upper,
                 int32_t* entry) const {
    const int ns = (int)up.size();
    int32_t* ids_dev = reinterpret_cast<int32_t*>(ws + p.ids_off);
    cudaError_t e = cudaMemcpyAsync(ids_dev, up.data(), (size_t)ns * 4, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e);
    std::vector<float> hx((size_t)ns * d);
    for (size_t off = 0; off < (size_t)ns; off += (size_t)p.batch_max) {
      const int cnt = (int)std::min((size_t)p.batch_max, (size_t)ns - off);
      float* q = reinterpret_cast<float*>(ws + p.q_off);
      const int64_t tot = (int64_t)cnt * (d / 4);
      gather_rows_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(d_x, d, ids_dev + off, cnt, q);
      e = cudaMemcpyAsync(hx.data() + off * d, q, (size_t)cnt * d * 4, cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return cuda_fail(e);
    }
    return kann_hnsw_build_dense(hx.data(), ns, d, metric, M, efc, seed, th, lvl, l0, us, upper, entry);
  }
  int upload(const kann_graph_desc& g, kann_index_t** idx) const {
    kann_vectors_desc v;
    std::memset(&v, 0, sizeof(v));
    v.dtype = KANN_F32;
    v.d = d;
    v.metric = metric;
    v.d_data = d_x;
    v.row_stride_bytes = (int64_t)d * 4;
    return kann_index_upload(idx, &g, &v, nullptr, nullptr, nullptr, 0);
  }
  int search(kann_index_t* idx, const int32_t* order, const std::vector<int32_t>& h_order, int64_t pos, int nb,
             unsigned char* ws, const BuildPlan& p, int efc, int32_t* cids, float* cdists, cudaStream_t s) const {
    (void)h_order;
    (void)pos;
    float* q = reinterpret_cast<float*>(ws + p.q_off);
    const int64_t tot = (int64_t)nb * (d / 4);
    gather_rows_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(d_x, d, order, nb, q);
    return kann_search(idx, q, nb, efc, efc, cids, cdists, s);
  }
};

struct SparseBuild {
  const int64_t* d_ip;
  const uint16_t* d_t;
  const float* d_w;
  int vocab;
  std::vector<int64_t> h_ip;  // the offsets, on the host
  SparseItems items() const { return SparseItems{d_ip, d_t, d_w}; }
  int host_build(const std::vector<int32_t>& up, unsigned char* ws, const BuildPlan& p, cudaStream_t s, int M, int efc,
                 uint64_t seed, int th, const int8_t* lvl, int32_t* l0, int32_t* us, int32_t* upper,
                 int32_t* entry) const {
    (void)ws;
    (void)p;
    const int ns = (int)up.size();
    const int64_t nnz = h_ip.back();
    std::vector<uint16_t> tt(nnz);
    std::vector<float> ww(nnz);
    cudaError_t e = cudaMemcpyAsync(tt.data(), d_t, (size_t)nnz * 2, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ww.data(), d_w, (size_t)nnz * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e);
    std::vector<int64_t> sip(ns + 1, 0);
    for (int j = 0; j < ns; ++j) sip[j + 1] = sip[j] + (h_ip[up[j] + 1] - h_ip[up[j]]);
    std::vector<uint16_t> st(sip[ns]);
    std::vector<float> sw(sip[ns]);
    for (int j = 0; j < ns; ++j) {
      std::copy(tt.begin() + h_ip[up[j]], tt.begin() + h_ip[up[j] + 1], st.begin() + sip[j]);
      std::copy(ww.begin() + h_ip[up[j]], ww.begin() + h_ip[up[j] + 1], sw.begin() + sip[j]);
    }
    return kann_hnsw_build_sparse(sip.data(), st.data(), sw.data(), ns, M, efc, seed, th, lvl, l0, us, upper, entry);
  }
  int upload(const kann_graph_desc& g, kann_index_t** idx) const {
    kann_sparse_desc sp;
    std::memset(&sp, 0, sizeof(sp));
    sp.d_indptr = d_ip;
    sp.d_terms = d_t;
    sp.d_weights = d_w;
    sp.vocab = vocab;
    return kann_index_upload(idx, &g, nullptr, nullptr, &sp, nullptr, 0);
  }
  int search(kann_index_t* idx, const int32_t* order, const std::vector<int32_t>& h_order, int64_t pos, int nb,
             unsigned char* ws, const BuildPlan& p, int efc, int32_t* cids, float* cdists, cudaStream_t s) const {
    std::vector<int64_t> qip(nb + 1, 0);
    for (int r = 0; r < nb; ++r) {
      const int32_t v = h_order[pos + r];
      qip[r + 1] = qip[r] + (h_ip[v + 1] - h_ip[v]);
    }
    int64_t* d_qip = reinterpret_cast<int64_t*>(ws + p.qip_off);
    uint16_t* qt = reinterpret_cast<uint16_t*>(ws + p.qt_off);
    float* qw = reinterpret_cast<float*>(ws + p.qw_off);
    cudaError_t e = cudaMemcpyAsync(d_qip, qip.data(), (size_t)(nb + 1) * 8, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e);
    gather_terms_kernel<<<(nb + 3) / 4, 128, 0, s>>>(d_ip, d_t, d_w, order, nb, d_qip, qt, qw);
    // the offsets' host buffer must outlive the copy
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e);
    return kann_search_sparse(idx, d_qip, qt, qw, nb, efc, efc, cids, cdists, nullptr, s);
  }
};

template <class BD>
int build_device(const BD& bd, int64_t n, int M, int ef_construction, uint64_t seed, int batch, int nthreads,
                 const int8_t* h_level, int32_t* d_l0, int32_t* d_upper_slot, int32_t* d_upper, int32_t* h_entry,
                 unsigned char* ws, const BuildPlan& p, cudaStream_t s) {
  const int M0 = 2 * M;
  (void)batch;
  // ---- 1. the upper-layer nodes on the host
  int L = 0;
  std::vector<int32_t> up, rest;
  for (int64_t i = 0; i < n; ++i) {
    L = std::max(L, (int)h_level[i]);
    (h_level[i] >= 1 ? up : rest).push_back((int32_t)i);
  }
  if (up.empty()) {  // every node on layer 0: node 0 starts the graph
    up.push_back(0);
    rest.erase(rest.begin());
  }
  if (L > 0 && !d_upper) return KANN_EINVAL;
  const int ns = (int)up.size();
  std::vector<int8_t> lvl_sub(ns);
  int64_t nu_sub = 0;
  for (int j = 0; j < ns; ++j) {
    lvl_sub[j] = h_level[up[j]];
    nu_sub += lvl_sub[j] >= 1;
  }
  std::vector<int32_t> l0_sub((size_t)ns * M0), us_sub(ns),
      upper_sub((size_t)std::max<int64_t>(nu_sub, 1) * std::max(L, 1) * M, -1);
  int32_t entry_sub = 0;
  // threads for the upper nodes: one per 4,096 of them at most -- they all go
  // to the same few layers, where concurrent insertions that miss each other
  // would otherwise leave nodes unreachable
  int th = nthreads > 0 ? nthreads : (int)std::thread::hardware_concurrency();
  th = std::max(1, std::min(th, ns / 4096));
  int rc = bd.host_build(up, ws, p, s, M, ef_construction, seed, th, lvl_sub.data(), l0_sub.data(), us_sub.data(),
                         upper_sub.data(), &entry_sub);
  if (rc != KANN_OK) return rc;
  for (auto& v : l0_sub)
    if (v >= 0) v = up[v];
  for (auto& v : upper_sub)
    if (v >= 0) v = up[v];
  // upper slots: every node of level >= 1 is an upper node, in the same order
  std::vector<int32_t> us_full((size_t)n, -1);
  for (int j = 0; j < ns; ++j) us_full[up[j]] = us_sub[j];
  int32_t* ids_dev = reinterpret_cast<int32_t*>(ws + p.ids_off);
  cudaError_t e = cudaMemcpyAsync(ids_dev, up.data(), (size_t)ns * 4, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_l0, 0xff, (size_t)n * M0 * 4, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_upper_slot, us_full.data(), (size_t)n * 4, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && L > 0)
    e = cudaMemcpyAsync(d_upper, upper_sub.data(), (size_t)nu_sub * L * M * 4, cudaMemcpyHostToDevice, s);
  // the upper nodes' layer-0 lists, scattered to their rows through the
  // candidate buffer (batch_max * efConstruction ints), piece by piece
  const size_t piece = std::max<size_t>(1, (size_t)p.batch_max * ef_construction / M0);
  for (size_t off = 0; off < (size_t)ns && e == cudaSuccess; off += piece) {
    const int cnt = (int)std::min(piece, (size_t)ns - off);
    int32_t* tmp = reinterpret_cast<int32_t*>(ws + p.cid_off);
    e = cudaMemcpyAsync(tmp, l0_sub.data() + off * M0, (size_t)cnt * M0 * 4, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) break;
    scatter_lists_kernel<<<(unsigned)(((int64_t)cnt * M0 + 255) / 256), 256, 0, s>>>(tmp, ids_dev + off, cnt, M0,
                                                                                     d_l0);
    e = cudaStreamSynchronize(s);  // the host buffers are reused / freed next
  }
  if (e != cudaSuccess) return cuda_fail(e);
  const int32_t entry = up[entry_sub];
  *h_entry = entry;

  // ---- 2. the level-0 nodes on the GPU, in batches
  int8_t* lvl_dev = reinterpret_cast<int8_t*>(ws + p.lvl_off);
  int32_t* cnt_in = reinterpret_cast<int32_t*>(ws + p.cnt_off);
  int32_t* inbox = reinterpret_cast<int32_t*>(ws + p.inbox_off);
  int32_t* touched = reinterpret_cast<int32_t*>(ws + p.touched_off);
  int32_t* ntouched = reinterpret_cast<int32_t*>(ws + p.nt_off);
  int32_t* order = ids_dev;  // reused: the level-0 insertion order
  int32_t* cids = reinterpret_cast<int32_t*>(ws + p.cid_off);
  float* cdists = reinterpret_cast<float*>(ws + p.cd_off);
  e = cudaMemcpyAsync(lvl_dev, h_level, (size_t)n, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && !rest.empty())
    e = cudaMemcpyAsync(order, rest.data(), rest.size() * 4, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(cnt_in, 0, (size_t)n * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(ntouched, 0, 4, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e);
  kann_graph_desc gdesc;
  std::memset(&gdesc, 0, sizeof(gdesc));
  gdesc.n = n;
  gdesc.M = M;
  gdesc.M0 = M0;
  gdesc.max_level = L;
  gdesc.entry = entry;
  gdesc.n_upper = nu_sub;
  gdesc.d_level = lvl_dev;
  gdesc.d_l0 = d_l0;
  gdesc.d_upper_slot = d_upper_slot;
  gdesc.d_upper = L > 0 ? d_upper : nullptr;
  kann_index_t* idx = nullptr;
  rc = bd.upload(gdesc, &idx);
  if (rc != KANN_OK) return rc;
  const auto items = bd.items();
  const int wpb = 4;
  const size_t sel_smem = (size_t)wpb * 64 * 4;
  const size_t mrg_smem = (size_t)wpb * MRG_WORDS * 8;
  int64_t inserted = ns, pos = 0;
  const int64_t nrest = (int64_t)rest.size();
  while (pos < nrest && rc == KANN_OK) {
    int64_t b = std::max<int64_t>(1, inserted / 32);
    b = std::min<int64_t>(b, p.batch_max);
    b = std::min<int64_t>(b, nrest - pos);
    const int nb = (int)b;
    // a. candidates among the nodes inserted so far
    rc = bd.search(idx, order + pos, rest, pos, nb, ws, p, ef_construction, cids, cdists, s);
    if (rc != KANN_OK) break;
    // b, c. selection, lists, reverse links
    select_new_kernel<<<(nb + wpb - 1) / wpb, wpb * 32, sel_smem, s>>>(items, order + pos, nb, cids, cdists,
                                                                      ef_construction, M, M0, d_l0, cnt_in, inbox,
                                                                      touched, ntouched);
    // d. the neighbours' lists (one warp per neighbour that received links)
    const int64_t maxt = (int64_t)nb * M;
    merge_inbox_kernel<<<(unsigned)((maxt + wpb - 1) / wpb), wpb * 32, mrg_smem, s>>>(items, touched, ntouched, M0,
                                                                                    d_l0, cnt_in, inbox);
    e = cudaMemsetAsync(ntouched, 0, 4, s);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
      rc = cuda_fail(e);
      break;
    }
    inserted += nb;
    pos += nb;
  }
  kann_index_destroy(idx);
  if (rc != KANN_OK) return rc;
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e);
  return KANN_OK;
}

}  // namespace
}  // namespace kann

using namespace kann;

extern "C" size_t kann_hnsw_build_device_workspace_bytes(int64_t n, int d, int M, int ef_construction, int batch) {
  if (n < 1 || d < 4 || M < 2 || ef_construction < 1) return 0;
  return plan(n, d, M, ef_construction, batch, 0).total;
}

extern "C" int kann_hnsw_build_device(const float* d_x, int64_t n, int d, int metric, int M, int ef_construction,
                                      uint64_t seed, int batch, int nthreads, const int8_t* h_level,
                                      int32_t* d_l0, int32_t* d_upper_slot, int32_t* d_upper, int32_t* h_entry,
                                      void* d_ws, size_t ws_bytes, void* stream) {
  if (!d_x || n < 1 || n >= ((int64_t)1 << 31) || d < 4 || d % 4 != 0 || M < 2 || M > 32) return KANN_EINVAL;
  if (ef_construction < 1 || ef_construction > KANN_MAX_EF || batch < 0) return KANN_EINVAL;
  if (metric != KANN_L2 && metric != KANN_IP) return KANN_EINVAL;
  if (!h_level || !d_l0 || !d_upper_slot || !h_entry || !d_ws) return KANN_EINVAL;
  if (((uintptr_t)d_x & 15u) != 0) return KANN_EINVAL;
  const BuildPlan p = plan(n, d, M, ef_construction, batch, 0);
  if (ws_bytes < p.total) return KANN_EINVAL;
  DenseBuild bd{d_x, d, metric};
  return build_device(bd, n, M, ef_construction, seed, batch, nthreads, h_level, d_l0, d_upper_slot, d_upper, h_entry,
                      static_cast<unsigned char*>(d_ws), p, (cudaStream_t)stream);
}

extern "C" size_t kann_hnsw_build_device_sparse_workspace_bytes(int64_t n, int64_t nnz, int M, int ef_construction,
                                                                int batch) {
  if (n < 1 || nnz < 0 || M < 2 || ef_construction < 1) return 0;
  return plan(n, 4, M, ef_construction, batch, nnz).total;
}

extern "C" int kann_hnsw_build_device_sparse(const int64_t* d_indptr, const uint16_t* d_terms, const float* d_weights,
                                             int64_t n, int vocab, int M, int ef_construction, uint64_t seed,
                                             int batch, int nthreads, const int8_t* h_level, int32_t* d_l0,
                                             int32_t* d_upper_slot, int32_t* d_upper, int32_t* h_entry, void* d_ws,
                                             size_t ws_bytes, void* stream) {
  if (!d_indptr || !d_terms || !d_weights || n < 1 || n >= ((int64_t)1 << 31) || M < 2 || M > 32) return KANN_EINVAL;
  if (vocab < 1 || vocab > 65536 || ef_construction < 1 || ef_construction > KANN_MAX_EF || batch < 0)
    return KANN_EINVAL;
  if (!h_level || !d_l0 || !d_upper_slot || !h_entry || !d_ws) return KANN_EINVAL;
  SparseBuild bd{d_indptr, d_terms, d_weights, vocab, std::vector<int64_t>((size_t)n + 1)};
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(bd.h_ip.data(), d_indptr, (size_t)(n + 1) * 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e);
  const BuildPlan p = plan(n, 4, M, ef_construction, batch, bd.h_ip.back());
  if (ws_bytes < p.total) return KANN_EINVAL;
  return build_device(bd, n, M, ef_construction, seed, batch, nthreads, h_level, d_l0, d_upper_slot, d_upper, h_entry,
                      static_cast<unsigned char*>(d_ws), p, s);
}
