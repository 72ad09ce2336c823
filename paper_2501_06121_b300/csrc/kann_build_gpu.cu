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
__device__ void select_heuristic(const float* X, int d, int metric, const int* cid, const float* cdist, int ncand,
                                 int cap, int* kept, int32_t* out, int lane) {
  int nk = 0;
  for (int c = 0; c < ncand && nk < cap; ++c) {
    const int e = cid[c];
    if (e < 0) break;
    const float de = cdist[c];
    const float* xe = X + (size_t)e * d;
    bool bad = false;
    for (int j = lane; j < nk; j += 32) bad |= !(de < row_dist(xe, X + (size_t)kept[j] * d, d, metric));
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
__global__ void select_new_kernel(const float* X, int d, int metric, const int32_t* batch, int nb, const int32_t* cids,
                                  const float* cdists, int efc, int M, int M0, int32_t* l0, int32_t* cnt_in,
                                  int32_t* inbox, int32_t* touched, int32_t* ntouched) {
  extern __shared__ int sm_kept[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int b = blockIdx.x * (blockDim.x >> 5) + w;
  if (b >= nb) return;
  int* kept = sm_kept + w * 64;
  const int node = batch[b];
  int32_t* row = l0 + (int64_t)node * M0;
  select_heuristic(X, d, metric, cids + (size_t)b * efc, cdists + (size_t)b * efc, efc, M, kept, row, lane);
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
__global__ void merge_inbox_kernel(const float* X, int d, int metric, const int32_t* touched, const int32_t* ntouched,
                                   int M0, int32_t* l0, int32_t* cnt_in, const int32_t* inbox) {
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
  const float* xe = X + (size_t)e * d;
  for (int j = lane; j < CMAX; j += 32) {
    u64 k = KEY_MAX;
    if (j < nc) {
      const int v = j < cur ? row[j] : inbox[(size_t)e * INBOX + (j - cur)];
      k = make_key(row_dist(xe, X + (size_t)v * d, d, metric), (uint32_t)v);
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
  select_heuristic(X, d, metric, ids, dists, nc, M0, cid, row, lane);
  if (lane == 0) cnt_in[e] = 0;
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
  size_t q_off, cid_off, cd_off, cnt_off, inbox_off, touched_off, nt_off, ids_off, lvl_off, total;
};

BuildPlan plan(int64_t n, int d, int M, int efc, int batch) {
  BuildPlan p;
  p.batch_max = batch > 0 ? batch : 65536;
  const size_t B = (size_t)p.batch_max;
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  size_t o = 0;
  p.q_off = o;
  o = al(o + B * d * 4);
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
  p.ids_off = o;  // the insertion order of the level-0 nodes, then the upper nodes' ids
  o = al(o + (size_t)n * 4);
  p.lvl_off = o;  // device copy of the levels
  o = al(o + (size_t)n);
  p.total = o;
  return p;
}

}  // namespace
}  // namespace kann

using namespace kann;

extern "C" size_t kann_hnsw_build_device_workspace_bytes(int64_t n, int d, int M, int ef_construction, int batch) {
  if (n < 1 || d < 4 || M < 2 || ef_construction < 1) return 0;
  return plan(n, d, M, ef_construction, batch).total;
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
  const BuildPlan p = plan(n, d, M, ef_construction, batch);
  if (ws_bytes < p.total) return KANN_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char* ws = static_cast<unsigned char*>(d_ws);
  const int M0 = 2 * M;
  auto fail = [](cudaError_t e) {
    set_cuda_error((int)e);
    return KANN_ECUDA;
  };

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
  int32_t* ids_dev = reinterpret_cast<int32_t*>(ws + p.ids_off);
  cudaError_t e = cudaMemcpyAsync(ids_dev, up.data(), (size_t)ns * 4, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return fail(e);
  // gather the upper nodes' rows (the query buffer is large enough only if ns
  // rows fit; else gather in pieces)
  std::vector<float> hx((size_t)ns * d);
  const size_t per = p.batch_max;
  for (size_t off = 0; off < (size_t)ns; off += per) {
    const int cnt = (int)std::min(per, (size_t)ns - off);
    float* q = reinterpret_cast<float*>(ws + p.q_off);
    const int64_t tot = (int64_t)cnt * (d / 4);
    gather_rows_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(d_x, d, ids_dev + off, cnt, q);
    e = cudaMemcpyAsync(hx.data() + off * d, q, (size_t)cnt * d * 4, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return fail(e);
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(e);
  }
  std::vector<int8_t> lvl_sub(ns);
  int64_t nu_sub = 0;
  for (int j = 0; j < ns; ++j) {
    lvl_sub[j] = h_level[up[j]];
    nu_sub += lvl_sub[j] >= 1;
  }
  std::vector<int32_t> l0_sub((size_t)ns * M0), us_sub(ns), upper_sub((size_t)std::max<int64_t>(nu_sub, 1) * std::max(L, 1) * M, -1);
  int32_t entry_sub = 0;
  // threads for the upper nodes: one per 4,096 of them at most -- they all go
  // to the same few layers, where concurrent insertions that miss each other
  // would otherwise leave nodes unreachable
  int th = nthreads > 0 ? nthreads : (int)std::thread::hardware_concurrency();
  th = std::max(1, std::min(th, ns / 4096));
  int rc = kann_hnsw_build_dense(hx.data(), ns, d, metric, M, ef_construction, seed, th, lvl_sub.data(),
                                 l0_sub.data(), us_sub.data(), upper_sub.data(), &entry_sub);
  if (rc != KANN_OK) return rc;
  for (auto& v : l0_sub)
    if (v >= 0) v = up[v];
  for (auto& v : upper_sub)
    if (v >= 0) v = up[v];
  // upper slots: every node of level >= 1 is an upper node, in the same order
  std::vector<int32_t> us_full((size_t)n, -1);
  for (int j = 0; j < ns; ++j) us_full[up[j]] = us_sub[j];
  e = cudaMemsetAsync(d_l0, 0xff, (size_t)n * M0 * 4, s);
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
  if (e != cudaSuccess) return fail(e);
  const int32_t entry = up[entry_sub];
  *h_entry = entry;

  // ---- 2. the level-0 nodes on the GPU, in batches
  int8_t* lvl_dev = reinterpret_cast<int8_t*>(ws + p.lvl_off);
  int32_t* cnt_in = reinterpret_cast<int32_t*>(ws + p.cnt_off);
  int32_t* inbox = reinterpret_cast<int32_t*>(ws + p.inbox_off);
  int32_t* touched = reinterpret_cast<int32_t*>(ws + p.touched_off);
  int32_t* ntouched = reinterpret_cast<int32_t*>(ws + p.nt_off);
  int32_t* order = ids_dev;  // reused: the level-0 insertion order
  float* qbuf = reinterpret_cast<float*>(ws + p.q_off);
  int32_t* cids = reinterpret_cast<int32_t*>(ws + p.cid_off);
  float* cdists = reinterpret_cast<float*>(ws + p.cd_off);
  e = cudaMemcpyAsync(lvl_dev, h_level, (size_t)n, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && !rest.empty())
    e = cudaMemcpyAsync(order, rest.data(), rest.size() * 4, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(cnt_in, 0, (size_t)n * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(ntouched, 0, 4, s);
  if (e != cudaSuccess) return fail(e);
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
  kann_vectors_desc vdesc;
  std::memset(&vdesc, 0, sizeof(vdesc));
  vdesc.dtype = KANN_F32;
  vdesc.d = d;
  vdesc.metric = metric;
  vdesc.d_data = d_x;
  vdesc.row_stride_bytes = (int64_t)d * 4;
  kann_index_t* idx = nullptr;
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(e);
  rc = kann_index_upload(&idx, &gdesc, &vdesc, nullptr, nullptr, nullptr, 0);
  if (rc != KANN_OK) return rc;
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
    const int64_t tot = (int64_t)nb * (d / 4);
    gather_rows_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(d_x, d, order + pos, nb, qbuf);
    // a. candidates among the nodes inserted so far
    rc = kann_search(idx, qbuf, nb, ef_construction, ef_construction, cids, cdists, stream);
    if (rc != KANN_OK) break;
    // b, c. selection, lists, reverse links
    select_new_kernel<<<(nb + wpb - 1) / wpb, wpb * 32, sel_smem, s>>>(d_x, d, metric, order + pos, nb, cids, cdists,
                                                                      ef_construction, M, M0, d_l0, cnt_in, inbox,
                                                                      touched, ntouched);
    // d. the neighbours' lists (one warp per neighbour that received links)
    const int64_t maxt = (int64_t)nb * M;
    merge_inbox_kernel<<<(unsigned)((maxt + wpb - 1) / wpb), wpb * 32, mrg_smem, s>>>(d_x, d, metric, touched,
                                                                                    ntouched, M0, d_l0, cnt_in, inbox);
    e = cudaMemsetAsync(ntouched, 0, 4, s);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
      rc = fail(e);
      break;
    }
    inserted += nb;
    pos += nb;
  }
  kann_index_destroy(idx);
  if (rc != KANN_OK) return rc;
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(e);
  return KANN_OK;
}
