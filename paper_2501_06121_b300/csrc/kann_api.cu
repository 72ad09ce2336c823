// kann_api.cu -- the C ABI: index upload/validation, search dispatch,
// storage-format conversion, status strings.
#include <cuda_runtime.h>

#include <cstdlib>
#include <cstring>
#include <new>

#include "kann_device.cuh"
#include "kann_internal.h"

struct kann_index {
  kann_graph_desc g;
  int kind;  // 0 dense, 1 PQ, 2 sparse
  kann_vectors_desc v;
  kann_pq_desc pq;
  kann_sparse_desc sp;
  int has_rr;
  kann_vectors_desc rr;
  int device;
};

namespace kann {

static thread_local int g_last_cuda = 0;
void set_cuda_error(int e) { g_last_cuda = e; }

namespace {

int elem_size(int dtype) {
  switch (dtype) {
    case KANN_F32: return 4;
    case KANN_F16:
    case KANN_BF16: return 2;
    case KANN_E4M3: return 1;
    default: return 0;
  }
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// Lanes that share one row: the largest power of two <= min(32, nchunks /
// chunks_per_lane), so that each lane reads `chunks_per_lane` 16-byte chunks
// of a row (more rows per warp pass, fewer per-row reductions).
int lanes_per_row(int nchunks, int chunks_per_lane = 1) {
  int target = nchunks / chunks_per_lane;
  if (target < 1) target = 1;
  int l = 1;
  while (l * 2 <= target && l * 2 <= 32) l *= 2;
  return l;
}

int check_cuda(cudaError_t e) {
  if (e != cudaSuccess) {
    set_cuda_error((int)e);
    return KANN_ECUDA;
  }
  return KANN_OK;
}

int validate_vectors(const kann_vectors_desc* v, int64_t n) {
  const int es = elem_size(v->dtype);
  if (es == 0 || v->d <= 0 || v->d > KANN_MAX_DIM) return KANN_EINVAL;
  if (v->metric != KANN_L2 && v->metric != KANN_IP) return KANN_EINVAL;
  if (!v->d_data || !aligned16(v->d_data)) return KANN_EINVAL;
  if (((int64_t)v->d * es) % 16 != 0) return KANN_EINVAL;
  if (v->row_stride_bytes < (int64_t)v->d * es || v->row_stride_bytes % 16 != 0) return KANN_EINVAL;
  if (v->dtype == KANN_E4M3 && !v->d_scale) return KANN_EINVAL;
  (void)n;
  return KANN_OK;
}

// Device-side scan of the adjacency arrays: ids must be -1 or in [0, n);
// a node has an upper slot exactly when its level is >= 1.
__global__ void validate_graph_kernel(kann_graph_desc g, int* bad) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int local = 0;
  for (int64_t i = tid; i < g.n * g.M0; i += stride) {
    const int32_t v = g.d_l0[i];
    if (v < -1 || v >= g.n) local = 1;
  }
  for (int64_t i = tid; i < g.n; i += stride) {
    const int lv = g.d_level[i];
    const int32_t s = g.d_upper_slot[i];
    if (lv < 0 || lv > g.max_level) local = 1;
    if ((lv >= 1) != (s >= 0) || s >= g.n_upper) local = 1;
  }
  const int64_t nu = g.n_upper * g.max_level * g.M;
  for (int64_t i = tid; i < nu; i += stride) {
    const int32_t v = g.d_upper[i];
    if (v < -1 || v >= g.n) local = 1;
  }
  if (tid == 0 && g.d_level[g.entry] != g.max_level) local = 1;
  if (local) atomicOr(bad, 1);
}

// Default visited-table size (log2 of its slots).  Wide (32-bit) table:
// 2^hbits >= 8 efmax, 10..13.  Compact (16-bit) table: 4,096 slots (8 KB),
// which holds the ~1,700-4,000 ids a search of 1M items visits at ef 56-512
// without filling up, and at ef <= 64 keeps six 4-warp CTAs per SM.
int default_hbits(int efmax, bool compact) {
  if (compact) return 12;
  int h = 10;
  while ((1 << h) < 8 * efmax && h < 13) ++h;
  return h;
}

int ceil_log2(int64_t n) {
  int k = 0;
  while (((int64_t)1 << k) < n) ++k;
  return k;
}

// Visited-table layout for 2^hbits slots over ids < n: compact when every id
// maps to a bucket of the table and a slot value of at most 16 bits
// (1 + the low vis_r <= 15 bits of the multiplied id), else wide.
bool set_visited(SearchArgs& a, int hbits, bool want_compact) {
  a.hbits = hbits;
  const int kb = ceil_log2(a.n), bb = hbits - 3;
  const int k = kb > bb ? kb : bb;
  if (want_compact && k - bb <= 15) {
    a.vis_k = k;
    a.vis_r = k - bb;
    return true;
  }
  a.vis_k = 0;
  a.vis_r = -1;
  return false;
}

int max_optin_smem() {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) v = 48 * 1024;
  return v;
}

int fill_search_args(const kann_index_t* idx, const float* d_q, int n, int k, int ef, int kmax, int efmax,
                     const int32_t* d_k, const int32_t* d_ef, int32_t* d_ids, float* d_dists,
                     const kann_search_opts* opts, SearchArgs& a, int& wpb) {
  if (!idx) return KANN_EINVAL;
  if (n < 0) return KANN_EINVAL;
  if (n > 0 && (!d_ids || !d_dists)) return KANN_EINVAL;
  const int efmax_eff = efmax > kmax ? efmax : kmax;
  if (kmax < 1 || efmax_eff > KANN_MAX_EF) return KANN_EINVAL;
  std::memset(&a, 0, sizeof(a));
  const kann_graph_desc& g = idx->g;
  a.l0 = g.d_l0;
  a.upper_slot = g.d_upper_slot;
  a.upper = g.d_upper;
  a.n = g.n;
  a.M0 = g.M0;
  a.M = g.M;
  a.max_level = g.max_level;
  a.entry = g.entry;
  a.q = d_q;
  a.nq = n;
  a.k = k;
  a.ef = ef > k ? ef : k;
  a.kmax = kmax;
  a.efmax = efmax_eff;
  a.k_arr = d_k;
  a.ef_arr = d_ef;
  a.out_ids = d_ids;
  a.out_d = d_dists;
  a.max_hops = 1000000;
  a.expand = 1;
  a.team = 1;
  int hbits = 0;
  int vformat = 0;
  wpb = 4;
  int R = 0;
  if (opts) {
    a.status = opts->d_status;
    a.counters = opts->d_counters;
    if (opts->max_hops > 0) a.max_hops = opts->max_hops;
    if (opts->max_hops < 0) return KANN_EINVAL;
    hbits = opts->hash_bits;
    if (hbits != 0 && (hbits < 5 || hbits > 16)) return KANN_EINVAL;
    if (opts->warps_per_block < 0 || opts->warps_per_block > 4) return KANN_EINVAL;
    if (opts->warps_per_block > 0) wpb = opts->warps_per_block;
    const int l = opts->lanes_per_row;
    if (l < 0 || l > 32 || (l & (l - 1)) != 0) return KANN_EINVAL;
    a.lpr_override = l;
    if (opts->lean < -1 || opts->lean > 1) return KANN_EINVAL;
    a.lean = opts->lean > 0 ? 1 : 0;
    if (opts->pq_lut < KANN_PQ_LUT_F32 || opts->pq_lut > KANN_PQ_LUT_U8) return KANN_EINVAL;
    a.lut = opts->pq_lut;
    if (opts->visited_format < 0 || opts->visited_format > 2) return KANN_EINVAL;
    vformat = opts->visited_format;
    if (opts->expand < 0 || opts->expand > KANN_MAX_EXPAND) return KANN_EINVAL;
    if (opts->expand > 1) a.expand = opts->expand;
    if (opts->team != 0 && opts->team != 1 && opts->team != 2 && opts->team != 4) return KANN_EINVAL;
    if (opts->team > 1) a.team = opts->team;
    R = opts->rerank;
    if (R < -1) return KANN_EINVAL;
    a.work_counter = opts->d_work_counter;
    a.d_n = opts->d_n;
    if (a.d_n && !a.work_counter) return KANN_EINVAL;
  }
  if (R != 0) {
    if (!idx->has_rr) return KANN_EINVAL;
    if (R > 0 && R < kmax) return KANN_EINVAL;
    a.R = R;
    a.rr_data = (const unsigned char*)idx->rr.d_data;
    a.rr_stride = idx->rr.row_stride_bytes;
    a.rr_dtype = idx->rr.dtype;
    a.rr_nchunks = idx->rr.d * elem_size(idx->rr.dtype) / 16;
    // the mapping a traversal of the same rows uses by default (bit-identical
    // distances to an FP32 traversal when the copy is FP32)
    a.rr_lpr = lanes_per_row(a.rr_nchunks, default_chunks_per_lane(idx->rr.dtype));
  }
  // visited table: compact unless asked for wide (or the ids do not fit it);
  // a PQ search with the uint8 table takes 2,048 slots so that four teams
  // fit an SM at m = 192
  int hb_compact = default_hbits(a.efmax, true);
  if (idx->kind == 1 && a.lut == KANN_PQ_LUT_U8) hb_compact = 11;
  const bool compact_ok = set_visited(a, hbits ? hbits : hb_compact, true);
  if (vformat == 1 && !compact_ok) return KANN_EINVAL;
  if (vformat == 2 || !compact_ok) set_visited(a, hbits ? hbits : default_hbits(a.efmax, false), false);
  a.efcap = (a.efmax + 31) / 32 * 32;  // beam capacity: efmax rounded up to whole warp rows
  return KANN_OK;
}

// Shared-memory plan of a search with the settings in `a` (efcap, hbits,
// lut filled in): bytes per warp (per team for PQ) and warps per CTA.  A
// PQ search drops visited-table bits (parity-safe: the table may forget)
// until its query region fits one CTA.  Both the search and the admission
// query (kann_search_workspace_bytes) take their answer from here.
int plan_shared(const kann_index_t* idx, SearchArgs& a, int& wpb) {
  const int optin = max_optin_smem();
  if (idx->kind != 0 && a.expand > 1) return KANN_EINVAL;  // multi-expansion: dense indices
  if (a.team > 1 && (idx->kind == 1 || a.expand > 1)) return KANN_EINVAL;  // teams: dense/sparse, one expansion
  if (idx->kind == 1) {
    const int m = idx->pq.m;
    a.warp_smem = search_warp_smem_pq(a.efcap, a.hbits, a.vis_r >= 0, m, a.lut);
    while (a.warp_smem + PQ_TEAM_CTL_BYTES > optin && a.hbits > 8) {
      set_visited(a, a.hbits - 1, a.vis_r >= 0);
      a.warp_smem = search_warp_smem_pq(a.efcap, a.hbits, a.vis_r >= 0, m, a.lut);
    }
    wpb = 1;  // one query per CTA (a team of warps sharing its table)
    return a.warp_smem + PQ_TEAM_CTL_BYTES > optin ? KANN_ENOMEM : KANN_OK;
  }
  const bool compact = a.vis_r >= 0;
  a.warp_smem = idx->kind == 2 ? search_warp_smem_sparse(a.efcap, a.hbits, compact, idx->sp.vocab)
                               : search_warp_smem(a.efcap, a.hbits, compact, a.expand);
  if (a.team > 1) {
    wpb = 1;  // one query per CTA of a.team warps, its control block after the region
    return a.warp_smem + PQ_TEAM_CTL_BYTES > optin ? KANN_ENOMEM : KANN_OK;
  }
  while (wpb > 1 && wpb * a.warp_smem > optin) --wpb;
  return a.warp_smem > optin ? KANN_ENOMEM : KANN_OK;
}

int run_dense(const kann_index_t* idx, SearchArgs& a, int wpb, void* stream) {
  const kann_vectors_desc& v = idx->v;
  a.data = (const unsigned char*)v.d_data;
  a.stride = v.row_stride_bytes;
  a.scale = v.d_scale;
  a.d = v.d;
  a.metric = v.metric;
  a.nchunks = v.d * elem_size(v.dtype) / 16;
  a.lpr = a.lpr_override ? a.lpr_override : lanes_per_row(a.nchunks, default_chunks_per_lane(v.dtype));
  if (a.lpr > a.nchunks && a.nchunks >= 1) a.lpr = lanes_per_row(a.nchunks);
  if ((a.nchunks + a.lpr - 1) / a.lpr > 8) return KANN_EINVAL;
  // lean: 2 chunks per lane, one expansion, one warp per query
  if ((a.nchunks + a.lpr - 1) / a.lpr != 2 || a.expand > 1 || a.team > 1) a.lean = 0;
  if (a.nq > 0 && (!a.q || !aligned16(a.q))) return KANN_EINVAL;
  const int rc = plan_shared(idx, a, wpb);
  if (rc != KANN_OK || a.nq == 0) return rc;
  return check_cuda((cudaError_t)launch_search_dense(a, v.dtype, wpb, stream));
}

int run_pq(const kann_index_t* idx, SearchArgs& a, int wpb, void* stream) {
  const kann_pq_desc& pq = idx->pq;
  a.codes = pq.d_codes;
  a.codebooks = pq.d_codebooks;
  a.pq_m = pq.m;
  a.pq_dsub = pq.dsub;
  a.stride = pq.m;
  a.d = pq.m * pq.dsub;
  a.metric = pq.metric;
  a.nchunks = pq.m / 16;
  a.lpr = a.lpr_override ? a.lpr_override : lanes_per_row(a.nchunks);
  if (a.lpr > a.nchunks) a.lpr = lanes_per_row(a.nchunks);
  if ((a.nchunks + a.lpr - 1) / a.lpr > 4) return KANN_EINVAL;
  if (a.nq > 0 && (!a.q || !aligned16(a.q))) return KANN_EINVAL;
  const int rc = plan_shared(idx, a, wpb);
  if (rc != KANN_OK || a.nq == 0) return rc;
  return check_cuda((cudaError_t)launch_search_pq(a, 1, stream));
}

int run_sparse(const kann_index_t* idx, SearchArgs& a, const SparseArgs& sa, int wpb, void* stream) {
  if (a.R != 0) return KANN_EINVAL;
  a.metric = KANN_IP;
  const int rc = plan_shared(idx, a, wpb);
  if (rc != KANN_OK || a.nq == 0) return rc;
  return check_cuda((cudaError_t)launch_search_sparse(a, sa, wpb, stream));
}

// ---- format conversion kernels ---------------------------------------------
__global__ void to_f16_kernel(const float* x, int64_t n, __half* y) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = __float2half_rn(x[i]);
}

__global__ void to_bf16_kernel(const float* x, int64_t n, __nv_bfloat16* y) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16_rn(x[i]);
}

// One warp per row: s = max|x| / 448 (IEEE division), code = RNE, satfinite
// E4M3 of x / s (IEEE division).
__global__ void to_e4m3_kernel(const float* x, int64_t n, int d, unsigned char* y, float* scale) {
  const int lane = threadIdx.x & 31;
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (row >= n) return;
  const float* r = x + row * d;
  float mx = 0.f;
  for (int k = lane; k < d; k += 32) mx = fmaxf(mx, fabsf(r[k]));
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(FULL, mx, o));
  const float s = __fdiv_rn(mx, 448.0f);
  if (lane == 0) scale[row] = s;
  for (int k = lane; k < d; k += 32) {
    unsigned char c = 0;
    if (s != 0.f) c = (unsigned char)__nv_cvt_float_to_fp8(__fdiv_rn(r[k], s), __NV_SATFINITE, __NV_E4M3);
    y[row * d + k] = c;
  }
}

}  // namespace
}  // namespace kann

using namespace kann;

extern "C" {

const char* kann_status_str(int s) {
  switch (s) {
    case KANN_OK: return "ok";
    case KANN_EINVAL: return "invalid argument";
    case KANN_ENOMEM: return "out of memory (host or shared-memory budget)";
    case KANN_ECUDA: return "CUDA runtime error";
    case KANN_EFORMAT: return "inconsistent index description";
    case KANN_ETIMEOUT: return "bounded device wait timed out";
    default: return "unknown status";
  }
}

int kann_last_cuda_error(void) { return g_last_cuda; }

int kann_index_upload(kann_index_t** out, const kann_graph_desc* g, const kann_vectors_desc* v,
                      const kann_pq_desc* pq, const kann_sparse_desc* sp, const kann_vectors_desc* rerank,
                      int validate_ids) {
  if (!out || !g) return KANN_EINVAL;
  *out = nullptr;
  const int nsrc = (v != nullptr) + (pq != nullptr) + (sp != nullptr);
  if (nsrc != 1) return KANN_EINVAL;
  if (g->n <= 0 || g->n >= (int64_t)1 << 31) return KANN_EINVAL;
  if (g->M < 1 || g->M > 32 || g->M0 < 1 || g->M0 > KANN_MAX_M0) return KANN_EFORMAT;
  if (g->max_level < 0 || g->max_level > 60) return KANN_EFORMAT;
  if (g->entry < 0 || g->entry >= g->n) return KANN_EFORMAT;
  if (g->max_level > 0 && (g->n_upper < 1 || !g->d_upper)) return KANN_EFORMAT;
  if (!g->d_l0 || !g->d_upper_slot || !g->d_level) return KANN_EINVAL;
  kann_index_t* idx = new (std::nothrow) kann_index_t;
  if (!idx) return KANN_ENOMEM;
  std::memset(idx, 0, sizeof(*idx));
  idx->g = *g;
  int rc = KANN_OK;
  if (v) {
    idx->kind = 0;
    idx->v = *v;
    rc = validate_vectors(v, g->n);
  } else if (pq) {
    idx->kind = 1;
    idx->pq = *pq;
    if (pq->m < 1 || pq->ksub != 256 || pq->dsub < 1 || !pq->d_codes || !pq->d_codebooks) rc = KANN_EINVAL;
    if (pq->metric != KANN_L2 && pq->metric != KANN_IP) rc = KANN_EINVAL;
    if ((pq->m * pq->dsub) % 4 != 0 || pq->m * pq->dsub > KANN_MAX_DIM) rc = KANN_EINVAL;
    if (pq->m % 16 != 0 || pq->m > 512 || !aligned16(pq->d_codes)) rc = KANN_EINVAL;
  } else {
    idx->kind = 2;
    idx->sp = *sp;
    if (!sp->d_indptr || !sp->d_terms || !sp->d_weights || sp->vocab < 1 || sp->vocab > 65536) rc = KANN_EINVAL;
  }
  if (rc == KANN_OK && rerank) {
    if (rerank->dtype != KANN_F32 && rerank->dtype != KANN_BF16) rc = KANN_EINVAL;
    else rc = validate_vectors(rerank, g->n);
    if (rc == KANN_OK && idx->kind == 0 && (rerank->d != v->d || rerank->metric != v->metric)) rc = KANN_EINVAL;
    if (rc == KANN_OK && idx->kind == 1 && (rerank->d != pq->m * pq->dsub || rerank->metric != pq->metric))
      rc = KANN_EINVAL;
    if (rc == KANN_OK && idx->kind == 2) rc = KANN_EINVAL;
    if (rc == KANN_OK && rerank->d / 4 > 32 * 8) rc = KANN_EINVAL;
    idx->has_rr = 1;
    idx->rr = *rerank;
  }
  if (rc == KANN_OK && validate_ids) {
    int* d_bad = nullptr;
    rc = check_cuda(cudaMalloc(&d_bad, sizeof(int)));
    if (rc == KANN_OK) {
      int h_bad = 0;
      rc = check_cuda(cudaMemset(d_bad, 0, sizeof(int)));
      if (rc == KANN_OK) {
        validate_graph_kernel<<<296, 256>>>(*g, d_bad);
        rc = check_cuda(cudaGetLastError());
      }
      if (rc == KANN_OK) rc = check_cuda(cudaMemcpy(&h_bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost));
      cudaFree(d_bad);
      if (rc == KANN_OK && h_bad) rc = KANN_EFORMAT;
    }
  }
  if (rc != KANN_OK) {
    delete idx;
    return rc;
  }
  cudaGetDevice(&idx->device);
  *out = idx;
  return KANN_OK;
}

int kann_index_destroy(kann_index_t* idx) {
  delete idx;
  return KANN_OK;
}

int kann_search_ex(const kann_index_t* idx, const float* d_queries, int n, int k, int ef, int32_t* d_ids,
                   float* d_dists, const kann_search_opts* opts, void* stream) {
  if (k < 1) return KANN_EINVAL;
  SearchArgs a;
  int wpb = 4;
  int rc = fill_search_args(idx, d_queries, n, k, ef, k, ef > k ? ef : k, nullptr, nullptr, d_ids, d_dists, opts, a,
                            wpb);
  if (rc != KANN_OK) return rc;
  if (idx->kind == 0) return run_dense(idx, a, wpb, stream);
  if (idx->kind == 1) return run_pq(idx, a, wpb, stream);
  return KANN_EINVAL;
}

int kann_search(const kann_index_t* idx, const float* d_queries, int n, int k, int ef, int32_t* d_ids,
                float* d_dists, void* stream) {
  return kann_search_ex(idx, d_queries, n, k, ef, d_ids, d_dists, nullptr, stream);
}

int kann_search_batch(const kann_index_t* idx, const float* d_queries, int n, const int32_t* d_k,
                      const int32_t* d_ef, int kmax, int efmax, int32_t* d_ids, float* d_dists,
                      const kann_search_opts* opts, void* stream) {
  if (n > 0 && (!d_k || !d_ef)) return KANN_EINVAL;
  SearchArgs a;
  int wpb = 4;
  int rc = fill_search_args(idx, d_queries, n, kmax, efmax, kmax, efmax, d_k, d_ef, d_ids, d_dists, opts, a, wpb);
  if (rc != KANN_OK) return rc;
  if (idx->kind == 0) return run_dense(idx, a, wpb, stream);
  if (idx->kind == 1) return run_pq(idx, a, wpb, stream);
  return KANN_EINVAL;
}

size_t kann_search_workspace_bytes_ex(const kann_index_t* idx, int n, int kmax, int efmax,
                                      const kann_search_opts* opts) {
  if (!idx || n < 0 || kmax < 1) return 0;
  // the search's own argument checks and shared-memory plan decide whether it
  // can run (the batch is sized by n below; no device pointer is needed)
  SearchArgs a;
  int wpb = 4;
  kann_search_opts o;
  if (opts) {
    o = *opts;
    o.d_n = nullptr;  // pointer options do not change what a batch needs
    o.d_work_counter = nullptr;
  }
  if (fill_search_args(idx, nullptr, 0, kmax, efmax, kmax, efmax, nullptr, nullptr, nullptr, nullptr,
                       opts ? &o : nullptr, a, wpb) != KANN_OK)
    return 0;
  if (idx->kind == 2 && a.R != 0) return 0;
  if (idx->kind == 0) {
    const int nchunks = idx->v.d * elem_size(idx->v.dtype) / 16;
    int lpr = a.lpr_override ? a.lpr_override : lanes_per_row(nchunks, default_chunks_per_lane(idx->v.dtype));
    if (lpr > nchunks && nchunks >= 1) lpr = lanes_per_row(nchunks);
    if ((nchunks + lpr - 1) / lpr > 8) return 0;
  }
  if (idx->kind == 1) {
    const int nchunks = idx->pq.m / 16;
    int lpr = a.lpr_override ? a.lpr_override : lanes_per_row(nchunks);
    if (lpr > nchunks) lpr = lanes_per_row(nchunks);
    if ((nchunks + lpr - 1) / lpr > 4) return 0;
  }
  if (plan_shared(idx, a, wpb) != KANN_OK) return 0;
  const int d = idx->kind == 1 ? idx->pq.m * idx->pq.dsub : idx->v.d;
  const size_t q = idx->kind == 2 ? (size_t)(n + 1) * 8 : (size_t)n * (size_t)d * 4;
  return q + (size_t)n * 8 + (size_t)n * (size_t)kmax * 8 + (size_t)n * 4 + 8;
}

size_t kann_search_workspace_bytes(const kann_index_t* idx, int n, int kmax, int efmax) {
  return kann_search_workspace_bytes_ex(idx, n, kmax, efmax, nullptr);
}

int kann_search_sparse(const kann_index_t* idx, const int64_t* d_q_indptr, const uint16_t* d_q_terms,
                       const float* d_q_weights, int n, int k, int ef, int32_t* d_ids, float* d_dists,
                       const kann_search_opts* opts, void* stream) {
  if (k < 1 || !idx || idx->kind != 2) return KANN_EINVAL;
  if (n > 0 && (!d_q_indptr || !d_q_terms || !d_q_weights)) return KANN_EINVAL;
  SearchArgs a;
  int wpb = 4;
  int rc = fill_search_args(idx, nullptr, n, k, ef, k, ef > k ? ef : k, nullptr, nullptr, d_ids, d_dists, opts, a,
                            wpb);
  if (rc != KANN_OK) return rc;
  SparseArgs sa;
  sa.indptr = idx->sp.d_indptr;
  sa.terms = idx->sp.d_terms;
  sa.w = idx->sp.d_weights;
  sa.q_indptr = d_q_indptr;
  sa.q_terms = d_q_terms;
  sa.q_w = d_q_weights;
  sa.vocab = idx->sp.vocab;
  return run_sparse(idx, a, sa, wpb, stream);
}

int kann_quantize(const float* d_x, int64_t n, int d, int dtype, void* d_out, float* d_scale, void* stream) {
  if (n < 0 || d < 1 || !d_x || !d_out) return KANN_EINVAL;
  if (n == 0) return KANN_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t total = n * (int64_t)d;
  const int blocks = (int)((total + 255) / 256 < 148 * 16 ? (total + 255) / 256 : 148 * 16);
  switch (dtype) {
    case KANN_F16: to_f16_kernel<<<blocks, 256, 0, s>>>(d_x, total, (__half*)d_out); break;
    case KANN_BF16: to_bf16_kernel<<<blocks, 256, 0, s>>>(d_x, total, (__nv_bfloat16*)d_out); break;
    case KANN_E4M3: {
      if (!d_scale) return KANN_EINVAL;
      const int64_t threads = n * 32;
      to_e4m3_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(d_x, n, d, (unsigned char*)d_out, d_scale);
      break;
    }
    default: return KANN_EINVAL;
  }
  return check_cuda(cudaGetLastError());
}

}  // extern "C"
