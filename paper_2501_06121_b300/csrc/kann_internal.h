// kann_internal.h -- definitions shared by the library's translation units.
#pragma once
#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/kann.h"

namespace kann {

// Arguments of one dense/PQ search launch (all device pointers).
struct SearchArgs {
  // graph (HNSW, fixed-width rows)
  const int32_t* l0;
  const int32_t* upper_slot;
  const int32_t* upper;
  int64_t n;
  int M0, M, max_level, entry;
  // traversal rows
  const unsigned char* data;
  int64_t stride;
  const float* scale;
  int d, nchunks, lpr, metric;
  // PQ traversal
  const unsigned char* codes;
  const float* codebooks;
  int pq_m, pq_dsub;
  // re-rank rows (FP32)
  const unsigned char* rr_data;
  int64_t rr_stride;
  int rr_nchunks, rr_lpr, R;
  int rr_dtype;        // KANN_F32 or KANN_BF16
  // queries and outputs
  const float* q;
  int nq, k, ef, kmax, efmax;
  const int32_t* k_arr;
  const int32_t* ef_arr;
  int32_t* out_ids;
  float* out_d;
  uint32_t* status;
  int32_t* counters;
  int hbits, max_hops;
  int vis_k, vis_r;      // compact visited table: id bits and slot-value bits; vis_r < 0: wide table
  int lpr_override;  // 0 = automatic lanes per row
  int* work_counter;     // persistent mode: next query index (zeroed before launch), or null
  const int32_t* d_n;    // persistent mode: device-side query count (<= nq), or null
  int lean;              // dense: half the rows in flight, 64-register budget
  int lut;               // PQ: per-query table format (KANN_PQ_LUT_F32 / F16 / U8)
  int efcap;       // W capacity (efmax rounded up to a multiple of 32)
  int expand;      // layer-0 entries expanded per step (1 = the HNSW step; 2..KANN_MAX_EXPAND: batched)
  int team;        // dense/sparse: warps per query (1 = one warp per query; 2 or 4 = a CTA per query)
  int warp_smem;   // bytes of shared memory per warp (per query region of a team)
};

// Sparse search additions.
struct SparseArgs {
  const int64_t* indptr;
  const uint16_t* terms;
  const float* w;
  const int64_t* q_indptr;
  const uint16_t* q_terms;
  const float* q_w;
  int vocab;
};

// Chunks (16 bytes) of a row per lane used for a storage format by default
// (measured on the 1M x 128 workload: 64 bytes of an FP32 or E4M3 row per
// lane, 32 bytes of an FP16 or BF16 row).
constexpr int default_chunks_per_lane(int dtype) { return (dtype == KANN_F16 || dtype == KANN_BF16) ? 2 : 4; }

// A dense/PQ search kernel.
typedef void (*SearchKernelFn)(const SearchArgs);

// Dense search kernel of one storage format for `cplt` chunks per lane
// (kann_search_{f32,f16,bf16,e4m3}.cu); lpr_exact > 0 when a row is exactly
// lpr_exact * cplt chunks; the _multi pickers give the multi-expansion
// kernels.  Null when no kernel exists for the settings.
SearchKernelFn pick_search_f32(int cplt, bool lean, int metric, int lpr_exact);
SearchKernelFn pick_search_f16(int cplt, bool lean, int metric, int lpr_exact);
SearchKernelFn pick_search_bf16(int cplt, bool lean, int metric, int lpr_exact);
SearchKernelFn pick_search_e4m3(int cplt, bool lean, int metric, int lpr_exact);
SearchKernelFn pick_search_f32_multi(int cplt, int metric, int lpr_exact);
SearchKernelFn pick_search_f16_multi(int cplt, int metric, int lpr_exact);
SearchKernelFn pick_search_bf16_multi(int cplt, int metric, int lpr_exact);
SearchKernelFn pick_search_e4m3_multi(int cplt, int metric, int lpr_exact);
// Team kernels (a CTA of `team` = 2 or 4 warps per query), compiled in
// kann_search_{f32,f16,bf16,e4m3}_team.cu.
SearchKernelFn pick_search_f32_team(int cplt, int metric, int lpr_exact, int team);
SearchKernelFn pick_search_f16_team(int cplt, int metric, int lpr_exact, int team);
SearchKernelFn pick_search_bf16_team(int cplt, int metric, int lpr_exact, int team);
SearchKernelFn pick_search_e4m3_team(int cplt, int metric, int lpr_exact, int team);

// Candidate keys a warp keeps per step: 64 per expanded entry, plus 64 for
// the ranked survivors of a batch when several entries are expanded at once.
__host__ __device__ constexpr int cand_keys(int expand) { return 64 * expand + (expand > 1 ? 64 : 0); }

// Per-warp shared memory needed by a dense search with these settings
// (compact: a visited table of 16-bit slots, else 32-bit).
int search_warp_smem(int efcap, int hbits, bool compact, int expand = 1);
int search_warp_smem_pq(int efcap, int hbits, bool compact, int m, int lut = KANN_PQ_LUT_F32);
// Shared memory of a search team's control block (after the query's region).
constexpr int PQ_TEAM_CTL_BYTES = 64;
int search_warp_smem_sparse(int efcap, int hbits, bool compact, int vocab);

// Launchers (kann_search.cu); return a cudaError_t.
int launch_search_dense(const SearchArgs& a, int dtype, int wpb, void* stream);
int launch_search_pq(const SearchArgs& a, int wpb, void* stream);
int launch_search_sparse(const SearchArgs& a, const SparseArgs& s, int wpb, void* stream);

void set_cuda_error(int e);

// Tensor-core exact k-NN (kann_exact_tc.cu).
bool exact_tc_supported(int dtype, int d, int k);
size_t exact_tc_workspace_bytes(int nq, int64_t nb, int k);
int exact_tc_run(const void* Q, const void* X, int nq, int64_t nb, int d, int metric, int dtype, int k, int32_t* ids,
                 float* dists, void* ws, cudaStream_t s);

}  // namespace kann
