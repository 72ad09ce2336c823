// kann_search.cu -- launchers of the batched HNSW search kernels, and the PQ
// and sparse kernels (the dense kernels are compiled per storage format in
// kann_search_{f32,f16,bf16,e4m3}.cu; the device code is kann_search_impl.cuh
// and, for the sparse back-end, kann_search_sparse.cuh).
#include "kann_search_impl.cuh"
#include "kann_search_sparse.cuh"

namespace kann {
namespace {

// Register budgets (measured on 1M documents, event times, identical results):
// 85 registers for a team (24 warps per SM) with 8 terms per lane in flight
// ran 7-21% faster than 128 registers (16 warps) with 16 terms per lane; the
// one-warp kernel keeps 102 so that it does not spill.
__global__ void __launch_bounds__(128, 5) search_sparse_kernel(const SearchArgs a, const __grid_constant__ SparseArgs sp) {
  SparseBackend be;
  be.sp = &sp;
  run_queries(a, be);
}

// A team kernel of the sparse back-end: one query per CTA of T warps.
template <int T>
__global__ void __launch_bounds__(T * 32, 24 / T)
    search_sparse_team_kernel(const SearchArgs a, const __grid_constant__ SparseArgs sp) {
  SparseBackend be;
  be.sp = &sp;
  run_queries_team<T>(a, be);
}

// Grid of a launch of CTAs of `warps` warps, `per_cta` queries each: one
// CTA per per_cta queries, or (persistent) as many CTAs as fit on the GPU at
// once.
template <class F>
int launch_grid(F fn, const SearchArgs& a, int warps, int per_cta, size_t smem) {
  const int plain = (a.nq + per_cta - 1) / per_cta;
  if (a.work_counter == nullptr) return plain;
  int dev = 0, sms = 148, per_sm = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, warps * 32, smem) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  const int full = sms * per_sm;
  return plain < full ? plain : full;
}

int start_counter(const SearchArgs& a, cudaStream_t s) {
  if (a.work_counter == nullptr) return 0;
  return (int)cudaMemsetAsync(a.work_counter, 0, sizeof(int), s);
}

int pow2_at_least(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

}  // namespace

// Every warp's (team's) region starts at a multiple of its size, and its
// 8-byte beam keys and 16-byte visited-table rows need that start aligned:
// region sizes are rounded up to 128 bytes.
int round_region(int bytes) { return (bytes + 127) / 128 * 128; }

int search_warp_smem(int efcap, int hbits, bool compact, int expand) {
  return round_region(efcap * 8 + cand_keys(expand) * 8 + 64 * expand * 4 + ((compact ? 2 : 4) << hbits));
}

int launch_search_dense(const SearchArgs& a, int dtype, int wpb, void* stream) {
  if (a.nq == 0) return 0;
  if (a.warp_smem % 16 != 0) return (int)cudaErrorInvalidValue;  // regions must stay 16-byte aligned
  const int cplt = pow2_at_least((a.nchunks + a.lpr - 1) / a.lpr);
  const int lpr_exact = a.nchunks == a.lpr * cplt ? a.lpr : 0;
  SearchKernelFn fn = nullptr;
  if (a.team > 1) {
    // one query per CTA of a.team warps, the team's control block after the
    // query's region
    switch (dtype) {
      case KANN_F32: fn = pick_search_f32_team(cplt, a.metric, lpr_exact, a.team); break;
      case KANN_F16: fn = pick_search_f16_team(cplt, a.metric, lpr_exact, a.team); break;
      case KANN_BF16: fn = pick_search_bf16_team(cplt, a.metric, lpr_exact, a.team); break;
      case KANN_E4M3: fn = pick_search_e4m3_team(cplt, a.metric, lpr_exact, a.team); break;
      default: break;
    }
    if (!fn || a.expand > 1) return (int)cudaErrorInvalidValue;
    const size_t smem = (size_t)a.warp_smem + PQ_TEAM_CTL_BYTES;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    const int grid = launch_grid(fn, a, a.team, 1, smem);
    int c = start_counter(a, (cudaStream_t)stream);
    if (c) return c;
    fn<<<grid, a.team * 32, smem, (cudaStream_t)stream>>>(a);
    return (int)cudaGetLastError();
  }
  switch (dtype) {
    case KANN_F32:
      fn = a.expand > 1 ? pick_search_f32_multi(cplt, a.metric, lpr_exact) : pick_search_f32(cplt, a.lean, a.metric, lpr_exact);
      break;
    case KANN_F16:
      fn = a.expand > 1 ? pick_search_f16_multi(cplt, a.metric, lpr_exact) : pick_search_f16(cplt, a.lean, a.metric, lpr_exact);
      break;
    case KANN_BF16:
      fn = a.expand > 1 ? pick_search_bf16_multi(cplt, a.metric, lpr_exact)
                        : pick_search_bf16(cplt, a.lean, a.metric, lpr_exact);
      break;
    case KANN_E4M3:
      fn = a.expand > 1 ? pick_search_e4m3_multi(cplt, a.metric, lpr_exact)
                        : pick_search_e4m3(cplt, a.lean, a.metric, lpr_exact);
      break;
    default: break;
  }
  if (!fn) return (int)cudaErrorInvalidValue;
  const size_t smem = (size_t)wpb * a.warp_smem;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  const int grid = launch_grid(fn, a, wpb, wpb, smem);
  int c = start_counter(a, (cudaStream_t)stream);
  if (c) return c;
  fn<<<grid, wpb * 32, smem, (cudaStream_t)stream>>>(a);
  return (int)cudaGetLastError();
}

int search_warp_smem_pq(int efcap, int hbits, bool compact, int m, int lut) {
  // uint8 table: the entries plus the subspace minima and ranges (8 m bytes)
  const int table = lut == KANN_PQ_LUT_U8 ? m * 256 + 8 * m : m * 256 * (lut == KANN_PQ_LUT_F16 ? 2 : 4);
  return round_region(search_warp_smem(efcap, hbits, compact) + table);
}

int search_warp_smem_sparse(int efcap, int hbits, bool compact, int vocab) {
  return round_region(search_warp_smem(efcap, hbits, compact) + sparse_query_bytes(vocab));
}

int launch_search_pq(const SearchArgs& a, int wpb, void* stream) {
  if (a.nq == 0) return 0;
  if (a.warp_smem % 16 != 0) return (int)cudaErrorInvalidValue;  // regions must stay 16-byte aligned
  const int cplt = pow2_at_least((a.nchunks + a.lpr - 1) / a.lpr);
  SearchKernelFn fn = nullptr;
  static_assert(PQ_LUT_F16 == KANN_PQ_LUT_F16 && PQ_LUT_U8 == KANN_PQ_LUT_U8, "table formats");
  switch (cplt * 4 + a.lut) {
    case 4 + PQ_LUT_F32: fn = search_pq_kernel<1, PQ_LUT_F32>; break;
    case 4 + PQ_LUT_F16: fn = search_pq_kernel<1, PQ_LUT_F16>; break;
    case 4 + PQ_LUT_U8: fn = search_pq_kernel<1, PQ_LUT_U8>; break;
    case 8 + PQ_LUT_F32: fn = search_pq_kernel<2, PQ_LUT_F32>; break;
    case 8 + PQ_LUT_F16: fn = search_pq_kernel<2, PQ_LUT_F16>; break;
    case 8 + PQ_LUT_U8: fn = search_pq_kernel<2, PQ_LUT_U8>; break;
    case 16 + PQ_LUT_F32: fn = search_pq_kernel<4, PQ_LUT_F32>; break;
    case 16 + PQ_LUT_F16: fn = search_pq_kernel<4, PQ_LUT_F16>; break;
    case 16 + PQ_LUT_U8: fn = search_pq_kernel<4, PQ_LUT_U8>; break;
    default: break;
  }
  if (!fn) return (int)cudaErrorInvalidValue;
  (void)wpb;  // one query per CTA of PQ_TEAM warps
  static_assert(sizeof(TeamCtl) <= PQ_TEAM_CTL_BYTES, "team control block");
  const size_t smem = (size_t)a.warp_smem + PQ_TEAM_CTL_BYTES;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  const int grid = launch_grid(fn, a, PQ_TEAM, 1, smem);
  int c = start_counter(a, (cudaStream_t)stream);
  if (c) return c;
  fn<<<grid, PQ_TEAM * 32, smem, (cudaStream_t)stream>>>(a);
  return (int)cudaGetLastError();
}

int launch_search_sparse(const SearchArgs& a, const SparseArgs& sp, int wpb, void* stream) {
  if (a.nq == 0) return 0;
  if (a.warp_smem % 16 != 0) return (int)cudaErrorInvalidValue;  // regions must stay 16-byte aligned
  if (a.team > 1) {
    void (*fn)(const SearchArgs, const SparseArgs) =
        a.team == 2 ? search_sparse_team_kernel<2> : (a.team == 4 ? search_sparse_team_kernel<4> : nullptr);
    if (!fn) return (int)cudaErrorInvalidValue;
    const size_t smem = (size_t)a.warp_smem + PQ_TEAM_CTL_BYTES;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    const int grid = launch_grid(fn, a, a.team, 1, smem);
    int c = start_counter(a, (cudaStream_t)stream);
    if (c) return c;
    fn<<<grid, a.team * 32, smem, (cudaStream_t)stream>>>(a, sp);
    return (int)cudaGetLastError();
  }
  const size_t smem = (size_t)wpb * a.warp_smem;
  cudaError_t e = cudaFuncSetAttribute(search_sparse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  const int grid = launch_grid(search_sparse_kernel, a, wpb, wpb, smem);
  int c = start_counter(a, (cudaStream_t)stream);
  if (c) return c;
  search_sparse_kernel<<<grid, wpb * 32, smem, (cudaStream_t)stream>>>(a, sp);
  return (int)cudaGetLastError();
}

}  // namespace kann
