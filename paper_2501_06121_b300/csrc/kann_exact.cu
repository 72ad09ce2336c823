// kann_exact.cu -- exact k-NN by brute force with a fused top-k (the ground
// truth against which search recall is measured; the paper's k-NN problem
// statement, Sec. 1).
//
// Pass 1 (exact_tile_kernel): grid = (query tiles of 64) x (S base splits).
// A CTA of 256 threads streams its split of the base in tiles of 64 rows,
// computes the 64 x 64 distance tile in the direct form (sum (q - x)^2 or
// -sum q x, FP32) with a 4 x 4 register micro-tile per thread, and keeps for
// each of its queries the k best (distance, id) keys in shared memory
// (threshold filter, then a warp-parallel sorted insert).  Each CTA writes
// its per-query lists to the caller's workspace.
// Pass 2 (exact_merge_kernel): one warp per query sorts the S * k partial keys
// and writes the k best.
#include <mutex>

#include "kann_device.cuh"
#include "kann_internal.h"

namespace kann {
namespace {

constexpr int QT = 64;   // queries per CTA
constexpr int BT = 64;   // base rows per tile
constexpr int DK = 32;   // dimensions staged per step
constexpr int LDS = DK + 4;

template <int DT>
__device__ __forceinline__ float4 load4(const void* base, int64_t row, int d, int col) {
  if (DT == KANN_F32) {
    return __ldg(reinterpret_cast<const float4*>(static_cast<const float*>(base) + row * d + col));
  } else {
    const uint2 v = __ldg(reinterpret_cast<const uint2*>(static_cast<const uint16_t*>(base) + row * d + col));
    float o[8];
    uint4 w = make_uint4(v.x, v.y, 0u, 0u);
    Fmt<DT>::unpack(w, o);
    return make_float4(o[0], o[1], o[2], o[3]);
  }
}

// Insert key x into the ascending list L[0..kp) (kp a multiple of 32),
// dropping the last entry.  Executed by a whole warp.
__device__ __forceinline__ void list_insert(u64* L, int kp, u64 x, int lane) {
  int pos = 0;
  for (int b = 0; b < kp; b += 32) pos += __popc(__ballot_sync(FULL, L[b + lane] < x));
  for (int b = kp - 32; b >= 0; b -= 32) {
    const int i = b + lane;
    const u64 prev = i > 0 ? L[i - 1] : KEY_MAX;
    __syncwarp();
    if (i > pos) L[i] = prev;
    else if (i == pos) L[i] = x;
    __syncwarp();
  }
}

template <int DT>
__global__ void __launch_bounds__(256) exact_tile_kernel(const void* __restrict__ Q, const void* __restrict__ X, int nq,
                                                         int64_t nb, int d, int metric, int k, int kp, int S,
                                                         u64* __restrict__ ws) {
  extern __shared__ __align__(16) unsigned char smem[];
  float* Qs = reinterpret_cast<float*>(smem);               // [QT][LDS]
  float* Xs = Qs + QT * LDS;                                // [BT][LDS]
  float* Ds = Xs + BT * LDS;                                // [QT][BT + 1]
  u64* Ls = reinterpret_cast<u64*>(Ds + QT * (BT + 1));     // [QT][kp]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ty = tid >> 4, tx = tid & 15;
  const int q0 = blockIdx.x * QT;
  const int split = blockIdx.y;
  const int64_t per = (nb + S - 1) / S;
  const int64_t b_begin = (int64_t)split * per;
  const int64_t b_end = b_begin + per < nb ? b_begin + per : nb;

  for (int i = tid; i < QT * kp; i += 256) Ls[i] = KEY_MAX;
  __syncthreads();

  for (int64_t b0 = b_begin; b0 < b_end; b0 += BT) {
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    for (int k0 = 0; k0 < d; k0 += DK) {
      // stage Q[q0.., k0..k0+DK) and X[b0.., k0..) (zero outside)
      for (int i = tid; i < QT * (DK / 4); i += 256) {
        const int r = i / (DK / 4), c = (i % (DK / 4)) * 4;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (q0 + r < nq && k0 + c < d) v = load4<DT>(Q, q0 + r, d, k0 + c);
        *reinterpret_cast<float4*>(Qs + r * LDS + c) = v;
      }
      for (int i = tid; i < BT * (DK / 4); i += 256) {
        const int r = i / (DK / 4), c = (i % (DK / 4)) * 4;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (b0 + r < b_end && k0 + c < d) v = load4<DT>(X, b0 + r, d, k0 + c);
        *reinterpret_cast<float4*>(Xs + r * LDS + c) = v;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < DK; kk += 4) {
        float4 qa[4], xb[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) qa[i] = *reinterpret_cast<const float4*>(Qs + (ty + 16 * i) * LDS + kk);
#pragma unroll
        for (int j = 0; j < 4; ++j) xb[j] = *reinterpret_cast<const float4*>(Xs + (tx + 16 * j) * LDS + kk);
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            if (metric == KANN_L2) {
              float t;
              t = qa[i].x - xb[j].x; acc[i][j] = fmaf(t, t, acc[i][j]);
              t = qa[i].y - xb[j].y; acc[i][j] = fmaf(t, t, acc[i][j]);
              t = qa[i].z - xb[j].z; acc[i][j] = fmaf(t, t, acc[i][j]);
              t = qa[i].w - xb[j].w; acc[i][j] = fmaf(t, t, acc[i][j]);
            } else {
              acc[i][j] = fmaf(qa[i].x, xb[j].x, acc[i][j]);
              acc[i][j] = fmaf(qa[i].y, xb[j].y, acc[i][j]);
              acc[i][j] = fmaf(qa[i].z, xb[j].z, acc[i][j]);
              acc[i][j] = fmaf(qa[i].w, xb[j].w, acc[i][j]);
            }
          }
      }
      __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j)
        Ds[(ty + 16 * i) * (BT + 1) + tx + 16 * j] = metric == KANN_L2 ? acc[i][j] : -acc[i][j];
    __syncthreads();
    // top-k upkeep: warp w owns queries w*8 .. w*8+7 of the tile
    for (int qq = warp * 8; qq < warp * 8 + 8; ++qq) {
      if (q0 + qq >= nq) break;
      u64* L = Ls + qq * kp;
      const int64_t i0 = b0 + lane, i1 = b0 + 32 + lane;
      u64 c0 = i0 < b_end ? make_key(Ds[qq * (BT + 1) + lane], (uint32_t)i0) : KEY_MAX;
      u64 c1 = i1 < b_end ? make_key(Ds[qq * (BT + 1) + 32 + lane], (uint32_t)i1) : KEY_MAX;
      u64 thr = L[k - 1];
      unsigned m0 = __ballot_sync(FULL, c0 < thr), m1 = __ballot_sync(FULL, c1 < thr);
      while (m0 | m1) {
        u64 x;
        if (m0) {
          const int src = __ffs(m0) - 1;
          x = __shfl_sync(FULL, c0, src);
          m0 &= m0 - 1;
        } else {
          const int src = __ffs(m1) - 1;
          x = __shfl_sync(FULL, c1, src);
          m1 &= m1 - 1;
        }
        if (x < thr) {
          list_insert(L, kp, x, lane);
          thr = L[k - 1];
        }
      }
      __syncwarp();
    }
    __syncthreads();
  }
  // partial lists -> workspace [nq][S][k]
  for (int i = tid; i < QT * k; i += 256) {
    const int qq = i / k, j = i % k;
    if (q0 + qq < nq) ws[((size_t)(q0 + qq) * S + split) * k + j] = Ls[qq * kp + j];
  }
}

__global__ void exact_merge_kernel(const u64* __restrict__ ws, int nq, int S, int k, int P, int32_t* ids,
                                   float* dists) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int q = blockIdx.x * (blockDim.x >> 5) + warp;
  if (q >= nq) return;
  u64* A = reinterpret_cast<u64*>(smem) + (size_t)warp * P;
  const int tot = S * k;
  for (int i = lane; i < P; i += 32) A[i] = i < tot ? ws[(size_t)q * tot + i] : KEY_MAX;
  __syncwarp();
  warp_smem_sort(A, P, lane);
  for (int j = lane; j < k; j += 32) {
    const u64 key = A[j];
    ids[(size_t)q * k + j] = key == KEY_MAX ? -1 : (int32_t)(uint32_t)key;
    dists[(size_t)q * k + j] = key == KEY_MAX ? __int_as_float(0x7f800000) : key_dist(key);
  }
}

int splits_for(int nq, int64_t nb) {
  const int qtiles = (nq + QT - 1) / QT;
  int S = (4 * 148 + qtiles - 1) / qtiles;
  const int64_t maxs = (nb + BT - 1) / BT;
  if (S > maxs) S = (int)maxs;
  if (S > 64) S = 64;
  if (S < 1) S = 1;
  return S;
}

}  // namespace
}  // namespace kann

using namespace kann;

extern "C" size_t kann_exact_knn_workspace_bytes(int nq, int64_t nb, int d, int k, int dtype) {
  if (nq <= 0 || nb <= 0 || k <= 0) return 0;
  if (exact_tc_supported(dtype, d, k)) return exact_tc_workspace_bytes(nq, nb, k);
  return (size_t)nq * splits_for(nq, nb) * k * sizeof(u64);
}

extern "C" int kann_exact_knn(const void* d_queries, const void* d_base, int nq, int64_t nb, int d, int metric,
                              int dtype, int k, int32_t* d_ids, float* d_dists, void* d_ws, size_t ws_bytes,
                              void* stream) {
  if (nq < 0 || nb < 0 || d < 1 || k < 1 || k > 256) return KANN_EINVAL;
  if (metric != KANN_L2 && metric != KANN_IP) return KANN_EINVAL;
  if (dtype != KANN_F32 && dtype != KANN_F16 && dtype != KANN_BF16) return KANN_EINVAL;
  if (d % 4 != 0) return KANN_EINVAL;
  if (nq == 0) return KANN_OK;
  if (!d_queries || !d_base || !d_ids || !d_dists || !d_ws) return KANN_EINVAL;
  // row loads are 16-byte vectors (FP32) or TMA boxes (tensor-core path);
  // the workspace holds 8-byte keys and a 16-byte aligned error word
  const auto misaligned = [](const void* p, uintptr_t a) { return ((uintptr_t)p & (a - 1)) != 0; };
  if (misaligned(d_queries, 16) || misaligned(d_base, 16) || misaligned(d_ws, 16)) return KANN_EINVAL;
  if (misaligned(d_ids, 4) || misaligned(d_dists, 4)) return KANN_EINVAL;
  if (nb == 0 || nb >= ((int64_t)1 << 31)) return KANN_EINVAL;
  if (ws_bytes < kann_exact_knn_workspace_bytes(nq, nb, d, k, dtype)) return KANN_EINVAL;
  if (exact_tc_supported(dtype, d, k)) {
    // BF16/FP16 inputs, k <= 32: tensor-core scores with the fused top-k
    const int e = exact_tc_run(d_queries, d_base, nq, nb, d, metric, dtype, k, d_ids, d_dists, d_ws,
                               (cudaStream_t)stream);
    if (e != cudaSuccess) {
      set_cuda_error(e);
      return KANN_ECUDA;
    }
    return KANN_OK;
  }
  const int S = splits_for(nq, nb);
  const int kp = (k + 31) / 32 * 32;
  const size_t smem = (size_t)(QT * LDS + BT * LDS + QT * (BT + 1)) * 4 + (size_t)QT * kp * 8;
  cudaStream_t s = (cudaStream_t)stream;
  void (*fn)(const void*, const void*, int, int64_t, int, int, int, int, int, u64*) =
      dtype == KANN_F32 ? exact_tile_kernel<KANN_F32>
                        : (dtype == KANN_F16 ? exact_tile_kernel<KANN_F16> : exact_tile_kernel<KANN_BF16>);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) {
    set_cuda_error((int)e);
    return KANN_ECUDA;
  }
  dim3 grid((nq + QT - 1) / QT, S);
  fn<<<grid, 256, smem, s>>>(d_queries, d_base, nq, nb, d, metric, k, kp, S, (u64*)d_ws);
  int P = 32;
  while (P < S * k) P <<= 1;
  int wpb = 4;
  while (wpb > 1 && (size_t)wpb * P * 8 > 160 * 1024) wpb >>= 1;
  const size_t msmem = (size_t)wpb * P * 8;
  e = cudaFuncSetAttribute(exact_merge_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)msmem);
  if (e == cudaSuccess) {
    exact_merge_kernel<<<(nq + wpb - 1) / wpb, wpb * 32, msmem, s>>>((const u64*)d_ws, nq, S, k, P, d_ids, d_dists);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    set_cuda_error((int)e);
    return KANN_ECUDA;
  }
  return KANN_OK;
}

// ---------------------------------------------------------------------------
// Exact k-NN without allocation, for callers that cannot call cudaMalloc (a
// host application whose device memory belongs to another allocator, or a
// latency-critical path where an allocation's implicit synchronisation is not
// allowed).  The split-N partial lists live in one static device array per
// GPU instead of caller scratch; its device address is looked up once per
// device, with that device current, by the first call there.
// ---------------------------------------------------------------------------
namespace kann {
namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[KANN_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};

int noalloc_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    set_cuda_error((int)e);
    return KANN_ECUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) return KANN_EINVAL;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (g_noalloc_ptr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) {
      set_cuda_error((int)e);
      return KANN_ECUDA;
    }
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return KANN_OK;
}

}  // namespace
}  // namespace kann

extern "C" int kann_exact_knn_noalloc(const void* d_queries, const void* d_base, int nq, int64_t nb, int d,
                                      int metric, int dtype, int k, int32_t* d_ids, float* d_dists, void* stream) {
  if (nq < 0 || nb < 0 || d < 1 || k < 1) return KANN_EINVAL;
  if (nq == 0) return KANN_OK;
  // the partial lists must fit the static array; nothing in it needs zeroing
  // (pass 1 writes every entry pass 2 reads)
  if (kann_exact_knn_workspace_bytes(nq, nb, d, k, dtype) > KANN_NOALLOC_SCRATCH_BYTES) return KANN_EINVAL;
  void* scratch = nullptr;
  const int rc = noalloc_scratch(&scratch);
  if (rc != KANN_OK) return rc;
  return kann_exact_knn(d_queries, d_base, nq, nb, d, metric, dtype, k, d_ids, d_dists, scratch,
                        KANN_NOALLOC_SCRATCH_BYTES, stream);
}
