// kann_exact_sparse.cu -- exact k-NN for sparse inner product (the ground
// truth of the sparse measure, Sec. 3 / Table 1): one CTA per query scatters
// the query's weights into a dense shared-memory table over the vocabulary,
// then its warps walk every document's term list (lanes over the terms, FP32
// sums of table[term] * weight, butterfly reduction) and keep the k best
// (distance = -IP, id) keys per warp; the warps' lists are merged at the end.
#include "kann_device.cuh"
#include "kann_internal.h"

namespace kann {
namespace {

constexpr int XS_WARPS = 16;
constexpr int XS_KMAX = 128;

// Insert x into the ascending warp-held list L[0..kp) in shared memory.
__device__ __forceinline__ void sorted_insert(u64* L, int kp, u64 x, int lane) {
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

__global__ void __launch_bounds__(XS_WARPS * 32) exact_sparse_kernel(
    const int64_t* __restrict__ indptr, const uint16_t* __restrict__ terms, const float* __restrict__ w, int64_t nb,
    const int64_t* __restrict__ q_indptr, const uint16_t* __restrict__ q_terms, const float* __restrict__ q_w,
    int vocab, int k, int kp, int32_t* ids, float* dists) {
  extern __shared__ __align__(16) unsigned char smem[];
  u64* lists = reinterpret_cast<u64*>(smem);                         // [XS_WARPS][kp]
  float* table = reinterpret_cast<float*>(lists + XS_WARPS * kp);    // [vocab]
  const int q = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < vocab; i += blockDim.x) table[i] = 0.f;
  for (int i = threadIdx.x; i < XS_WARPS * kp; i += blockDim.x) lists[i] = KEY_MAX;
  __syncthreads();
  for (int64_t t = q_indptr[q] + threadIdx.x; t < q_indptr[q + 1]; t += blockDim.x)
    if (q_terms[t] < vocab) table[q_terms[t]] = q_w[t];
  __syncthreads();
  u64* L = lists + warp * kp;
  u64 thr = KEY_MAX;
  for (int64_t doc = warp; doc < nb; doc += XS_WARPS) {
    const int64_t b = __ldg(indptr + doc), e = __ldg(indptr + doc + 1);
    float acc = 0.f;
    for (int64_t t = b + lane; t < e; t += 32) {
      const uint32_t tm = __ldg(terms + t);
      if (tm < (uint32_t)vocab) acc = fmaf(table[tm], __ldg(w + t), acc);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
    const u64 key = make_key(-acc, (uint32_t)doc);
    if (key < thr) {
      sorted_insert(L, kp, key, lane);
      thr = L[k - 1];
    }
  }
  __syncthreads();
  // merge the warps' lists: warp 0 sorts all of them
  if (warp == 0) {
    int P = 32;
    while (P < XS_WARPS * kp) P <<= 1;
    // lists occupy XS_WARPS * kp slots; pad to P in place is not possible, so
    // repeatedly take the minimum head (k rounds)
    for (int j = 0; j < k; ++j) {
      u64 best = KEY_MAX;
      int bw = 0;
      if (lane < XS_WARPS) {
        best = lists[lane * kp];
        bw = lane;
      }
      for (int o = 16; o > 0; o >>= 1) {
        const u64 ob = __shfl_xor_sync(FULL, best, o);
        const int ow = __shfl_xor_sync(FULL, bw, o);
        if (ob < best || (ob == best && ow < bw)) {
          best = ob;
          bw = ow;
        }
      }
      if (lane == 0) {
        ids[(size_t)q * k + j] = best == KEY_MAX ? -1 : (int32_t)(uint32_t)best;
        dists[(size_t)q * k + j] = best == KEY_MAX ? __int_as_float(0x7f800000) : key_dist(best);
      }
      // pop the head of list bw
      u64* Lb = lists + bw * kp;
      for (int b = 0; b < kp; b += 32) {
        const int i = b + lane;
        const u64 nxt = i + 1 < kp ? Lb[i + 1] : KEY_MAX;
        __syncwarp();
        Lb[i] = nxt;
        __syncwarp();
      }
    }
  }
}

}  // namespace
}  // namespace kann

using namespace kann;

extern "C" int kann_exact_knn_sparse(const int64_t* d_indptr, const uint16_t* d_terms, const float* d_weights,
                                     int64_t nb, const int64_t* d_q_indptr, const uint16_t* d_q_terms,
                                     const float* d_q_weights, int nq, int vocab, int k, int32_t* d_ids,
                                     float* d_dists, void* stream) {
  if (nq < 0 || nb < 1 || k < 1 || k > XS_KMAX || vocab < 1) return KANN_EINVAL;
  if (nq == 0) return KANN_OK;
  if (!d_indptr || !d_terms || !d_weights || !d_q_indptr || !d_q_terms || !d_q_weights || !d_ids || !d_dists)
    return KANN_EINVAL;
  const int kp = (k + 31) / 32 * 32;
  const size_t smem = (size_t)XS_WARPS * kp * 8 + (size_t)vocab * 4;
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (smem > (size_t)optin) return KANN_EINVAL;  // vocabulary too large for the shared table
  cudaError_t e = cudaFuncSetAttribute(exact_sparse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) {
    exact_sparse_kernel<<<nq, XS_WARPS * 32, smem, (cudaStream_t)stream>>>(
        d_indptr, d_terms, d_weights, nb, d_q_indptr, d_q_terms, d_q_weights, vocab, k, kp, d_ids, d_dists);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    set_cuda_error((int)e);
    return KANN_ECUDA;
  }
  return KANN_OK;
}
