// kann_pq.cu -- Product Quantization training and encoding on the GPU (the
// quantizer of kANNolo Sec. 2, citing Jegou et al.): per subspace j of dsub
// dimensions, Lloyd k-means with ksub = 256 centroids, then every vector's
// code byte j = its nearest centroid of subspace j (ties to the lowest index).
//
// This is index preparation, not the search path.  Initial centroids are
// distinct training vectors picked by a counter-based SplitMix64 draw keyed
// by (seed, subspace, draw); a centroid that loses all its points keeps its
// previous position.
#include "kann_device.cuh"
#include "kann_internal.h"

namespace kann {
namespace {

constexpr int PQ_K = 256;

__host__ __device__ inline uint64_t mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// Nearest centroid of subspace j for points [i0, i0 + blockDim) ; one CTA
// handles one subspace and a run of points, with the subspace's codebook in
// shared memory.  With `sums` non-null the chosen centroid's running sum and
// count are updated (training); codes may be null.
__global__ void assign_kernel(const float* __restrict__ x, int64_t n, int d, int m, int dsub,
                              const float* __restrict__ cb, uint8_t* __restrict__ codes, float* sums, int* counts) {
  extern __shared__ float scb[];  // [256][dsub]
  const int j = blockIdx.y;
  for (int i = threadIdx.x; i < PQ_K * dsub; i += blockDim.x) scb[i] = cb[(size_t)j * PQ_K * dsub + i];
  __syncthreads();
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const float* xp = x + p * d + (int64_t)j * dsub;
    float v[16];
    for (int t = 0; t < dsub; ++t) v[t] = xp[t];
    float best = __int_as_float(0x7f800000);
    int bc = 0;
    for (int c = 0; c < PQ_K; ++c) {
      float s = 0.f;
      for (int t = 0; t < dsub; ++t) {
        const float u = v[t] - scb[c * dsub + t];
        s = fmaf(u, u, s);
      }
      if (s < best) {
        best = s;
        bc = c;
      }
    }
    if (codes) codes[p * m + j] = (uint8_t)bc;
    if (sums) {
      for (int t = 0; t < dsub; ++t) atomicAdd(&sums[((size_t)j * PQ_K + bc) * dsub + t], v[t]);
      atomicAdd(&counts[(size_t)j * PQ_K + bc], 1);
    }
  }
}

__global__ void update_kernel(float* cb, const float* sums, const int* counts, int m, int dsub) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;  // (j, c)
  if (i >= m * PQ_K) return;
  const int cnt = counts[i];
  if (cnt > 0)
    for (int t = 0; t < dsub; ++t) cb[(size_t)i * dsub + t] = sums[(size_t)i * dsub + t] / (float)cnt;
}

__global__ void init_kernel(const float* x, int64_t n, int d, int m, int dsub, uint64_t seed, float* cb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;  // (j, c)
  if (i >= m * PQ_K) return;
  const int j = i / PQ_K, c = i % PQ_K;
  // c-th of PQ_K distinct points: stratified draw, one point per stratum
  const int64_t stratum = n / PQ_K > 0 ? n / PQ_K : 1;
  const uint64_t r = mix64(seed ^ ((uint64_t)(j + 1) * 0xD1B54A32D192ED03ULL) ^ ((uint64_t)c * 0x9E3779B97F4A7C15ULL));
  int64_t p = (int64_t)c * stratum + (int64_t)(r % (uint64_t)stratum);
  if (p >= n) p = n - 1;
  for (int t = 0; t < dsub; ++t) cb[(size_t)i * dsub + t] = x[p * d + (int64_t)j * dsub + t];
}

int check(cudaError_t e) {
  if (e != cudaSuccess) {
    set_cuda_error((int)e);
    return KANN_ECUDA;
  }
  return KANN_OK;
}

}  // namespace
}  // namespace kann

using namespace kann;

extern "C" size_t kann_pq_train_workspace_bytes(int d, int m) {
  if (m < 1 || d % m != 0) return 0;
  return (size_t)m * PQ_K * (d / m) * 4 + (size_t)m * PQ_K * 4;
}

extern "C" int kann_pq_train(const float* d_x, int64_t n, int d, int m, int iters, uint64_t seed, float* d_codebooks,
                             void* d_ws, size_t ws_bytes, void* stream) {
  if (!d_x || !d_codebooks || n < PQ_K || m < 1 || d % m != 0 || d / m > 16 || iters < 0) return KANN_EINVAL;
  if (!d_ws || ws_bytes < kann_pq_train_workspace_bytes(d, m)) return KANN_EINVAL;
  const int dsub = d / m;
  cudaStream_t s = (cudaStream_t)stream;
  float* sums = static_cast<float*>(d_ws);
  int* counts = reinterpret_cast<int*>(sums + (size_t)m * PQ_K * dsub);
  init_kernel<<<(m * PQ_K + 255) / 256, 256, 0, s>>>(d_x, n, d, m, dsub, seed, d_codebooks);
  int rc = check(cudaGetLastError());
  const dim3 grid((unsigned)((n + 255) / 256 < 64 ? (n + 255) / 256 : 64), m);
  for (int it = 0; it < iters && rc == KANN_OK; ++it) {
    rc = check(cudaMemsetAsync(d_ws, 0, kann_pq_train_workspace_bytes(d, m), s));
    if (rc) break;
    assign_kernel<<<grid, 256, PQ_K * dsub * 4, s>>>(d_x, n, d, m, dsub, d_codebooks, nullptr, sums, counts);
    update_kernel<<<(m * PQ_K + 255) / 256, 256, 0, s>>>(d_codebooks, sums, counts, m, dsub);
    rc = check(cudaGetLastError());
  }
  return rc;
}

extern "C" int kann_pq_encode(const float* d_x, int64_t n, int d, int m, const float* d_codebooks, uint8_t* d_codes,
                              void* stream) {
  if (!d_x || !d_codebooks || !d_codes || n < 0 || m < 1 || d % m != 0 || d / m > 16) return KANN_EINVAL;
  if (n == 0) return KANN_OK;
  const int dsub = d / m;
  const dim3 grid((unsigned)((n + 255) / 256 < 512 ? (n + 255) / 256 : 512), m);
  assign_kernel<<<grid, 256, PQ_K * dsub * 4, (cudaStream_t)stream>>>(d_x, n, d, m, dsub, d_codebooks, d_codes,
                                                                       nullptr, nullptr);
  return check(cudaGetLastError());
}
