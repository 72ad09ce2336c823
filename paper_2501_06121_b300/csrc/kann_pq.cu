// kann_pq.cu -- Product Quantization training and encoding on the GPU (the
// quantizer of kANNolo Sec. 2, citing Jegou et al.): per subspace j of dsub
// dimensions, k-means with ksub = 256 centroids, then every vector's code
// byte j = its nearest centroid of subspace j (ties to the lowest index).
//
// This is index preparation, not the search path.  Training takes the steps
// of the reading the oracle states, in FP64 on the CUDA cores:
//   * k-means++ seeding: the first centroid is training row
//     floor(u_0 * n), u_c = the counter-based SplitMix64 uniform keyed by
//     (seed ^ (j + 1) * 0xD1B54A32D192ED03, c); centroid c is the first row
//     i whose running sum of D^2 (squared distance to the nearest centroid
//     so far) reaches u_c * sum D^2 (or row floor(u_c * n) when every D^2 is
//     0);
//   * Lloyd iterations: every row to its nearest centroid (strictly smaller
//     distance wins, so ties go to the lowest index), then every centroid to
//     the mean of its rows; a centroid with no rows is moved to the row
//     farthest from its centroid (the first such row), whose distance then
//     counts as 0 for the next empty centroid.
// Distances are sum_t (x_t - c_t)^2 in FP64, each operation rounded on its
// own (no fused multiply-add), as the oracle computes them.  Sums are exact
// on integer data, where the codebooks therefore equal the oracle's bit for
// bit; on other data the parallel sums may round differently.  A subspace's
// distance product has only dsub (<= 16) terms per pair, far too short for
// a tensor-core contraction, and the decisions must be the oracle's: FP64
// CUDA cores serve both.
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

// The counter-based uniform in (0, 1]: one SplitMix64 step from state
// key ^ i * 0x9E3779B97F4A7C15, its top 53 bits plus one over 2^53.
__device__ __forceinline__ double uniform53(uint64_t key, uint64_t i) {
  const uint64_t u = mix64(key ^ (i * 0x9E3779B97F4A7C15ULL)) >> 11;
  return ((double)u + 1.0) / 9007199254740992.0;
}

__device__ __forceinline__ double sqdist64(const float* x, const double* c, int dsub) {
  double s = 0.0;
  for (int t = 0; t < dsub; ++t) {
    const double u = __dsub_rn((double)x[t], c[t]);
    s = __dadd_rn(s, __dmul_rn(u, u));
  }
  return s;
}

// Exclusive scan of one double per thread over a block of 1024 threads;
// returns the exclusive prefix, *total gets the block's sum.
__device__ double block_exscan(double v, double* smem, double* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  double incl = v;
  for (int o = 1; o < 32; o <<= 1) {
    const double y = __shfl_up_sync(FULL, incl, o);
    if (lane >= o) incl = __dadd_rn(incl, y);
  }
  if (lane == 31) smem[w] = incl;
  __syncthreads();
  if (w == 0) {
    double t = smem[lane], ti = t;
    for (int o = 1; o < 32; o <<= 1) {
      const double y = __shfl_up_sync(FULL, ti, o);
      if (lane >= o) ti = __dadd_rn(ti, y);
    }
    smem[32 + lane] = __dsub_rn(ti, t);  // exclusive warp prefix
    if (lane == 31) smem[64] = ti;
  }
  __syncthreads();
  const double ex = __dadd_rn(smem[32 + w], __dsub_rn(incl, v));
  *total = smem[64];
  __syncthreads();
  return ex;
}

// k-means++ seeding, one CTA of 1024 threads per subspace; thread t owns
// training rows [t * chunk, (t + 1) * chunk).
__global__ void __launch_bounds__(1024) pp_init_kernel(const float* __restrict__ x, int64_t n, int d, int dsub,
                                                       uint64_t seed, double* C, double* D2) {
  __shared__ double red[72];
  __shared__ double cen[16];
  __shared__ long long pick_s;
  const int j = blockIdx.x, tid = threadIdx.x;
  const uint64_t key = seed ^ ((uint64_t)(j + 1) * 0xD1B54A32D192ED03ULL);
  const int64_t chunk = (n + 1023) / 1024, i0 = min(n, (int64_t)tid * chunk), i1 = min(n, i0 + chunk);
  double* d2 = D2 + (size_t)j * n;
  double* Cj = C + (size_t)j * PQ_K * dsub;
  if (tid == 0) {
    const double f = floor(uniform53(key, 0) * (double)n);
    pick_s = (long long)(f < (double)(n - 1) ? f : (double)(n - 1));
  }
  __syncthreads();
  // centroid 0
  if (tid < dsub) cen[tid] = (double)x[(size_t)pick_s * d + (size_t)j * dsub + tid];
  __syncthreads();
  if (tid < dsub) Cj[tid] = cen[tid];
  double csum = 0.0;
  for (int64_t i = i0; i < i1; ++i) {
    const double v = sqdist64(x + (size_t)i * d + (size_t)j * dsub, cen, dsub);
    d2[i] = v;
    csum = __dadd_rn(csum, v);
  }
  for (int c = 1; c < PQ_K; ++c) {
    double tot;
    const double ex = block_exscan(csum, red, &tot);
    if (tid == 0) pick_s = n - 1;
    __syncthreads();
    if (tot > 0.0) {
      const double r = __dmul_rn(uniform53(key, (uint64_t)c), tot);
      if (ex < r && __dadd_rn(ex, csum) >= r) {
        double acc = ex;
        for (int64_t i = i0; i < i1; ++i) {
          acc = __dadd_rn(acc, d2[i]);
          if (acc >= r) {
            pick_s = i;
            break;
          }
        }
      }
    } else if (tid == 0) {
      const double f = floor(uniform53(key, (uint64_t)c) * (double)n);
      pick_s = (long long)(f < (double)(n - 1) ? f : (double)(n - 1));
    }
    __syncthreads();
    if (tid < dsub) {
      cen[tid] = (double)x[(size_t)pick_s * d + (size_t)j * dsub + tid];
      Cj[(size_t)c * dsub + tid] = cen[tid];
    }
    __syncthreads();
    csum = 0.0;
    for (int64_t i = i0; i < i1; ++i) {
      const double v = fmin(d2[i], sqdist64(x + (size_t)i * d + (size_t)j * dsub, cen, dsub));
      d2[i] = v;
      csum = __dadd_rn(csum, v);
    }
  }
}

// Lloyd assignment in FP64: nearest centroid (strictly smaller wins), its
// distance into D2, and the row's coordinates added to its centroid's sums.
__global__ void assign64_kernel(const float* __restrict__ x, int64_t n, int d, int dsub, const double* C, double* D2,
                                double* sums, int* counts) {
  extern __shared__ double sc64[];  // [256][dsub]
  const int j = blockIdx.y;
  for (int i = threadIdx.x; i < PQ_K * dsub; i += blockDim.x) sc64[i] = C[(size_t)j * PQ_K * dsub + i];
  __syncthreads();
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const float* xp = x + (size_t)p * d + (size_t)j * dsub;
    double best = __longlong_as_double(0x7ff0000000000000LL);
    int bc = 0;
    for (int c = 0; c < PQ_K; ++c) {
      const double s = sqdist64(xp, sc64 + c * dsub, dsub);
      if (s < best) {
        best = s;
        bc = c;
      }
    }
    D2[(size_t)j * n + p] = best;
    for (int t = 0; t < dsub; ++t) atomicAdd(&sums[((size_t)j * PQ_K + bc) * dsub + t], (double)xp[t]);
    atomicAdd(&counts[(size_t)j * PQ_K + bc], 1);
  }
}

// Centroids to their means; then, in centroid order, each empty centroid to
// the farthest row (the first of the farthest), whose D2 becomes 0.  One CTA
// of 1024 threads per subspace.
__global__ void __launch_bounds__(1024) update64_kernel(const float* __restrict__ x, int64_t n, int d, int dsub,
                                                        double* C, double* D2, const double* sums,
                                                        const int* counts) {
  __shared__ double bv[32];
  __shared__ long long bi[32];
  const int j = blockIdx.x, tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  double* Cj = C + (size_t)j * PQ_K * dsub;
  double* d2 = D2 + (size_t)j * n;
  const int* cnt = counts + (size_t)j * PQ_K;
  for (int c = tid; c < PQ_K; c += blockDim.x)
    if (cnt[c] > 0)
      for (int t = 0; t < dsub; ++t)
        Cj[(size_t)c * dsub + t] = __ddiv_rn(sums[((size_t)j * PQ_K + c) * dsub + t], (double)cnt[c]);
  __syncthreads();
  for (int c = 0; c < PQ_K; ++c) {
    if (cnt[c] > 0) continue;  // uniform across the block
    double v = -1.0;
    long long vi = 0;
    for (int64_t i = tid; i < n; i += blockDim.x)
      if (d2[i] > v) {
        v = d2[i];
        vi = i;
      }
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(FULL, v, o);
      const long long oi = __shfl_xor_sync(FULL, vi, o);
      if (ov > v || (ov == v && oi < vi)) {
        v = ov;
        vi = oi;
      }
    }
    if (lane == 0) {
      bv[w] = v;
      bi[w] = vi;
    }
    __syncthreads();
    if (tid == 0) {
      double b = bv[0];
      long long bix = bi[0];
      for (int k = 1; k < 32; ++k)
        if (bv[k] > b || (bv[k] == b && bi[k] < bix)) {
          b = bv[k];
          bix = bi[k];
        }
      d2[bix] = 0.0;
      for (int t = 0; t < dsub; ++t) Cj[(size_t)c * dsub + t] = (double)x[(size_t)bix * d + (size_t)j * dsub + t];
    }
    __syncthreads();
  }
}

__global__ void round_codebooks_kernel(const double* C, int64_t total, float* cb) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < total) cb[i] = (float)C[i];
}

struct PQTrainPlan {
  size_t d2_off, c_off, sum_off, cnt_off, total;
};

PQTrainPlan pq_train_plan(int64_t n, int d, int m) {
  const int dsub = d / m;
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  PQTrainPlan p;
  size_t o = 0;
  p.d2_off = o;
  o = al(o + (size_t)m * n * 8);
  p.c_off = o;
  o = al(o + (size_t)m * PQ_K * dsub * 8);
  p.sum_off = o;
  o = al(o + (size_t)m * PQ_K * dsub * 8);
  p.cnt_off = o;
  o = al(o + (size_t)m * PQ_K * 4);
  p.total = o;
  return p;
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

extern "C" size_t kann_pq_train_workspace_bytes(int64_t n, int d, int m) {
  if (n < 1 || m < 1 || d % m != 0) return 0;
  return pq_train_plan(n, d, m).total;
}

extern "C" int kann_pq_train(const float* d_x, int64_t n, int d, int m, int iters, uint64_t seed, float* d_codebooks,
                             void* d_ws, size_t ws_bytes, void* stream) {
  if (!d_x || !d_codebooks || n < PQ_K || m < 1 || d % m != 0 || d / m > 16 || iters < 0) return KANN_EINVAL;
  const PQTrainPlan p = pq_train_plan(n, d, m);
  if (!d_ws || ws_bytes < p.total) return KANN_EINVAL;
  const int dsub = d / m;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char* ws = static_cast<unsigned char*>(d_ws);
  double* D2 = reinterpret_cast<double*>(ws + p.d2_off);
  double* C = reinterpret_cast<double*>(ws + p.c_off);
  double* sums = reinterpret_cast<double*>(ws + p.sum_off);
  int* counts = reinterpret_cast<int*>(ws + p.cnt_off);
  pp_init_kernel<<<m, 1024, 0, s>>>(d_x, n, d, dsub, seed, C, D2);
  int rc = check(cudaGetLastError());
  const dim3 grid((unsigned)((n + 255) / 256 < 256 ? (n + 255) / 256 : 256), m);
  const size_t csz = (size_t)m * PQ_K * dsub * 8, nsz = (size_t)m * PQ_K * 4;
  for (int it = 0; it < iters && rc == KANN_OK; ++it) {
    rc = check(cudaMemsetAsync(sums, 0, csz, s));
    if (rc == KANN_OK) rc = check(cudaMemsetAsync(counts, 0, nsz, s));
    if (rc) break;
    assign64_kernel<<<grid, 256, PQ_K * dsub * 8, s>>>(d_x, n, d, dsub, C, D2, sums, counts);
    update64_kernel<<<m, 1024, 0, s>>>(d_x, n, d, dsub, C, D2, sums, counts);
    rc = check(cudaGetLastError());
  }
  if (rc == KANN_OK) {
    const int64_t total = (int64_t)m * PQ_K * dsub;
    round_codebooks_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(C, total, d_codebooks);
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
