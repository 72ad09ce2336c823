// kann_device.cuh -- device helpers shared by the search and exact-k-NN kernels:
// (distance, id) keys, warp sorting networks, global loads.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/kann.h"

namespace kann {

typedef unsigned long long u64;
constexpr unsigned FULL = 0xffffffffu;
constexpr u64 KEY_MAX = ~0ull;

// A result is ordered by (distance, id): distance first (NaN as +inf, -0 as
// +0), then id.  Both are packed into one unsigned 64-bit key whose integer
// order is that total order: the high word is the distance's bits mapped to
// an order-preserving unsigned code, the low word the id (< 2^31).
__device__ __forceinline__ uint32_t ordered_bits(float d) {
  uint32_t u = __float_as_uint(d);
  if ((u & 0x7fffffffu) > 0x7f800000u) u = 0x7f800000u;  // NaN -> +inf
  if ((u << 1) == 0u) u = 0u;                             // -0 -> +0
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ float key_dist(u64 key) {
  uint32_t b = (uint32_t)(key >> 32);
  uint32_t u = (b & 0x80000000u) ? (b & 0x7fffffffu) : ~b;
  return __uint_as_float(u);
}

__device__ __forceinline__ u64 make_key(float d, uint32_t id) { return ((u64)ordered_bits(d) << 32) | id; }

__device__ __forceinline__ u64 umin64(u64 a, u64 b) { return a < b ? a : b; }
__device__ __forceinline__ u64 umax64(u64 a, u64 b) { return a < b ? b : a; }

__device__ __forceinline__ u64 warp_min64(u64 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = umin64(v, __shfl_xor_sync(FULL, v, o));
  return v;
}

// Bitonic sort of one key per lane, ascending by lane.
__device__ __forceinline__ u64 warp_sort32(u64 v, int lane) {
#pragma unroll
  for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      u64 w = __shfl_xor_sync(FULL, v, j);
      bool up = (lane & k) == 0;
      bool lower = (lane & j) == 0;
      v = (lower == up) ? umin64(v, w) : umax64(v, w);
    }
  }
  return v;
}

// A bitonic sequence across the warp -> ascending.
__device__ __forceinline__ u64 warp_bitonic_merge32(u64 v, int lane) {
#pragma unroll
  for (int j = 16; j > 0; j >>= 1) {
    u64 w = __shfl_xor_sync(FULL, v, j);
    v = ((lane & j) == 0) ? umin64(v, w) : umax64(v, w);
  }
  return v;
}

// Sort 64 keys held as a (elements 0..31 by lane) and b (32..63).
__device__ __forceinline__ void warp_sort64(u64& a, u64& b, int lane) {
  a = warp_sort32(a, lane);
  b = warp_sort32(b, lane);
  u64 br = __shfl_sync(FULL, b, 31 - lane);
  u64 lo = umin64(a, br), hi = umax64(a, br);
  a = warp_bitonic_merge32(lo, lane);
  b = warp_bitonic_merge32(hi, lane);
}

// Ascending bitonic sort of P (a power of two) keys in shared memory by one warp.
__device__ __forceinline__ void warp_smem_sort(u64* A, int P, int lane) {
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = lane; i < P; i += 32) {
        int l = i ^ j;
        if (l > i) {
          u64 x = A[i], y = A[l];
          bool up = (i & k) == 0;
          if ((x > y) == up) { A[i] = y; A[l] = x; }
        }
      }
      __syncwarp();
    }
  }
}

// Ascending sort of A[0..n), any n, by one warp.  A bitonic network in the
// form whose comparators always put the smaller key at the lower index (each
// merge stage of block size k starts by comparing i with its mirror
// i ^ (k - 1), then halves as usual).  Positions n .. P - 1 (P the next power
// of two) act as +inf padding: a comparator never moves the larger key to
// the lower index, so one that reaches past n would leave both keys in place
// and is skipped -- nothing beyond A[n) is read or written.
__device__ __forceinline__ void warp_smem_sort_n(u64* A, int n, int lane) {
  int P = 1;
  while (P < n) P <<= 1;
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      const int flip = (j == (k >> 1)) ? (k - 1) : j;
      for (int i = lane; i < n; i += 32) {
        const int l = i ^ flip;
        if (l > i && l < n) {
          const u64 x = A[i], y = A[l];
          if (x > y) {
            A[i] = y;
            A[l] = x;
          }
        }
      }
      __syncwarp();
    }
  }
}

// Packed FP32 pair arithmetic (the sm_100 f32x2 forms: each half is rounded
// exactly as the scalar instruction would round it).  A distance kept as two
// partial sums, a0 over the even and a1 over the odd elements of a lane's
// chunks, costs half the accumulation instructions.
//   acc_sq2:      (a0, a1) += (t0 * t0, t1 * t1)
//   acc_diff_sq2: t = (q0 - x0, q1 - x1); (a0, a1) += (t0 * t0, t1 * t1)
//   acc_mul2:     (a0, a1) += (q0 * x0, q1 * x1)
__device__ __forceinline__ void acc_sq2(float& a0, float& a1, float t0, float t1) {
  asm("{.reg .b64 A, T;\n\tmov.b64 A, {%0, %1};\n\tmov.b64 T, {%2, %3};\n\t"
      "fma.rn.f32x2 A, T, T, A;\n\tmov.b64 {%0, %1}, A;}"
      : "+f"(a0), "+f"(a1)
      : "f"(t0), "f"(t1));
}

__device__ __forceinline__ void acc_diff_sq2(float& a0, float& a1, float q0, float q1, float x0, float x1) {
  asm("{.reg .b64 A, Q, X, T;\n\tmov.b64 A, {%0, %1};\n\tmov.b64 Q, {%2, %3};\n\tmov.b64 X, {%4, %5};\n\t"
      "sub.rn.f32x2 T, Q, X;\n\tfma.rn.f32x2 A, T, T, A;\n\tmov.b64 {%0, %1}, A;}"
      : "+f"(a0), "+f"(a1)
      : "f"(q0), "f"(q1), "f"(x0), "f"(x1));
}

__device__ __forceinline__ void acc_mul2(float& a0, float& a1, float q0, float q1, float x0, float x1) {
  asm("{.reg .b64 A, Q, X;\n\tmov.b64 A, {%0, %1};\n\tmov.b64 Q, {%2, %3};\n\tmov.b64 X, {%4, %5};\n\t"
      "fma.rn.f32x2 A, Q, X, A;\n\tmov.b64 {%0, %1}, A;}"
      : "+f"(a0), "+f"(a1)
      : "f"(q0), "f"(q1), "f"(x0), "f"(x1));
}

// 16-byte read-only global load that does not allocate in L1 (random rows).
__device__ __forceinline__ uint4 ldg_stream16(const void* p) {
  uint4 r;
  asm("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
      : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
      : "l"(p));
  return r;
}

// Storage formats: elements per 16-byte chunk and their FP32 values.
template <int DT>
struct Fmt;

template <>
struct Fmt<KANN_F32> {
  static constexpr int EPC = 4;
  __device__ __forceinline__ static void unpack(const uint4& v, float* o) {
    o[0] = __uint_as_float(v.x);
    o[1] = __uint_as_float(v.y);
    o[2] = __uint_as_float(v.z);
    o[3] = __uint_as_float(v.w);
  }
};

template <>
struct Fmt<KANN_F16> {
  static constexpr int EPC = 8;
  __device__ __forceinline__ static void unpack(const uint4& v, float* o) {
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      __half2_raw r;
      r.x = (unsigned short)(w[i] & 0xffffu);
      r.y = (unsigned short)(w[i] >> 16);
      float2 f = __half22float2(__half2(r));
      o[2 * i] = f.x;
      o[2 * i + 1] = f.y;
    }
  }
};

template <>
struct Fmt<KANN_BF16> {
  static constexpr int EPC = 8;
  __device__ __forceinline__ static void unpack(const uint4& v, float* o) {
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      o[2 * i] = __uint_as_float(w[i] << 16);
      o[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
    }
  }
};

template <>
struct Fmt<KANN_E4M3> {
  static constexpr int EPC = 16;
  __device__ __forceinline__ static void unpack(const uint4& v, float* o) {
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        __nv_fp8x2_storage_t pair = (__nv_fp8x2_storage_t)((w[i] >> (16 * h)) & 0xffffu);
        __half2_raw r = __nv_cvt_fp8x2_to_halfraw2(pair, __NV_E4M3);
        float2 f = __half22float2(__half2(r));
        o[4 * i + 2 * h] = f.x;
        o[4 * i + 2 * h + 1] = f.y;
      }
    }
  }
};

}  // namespace kann
