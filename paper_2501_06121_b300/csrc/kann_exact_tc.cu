// kann_exact_tc.cu -- exact k-NN on the 5th-generation tensor cores (tcgen05).
//
// The ground truth for recall (the paper's k-NN problem, Sec. 1) over BF16 or
// FP16 inputs: S = Q X^T accumulates in FP32 in tensor memory, the epilogue
// turns a row of S into distances (L2: ||x||^2 - 2 q.x + ||q||^2, IP: -q.x)
// and keeps each query's k best (distance, id) pairs in registers; the scores
// are never written to HBM.
//
// One persistent CTA per SM walks work items (two tiles of 128 queries x one
// split of the base: both query blocks use each staged base tile, which halves
// the base traffic from L2 per score).  Roles inside a CTA (320 threads):
//   warp 0      TMA producer: per base tile of 128 rows and per 64-element K
//               chunk, loads the base chunk (128 x 64), 128-byte swizzled,
//               into a stage ring; for d <= 256 (when shared memory allows)
//               the item's two 128 x d query blocks are loaded once per item
//               and stay resident (the MMAs of every tile read them),
//               otherwise each stage carries their two query chunks
//               (2 x 128 x 64) too;
//   warp 1      allocates 512 TMEM columns (two buffers, each holding one
//               128 x 128 FP32 accumulator per query block) and issues
//               tcgen05.mma (M=128, N=128, K=16) from one lane, one per query
//               block and K step on the same base chunk; tcgen05.commit frees
//               a ring stage when its MMAs are done and signals a full buffer;
//   warps 2..9  two epilogue warpgroups: thread r of group g owns row r of
//               query block g (TMEM lane r) over the 128 columns of each tile,
//               reads its scores with tcgen05.ld into registers, filters them
//               against its current k-th distance and inserts the survivors
//               into its own top-k list in shared memory.
// The scans of one query (its S split lists, on different CTAs) share an
// upper bound on its k-th score in global memory: it starts
// from tc_threshold_kernel's bound (a strided sample of the base scored on the
// CUDA cores), every list that is full lowers it (atomicMin) to just above its
// own k-th score, and each scan filters against the smaller of that bound and
// its own k-th.  Any list's k-th bounds the union's from above, so nothing
// that belongs in the top k is dropped, and the insert path stays rare.
// Accumulators are double-buffered so the epilogue of tile t overlaps the
// MMAs of tile t+1.  Every mbarrier wait is bounded by a %globaltimer
// deadline; on expiry the CTA raises an error flag and all roles wind down,
// and the merge pass then reports id -1 for every query.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "kann_device.cuh"
#include "kann_internal.h"

namespace kann {
namespace {

constexpr int TC_M = 128;       // queries per work item (TMEM lanes)
constexpr int TC_N = 128;       // base rows per tile (accumulator columns)
constexpr int TC_QB = 2;        // query blocks of TC_M rows per work item (share each base tile)
constexpr int TC_K = 64;        // K elements per stage: one 128-byte swizzle row
constexpr int TC_MAX_STAGES = 6;
constexpr int TC_QRES_MAX_KCHUNKS = 4;  // resident query block up to d = 256
constexpr int A_BYTES = TC_M * TC_K * 2;
constexpr int B_BYTES = TC_N * TC_K * 2;
constexpr int STAGE_BYTES = TC_QB * A_BYTES + B_BYTES;
constexpr int TC_EPI_WARPS = 8;     // two warpgroups, one per half of a tile's columns
constexpr int TC_THREADS = 64 + 32 * TC_EPI_WARPS;
constexpr uint32_t TMEM_COLS = 512;
constexpr int TC_KMAX = 32;     // largest k of the tensor-core path (top-k lists in shared memory)
constexpr unsigned long long WAIT_NS = 2000000000ull;  // 2 s per wait

struct TcArgs {
  int nq;
  int64_t nb;
  int d, metric, k, S, kchunks;
  int64_t per;          // base rows per split (a multiple of TC_N)
  int n_items;
  int stages;           // ring depth (by shared memory left for the query block and the top-k lists)
  int qres;             // 1: the item's query block is resident, stages hold base chunks only
  int stage_bytes;      // B_BYTES (qres) or A_BYTES + B_BYTES
  int qbytes;           // kchunks * A_BYTES (qres) or 0
  uint32_t idesc;
  const float* xnorm;   // [nb]
  const float* qnorm;   // [nq]
  unsigned* thr;        // [nq] shared upper bound on each query's k-th score (ordered_bits code)
  u64* out;             // [nq][S][k] partial lists
  int* err;
};

// ---- PTX wrappers ----------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// Wait for the phase of `bar` with the given parity; false if the deadline
// passed or another role raised the error flag.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* err) {
  unsigned long long t0 = 0;
  for (uint32_t it = 0;; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if ((it & 255u) == 255u) {
      if (*(volatile int*)err) return false;
      const unsigned long long t = gtimer();
      if (t0 == 0) t0 = t;
      else if (t - t0 > WAIT_NS) {
        atomicOr(err, 1);
        return false;
      }
    }
  }
}

// The same wait taken by a whole warp with one outcome for every lane.
__device__ __forceinline__ bool mbar_wait_warp(uint32_t bar, uint32_t parity, int* err, int lane) {
  unsigned long long t0 = 0;
  for (uint32_t it = 0;; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (__all_sync(FULL, ok)) return true;
    if ((it & 255u) == 255u) {
      int stop = 0;
      if (lane == 0) {
        if (*(volatile int*)err) stop = 1;
        const unsigned long long t = gtimer();
        if (t0 == 0) t0 = t;
        else if (t - t0 > WAIT_NS) {
          atomicOr(err, 1);
          stop = 1;
        }
      }
      if (__shfl_sync(FULL, stop, 0)) return false;
    }
  }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(dst),
      "l"(map), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor of a K-major operand staged with the
// 128-byte swizzle: rows of 128 bytes, 8-row groups 1024 bytes apart.
__device__ __forceinline__ u64 smem_desc(uint32_t saddr) {
  u64 d = 0;
  d |= (u64)((saddr & 0x3FFFFu) >> 4);   // start address
  d |= (u64)(16u >> 4) << 16;            // leading byte offset (unused with this swizzle)
  d |= (u64)(1024u >> 4) << 32;          // stride byte offset: next 8-row group
  d |= (u64)1 << 46;                     // descriptor version for tcgen05
  d |= (u64)2 << 61;                     // 128-byte swizzle
  return d;
}

__device__ __forceinline__ void tc_mma(uint32_t dtmem, u64 adesc, u64 bdesc, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// 64 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tc_ld64(uint32_t taddr, float* v) {
  uint32_t r[64];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x64.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,"
      "%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,"
      "%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%64];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]),
        "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]),
        "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]),
        "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]),
        "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 64; ++i) v[i] = __uint_as_float(r[i]);
}

// (x0, x1) = (m x0 + c0, m x1 + c1) in one packed FP32 FMA (each lane rounds
// as fmaf does).
__device__ __forceinline__ void fma2(float& x0, float& x1, float m, float c0, float c1) {
  asm("{.reg .b64 A, C, M, R;\n\tmov.b64 A, {%0, %1};\n\tmov.b64 C, {%3, %4};\n\tmov.b64 M, {%2, %2};\n\t"
      "fma.rn.f32x2 R, A, M, C;\n\tmov.b64 {%0, %1}, R;}"
      : "+f"(x0), "+f"(x1)
      : "f"(m), "f"(c0), "f"(c1));
}

// Three-input minimum (the same value as fminf(fminf(a, b), c)).
__device__ __forceinline__ float min3(float a, float b, float c) {
  float r;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}

// Inverse of ordered_bits.
__device__ __forceinline__ float from_ordered(unsigned b) {
  return __uint_as_float((b & 0x80000000u) ? (b & 0x7fffffffu) : ~b);
}

// A thread's top-k list lives in shared memory (its own k slots); the
// registers hold the current worst entry's distance and slot.
// Scan state of one thread: its own list's k-th score and slot, and the
// query's shared bound as last seen.
struct ScanState {
  float thr;    // own list's k-th score (+inf until the list is full)
  int slot;     // slot holding it (the heap root)
  float thr_g;  // shared bound on the query's k-th score
};

// A thread's list is a max-heap by (d, id) in its k slots (root = the current
// k-th, empty slots (+inf, -1)): put (dist, col) in place of the root and sift
// it down, and when the list is full publish just above its new k-th as the
// query's bound.
__device__ __noinline__ ScanState topk_insert(float* ld, int* li, int k, ScanState w, float dist, int col,
                                              unsigned* thr_q) {
  int i = 0;
  for (;;) {
    int c = 2 * i + 1;
    if (c >= k) break;
    float cd = ld[c];
    int cx = li[c];
    if (c + 1 < k) {
      const float d2 = ld[c + 1];
      const int x2 = li[c + 1];
      if (d2 > cd || (d2 == cd && x2 > cx)) {
        ++c;
        cd = d2;
        cx = x2;
      }
    }
    if (!(cd > dist || (cd == dist && cx > col))) break;
    ld[i] = cd;
    li[i] = cx;
    i = c;
  }
  ld[i] = dist;
  li[i] = col;
  const float wd = ld[0];
  w.thr = wd;
  w.slot = 0;
  if (wd != __int_as_float(0x7f800000)) {
    const float up = nextafterf(wd, __int_as_float(0x7f800000));
    if (up < w.thr_g) {
      w.thr_g = up;
      atomicMin(thr_q, ordered_bits(up));
    }
  }
  return w;
}

// ---- the kernel ------------------------------------------------------------
__global__ void __launch_bounds__(TC_THREADS, 1)
    exact_tc_kernel(const __grid_constant__ CUtensorMap tmQ, const __grid_constant__ CUtensorMap tmX, const TcArgs a) {
  extern __shared__ unsigned char smem_raw[];
  // 1024-byte alignment for the swizzled stages
  unsigned char* smem = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int NS = a.stages;
  unsigned char* qblock = smem;                 // resident query block (qres)
  unsigned char* stage_base = smem + a.qbytes;
  u64* bars = reinterpret_cast<u64*>(stage_base + NS * a.stage_bytes);
  // bars: full[NS], empty[NS], tfull[2], tempty[2], qfull, qempty
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * TC_MAX_STAGES + 6);
  float* xn_s = reinterpret_cast<float*>(tmem_slot + 4);        // [8][128] per-warp tile norms
  float* list_d = xn_s + TC_EPI_WARPS * 128;                    // [2][128][k] top-k distances
  int* list_i = reinterpret_cast<int*>(list_d + 2 * TC_M * a.k); // [2][128][k] top-k ids

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + TC_MAX_STAGES);
  const uint32_t tfull0 = smem_u32(bars + 2 * TC_MAX_STAGES), tempty0 = smem_u32(bars + 2 * TC_MAX_STAGES + 2);
  const uint32_t qfull0 = smem_u32(bars + 2 * TC_MAX_STAGES + 4), qempty0 = smem_u32(bars + 2 * TC_MAX_STAGES + 5);

  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull0 + 8 * b, 1);
      mbar_init(tempty0 + 8 * b, TC_EPI_WARPS);
    }
    mbar_init(qfull0, 1);
    mbar_init(qempty0, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      uint32_t it = 0, iq = 0;
      bool ok = true;
      for (int item = blockIdx.x; item < a.n_items && ok; item += gridDim.x) {
        const int q0 = (item / a.S) * (TC_M * TC_QB);
        const int64_t b_begin = (int64_t)(item % a.S) * a.per;
        const int64_t b_end = b_begin + a.per < a.nb ? b_begin + a.per : a.nb;
        if (a.qres) {
          // the previous item's MMAs must be done with the resident block
          ok = mbar_wait(qempty0, (iq & 1u) ^ 1u, a.err);
          if (!ok) break;
          mbar_expect_tx(qfull0, (uint32_t)a.qbytes);
          for (int qb = 0; qb < TC_QB; ++qb)
            for (int kc = 0; kc < a.kchunks; ++kc)
              tma_load_2d(smem_u32(qblock + (qb * a.kchunks + kc) * A_BYTES), &tmQ, kc * TC_K, q0 + qb * TC_M, qfull0);
          ++iq;
        }
        for (int64_t b0 = b_begin; b0 < b_end && ok; b0 += TC_N) {
          for (int kc = 0; kc < a.kchunks && ok; ++kc, ++it) {
            const uint32_t s = it % NS, ph = (it / NS) & 1u;
            ok = mbar_wait(empty0 + 8 * s, ph ^ 1u, a.err);
            if (!ok) break;
            const uint32_t sa = smem_u32(stage_base + s * a.stage_bytes);
            mbar_expect_tx(full0 + 8 * s, (uint32_t)a.stage_bytes);
            if (a.qres) {
              tma_load_2d(sa, &tmX, kc * TC_K, (int)b0, full0 + 8 * s);
            } else {
              for (int qb = 0; qb < TC_QB; ++qb)
                tma_load_2d(sa + qb * A_BYTES, &tmQ, kc * TC_K, q0 + qb * TC_M, full0 + 8 * s);
              tma_load_2d(sa + TC_QB * A_BYTES, &tmX, kc * TC_K, (int)b0, full0 + 8 * s);
            }
          }
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer (one lane) ----------------
    if (lane == 0) {
      uint32_t it = 0, t = 0, iq = 0;
      bool ok = true;
      for (int item = blockIdx.x; item < a.n_items && ok; item += gridDim.x) {
        const int64_t b_begin = (int64_t)(item % a.S) * a.per;
        const int64_t b_end = b_begin + a.per < a.nb ? b_begin + a.per : a.nb;
        if (a.qres) {
          ok = mbar_wait(qfull0, iq & 1u, a.err);
          if (!ok) break;
          tc_fence_after();
        }
        for (int64_t b0 = b_begin; b0 < b_end && ok; b0 += TC_N, ++t) {
          const uint32_t buf = t & 1u, use = t >> 1;
          ok = mbar_wait(tempty0 + 8 * buf, (use & 1u) ^ 1u, a.err);
          if (!ok) break;
          tc_fence_after();
          const uint32_t dt = tmem + buf * (TC_QB * TC_N);
          for (int kc = 0; kc < a.kchunks; ++kc, ++it) {
            const uint32_t s = it % NS, ph = (it / NS) & 1u;
            ok = mbar_wait(full0 + 8 * s, ph, a.err);
            if (!ok) break;
            tc_fence_after();
            const uint32_t sa = smem_u32(stage_base + s * a.stage_bytes);
            const uint32_t xa = a.qres ? sa : sa + TC_QB * A_BYTES;
#pragma unroll
            for (int qb = 0; qb < TC_QB; ++qb) {
              const uint32_t qa = a.qres ? smem_u32(qblock + (qb * a.kchunks + kc) * A_BYTES) : sa + qb * A_BYTES;
#pragma unroll
              for (int kk = 0; kk < TC_K / 16; ++kk)
                tc_mma(dt + qb * TC_N, smem_desc(qa + kk * 32), smem_desc(xa + kk * 32), a.idesc, (kc | kk) != 0);
            }
            tc_commit(empty0 + 8 * s);
          }
          if (!ok) break;
          tc_commit(tfull0 + 8 * buf);
        }
        if (a.qres && ok) {
          tc_commit(qempty0);  // the resident block is free once this item's MMAs are done
          ++iq;
        }
      }
    }
  } else {
    // ---------------- epilogue warpgroups ----------------
    const int quarter = warp & 3;            // TMEM lanes 32*quarter .. +31
    const int row = quarter * 32 + lane;
    const int grp = (warp - 2) >> 2;         // query block of the item
    float* xw = xn_s + (warp - 2) * 128;     // this warp's copy of its columns' norms
    float* ld = list_d + ((size_t)grp * TC_M + row) * a.k;
    int* li = list_i + ((size_t)grp * TC_M + row) * a.k;
    uint32_t t = 0;
    bool ok = true;
    for (int item = blockIdx.x; item < a.n_items && ok; item += gridDim.x) {
      const int q = (item / a.S) * (TC_M * TC_QB) + grp * TC_M + row;
      const int split = item % a.S;
      const int64_t b_begin = (int64_t)split * a.per;
      const int64_t b_end = b_begin + a.per < a.nb ? b_begin + a.per : a.nb;
      for (int j = 0; j < a.k; ++j) {
        ld[j] = __int_as_float(0x7f800000);
        li[j] = -1;
      }
      // rows past nq (the zero-filled tail of the last query tile) never
      // insert, so they never publish a bound
      ScanState w{q < a.nq ? __int_as_float(0x7f800000) : -__int_as_float(0x7f800000), 0,
                  q < a.nq ? from_ordered(__ldcg(a.thr + q)) : __int_as_float(0x7f800000)};
      unsigned* thr_q = a.thr + (q < a.nq ? q : 0);
      for (int64_t b0 = b_begin; b0 < b_end; b0 += TC_N, ++t) {
        const uint32_t buf = t & 1u, use = t >> 1;
        const int64_t c_base = b0;
        const unsigned thr_code = q < a.nq ? __ldcg(a.thr + q) : 0xff800000u;  // other lists' progress (+inf)
        if (a.metric == KANN_L2)
          for (int j = lane; j < 128; j += 32) xw[j] = (c_base + j < b_end) ? __ldg(a.xnorm + c_base + j) : 0.f;
        __syncwarp();
        ok = mbar_wait_warp(tfull0 + 8 * buf, use & 1u, a.err, lane);
        if (!ok) break;
        tc_fence_after();
#pragma unroll 1
        for (int c0 = 0; c0 < 128; c0 += 64) {
          float v[64];
          tc_ld64(tmem + ((uint32_t)(quarter * 32) << 16) + buf * (TC_QB * TC_N) + grp * TC_N + c0, v);
          const int64_t cb = c_base + c0;
          // pass 1: scores and the minimum of each group of 16 columns
          float mn[4];
#pragma unroll
          for (int g = 0; g < 4; ++g) {
            mn[g] = __int_as_float(0x7f800000);
#pragma unroll
            for (int j = 16 * g; j < 16 * g + 16; j += 4) {
              if (a.metric == KANN_L2) {
                const float4 n4 = *reinterpret_cast<const float4*>(xw + c0 + j);
                fma2(v[j], v[j + 1], -2.f, n4.x, n4.y);
                fma2(v[j + 2], v[j + 3], -2.f, n4.z, n4.w);
              } else {
                v[j] = -v[j];
                v[j + 1] = -v[j + 1];
                v[j + 2] = -v[j + 2];
                v[j + 3] = -v[j + 3];
              }
              mn[g] = min3(min3(mn[g], v[j], v[j + 1]), v[j + 2], v[j + 3]);
            }
          }
          // pass 2 (rare: a score beats the current bound), per group of 16
          // columns: insert in column order; columns arrive in increasing id
          // order, so a tie with this list's own k-th never enters
          w.thr_g = fminf(w.thr_g, from_ordered(thr_code));
          float eff = fminf(w.thr, w.thr_g);
          const bool tail = cb + 64 > b_end;
#pragma unroll
          for (int g = 0; g < 4; ++g) {
            if (mn[g] < eff) {
#pragma unroll
              for (int j = 16 * g; j < 16 * g + 16; ++j) {
                if (v[j] < eff && (!tail || cb + j < b_end)) {
                  w = topk_insert(ld, li, a.k, w, v[j], (int)(cb + j), thr_q);
                  eff = fminf(w.thr, w.thr_g);
                }
              }
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(tempty0 + 8 * buf);
      }
      if (!ok) break;
      if (q < a.nq) {
        const float qn = a.metric == KANN_L2 ? a.qnorm[q] : 0.f;
        u64* o = a.out + ((size_t)q * a.S + split) * a.k;
        for (int j = 0; j < a.k; ++j)
          o[j] = li[j] < 0 ? ((u64)ordered_bits(__int_as_float(0x7f800000)) << 32) | 0xffffffffull
                           : make_key(ld[j] + qn, (uint32_t)li[j]);
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

// Squared norms of BF16/FP16 rows in FP32 (one warp per row).
template <int DT>
__global__ void row_norms_kernel(const uint16_t* __restrict__ x, int64_t n, int d, float* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (row >= n) return;
  float s = 0.f;
  for (int k = lane * 8; k < d; k += 256) {
    const uint4 w = *reinterpret_cast<const uint4*>(x + row * d + k);
    float v[8];
    Fmt<DT>::unpack(w, v);
#pragma unroll
    for (int e = 0; e < 8; ++e) s = fmaf(v[e], v[e], s);
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
  if (lane == 0) out[row] = s;
}

constexpr int TH_SAMPLE = 1024;  // base rows scored per query for the starting threshold

// Starting threshold of each query's scan (one warp per query).  Every lane
// scores a strided sample of base rows exactly as the epilogue does (L2:
// ||x||^2 - 2 q.x, IP: -q.x; the query's own constant left out) but in FP32
// on the CUDA cores, raises each score by a bound on the difference between
// two FP32 evaluations of the same dot product in any summation order (the
// products of 16-bit inputs are exact; with unit roundoff taken as 2^-23,
// d terms, S = sum |q_i x_i|: 2 * d * 2^-23 * S per evaluation, doubled for
// L2's factor 2, plus the final roundings), and keeps its minimum.  The k-th
// smallest lane minimum comes from k distinct rows, so it is at least the
// k-th smallest tensor-core score of the whole base: no neighbour that
// belongs in the top k is pruned.  thr (an ordered_bits code) is stored just
// above it because the scan keeps scores strictly below the threshold.
template <int DT>
__global__ void tc_threshold_kernel(const uint16_t* __restrict__ Q, const uint16_t* __restrict__ X, int nq,
                                    int64_t nb, int d, int metric, int k, const float* __restrict__ xnorm,
                                    unsigned* __restrict__ thr) {
  const int lane = threadIdx.x & 31;
  const int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (q >= nq) return;
  const float inf = __int_as_float(0x7f800000);
  const float u = 1.0f / 8388608.0f;  // 2^-23
  const int64_t T = nb < TH_SAMPLE ? nb : TH_SAMPLE;
  const uint16_t* qp = Q + q * d;
  float mn = inf;
  for (int64_t j = lane; j < T; j += 32) {
    const int64_t r = j * nb / T;  // distinct rows, since T <= nb
    const uint16_t* xp = X + r * d;
    float dot = 0.f, sab = 0.f;
    for (int c = 0; c < d; c += 8) {
      float xv[8], qv[8];
      Fmt<DT>::unpack(*reinterpret_cast<const uint4*>(xp + c), xv);
      Fmt<DT>::unpack(*reinterpret_cast<const uint4*>(qp + c), qv);
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        dot = fmaf(xv[e], qv[e], dot);
        sab += fabsf(xv[e] * qv[e]);
      }
    }
    float v, margin;
    if (metric == KANN_L2) {
      const float xn = xnorm[r];
      v = fmaf(-2.f, dot, xn);
      margin = 8.f * (float)d * u * sab + 4.f * u * (fabsf(v) + xn + 2.f * sab);
    } else {
      v = -dot;
      margin = 4.f * (float)d * u * sab + 4.f * u * sab;
    }
    float vu = v + margin;
    vu = vu + 4.f * u * fabsf(vu) + 1e-30f;
    if (!(vu == vu)) vu = inf;  // NaN input: no pruning
    mn = fminf(mn, vu);
  }
  // k-th smallest of the 32 lane minima
  const u64 key = warp_sort32(((u64)ordered_bits(mn) << 32) | (uint32_t)lane, lane);
  const u64 kth = __shfl_sync(FULL, key, k - 1);
  if (lane == 0) {
    const float t = key_dist(kth);
    thr[q] = ordered_bits(t == inf ? inf : nextafterf(t, inf));
  }
}

// Final merge: sort each query's S*k partial keys, keep k (an error flag
// from the main pass turns every output into id -1 / +inf).
__global__ void exact_tc_merge_kernel(const u64* __restrict__ ws, const int* err, int nq, int S, int k, int P,
                                      int32_t* ids, float* dists) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int q = blockIdx.x * (blockDim.x >> 5) + warp;
  if (q >= nq) return;
  const bool bad = *err != 0;
  u64* A = reinterpret_cast<u64*>(smem) + (size_t)warp * P;
  const int tot = S * k;
  for (int i = lane; i < P; i += 32) A[i] = (i < tot && !bad) ? ws[(size_t)q * tot + i] : KEY_MAX;
  __syncwarp();
  warp_smem_sort(A, P, lane);
  for (int j = lane; j < k; j += 32) {
    const u64 key = A[j];
    const uint32_t id = (uint32_t)key;
    ids[(size_t)q * k + j] = (key == KEY_MAX || id == 0xffffffffu) ? -1 : (int32_t)id;
    dists[(size_t)q * k + j] = (key == KEY_MAX || id == 0xffffffffu) ? __int_as_float(0x7f800000) : key_dist(key);
  }
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

bool make_map(CUtensorMap* m, const void* base, int dtype, int d, int64_t rows, int box_rows) {
  auto enc = get_encode();
  if (!enc) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)d, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)d * 2};
  const cuuint32_t box[2] = {(cuuint32_t)TC_K, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUtensorMapDataType t = dtype == KANN_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
  return enc(m, t, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Instruction descriptor of tcgen05.mma kind::f16: FP32 accumulator, A and B
// in the same 16-bit format, both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
uint32_t make_idesc(int dtype) {
  const uint32_t ab = dtype == KANN_BF16 ? 1u : 0u;
  return (1u << 4) | (ab << 7) | (ab << 10) | ((uint32_t)(TC_N >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
}

int num_sms() {
  int dev = 0, n = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n;
}

}  // namespace

// Work split of the tensor-core path: queries in pairs of 128-row tiles, the
// base in S splits (multiples of 128 rows) so that there are >= 4 work items
// per SM.
void exact_tc_plan(int nq, int64_t nb, int* S_out, int64_t* per_out) {
  const int qtiles = (nq + TC_M * TC_QB - 1) / (TC_M * TC_QB);
  const int64_t ntiles = (nb + TC_N - 1) / TC_N;
  int S = (4 * 148 + qtiles - 1) / qtiles;
  if (S > 64) S = 64;
  if (S > ntiles) S = (int)ntiles;
  if (S < 1) S = 1;
  const int64_t tiles_per = (ntiles + S - 1) / S;
  S = (int)((ntiles + tiles_per - 1) / tiles_per);
  *S_out = S;
  *per_out = tiles_per * TC_N;
}

size_t exact_tc_workspace_bytes(int nq, int64_t nb, int k) {
  int S;
  int64_t per;
  exact_tc_plan(nq, nb, &S, &per);
  return (size_t)nq * S * k * 8 + (size_t)nb * 4 + (size_t)nq * 8 + 256;
}

bool exact_tc_supported(int dtype, int d, int k) {
  return (dtype == KANN_BF16 || dtype == KANN_F16) && d % 8 == 0 && k >= 1 && k <= TC_KMAX;
}

int exact_tc_run(const void* Q, const void* X, int nq, int64_t nb, int d, int metric, int dtype, int k, int32_t* ids,
                 float* dists, void* ws, cudaStream_t s) {
  int S;
  int64_t per;
  exact_tc_plan(nq, nb, &S, &per);
  unsigned char* w = static_cast<unsigned char*>(ws);
  u64* part = reinterpret_cast<u64*>(w);
  float* xn = reinterpret_cast<float*>(w + (size_t)nq * S * k * 8);
  float* qn = xn + nb;
  unsigned* th = reinterpret_cast<unsigned*>(qn + nq);
  int* err = reinterpret_cast<int*>(((uintptr_t)(th + nq) + 15) & ~(uintptr_t)15);
  CUtensorMap mq, mx;
  if (!make_map(&mq, Q, dtype, d, nq, TC_M) || !make_map(&mx, X, dtype, d, nb, TC_N)) return (int)cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), s);
  if (e != cudaSuccess) return (int)e;
  void (*nfn)(const uint16_t*, int64_t, int, float*) =
      dtype == KANN_BF16 ? row_norms_kernel<KANN_BF16> : row_norms_kernel<KANN_F16>;
  nfn<<<(unsigned)((nb * 32 + 255) / 256), 256, 0, s>>>((const uint16_t*)X, nb, d, xn);
  nfn<<<(unsigned)(((int64_t)nq * 32 + 255) / 256), 256, 0, s>>>((const uint16_t*)Q, nq, d, qn);
  void (*tfn)(const uint16_t*, const uint16_t*, int, int64_t, int, int, int, const float*, unsigned*) =
      dtype == KANN_BF16 ? tc_threshold_kernel<KANN_BF16> : tc_threshold_kernel<KANN_F16>;
  tfn<<<(unsigned)(((int64_t)nq * 32 + 255) / 256), 256, 0, s>>>((const uint16_t*)Q, (const uint16_t*)X, nq, nb, d,
                                                                  metric, k, xn, th);
  TcArgs a;
  a.nq = nq;
  a.nb = nb;
  a.d = d;
  a.metric = metric;
  a.k = k;
  a.S = S;
  a.kchunks = (d + TC_K - 1) / TC_K;
  a.per = per;
  a.n_items = ((nq + TC_M * TC_QB - 1) / (TC_M * TC_QB)) * S;
  a.idesc = make_idesc(dtype);
  a.xnorm = xn;
  a.qnorm = qn;
  a.thr = th;
  a.out = part;
  a.err = err;
  // shared memory: alignment pad, stage ring, barriers, norms, top-k lists
  const size_t fixed = 1024 + (2 * TC_MAX_STAGES + 6) * 8 + 16 + TC_EPI_WARPS * 128 * 4 + (size_t)2 * TC_M * k * 8;
  int optin = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  // resident query block when it and a ring of at least 3 base stages fit
  a.qres = a.kchunks <= TC_QRES_MAX_KCHUNKS &&
           fixed + (size_t)TC_QB * a.kchunks * A_BYTES + 3 * (size_t)B_BYTES <= (size_t)optin;
  a.qbytes = a.qres ? TC_QB * a.kchunks * A_BYTES : 0;
  a.stage_bytes = a.qres ? B_BYTES : STAGE_BYTES;
  a.stages = TC_MAX_STAGES;
  while (a.stages > 2 && fixed + (size_t)a.qbytes + (size_t)a.stages * a.stage_bytes > (size_t)optin) --a.stages;
  const size_t smem = fixed + (size_t)a.qbytes + (size_t)a.stages * a.stage_bytes;
  e = cudaFuncSetAttribute(exact_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  const int grid = a.n_items < num_sms() ? a.n_items : num_sms();
  exact_tc_kernel<<<grid, TC_THREADS, smem, s>>>(mq, mx, a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return (int)e;
  int P = 32;
  while (P < S * k) P <<= 1;
  int wpb = 4;
  while (wpb > 1 && (size_t)wpb * P * 8 > 160 * 1024) wpb >>= 1;
  const size_t msmem = (size_t)wpb * P * 8;
  e = cudaFuncSetAttribute(exact_tc_merge_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)msmem);
  if (e != cudaSuccess) return (int)e;
  exact_tc_merge_kernel<<<(nq + wpb - 1) / wpb, wpb * 32, msmem, s>>>(part, err, nq, S, k, P, ids, dists);
  return (int)cudaGetLastError();
}

}  // namespace kann
