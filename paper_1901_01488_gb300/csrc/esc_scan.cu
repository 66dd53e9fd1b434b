// The selectivity sub-query on the GPU (paper Sec. 2): evaluate a compiled
// selection predicate over resident columns, count the qualifying rows
// exactly, and optionally materialise them with their projected columns in
// row order (Sec. 2.1), or emit a dense-key bitmap (for the semi-join
// counts of esc_semijoin.cu).
//
// Kernel shape (sm_103a):
//  * scan_kernel, persistent: one CTA per SM, 1 producer warp + 15 to 23
//    consumer warps (one instance per block shape of kScanShapes: fewer
//    warps where the udf path's registers are compiled in, more with one
//    group per pass); work units (a few consecutive tiles; the last tiles of
//    a query one per unit) are claimed in order from a global ticket;
//  * the producer stages every column the predicate reads into shared memory
//    with 1-D bulk TMA copies (cp.async.bulk ... mbarrier::complete_tx) into a
//    ring of kStages stages; the ragged tail of the last tile (< 16 bytes per
//    column) is copied with plain loads;
//  * consumers claim runs of one, two or four 256-row groups of a stage from a
//    shared counter and interpret the postfix program on 8 rows per lane per
//    group (one decode per instruction for the run), keeping the
//    boolean evaluation stack as 8-bit masks in one 64-bit register;
//  * counts: popc per lane, one atomic per warp and query;
//  * ordered compaction, first pass: the selection bitmap (lane-major, one
//    byte per lane and group, a coalesced 32-byte store per warp) and a
//    total per compaction unit of 65536 rows; second pass (write_kernel,
//    one block per compaction unit): a decoupled look-back over the unit
//    totals (Merrill & Garland, "Single-pass Parallel Prefix Scan with
//    Decoupled Look-back", 2016), a block scan of the group counts, then ids
//    and projected values to consecutive output slots.
// Every wait on an mbarrier is bounded by %globaltimer; on expiry the kernel
// records ESC_ETIMEOUT in the scratch header and all CTAs wind down.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "esc_internal.h"

namespace esc {

constexpr int kConsumers = 15;                   // consumer warps per CTA of the shared scan
constexpr int kThreads = 32 * (kConsumers + 1);  // + the producer warp: 16 warps, 4 per SM sub-partition
// The scan kernel's instances are the block shapes of kScanShapes: the udf
// remainder sets the register demand (128 per thread at 16 warps, two groups
// per pass), so the instances without it, or with one group per pass, run
// more consumer warps per SM.
constexpr int kStages = 3;
constexpr uint32_t kStageBytes = 64 * 1024;
constexpr int kTailTilesPerSm = 8;      // single-tile work units at the end of a query (per SM)
constexpr int kMaxUnitGroups = kMaxUnitRows / kGroup;  // 256: one write-kernel thread per group
constexpr uint64_t kWaitLimitNs = 2000000000ull;   // 2 s per bounded wait
constexpr uint32_t FULL = 0xffffffffu;
static_assert(kStageBytes <= 65536, "stage column offsets are 16-bit");

// ------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_addr(bar))
               : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(
                   smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed(unsigned long long *p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ void raise_status(ScratchHdr *hdr, unsigned status) {
  atomicCAS(&hdr->status, 0u, status);
  atomicExch(&hdr->abort, 1u);
}
__device__ __forceinline__ bool aborted(const ScratchHdr *hdr) {
  return *(volatile const unsigned *)&hdr->abort != 0u;
}

// Warp-collective bounded wait for the phase of parity `parity` of an
// mbarrier: every lane must observe the completion itself (so that every lane
// has acquire ordering), the warp leaves together, and the decision to give
// up is lane 0's, broadcast.  With `abortable` the wait also gives up as
// soon as the launch is aborting (used for every wait that does not guard an
// in-flight bulk copy, so that one timeout cannot cascade into more).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, ScratchHdr *hdr,
                                          uint64_t limit_ns = kWaitLimitNs, bool abortable = false) {
  bool seen = mbar_try_wait(bar, parity);
  if (__all_sync(FULL, seen)) return true;
  const uint64_t t0 = globaltimer();
  for (uint32_t it = 1;; ++it) {
    if (!seen) seen = mbar_try_wait(bar, parity);
    if (__all_sync(FULL, seen)) return true;
    if ((it & 63u) == 0) {
      int give_up = 0;
      if ((threadIdx.x & 31) == 0) give_up = (abortable && aborted(hdr)) ? 1 : (globaltimer() - t0 > limit_ns) ? 2 : 0;
      give_up = __shfl_sync(FULL, give_up, 0);
      if (give_up) {
        if (give_up == 2 && (threadIdx.x & 31) == 0) raise_status(hdr, ESC_ETIMEOUT);
        return false;
      }
    }
  }
}

// Warp-collective non-blocking test: true only if every lane observed it.
__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return __all_sync(FULL, ok != 0);
}

// ------------------------------------------------------------------ loads
// Values of this lane's 8 rows of a group, for each element type (see the
// row-to-lane map in esc_internal.h).  `g` points at the group's first
// element in shared memory.
__device__ __forceinline__ void load8(int32_t dt, const uint8_t *g, int lane, int64_t v[8]) {
  switch (dt) {
    case ESC_U8: {
      const uint16_t *p = reinterpret_cast<const uint16_t *>(g) + lane;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        uint32_t x = p[32 * j];
        v[2 * j] = x & 0xffu;
        v[2 * j + 1] = x >> 8;
      }
      break;
    }
    case ESC_U16: {
      const uint32_t *p = reinterpret_cast<const uint32_t *>(g) + lane;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        uint32_t x = p[32 * j];
        v[2 * j] = x & 0xffffu;
        v[2 * j + 1] = x >> 16;
      }
      break;
    }
    case ESC_I32: {
      const int2 *p = reinterpret_cast<const int2 *>(g) + lane;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        int2 x = p[32 * j];
        v[2 * j] = x.x;
        v[2 * j + 1] = x.y;
      }
      break;
    }
    default: {
      const longlong2 *p = reinterpret_cast<const longlong2 *>(g) + lane;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        longlong2 x = p[32 * j];
        v[2 * j] = x.x;
        v[2 * j + 1] = x.y;
      }
      break;
    }
  }
}

// 32-bit variant for the narrow types (values fit in int32 exactly).
__device__ __forceinline__ void load8_32(int32_t dt, const uint8_t *g, int lane, int32_t v[8]) {
  switch (dt) {
    case ESC_U8: {
      const uint16_t *p = reinterpret_cast<const uint16_t *>(g) + lane;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        uint32_t x = p[32 * j];
        v[2 * j] = (int32_t)(x & 0xffu);
        v[2 * j + 1] = (int32_t)(x >> 8);
      }
      break;
    }
    case ESC_U16: {
      const uint32_t *p = reinterpret_cast<const uint32_t *>(g) + lane;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        uint32_t x = p[32 * j];
        v[2 * j] = (int32_t)(x & 0xffffu);
        v[2 * j + 1] = (int32_t)(x >> 16);
      }
      break;
    }
    default: {
      const int2 *p = reinterpret_cast<const int2 *>(g) + lane;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        int2 x = p[32 * j];
        v[2 * j] = x.x;
        v[2 * j + 1] = x.y;
      }
      break;
    }
  }
}

__device__ __forceinline__ int width_of(int32_t dt) {
  return dt == ESC_U8 ? 1 : dt == ESC_U16 ? 2 : dt == ESC_I32 ? 4 : 8;
}

// (a * b) mod d, product wrapping in 64 bits, remainder truncated toward
// zero; the unsigned quotient uses Granlund & Montgomery's multiply-high
// (PLDI 1994, Fig. 4.1) with host-precomputed mult/sh1/sh2.
__device__ __forceinline__ int64_t udf_rem(int64_t a, int64_t b, uint64_t d, uint64_t mult, int sh1, int sh2) {
  const int64_t p = (int64_t)((uint64_t)a * (uint64_t)b);
  const uint64_t n = p < 0 ? 0ull - (uint64_t)p : (uint64_t)p;
  const uint64_t t = __umul64hi(mult, n);
  const uint64_t q = (t + ((n - t) >> sh1)) >> sh2;
  const int64_t r = (int64_t)(n - q * d);
  return p < 0 ? -r : r;
}

// x mod d for 32-bit x and 1 <= d < 2^32, with M = ceil(2^64 / d): the low 64
// bits of M * x, times d, high 64 bits (Lemire, Kaser & Kurz 2019, direct
// remainder; exact for every 32-bit x and d).
__device__ __forceinline__ uint32_t fastmod32(uint32_t x, uint64_t M, uint32_t d) {
  const uint64_t low = M * (uint64_t)x;
  const uint64_t u = (uint64_t)(uint32_t)(low >> 32) * d + __umulhi((uint32_t)low, d);
  return (uint32_t)(u >> 32);
}

// Remainders of 8 udf products for a modulus d < 2^16, as 32-bit signed
// values (truncated: the sign of the product).  With |p| = H 2^32 + L,
// |p| mod d = ((H mod d) (2^32 mod d) + L mod d) mod d, the inner sum staying
// below d^2 < 2^32 (K = 2^32 mod d); when every |p| of the warp's rows is
// below 2^32 (H = 0), one remainder per row suffices.
__device__ __forceinline__ void udf_rem_small8(const int64_t (&a)[8], const int64_t (&b)[8], uint32_t d, uint64_t M,
                                               uint32_t K, int32_t (&r)[8]) {
  uint64_t n[8];
  uint32_t s[8], hi = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const uint64_t p = (uint64_t)a[k] * (uint64_t)b[k];
    s[k] = (uint32_t)((int64_t)p >> 63);  // 0 or all ones
    const uint64_t s64 = (uint64_t)(int64_t)(int32_t)s[k];
    n[k] = (p ^ s64) - s64;               // |p|, 2^63 included
    hi |= (uint32_t)(n[k] >> 32);
  }
  if (__any_sync(FULL, hi != 0)) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const uint32_t r1 = fastmod32((uint32_t)(n[k] >> 32), M, d);
      const uint32_t r2 = fastmod32((uint32_t)n[k], M, d);
      const uint32_t x = fastmod32(r1 * K + r2, M, d);
      r[k] = (int32_t)((x ^ s[k]) - s[k]);
    }
  } else {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const uint32_t x = fastmod32((uint32_t)n[k], M, d);
      r[k] = (int32_t)((x ^ s[k]) - s[k]);
    }
  }
}

// ------------------------------------------------------------------ evaluation
// Runs the program on this lane's 8 rows of NG groups of the staged tile at
// once (one decode per instruction for all of them, NG independent chains).
// Q (program included) lives in shared memory.
template <int NG, bool UDF>
__device__ __forceinline__ void eval_groups(const Query *Q, const uint8_t *stage, const int (&grp)[NG], int lane,
                                            uint32_t (&out)[NG]) {
  uint64_t S[NG];  // evaluation stacks: entry k in bits [8k, 8k+8), top at bits 0..7
#pragma unroll
  for (int i = 0; i < NG; ++i) S[i] = 0;
  const int n = Q->ninstr;
  for (int pc = 0; pc < n; ++pc) {
    const uint4 h = *reinterpret_cast<const uint4 *>(&Q->code[pc]);
    const uint32_t op = h.x & 0xffu;
    if (op == OP_JZ || op == OP_JNZ) {
      // the connective's result is already known for every row this warp holds
      bool done = true;
      const uint64_t want = op == OP_JZ ? 0u : 0xffu;
#pragma unroll
      for (int i = 0; i < NG; ++i) done = done && ((S[i] & 0xffu) == want);
      if (__all_sync(FULL, done)) pc = (int)(h.z & 0xffffu) - 1;
      continue;
    }
    if (op == OP_INSET) {
      // membership in a 256-bit set of the values 0..255
      const int dt = (int)((h.x >> 8) & 0xffu);
      const int w = width_of(dt);
      const uint8_t *col = stage + (h.z >> 16);
      const uint32_t *set = reinterpret_cast<const uint32_t *>(&Q->pool[h.z & 0xffffu]);
      uint32_t m[NG];
#pragma unroll
      for (int i = 0; i < NG; ++i) m[i] = 0;
      if (dt == ESC_I64) {
#pragma unroll
        for (int i = 0; i < NG; ++i) {
          int64_t v[8];
          load8(dt, col + (size_t)grp[i] * kGroup * 8, lane, v);
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const uint64_t x = (uint64_t)v[k];
            const uint32_t b = x < 256u ? (set[x >> 5] >> (x & 31u)) & 1u : 0u;
            m[i] |= b << k;
          }
        }
      } else {
#pragma unroll
        for (int i = 0; i < NG; ++i) {
          int32_t v[8];
          load8_32(dt, col + (size_t)grp[i] * kGroup * w, lane, v);
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const uint32_t x = (uint32_t)v[k];
            const uint32_t b = x < 256u ? (set[x >> 5] >> (x & 31u)) & 1u : 0u;
            m[i] |= b << k;
          }
        }
      }
#pragma unroll
      for (int i = 0; i < NG; ++i) S[i] = (S[i] << 8) | m[i];
      continue;
    }
    if (op <= OP_UDF) {
      const longlong2 lh = *reinterpret_cast<const longlong2 *>(&Q->code[pc].lo);
      const int dt = (int)((h.x >> 8) & 0xffu);
      const int w = width_of(dt);
      const uint8_t *col = stage + (h.z >> 16);
      uint32_t m[NG];
#pragma unroll
      for (int i = 0; i < NG; ++i) m[i] = 0;
      if (op == OP_RANGE) {
        if (dt == ESC_I64) {
          int64_t v[NG][8];
#pragma unroll
          for (int i = 0; i < NG; ++i) load8(dt, col + (size_t)grp[i] * kGroup * 8, lane, v[i]);
          const uint64_t span = (uint64_t)lh.y - (uint64_t)lh.x;
#pragma unroll
          for (int i = 0; i < NG; ++i)
#pragma unroll
            for (int k = 0; k < 8; ++k) m[i] |= (uint32_t)((uint64_t)v[i][k] - (uint64_t)lh.x <= span) << k;
        } else {
          int32_t v[NG][8];
#pragma unroll
          for (int i = 0; i < NG; ++i) load8_32(dt, col + (size_t)grp[i] * kGroup * w, lane, v[i]);
          const uint32_t lo = (uint32_t)lh.x;
          const uint32_t span = (uint32_t)((uint64_t)lh.y - (uint64_t)lh.x);
#pragma unroll
          for (int i = 0; i < NG; ++i)
#pragma unroll
            for (int k = 0; k < 8; ++k) m[i] |= (uint32_t)((uint32_t)v[i][k] - lo <= span) << k;
        }
      } else if (op == OP_IN) {
        const int64_t *vals = &Q->pool[h.z & 0xffffu];
        const int nv = (int)(h.y >> 16);
        if (dt == ESC_I64) {
          int64_t v[NG][8];
#pragma unroll
          for (int i = 0; i < NG; ++i) load8(dt, col + (size_t)grp[i] * kGroup * 8, lane, v[i]);
          for (int t = 0; t < nv; ++t) {
            const int64_t c = vals[t];
#pragma unroll
            for (int i = 0; i < NG; ++i)
#pragma unroll
              for (int k = 0; k < 8; ++k) m[i] |= (uint32_t)(v[i][k] == c) << k;
          }
        } else {
          int32_t v[NG][8];
#pragma unroll
          for (int i = 0; i < NG; ++i) load8_32(dt, col + (size_t)grp[i] * kGroup * w, lane, v[i]);
          for (int t = 0; t < nv; ++t) {
            const int32_t c = (int32_t)vals[t];
#pragma unroll
            for (int i = 0; i < NG; ++i)
#pragma unroll
              for (int k = 0; k < 8; ++k) m[i] |= (uint32_t)(v[i][k] == c) << k;
          }
        }
      } else if constexpr (UDF) {  // OP_UDF (a program with one runs only on an instance with the udf path)
        const int dt2 = (int)((h.x >> 16) & 0xffu);
        const int w2 = width_of(dt2);
        const uint8_t *col2 = stage + (h.w & 0xffffu);
        const int64_t *P = &Q->pool[h.z & 0xffffu];
        const uint64_t d = (uint64_t)P[0];
        if (d < 65536u) {
          // remainder and range in 32 bits (the range lies inside (-d, d))
          const uint64_t M = (uint64_t)P[4];
          const uint32_t K = (uint32_t)P[5], d32 = (uint32_t)d;
          const uint32_t lo = (uint32_t)lh.x, span = (uint32_t)((uint64_t)lh.y - (uint64_t)lh.x);
#pragma unroll
          for (int i = 0; i < NG; ++i) {
            int64_t a[8], b[8];
            load8(dt, col + (size_t)grp[i] * kGroup * w, lane, a);
            load8(dt2, col2 + (size_t)grp[i] * kGroup * w2, lane, b);
            int32_t r[8];
            udf_rem_small8(a, b, d32, M, K, r);
#pragma unroll
            for (int k = 0; k < 8; ++k) m[i] |= (uint32_t)((uint32_t)r[k] - lo <= span) << k;
          }
        } else {
          const uint64_t mult = (uint64_t)P[1];
          const int sh1 = (int)P[2], sh2 = (int)P[3];
          const uint64_t span = (uint64_t)lh.y - (uint64_t)lh.x;
#pragma unroll
          for (int i = 0; i < NG; ++i) {
            int64_t a[8], b[8];
            load8(dt, col + (size_t)grp[i] * kGroup * w, lane, a);
            load8(dt2, col2 + (size_t)grp[i] * kGroup * w2, lane, b);
#pragma unroll
            for (int k = 0; k < 8; ++k) {
              const int64_t r = udf_rem(a[k], b[k], d, mult, sh1, sh2);
              m[i] |= (uint32_t)((uint64_t)r - (uint64_t)lh.x <= span) << k;
            }
          }
        }
      }
#pragma unroll
      for (int i = 0; i < NG; ++i) S[i] = (S[i] << 8) | m[i];
    } else if (op == OP_AND) {
#pragma unroll
      for (int i = 0; i < NG; ++i) S[i] = (S[i] >> 8) & ((S[i] & 0xffu) | ~0xffull);
    } else if (op == OP_OR) {
#pragma unroll
      for (int i = 0; i < NG; ++i) S[i] = (S[i] >> 8) | (S[i] & 0xffu);
    } else if (op == OP_NOT) {
#pragma unroll
      for (int i = 0; i < NG; ++i) S[i] ^= 0xffu;
    } else if (op == OP_TRUE) {
#pragma unroll
      for (int i = 0; i < NG; ++i) S[i] = (S[i] << 8) | 0xffu;
    } else {  // OP_FALSE
#pragma unroll
      for (int i = 0; i < NG; ++i) S[i] = S[i] << 8;
    }
  }
#pragma unroll
  for (int i = 0; i < NG; ++i) out[i] = (uint32_t)(S[i] & 0xffu);
}

// Bits of this lane's 8 rows that lie inside the tile's `rows` valid rows.
__device__ __forceinline__ uint32_t valid_mask(int grp, int lane, uint32_t rows) {
  const uint32_t base = (uint32_t)grp * kGroup + 2u * lane;
  if (base + 193u < rows) return 0xffu;  // row 64*3 + 2*lane + 1 is the lane's last
  uint32_t m = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) m |= (uint32_t)(base + 64u * (k >> 1) + (k & 1) < rows) << k;
  return m;
}

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}

// Tiles [t0, t1) of work unit u of a query: the first unit_big units hold
// unit_tiles tiles each, the rest one tile each, so that the last work of a
// launch comes in small pieces and the SMs finish together.
__device__ __forceinline__ void unit_range(const Query &Q, uint32_t u, uint32_t &t0, uint32_t &t1) {
  const uint32_t nb = Q.unit_big, ut = Q.unit_tiles;
  t0 = u < nb ? u * ut : nb * ut + (u - nb);
  t1 = min(u < nb ? t0 + ut : t0 + 1u, Q.ntiles);
}

struct StageMeta {
  int32_t q;       // query index, -1 = end of work
  uint32_t tile;   // tile index within the query
  uint32_t rows;   // valid rows in this tile
  uint32_t dead;   // 1: the launch is aborting, skip the work (same for every reader)
  uint32_t pad[4];
};

struct Launch {
  const Query *queries;  // device array of nq queries, or null: use q0
  int32_t nq;
  uint32_t total_units;  // work units (scan tickets) of all queries
  ScratchHdr *hdr;
  // single sub-query: where the scan's last consumer warp stores the final
  // count (the caller's word, which then needs no zeroing); null: none
  unsigned long long *count_out;
  uint32_t pad[2];
  Query q0;
};

__device__ __forceinline__ const Query *query_ptr(const Launch &L, int q) {
  return L.queries ? &L.queries[q] : &L.q0;
}

__device__ __forceinline__ void retire_tile(unsigned int *tiles_left, unsigned long long *done_ns, int lane) {
  // Per-query completion time: every consumer warp retires each tile once.
  if (done_ns && lane == 0) {
    __threadfence();
    if (atomicSub(tiles_left, 1u) == 1u) *done_ns = globaltimer();
  }
}

// Groups of a full tile at most (checked build).
[[maybe_unused]] constexpr size_t kTileGroups = kMaxTileRows / kGroup;

// Shared-memory layout of the scan kernel (offsets in bytes).
struct SmemLayout {
  static constexpr size_t stages = 0;
  static constexpr size_t qslot = stages + (size_t)kStages * kStageBytes;
  static constexpr size_t bars = qslot + (size_t)kStages * sizeof(Query);  // full[S] empty[S]
  static constexpr size_t meta = bars + 2 * kStages * 8;
  static constexpr size_t slotq = meta + kStages * sizeof(StageMeta);      // [S] int32
  static constexpr size_t take = slotq + kStages * 4;                       // [S] u32 run claims
  static constexpr size_t total = take + kStages * 4;
};

// Checked build: everything the evaluation of a stage will index -- every
// operand slice of the staged tile, the constant pool entries of IN lists,
// sets and udf moduli, jump targets, the groups' result bytes -- lies inside
// its buffer (warp-collective; lanes take instructions).  True in the
// release build.
__device__ __forceinline__ bool stage_in_bounds(const Query *Q, int ngroups, ScratchHdr *hdr, int lane) {
#ifdef ESC_CHECKED
  bool ok = ESC_INB(hdr, ngroups >= 0 && (uint32_t)ngroups <= Q->gmax && Q->gmax <= (uint32_t)kTileGroups, 10, ngroups);
  ok = ok && ESC_INB(hdr, Q->ninstr >= 0 && Q->ninstr <= kMaxInstr && Q->nref <= kMaxRef, 11, Q->ninstr);
  const uint64_t span = (uint64_t)ngroups * kGroup;
  for (int pc = lane; ok && pc < Q->ninstr; pc += 32) {
    const Instr &I = Q->code[pc];
    const bool opd = I.op == OP_RANGE || I.op == OP_IN || I.op == OP_INSET || I.op == OP_UDF;
    if (opd) {
      ok = ok && ESC_INB(hdr, I.ref < Q->nref, 12, pc);
      ok = ok && ESC_INB(hdr, I.soff + span * width_of(I.dtype) <= kStageBytes, 13, pc);
    }
    if (I.op == OP_UDF) {
      ok = ok && ESC_INB(hdr, I.ref2 < Q->nref, 12, pc);
      ok = ok && ESC_INB(hdr, I.soff2 + span * width_of(I.dtype2) <= kStageBytes, 13, pc);
      ok = ok && ESC_INB(hdr, I.off + 6u <= (uint32_t)kMaxPool, 14, pc);
    }
    if (I.op == OP_IN) ok = ok && ESC_INB(hdr, (uint32_t)I.off + I.n <= (uint32_t)kMaxPool, 14, pc);
    if (I.op == OP_INSET) ok = ok && ESC_INB(hdr, I.off + 4u <= (uint32_t)kMaxPool, 14, pc);
    if (I.op == OP_JZ || I.op == OP_JNZ) ok = ok && ESC_INB(hdr, I.off <= (uint32_t)Q->ninstr, 15, pc);
  }
  return __all_sync(FULL, ok);
#else
  (void)Q;
  (void)ngroups;
  (void)hdr;
  (void)lane;
  return true;
#endif
}

// ------------------------------------------------------------------ the scan kernel
// Warp 0: producer (unit tickets, bulk copies).  Warps 1..: consumers
// (evaluate; count; compaction: bitmap words and unit totals; bitmap mode:
// the caller's bitmap words).
// NC consumer warps; UDF: the instance can run programs with a udf.
template <int NC, bool UDF, int NG>
__global__ void __launch_bounds__(32 * (NC + 1), 1) scan_kernel(const __grid_constant__ Launch L) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t *stages = smem + SmemLayout::stages;
  Query *qslot = reinterpret_cast<Query *>(smem + SmemLayout::qslot);
  uint64_t *full_bar = reinterpret_cast<uint64_t *>(smem + SmemLayout::bars);
  uint64_t *empty_bar = full_bar + kStages;
  StageMeta *meta = reinterpret_cast<StageMeta *>(smem + SmemLayout::meta);
  int32_t *slotq = reinterpret_cast<int32_t *>(smem + SmemLayout::slotq);
  uint32_t *take = reinterpret_cast<uint32_t *>(smem + SmemLayout::take);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  ScratchHdr *hdr = L.hdr;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], NC);
      slotq[s] = -1;
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  if (warp == 0) {
    // ---------------------------------------------------------------- producer
    int s = 0;
    uint32_t phase = 0;
    int qc = 0;  // cursor over queries: tickets of one CTA only increase
    bool done = false;
    // The next unit's ticket and the abort flag are fetched one unit ahead,
    // so that neither round trip delays the bulk copies of the current unit.
    uint32_t u_next = 0, dead_next = 0;
    if (lane == 0) u_next = atomicAdd(&hdr->ticket, 1u);
    while (!done) {
      uint32_t u = 0, dead = 0;
      if (lane == 0) {
        u = u_next;
        dead = dead_next;
        if (u < L.total_units && !dead) {
          u_next = atomicAdd(&hdr->ticket, 1u);
          dead_next = aborted(hdr) ? 1u : 0u;
        }
      }
      u = __shfl_sync(FULL, u, 0);
      dead = __shfl_sync(FULL, dead, 0);
      if (u >= L.total_units || dead) {
        if (mbar_wait(&empty_bar[s], phase ^ 1u, hdr, kWaitLimitNs, true) && lane == 0) {
          meta[s].q = -1;
          mbar_arrive(&full_bar[s]);
        }
        break;
      }
      while (qc + 1 < L.nq && u >= query_ptr(L, qc + 1)->unit_base) ++qc;
      const Query *Qg = query_ptr(L, qc);
      const uint32_t unit = u - Qg->unit_base;
      uint32_t t0, t1;
      unit_range(*Qg, unit, t0, t1);
      for (uint32_t tile = t0; tile < t1; ++tile) {
        if (!mbar_wait(&empty_bar[s], phase ^ 1u, hdr, kWaitLimitNs, true)) {
          done = true;
          break;
        }
        Query *Q = &qslot[s];
        if (slotq[s] != qc) {  // stage the query (program included) in shared memory
          const uint2 *src = reinterpret_cast<const uint2 *>(Qg);
          uint2 *dst = reinterpret_cast<uint2 *>(Q);
          for (int i = lane; i < (int)(sizeof(Query) / 8); i += 32) dst[i] = src[i];
          __syncwarp();
          if (lane == 0) slotq[s] = qc;
        }
        __syncwarp();
        const uint32_t r0 = tile * Q->tile_rows;
        const uint32_t rows = min(Q->tile_rows, Q->nrows - r0);
        uint8_t *stage = stages + (size_t)s * kStageBytes;
        // bytes of each read column: a 16-byte multiple by bulk copy, the rest by hand
        uint32_t bulk = 0, tail = 0;
        const uint8_t *src = nullptr;
        uint8_t *dst = nullptr;
        const int nref = Q->nref;
        if (lane < nref) {
          const uint32_t w = Q->ref_w[lane];
          const uint32_t bytes = rows * w;
          bulk = bytes & ~15u;
          tail = bytes - bulk;
          src = Q->ref_ptr[lane] + (size_t)r0 * w;
          dst = stage + Q->stage_off[lane];
          // checked build: the copy stays inside the stage and the column
          if (!ESC_INB(hdr, Q->stage_off[lane] + bytes <= kStageBytes, 1, Q->stage_off[lane] + bytes) ||
              !ESC_INB(hdr, (uint64_t)r0 + rows <= Q->nrows, 2, r0 + rows))
            bulk = tail = 0;
        }
        if (__ballot_sync(FULL, tail != 0)) {
          for (int c = 0; c < nref; ++c) {
            const uint32_t tb = __shfl_sync(FULL, tail, c);
            const uint32_t bb = __shfl_sync(FULL, bulk, c);
            const uint8_t *sp = reinterpret_cast<const uint8_t *>(__shfl_sync(FULL, (unsigned long long)src, c));
            uint8_t *dp = reinterpret_cast<uint8_t *>(__shfl_sync(FULL, (unsigned long long)dst, c));
            if ((uint32_t)lane < tb) dp[bb + lane] = sp[bb + lane];
          }
          fence_proxy_async_smem();
        }
        const uint32_t tot = __reduce_add_sync(FULL, bulk);
        __syncwarp();
        if (lane == 0) {
          StageMeta &m = meta[s];
          take[s] = 0;  // every consumer has left the stage (empty barrier)
          m.q = qc;
          m.tile = tile;
          m.rows = rows;
          m.dead = dead;
          mbar_arrive_expect_tx(&full_bar[s], tot);
        }
        __syncwarp();
        if (bulk) bulk_load(dst, src, bulk, &full_bar[s]);
        if (++s == kStages) {
          s = 0;
          phase ^= 1u;
        }
      }
    }
    return;
  }

  // ---------------------------------------------------------------- consumers
  int s = 0;
  uint32_t phase = 0;
  // Running sums flushed with one atomic when the query / unit changes.
  unsigned long long *acc_ptr = nullptr;  // query count being accumulated
  int acc_q = -1;
  uint32_t acc = 0;                       // this lane's share
  unsigned long long *uacc_ptr = nullptr; // compaction-unit total being accumulated (MODE_SELECT)
  uint32_t uacc = 0;
  while (true) {
    const bool got = mbar_wait(&full_bar[s], phase, hdr);
    const StageMeta mt = meta[s];
    const bool end = !got || mt.q < 0;
    const Query *Q = &qslot[s];
    if (uacc_ptr && end) {
      const uint32_t t = __reduce_add_sync(FULL, uacc);
      if (lane == 0 && t) atomicAdd(uacc_ptr, (unsigned long long)t);
      uacc = 0;
      uacc_ptr = nullptr;
    }
    if (acc_ptr && (end || acc_q != mt.q)) {
      const uint32_t t = __reduce_add_sync(FULL, acc);
      if (lane == 0 && t) atomicAdd(acc_ptr, (unsigned long long)t);
      acc = 0;
      acc_ptr = nullptr;
      acc_q = -1;
    }
    if (end) break;
    const uint8_t *stage = stages + (size_t)s * kStageBytes;
    const uint32_t rows = mt.rows;
    const int ngroups = (int)((rows + kGroup - 1) / kGroup);
    const int mode = Q->mode;
    const uint32_t r0 = mt.tile * Q->tile_rows;
    acc_q = mt.q;
    acc_ptr = Q->count;
    // Consumers claim runs of NG adjacent groups of the stage from a shared
    // counter until none is left, then move on to the next stage: the work of
    // a stage spreads over every consumer whatever its group count, and a warp
    // that finishes early starts on the next stage.
    const int nruns = (ngroups + NG - 1) / NG;
    auto claim = [&]() {
      int j = 0;
      if (lane == 0) j = (int)atomicAdd(&take[s], 1u);
      return __shfl_sync(FULL, j, 0);
    };
    if (mt.dead == 0 && stage_in_bounds(Q, ngroups, hdr, lane)) {
      // one evaluation loop for every mode (a single inlined copy of the
      // interpreter); the per-group epilogue branches on the mode (uniform)
      const uint32_t nwords = (Q->nrows + 31u) / 32u;
      uint32_t *bm = Q->bitmap;
      for (int j = claim(); j < nruns; j = claim()) {
        // the run's groups; past the stage's last group, that group again
        // (evaluated, not counted)
        int gs[NG];
#pragma unroll
        for (int i = 0; i < NG; ++i) gs[i] = min(NG * j + i, ngroups - 1);
        uint32_t mm[NG];
        eval_groups<NG, UDF>(Q, stage, gs, lane, mm);
#pragma unroll
        for (int i = 0; i < NG; ++i) {
          if (NG * j + i >= ngroups) break;
          const uint32_t m = mm[i] & valid_mask(gs[i], lane, rows);
          const uint32_t c = __popc(m);
          acc += c;
          if (mode == MODE_COUNT) continue;
          uint32_t word = 0;
          if (mode == MODE_SELECT) {
            // the group's compaction unit (wunit_groups groups): flush the
            // running total when it changes (warp-uniform)
            const uint32_t gix = mt.tile * Q->gmax + (uint32_t)gs[i];
            const uint32_t wu = Q->wunit_recip ? __umulhi(gix, Q->wunit_recip) : gix;
            if (!ESC_INB(hdr, wu < Q->nwunits, 16, wu)) continue;
            unsigned long long *up = Q->unit_total + wu;
            if (up != uacc_ptr) {
              if (uacc_ptr) {
                const uint32_t t = __reduce_add_sync(FULL, uacc);
                if (lane == 0 && t) atomicAdd(uacc_ptr, (unsigned long long)t);
              }
              uacc = 0;
              uacc_ptr = up;
            }
            uacc += c;
            // selection bitmap, lane-major: byte l of the group's 32 bytes is
            // lane l's mask (bit 2j+i: row 64*j + 2*l + i of the group), one
            // coalesced 32-byte store per warp; the write kernel counts a
            // group's rows from its bytes
            const uint64_t gi = (uint64_t)mt.tile * Q->gmax + (uint32_t)gs[i];
            if (ESC_INB(hdr, gi < (uint64_t)Q->ntiles * Q->gmax, 17, gi))
              reinterpret_cast<uint8_t *>(Q->bitmap)[gi * 32 + lane] = (uint8_t)m;
            continue;
          }
          const uint32_t gidx = (r0 + (uint32_t)gs[i] * kGroup) / kGroup;
#pragma unroll
          for (int p = 0; p < 8; ++p) {  // caller's bitmap: words of rows 32p .. 32p+31 of the group
            const int src = 16 * (p & 1) + (lane >> 1);
            const int bit = 2 * (p >> 1) + (lane & 1);
            const uint32_t bb = __ballot_sync(FULL, (__shfl_sync(FULL, m, src) >> bit) & 1u);
            if (lane == p) word = bb;
          }
          const uint32_t wi = gidx * 8u + (uint32_t)lane;
          if (lane < 8 && wi < nwords) bm[wi] = word;
        }
      }
    }
    if (mode != MODE_SELECT) retire_tile(Q->tiles_left, Q->done_ns, lane);
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty_bar[s]);
    if (++s == kStages) {
      s = 0;
      phase ^= 1u;
    }
  }
  // Single sub-query: the last consumer warp of the grid to finish (every
  // warp has flushed its count by now) stores the final count in the
  // caller's word.
  if (L.count_out && lane == 0) {
    __threadfence();
    if (atomicAdd(&hdr->warps_done, 1u) == gridDim.x * (uint32_t)NC - 1u) {
      __threadfence();
      *L.count_out = atomicAdd(L.q0.count, 0ull);
    }
  }
}

// ------------------------------------------------------------------ the write kernel
// Second pass of ordered compaction, one block per compaction unit (at most
// kMaxUnitGroups = 256 groups of 256 rows: one thread per group; sized per
// query so that the blocks fill whole waves of the GPU, see
// layout_write_units; independent of the scan's work units, whatever the
// predicate's read width).
//  1. The unit's first output slot: a decoupled look-back over the units
//     before it (Merrill & Garland 2016).  Every unit's aggregate is already
//     final (written by the scan kernel), so the look-back adds aggregates
//     until it meets a unit whose inclusive prefix another block published,
//     and never waits.
//  2. Each group's first slot: a block-wide exclusive scan of the group
//     counts of the unit.
//  3. The unit's groups are split evenly over the warps (at most 32 each).
//     A dense group (at least kDenseMin qualifying rows, all 256 rows inside
//     the table) takes the whole warp: its projected columns arrive in shared
//     memory by asynchronous copies and each output slot takes its row's
//     value from there, so that stores coalesce.  Every other group takes one
//     lane, which walks its group's rows in order and stages (row, slot)
//     entries; the warp then copies the staged entries, 4 per lane, loads
//     before stores.
// The selection bitmap is lane-major (see the scan kernel): bit 2j+i of the
// group's byte l is its row 64*j + 2*l + i.

constexpr int kWriteThreads = 256;
constexpr int kWriteWarps = kWriteThreads / 32;
constexpr int kWriteBlocksPerSm = 4;     // resident write-kernel blocks per SM (registers and shared memory)
static_assert(kMaxUnitGroups <= kWriteThreads, "one write-kernel thread per group of a unit");
constexpr uint32_t kDenseMin = 64;       // qualifying rows of a group for the dense path
constexpr uint32_t kRawBytes = 2048;     // per warp: a dense group's projected values (<= 8 B per row at once)
constexpr uint32_t kStageEntries = kRawBytes / 4;  // sparse entries staged per warp (same buffer)

// Shared memory of one warp of the write kernel.
struct WriteWarpSmem {
  uint32_t words[32][8];                 // bitmap words of the warp's groups
  uint32_t sids[kGroup];                 // dense group: row (within the group) of each output slot
  __align__(16) uint8_t raw[kRawBytes];  // dense group: projected columns in row order; else sparse entries
};
constexpr size_t kWriteSmem = sizeof(WriteWarpSmem) * kWriteWarps;

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

__device__ __forceinline__ uint64_t load_elem(const uint8_t *base, uint32_t row, int w) {
  switch (w) {
    case 1: return base[row];
    case 2: return reinterpret_cast<const uint16_t *>(base)[row];
    case 4: return reinterpret_cast<const uint32_t *>(base)[row];
    default: return reinterpret_cast<const unsigned long long *>(base)[row];
  }
}

__device__ __forceinline__ void store_elem(void *base, unsigned long long pos, uint64_t v, int w) {
  switch (w) {
    case 1: static_cast<uint8_t *>(base)[pos] = (uint8_t)v; break;
    case 2: static_cast<uint16_t *>(base)[pos] = (uint16_t)v; break;
    case 4: static_cast<uint32_t *>(base)[pos] = (uint32_t)v; break;
    default: static_cast<unsigned long long *>(base)[pos] = v; break;
  }
}

// Finds the query a block belongs to: the last one whose first block (the
// field `base` selects) is <= blockIdx.x.
template <typename F>
__device__ __forceinline__ int block_query(const Launch &L, F base) {
  int lo = 0, hi = L.nq - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (base(query_ptr(L, mid)) <= blockIdx.x) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// What the write kernel needs of a query, in shared memory.
struct GatherInfo {
  uint64_t capacity;
  uint32_t *out_ids;
  unsigned int *tiles_left;
  unsigned long long *done_ns;
  uint32_t nrows;
  int32_t nproj;
  uint8_t proj_w[kMaxProj];
  const uint8_t *proj_ptr[kMaxProj];
  void *out_proj[kMaxProj];
};

// Copies staged sparse entries (row within the warp's groups << 16 | output
// slot relative to the warp's first group) to the outputs: 4 entries per
// lane, each column's loads issued before its stores.
__device__ __forceinline__ void flush_sparse(const GatherInfo &G, const uint32_t *ent, uint32_t n, uint32_t row_ref,
                                             unsigned long long pos_ref, int lane, ScratchHdr *hdr) {
  const uint64_t cap = G.capacity;
  for (uint32_t t0 = 0; t0 < n; t0 += 128) {
    uint32_t row[4];
    unsigned long long pos[4];
    uint32_t ok = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint32_t t = t0 + 32u * k + (uint32_t)lane;
      row[k] = 0;
      pos[k] = 0;
      if (t < n) {
        const uint32_t e = ent[t];
        row[k] = row_ref + (e >> 16);
        pos[k] = pos_ref + (e & 0xffffu);
        if (pos[k] < cap && ESC_INB(hdr, row[k] < G.nrows, 22, row[k])) ok |= 1u << k;
      }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if ((ok >> k) & 1u) G.out_ids[pos[k]] = row[k];
    for (int c = 0; c < G.nproj; ++c) {
      const int w = G.proj_w[c];
      const uint8_t *src = G.proj_ptr[c];
      void *dst = G.out_proj[c];
      uint64_t v[4];
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if ((ok >> k) & 1u) v[k] = load_elem(src, row[k], w);
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if ((ok >> k) & 1u) store_elem(dst, pos[k], v[k], w);
    }
  }
}

// One dense group, the whole warp.  The projected columns of all 256 rows
// arrive together (16-byte asynchronous copies, at most kRawBytes at a
// time; a column wider than that is read in place); each output slot then
// takes its row's value from shared memory, so that the stores coalesce.
__device__ __forceinline__ void dense_group(const GatherInfo &G, WriteWarpSmem &W, int j, uint32_t g, uint32_t cnt,
                                            unsigned long long base, int lane, ScratchHdr *hdr) {
  const uint64_t cap = G.capacity;
  // rows 8l .. 8l+7 of the group: bits 2(l/8), 2(l/8)+1 of bytes 4(l%8) ..
  // 4(l%8)+3 (word l%8 of the lane-major bitmap), packed in row order
  uint32_t x = (W.words[j][lane & 7] >> (2u * ((uint32_t)lane >> 3))) & 0x03030303u;
  x = (x | (x >> 6)) & 0x000f000fu;
  const uint32_t bits8 = (x | (x >> 12)) & 0xffu;
  const uint32_t cl = __popc(bits8);
  uint32_t incl = cl;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(FULL, incl, o);
    if (lane >= o) incl += y;
  }
  uint32_t r = incl - cl;
#pragma unroll
  for (int k = 0; k < 8; ++k)
    if (((bits8 >> k) & 1u) && ESC_INB(hdr, r < (uint32_t)kGroup, 24, r)) W.sids[r++] = 8u * (uint32_t)lane + (uint32_t)k;
  const uint32_t grow = g * kGroup;
  const int np = G.nproj;
  int c0 = 0;
  do {
    // columns c0 .. c1-1 share the buffer (a single column always goes, in place if too wide)
    int c1 = c0;
    uint32_t off = 0;
    while (c1 < np && (c1 == c0 || off + kGroup * G.proj_w[c1] <= kRawBytes)) off += kGroup * G.proj_w[c1++];
    const bool staged = off <= kRawBytes;
    if (staged) {
      off = 0;
      for (int c = c0; c < c1; ++c) {
        const uint32_t bytes = kGroup * G.proj_w[c];
        const uint8_t *src = G.proj_ptr[c] + (size_t)grow * G.proj_w[c];
        for (uint32_t x = 16u * (uint32_t)lane; x < bytes; x += 512u) cp_async16(W.raw + off + x, src + x);
        off += bytes;
      }
    }
    if (c0 == 0) {
      __syncwarp();
      for (uint32_t t = (uint32_t)lane; t < cnt; t += 32)
        if (base + t < cap) G.out_ids[base + t] = grow + W.sids[t];
    }
    if (staged) cp_async_wait_all();
    __syncwarp();
    off = 0;
    for (int c = c0; c < c1; ++c) {
      const int w = G.proj_w[c];
      void *dst = G.out_proj[c];
      const uint8_t *col = staged ? W.raw + off : G.proj_ptr[c] + (size_t)grow * w;
      for (uint32_t t = (uint32_t)lane; t < cnt; t += 32)
        if (base + t < cap) store_elem(dst, base + t, load_elem(col, W.sids[t], w), w);
      off += kGroup * w;
    }
    __syncwarp();
    c0 = c1;
  } while (c0 < np);
}

// Look-back words: flag in bits 63..62 (2 = inclusive prefix published),
// the value below.
constexpr unsigned long long kLookFinal = 2ull << 62, kLookValue = (1ull << 62) - 1;
constexpr int kLookPerThread = 4;

// One look-back window: this thread's units idx - kLookPerThread*t - k; a
// unit before the first reads as a published prefix of 0.
__device__ __forceinline__ void lookback_load(const unsigned long long *st, const unsigned long long *tot,
                                              long long idx, unsigned long long (&w)[kLookPerThread],
                                              unsigned long long (&t)[kLookPerThread]) {
#pragma unroll
  for (int k = 0; k < kLookPerThread; ++k) {
    const long long j = idx - (long long)kLookPerThread * threadIdx.x - k;
    w[k] = kLookFinal;
    t[k] = 0;
    if (j >= 0) {
      w[k] = ld_relaxed(&st[j]);
      t[k] = __ldcg(&tot[j]);
    }
  }
}

__global__ void __launch_bounds__(kWriteThreads, kWriteBlocksPerSm) write_kernel(const __grid_constant__ Launch L) {
  extern __shared__ __align__(16) uint8_t wsmem[];
  __shared__ GatherInfo G;
  __shared__ uint32_t wsum[kWriteWarps];
  __shared__ unsigned long long lb_val[2][kWriteWarps];  // look-back rounds, by parity
  __shared__ uint32_t lb_hit[2][kWriteWarps];
  __shared__ int s_q;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  WriteWarpSmem &W = reinterpret_cast<WriteWarpSmem *>(wsmem)[warp];
  if (threadIdx.x == 0) s_q = block_query(L, [](const Query *q) { return q->wunit_base; });
  __syncthreads();
  const Query *Q = query_ptr(L, s_q);
  if (warp == 1) {
    const int np = Q->nproj;
    if (lane == 0) {
      G.capacity = Q->capacity;
      G.out_ids = Q->out_ids;
      G.tiles_left = Q->tiles_left;
      G.done_ns = Q->done_ns;
      G.nrows = Q->nrows;
      G.nproj = np;
    }
    if (lane < np) {
      G.proj_w[lane] = Q->proj_w[lane];
      G.proj_ptr[lane] = Q->proj_ptr[lane];
      G.out_proj[lane] = Q->out_proj[lane];
    }
  }
  const uint32_t u = blockIdx.x - Q->wunit_base;
  if (!ESC_INB(L.hdr, u < Q->nwunits, 20, u)) return;  // uniform: the whole block
  const uint32_t urows = Q->wunit_groups * kGroup;
  const uint32_t urow0 = u * urows;
  const uint32_t rows = min(urows, Q->nrows - urow0);
  const int ng = (int)((rows + kGroup - 1) / kGroup);
  const uint32_t g0 = urow0 / kGroup;
  // warp w: groups w*gpw .. w*gpw+gpw-1 of the unit, lane = group
  const int gpw = (ng + kWriteWarps - 1) / kWriteWarps;
  const int gi = warp * gpw + lane;
  const bool valid = lane < gpw && gi < ng;
  const uint32_t grp_l = g0 + (uint32_t)gi;
  // Everything the block reads of the scan's output is requested at once:
  // the unit's total, the bitmap words of this thread's group (the scan
  // wrote all 8 words of every group) and the first look-back window.
  const unsigned long long *tot = Q->unit_total;
  unsigned long long *st = Q->unit_status;
  const unsigned long long utot = __ldcg(&tot[u]);
  uint4 wlo = make_uint4(0, 0, 0, 0), whi = wlo;
  if (valid && ESC_INB(L.hdr, grp_l < (uint64_t)Q->ntiles * Q->gmax, 21, grp_l)) {
    const uint4 *bw = reinterpret_cast<const uint4 *>(Q->bitmap + (size_t)grp_l * 8);
    wlo = __ldcg(bw);
    whi = __ldcg(bw + 1);
  }
  long long idx = (long long)u - 1;  // closest predecessor not yet accounted
  unsigned long long lw[kLookPerThread], lt[kLookPerThread];
  lookback_load(st, tot, idx, lw, lt);
  if (utot == 0) {
    // no qualifying row in this unit: nothing to write, nothing to publish
    if (Q->done_ns && threadIdx.x == 0) {
      __threadfence();
      if (atomicSub(Q->tiles_left, 1u) == 1u) *Q->done_ns = globaltimer();
    }
    return;
  }
  const uint32_t c = __popc(wlo.x) + __popc(wlo.y) + __popc(wlo.z) + __popc(wlo.w) + __popc(whi.x) +
                     __popc(whi.y) + __popc(whi.z) + __popc(whi.w);
  uint32_t inc = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(FULL, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) wsum[warp] = inc;
  // The unit's first slot: a decoupled look-back over the unit totals, all
  // of them final (the scan wrote them), so it never waits.  Each round the
  // whole block covers kLookPerThread * kWriteThreads predecessors (thread t:
  // units idx - kLookPerThread*t - k, closest first) and stops at the
  // closest one whose inclusive prefix another block has published.
  unsigned long long excl = 0;
  for (int r = 0;; ++r) {
    if (r > 0) lookback_load(st, tot, idx, lw, lt);
    unsigned long long sum = 0, pval = 0;  // totals before the thread's closest published prefix
    int kp = kLookPerThread;               // that prefix among the thread's units (none: kLookPerThread)
#pragma unroll
    for (int k = 0; k < kLookPerThread; ++k) {
      if (kp == kLookPerThread) {
        if ((lw[k] >> 62) == 2) {
          kp = k;
          pval = lw[k] & kLookValue;
        } else {
          sum += lt[k];
        }
      }
    }
    const uint32_t pm = __ballot_sync(FULL, kp < kLookPerThread);
    const int first = pm ? __ffs(pm) - 1 : 32;
    const unsigned long long v = warp_sum(lane < first ? sum : lane == first ? sum + pval : 0ull);
    if (lane == 0) {
      lb_val[r & 1][warp] = v;
      lb_hit[r & 1][warp] = pm != 0u;
    }
    __syncthreads();  // also publishes wsum and G
    bool found = false;
#pragma unroll 1
    for (int w = 0; w < kWriteWarps && !found; ++w) {
      excl += lb_val[r & 1][w];
      found = lb_hit[r & 1][w] != 0;
    }
    if (found) break;
    idx -= (long long)kLookPerThread * kWriteThreads;
  }
  if (threadIdx.x == 0) st_relaxed(&st[u], kLookFinal | (excl + utot));
  uint32_t wbase = 0;
  for (int i = 0; i < warp; ++i) wbase += wsum[i];
  if (wsum[warp] != 0) {
    const unsigned long long pos_ref = excl + wbase;        // first slot of the warp's groups
    const unsigned long long base_l = pos_ref + inc - c;    // first slot of this lane's group
    const uint32_t grow_l = grp_l * kGroup;
    const bool dense_l = valid && c >= kDenseMin && grow_l + kGroup <= G.nrows;
    const uint32_t dm0 = __ballot_sync(FULL, dense_l);
    if (dm0) {
      *reinterpret_cast<uint4 *>(&W.words[lane][0]) = wlo;
      *reinterpret_cast<uint4 *>(&W.words[lane][4]) = whi;
      __syncwarp();
    }
    for (uint32_t dm = dm0; dm; dm &= dm - 1) {
      const int j = __ffs(dm) - 1;
      const unsigned long long base = __shfl_sync(FULL, base_l, j);
      if (base < G.capacity)
        dense_group(G, W, j, __shfl_sync(FULL, grp_l, j), __shfl_sync(FULL, c, j), base, lane, L.hdr);
    }
    // the other groups: lane = group, entries staged in slot order
    const uint32_t sc = dense_l ? 0u : c;
    uint32_t sx = sc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(FULL, sx, o);
      if (lane >= o) sx += y;
    }
    const uint32_t stot = __shfl_sync(FULL, sx, 31);
    sx -= sc;
    if (stot != 0) {
      const uint32_t row_ref = (g0 + (uint32_t)(warp * gpw)) * kGroup;
      const uint32_t rrel = grow_l - row_ref;
      const uint32_t srel = (uint32_t)(base_l - pos_ref);
      uint32_t *ent = reinterpret_cast<uint32_t *>(W.raw);
      for (uint32_t win = 0; win < stot; win += kStageEntries) {
        const uint32_t wend = win + kStageEntries;
        if (sc != 0 && sx < wend && sx + sc > win) {
          // the group's first sc set bits are its rows: never read past sc
          const uint32_t eend = min(wend, sx + sc);
          uint32_t e = sx;  // staged index of this lane's next entry
          // rows in order: block j (rows 64j .. 64j+63) is bits 2j, 2j+1 of the
          // 32 bytes (byte l: rows 64j + 2l + {0, 1}); words in order, bits
          // ascending within a word, is row order
#pragma unroll 1
          for (uint32_t jb = 0; jb < 4; ++jb) {
#pragma unroll
            for (uint32_t wi = 0; wi < 8; ++wi) {
              const uint4 &h = wi < 4 ? wlo : whi;
              const uint32_t wv = (wi & 3) == 0 ? h.x : (wi & 3) == 1 ? h.y : (wi & 3) == 2 ? h.z : h.w;
              for (uint32_t xm = wv & (0x03030303u << (2 * jb)); xm != 0u && e < eend; xm &= xm - 1u, ++e) {
                const uint32_t bpos = (uint32_t)__ffs(xm) - 1u;  // 8 * byte + 2j + i
                const uint32_t rr = 64u * jb + 2u * (4u * wi + (bpos >> 3)) + ((bpos & 7u) - 2u * jb);
                if (e >= win && ESC_INB(L.hdr, e - win < kStageEntries, 23, e - win))
                  ent[e - win] = ((rrel + rr) << 16) | (srel + e - sx);
              }
            }
          }
        }
        __syncwarp();
        flush_sparse(G, ent, min(stot - win, kStageEntries), row_ref, pos_ref, lane, L.hdr);
        __syncwarp();
      }
    }
  }
  // per-query completion time: the query's last write block
  if (G.done_ns) {
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      if (atomicSub(G.tiles_left, 1u) == 1u) *G.done_ns = globaltimer();
    }
  }
}

// ------------------------------------------------------------------ the shared scan
// Count-only sub-queries of several predicates on one table with one pass
// over it: each tile of the union of the columns they read is staged once
// (the scan kernel's producer), and every predicate is evaluated on it.
// L.q0 is the union layout (columns, tile and unit sizes; no program);
// L.queries holds the nq predicates, compiled against that layout (their
// stage offsets point into the union stage).  Consumers claim (predicate,
// pair of groups) items of a stage predicate-major -- consecutive items of a
// warp share a program, which stays in L1 -- and add each predicate's count
// into shared counters, flushed once per CTA into L.queries[k].count.
constexpr int kSharedMaxQueries = 2048;

struct SharedSmem {
  static constexpr size_t stages = 0;
  static constexpr size_t bars = stages + (size_t)kStages * kStageBytes;
  static constexpr size_t meta = bars + 2 * kStages * 8;
  static constexpr size_t take = meta + kStages * sizeof(StageMeta);
  static constexpr size_t cnt = (take + kStages * 4 + 15) & ~(size_t)15;
  static constexpr size_t total = cnt + kSharedMaxQueries * 4;
};

__global__ void __launch_bounds__(kThreads, 1) shared_kernel(const __grid_constant__ Launch L) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t *stages = smem + SharedSmem::stages;
  uint64_t *full_bar = reinterpret_cast<uint64_t *>(smem + SharedSmem::bars);
  uint64_t *empty_bar = full_bar + kStages;
  StageMeta *meta = reinterpret_cast<StageMeta *>(smem + SharedSmem::meta);
  uint32_t *take = reinterpret_cast<uint32_t *>(smem + SharedSmem::take);
  uint32_t *cnt = reinterpret_cast<uint32_t *>(smem + SharedSmem::cnt);
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  ScratchHdr *hdr = L.hdr;
  const Query &Y = L.q0;  // the union layout
  const int nq = L.nq;
  for (int k = threadIdx.x; k < nq; k += blockDim.x) cnt[k] = 0;
  if (threadIdx.x == 0) {
    for (int st = 0; st < kStages; ++st) {
      mbar_init(&full_bar[st], 1);
      mbar_init(&empty_bar[st], kConsumers);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  if (warp == 0) {
    // ---------------------------------------------------------------- producer
    int s = 0;
    uint32_t phase = 0;
    bool done = false;
    uint32_t u_next = 0, dead_next = 0;
    if (lane == 0) u_next = atomicAdd(&hdr->ticket, 1u);
    while (!done) {
      uint32_t u = 0, dead = 0;
      if (lane == 0) {
        u = u_next;
        dead = dead_next;
        if (u < L.total_units && !dead) {
          u_next = atomicAdd(&hdr->ticket, 1u);
          dead_next = aborted(hdr) ? 1u : 0u;
        }
      }
      u = __shfl_sync(FULL, u, 0);
      dead = __shfl_sync(FULL, dead, 0);
      if (u >= L.total_units || dead) {
        if (mbar_wait(&empty_bar[s], phase ^ 1u, hdr, kWaitLimitNs, true) && lane == 0) {
          meta[s].q = -1;
          mbar_arrive(&full_bar[s]);
        }
        break;
      }
      uint32_t t0, t1;
      unit_range(Y, u, t0, t1);
      for (uint32_t tile = t0; tile < t1; ++tile) {
        if (!mbar_wait(&empty_bar[s], phase ^ 1u, hdr, kWaitLimitNs, true)) {
          done = true;
          break;
        }
        const uint32_t r0 = tile * Y.tile_rows;
        const uint32_t rows = min(Y.tile_rows, Y.nrows - r0);
        uint8_t *stage = stages + (size_t)s * kStageBytes;
        uint32_t bulk = 0, tail = 0;
        const uint8_t *src = nullptr;
        uint8_t *dst = nullptr;
        const int nref = Y.nref;
        if (lane < nref) {
          const uint32_t w = Y.ref_w[lane];
          const uint32_t bytes = rows * w;
          bulk = bytes & ~15u;
          tail = bytes - bulk;
          src = Y.ref_ptr[lane] + (size_t)r0 * w;
          dst = stage + Y.stage_off[lane];
        }
        if (__ballot_sync(FULL, tail != 0)) {
          for (int c = 0; c < nref; ++c) {
            const uint32_t tb = __shfl_sync(FULL, tail, c);
            const uint32_t bb = __shfl_sync(FULL, bulk, c);
            const uint8_t *sp = reinterpret_cast<const uint8_t *>(__shfl_sync(FULL, (unsigned long long)src, c));
            uint8_t *dp = reinterpret_cast<uint8_t *>(__shfl_sync(FULL, (unsigned long long)dst, c));
            if ((uint32_t)lane < tb) dp[bb + lane] = sp[bb + lane];
          }
          fence_proxy_async_smem();
        }
        const uint32_t tot = __reduce_add_sync(FULL, bulk);
        __syncwarp();
        if (lane == 0) {
          StageMeta &m = meta[s];
          take[s] = 0;
          m.q = 0;
          m.tile = tile;
          m.rows = rows;
          m.dead = dead;
          mbar_arrive_expect_tx(&full_bar[s], tot);
        }
        __syncwarp();
        if (bulk) bulk_load(dst, src, bulk, &full_bar[s]);
        if (++s == kStages) {
          s = 0;
          phase ^= 1u;
        }
      }
    }
    return;
  }

  // ---------------------------------------------------------------- consumers
  int s = 0;
  uint32_t phase = 0;
  int acc_q = -1;
  uint32_t acc = 0;
  while (true) {
    const bool got = mbar_wait(&full_bar[s], phase, hdr);
    const StageMeta mt = meta[s];
    if (!got || mt.q < 0) break;
    if (mt.dead == 0) {
      const uint8_t *stage = stages + (size_t)s * kStageBytes;
      const uint32_t rows = mt.rows;
      const int ngroups = (int)((rows + kGroup - 1) / kGroup);
      const int npairs = (ngroups + 1) >> 1;
      const int items = npairs * nq;
      for (;;) {
        int j = 0;
        if (lane == 0) j = (int)atomicAdd(&take[s], 1u);
        j = __shfl_sync(FULL, j, 0);
        if (j >= items) break;
        const int qi = j / npairs;
        const int g = 2 * (j - qi * npairs), g1 = g + 1;
        if (qi != acc_q) {
          const uint32_t t = __reduce_add_sync(FULL, acc);
          if (lane == 0 && t) atomicAdd(&cnt[acc_q], t);
          acc = 0;
          acc_q = qi;
        }
        const int gs[2] = {g, g1 < ngroups ? g1 : g};
        uint32_t mm[2];
        eval_groups<2, true>(&L.queries[qi], stage, gs, lane, mm);
        acc += __popc(mm[0] & valid_mask(g, lane, rows));
        if (g1 < ngroups) acc += __popc(mm[1] & valid_mask(g1, lane, rows));
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty_bar[s]);
    if (++s == kStages) {
      s = 0;
      phase ^= 1u;
    }
  }
  if (acc_q >= 0) {
    const uint32_t t = __reduce_add_sync(FULL, acc);
    if (lane == 0 && t) atomicAdd(&cnt[acc_q], t);
  }
  // the consumer warps only (the producer has returned): then flush
  asm volatile("bar.sync 1, %0;" ::"r"(kConsumers * 32) : "memory");
  for (int k = (int)threadIdx.x - 32; k < nq; k += kConsumers * 32)
    if (cnt[k]) atomicAdd(L.queries[k].count, (unsigned long long)cnt[k]);
}

// A program that reads no column is a constant (the compiler folded it:
// e.g. a conjunction of contradictory tests): its result needs no scan.
// Writes the count, and for a constant TRUE the caller's bitmap words or the
// materialised rows (ids 0.., projected columns copied); FALSE leaves rows
// unwritten and the bitmap zero.
__device__ __forceinline__ void const_body(const Query &q, uint32_t value, uint64_t tid, uint64_t stride) {
  const uint64_t n = value ? q.nrows : 0u;
  if (tid == 0) *q.count = n;
  if (q.mode == MODE_BITMAP) {
    const uint32_t nwords = (q.nrows + 31u) / 32u, tail = q.nrows & 31u;
    for (uint64_t w = tid; w < nwords; w += stride)
      q.bitmap[w] = !value ? 0u : (w + 1 == nwords && tail) ? (1u << tail) - 1u : ~0u;
  } else if (q.mode == MODE_SELECT && value) {
    const uint64_t m = min(n, (uint64_t)q.capacity);
    for (uint64_t i = tid; i < m; i += stride) {
      q.out_ids[i] = (uint32_t)i;
      for (int c = 0; c < q.nproj; ++c)
        store_elem(q.out_proj[c], i, load_elem(q.proj_ptr[c], (uint32_t)i, q.proj_w[c]), q.proj_w[c]);
    }
  }
}

__global__ void __launch_bounds__(256) const_kernel(const __grid_constant__ Launch L, uint32_t value) {
  const_body(L.q0, value, (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, (uint64_t)gridDim.x * blockDim.x);
}

// The constant sub-queries of a batch: blockIdx.y indexes cidx (the batch's
// constant queries), kConstBlocks blocks each; the last block of a query
// records its completion time.
constexpr int kConstBlocks = 32;
__global__ void __launch_bounds__(256) const_batch_kernel(const Query *queries, const uint32_t *cidx, uint32_t y0) {
  const Query &q = queries[cidx[y0 + blockIdx.y]];
  const_body(q, q.const_value, (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, (uint64_t)gridDim.x * blockDim.x);
  if (q.done_ns) {
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      if (atomicSub(q.tiles_left, 1u) == 1u) *q.done_ns = globaltimer();
    }
  }
}

// A kernel whose only job is a bounded wait on a flag that nothing sets.
__global__ void wait_selftest_kernel(const unsigned *flag, ScratchHdr *hdr, uint64_t limit_ns) {
  const uint64_t t0 = globaltimer();
  while (*(volatile const unsigned *)flag == 0u) {
    __nanosleep(1000);
    if (globaltimer() - t0 > limit_ns) {
      if (threadIdx.x == 0) raise_status(hdr, ESC_ETIMEOUT);
      return;
    }
  }
}

__global__ void timestamp_kernel(unsigned long long *out) { *out = globaltimer(); }

// ------------------------------------------------------------------ host side
namespace {

std::mutex g_mu;
struct DeviceState {
  bool ready = false;
  int sms = 0;
  int blocks_per_sm = 0;
  cudaMemPool_t pool = nullptr;
};
DeviceState g_dev[64];

size_t smem_bytes() { return SmemLayout::total; }

#define ESC_CK(call)                                                                      \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(ESC_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));          \
  } while (0)

// The scan kernel instance of block shape S (an index into kScanShapes).
template <int S>
struct ScanInstance {
  static constexpr ScanShape sh = kScanShapes[S];
  static constexpr int threads = 32 * (sh.consumers + 1);
  static const void *fn() { return reinterpret_cast<const void *>(scan_kernel<sh.consumers, sh.udf, sh.groups>); }
  static void launch(uint32_t grid, const Launch &L, cudaStream_t st) {
    scan_kernel<sh.consumers, sh.udf, sh.groups><<<grid, threads, smem_bytes(), st>>>(L);
  }
};
static_assert(kNumScanShapes == 5, "one ScanInstance per shape below");

// Launches the scan kernel instance of block shape `shape`.
void launch_scan_shape(int shape, uint32_t grid, const Launch &L, cudaStream_t st) {
  switch (shape) {
    case 0: ScanInstance<0>::launch(grid, L, st); break;
    case 1: ScanInstance<1>::launch(grid, L, st); break;
    case 2: ScanInstance<2>::launch(grid, L, st); break;
    case 3: ScanInstance<3>::launch(grid, L, st); break;
    default: ScanInstance<4>::launch(grid, L, st); break;
  }
}

// Kernel attributes (dynamic shared memory) of every kernel of this file,
// and the CTAs per SM that every scan instance reaches.
esc_status configure_kernels(int *blocks_per_sm) {
  const void *fns[kNumScanShapes] = {ScanInstance<0>::fn(), ScanInstance<1>::fn(), ScanInstance<2>::fn(),
                                     ScanInstance<3>::fn(), ScanInstance<4>::fn()};
  const int threads[kNumScanShapes] = {ScanInstance<0>::threads, ScanInstance<1>::threads, ScanInstance<2>::threads,
                                       ScanInstance<3>::threads, ScanInstance<4>::threads};
  int b = 1 << 30;
  for (int i = 0; i < kNumScanShapes; ++i) {
    ESC_CK(cudaFuncSetAttribute(fns[i], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes()));
    int k = 0;
    ESC_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&k, fns[i], threads[i], smem_bytes()));
    b = std::min(b, k);
  }
  if (b < 1) return fail(ESC_ECUDA, "a scan kernel instance does not fit on an SM");
  ESC_CK(cudaFuncSetAttribute(write_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWriteSmem));
  ESC_CK(cudaFuncSetAttribute(shared_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SharedSmem::total));
  *blocks_per_sm = b;
  return ESC_OK;
}

}  // namespace

esc_status device_state(DeviceState **out) {
  int dev = 0;
  ESC_CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(ESC_EINVAL, "device index out of range");
  std::lock_guard<std::mutex> lk(g_mu);
  DeviceState &d = g_dev[dev];
  if (!d.ready) {
    ESC_CK(cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev));
    esc_status cs = configure_kernels(&d.blocks_per_sm);
    if (cs != ESC_OK) return cs;
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof props);
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    ESC_CK(cudaMemPoolCreate(&d.pool, &props));
    uint64_t thr = ~0ull;
    ESC_CK(cudaMemPoolSetAttribute(d.pool, cudaMemPoolAttrReleaseThreshold, &thr));
    d.ready = true;
  }
  *out = &d;
  return ESC_OK;
}

// Tile size for a query: as many rows as fit in one stage, a multiple of the
// 256-row group, at most kMaxTileRows.
// The value of a program that reads no column (TRUE, FALSE and connectives
// only); false when the program reads a column.
// Whether the program has a udf test: it then needs a scan kernel instance
// with the udf path.
bool program_has_udf(const Query &q) {
  for (int i = 0; i < q.ninstr; ++i)
    if (q.code[i].op == OP_UDF) return true;
  return false;
}

uint32_t read_bytes_per_row(const Query &q) {
  uint32_t b = 0;
  for (int i = 0; i < q.nref; ++i) b += q.ref_w[i];
  return b;
}

// The block shape a single sub-query's scan uses: the predicate's tuning
// (validated when it was set), else the automatic one.
int query_shape(const Query &q, const esc_tuning &tu) {
  const bool udf = program_has_udf(q);
  const uint32_t b = read_bytes_per_row(q);
  const int s = scan_shape_for(tu.consumer_warps, tu.rows_per_pass, udf, b);
  return s >= 0 ? s : auto_scan_shape(udf, b > kWideBytes);
}

// The block shape of a launch that scans several queries (a batch or one
// of its waves): the automatic shape, with the udf path if any program has
// a udf, for wide programs if they hold most of the launch's bytes.
int launch_shape(const Query *qs, int n) {
  bool udf = false;
  uint64_t wide = 0, all = 0;
  for (int i = 0; i < n; ++i) {
    if (qs[i].is_const) continue;
    udf = udf || program_has_udf(qs[i]);
    const uint64_t w = (uint64_t)qs[i].nrows * read_bytes_per_row(qs[i]);
    all += w;
    if (read_bytes_per_row(qs[i]) > kWideBytes) wide += w;
  }
  return auto_scan_shape(udf, 2 * wide > all);
}

bool program_constant(const Query &q, uint32_t *value) {
  if (q.nref != 0) return false;
  uint8_t stack[kMaxDepth + 1];
  int sp = 0;
  for (int pc = 0; pc < q.ninstr; ++pc) {
    switch (q.code[pc].op) {
      case OP_TRUE:
      case OP_FALSE:
        if (sp > kMaxDepth) return false;
        stack[sp++] = q.code[pc].op == OP_TRUE ? 1 : 0;
        break;
      case OP_NOT:
        if (sp < 1) return false;
        stack[sp - 1] ^= 1;
        break;
      case OP_AND:
      case OP_OR:
        if (sp < 2) return false;
        --sp;
        stack[sp - 1] = q.code[pc].op == OP_AND ? (stack[sp - 1] & stack[sp]) : (stack[sp - 1] | stack[sp]);
        break;
      case OP_JZ:
      case OP_JNZ:
        break;  // a jump only skips work whose result is already decided
      default:
        return false;
    }
  }
  if (sp != 1) return false;
  *value = stack[0];
  return true;
}

// Batch builders: a query whose program is constant gets no work units (the
// scan and write kernels skip it) and is answered by const_batch_kernel.
void mark_constant(Query &q) {
  uint32_t v = 0;
  if (!program_constant(q, &v)) return;
  q.is_const = 1;
  q.const_value = v;
  q.nunits = 0;
  q.nwunits = 0;
  q.ntiles = 0;
}

esc_status launch_const_batch(const Query *dev_queries, const uint32_t *dev_cidx, uint32_t nconst, cudaStream_t st) {
  for (uint32_t y0 = 0; y0 < nconst; y0 += 65535u) {
    const dim3 grid(kConstBlocks, std::min<uint32_t>(65535u, nconst - y0));
    const_batch_kernel<<<grid, 256, 0, st>>>(dev_queries, dev_cidx, y0);
    ESC_CK(cudaGetLastError());
  }
  return ESC_OK;
}

esc_status launch_const(const Launch &L, uint32_t value, cudaStream_t st) {
  DeviceState *d;
  esc_status s = device_state(&d);
  if (s != ESC_OK) return s;
  const Query &q = L.q0;
  const uint64_t work = q.mode == MODE_BITMAP ? (q.nrows + 31u) / 32u
                        : (q.mode == MODE_SELECT && value) ? std::min<uint64_t>(q.nrows, q.capacity) : 0;
  const uint32_t grid = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)d->sms * 8, (work + 255) / 256));
  const_kernel<<<grid, 256, 0, st>>>(L, value);
  ESC_CK(cudaGetLastError());
  return ESC_OK;
}

uint32_t tile_rows_for(const Query &q, const esc_tuning &tu) {
  uint32_t bpr = 0;
  for (int i = 0; i < q.nref; ++i) bpr += q.ref_w[i];
  if (bpr == 0) bpr = 1;
  uint32_t t = (kStageBytes / bpr / kGroup) * kGroup;
  t = std::max<uint32_t>(t, kGroup);
  return std::min<uint32_t>(std::min<uint32_t>(t, kMaxTileRows), tu.max_tile_rows);
}

// Compaction units: one write-kernel block each.  slots == 0: units of
// kMaxUnitGroups groups.  Otherwise the fewest whole waves of `slots` blocks
// that full-size units need, with units just large enough to fill them: the
// write kernel's blocks take about equal time, so a last wave only partly
// full would leave that share of the GPU idle for a whole block's time.
void layout_write_units(Query &q, int slots) {
  const uint64_t ngroups = ((uint64_t)q.nrows + kGroup - 1) / kGroup;
  uint64_t ug = kMaxUnitGroups;
  if (slots > 0) {
    const uint64_t wave = (uint64_t)slots * kMaxUnitGroups;
    const uint64_t waves = std::max<uint64_t>(1, (ngroups + wave - 1) / wave);
    ug = std::min<uint64_t>(kMaxUnitGroups, std::max<uint64_t>(1, (ngroups + waves * slots - 1) / (waves * slots)));
  }
  q.wunit_groups = (uint32_t)ug;
  // group g's unit is g / ug = umulhi(g, ceil(2^32 / ug)): with ug * M = 2^32 + e,
  // e < ug, the quotient is exact while g * e < 2^32, and every group index
  // (< ESC_MAX_ROWS / 256 < 2^24) keeps g * 255 below 2^32
  q.wunit_recip = ug > 1 ? (uint32_t)(((1ull << 32) + ug - 1) / ug) : 0u;
  q.nwunits = (uint32_t)((ngroups + ug - 1) / ug);
}

// Stage layout (read columns back to back, each slice 128-byte aligned), the
// work units (consecutive tiles claimed with one ticket: at most ~512 KB of
// staged columns, >= 8 per SM when the table is large enough), and the
// compaction units (layout_write_units).
void layout_stage(Query &q, int sms, const esc_tuning &tu = kDefaultTuning) {
  q.tile_rows = tile_rows_for(q, tu);
  uint32_t off = 0, bpr = 0;
  for (int i = 0; i < q.nref; ++i) {
    q.stage_off[i] = off;
    off += (q.tile_rows * q.ref_w[i] + 127u) & ~127u;
    bpr += q.ref_w[i];
  }
  for (int pc = 0; pc < q.ninstr; ++pc) {  // resolve operand slots to stage offsets
    Instr &I = q.code[pc];
    if (I.op == OP_RANGE || I.op == OP_IN || I.op == OP_INSET || I.op == OP_UDF) I.soff = (uint16_t)q.stage_off[I.ref];
    if (I.op == OP_UDF) I.soff2 = (uint16_t)q.stage_off[I.ref2];
  }
  // nrows <= ESC_MAX_ROWS (2^32 - 2^16): the rounded-up extents here and in
  // the kernels (tiles, groups, 32-bit words, compaction units) stay below 2^32
  q.ntiles = (q.nrows + q.tile_rows - 1) / q.tile_rows;
  q.gmax = q.tile_rows / kGroup;
  const uint64_t tile_bytes = (uint64_t)q.tile_rows * std::max<uint32_t>(bpr, 1);
  const uint32_t max_ut = (uint32_t)std::max<uint64_t>(
      1, std::min<uint64_t>((uint64_t)tu.max_unit_kb * 1024 / tile_bytes, (uint64_t)kMaxUnitRows / q.tile_rows));
  const uint32_t want = q.ntiles / (uint32_t)std::max(1, sms * tu.units_per_sm);
  q.unit_tiles = std::min(std::max<uint32_t>(want, 1), max_ut);
  // the last kTailTilesPerSm tiles per SM go out one tile per unit
  const uint32_t tail = std::min<uint32_t>(q.ntiles, (uint32_t)(kTailTilesPerSm * sms));
  q.unit_big = (q.ntiles - tail) / q.unit_tiles;
  q.nunits = q.unit_big + (q.ntiles - q.unit_big * q.unit_tiles);
  layout_write_units(q, sms * kWriteBlocksPerSm);
}


esc_status alloc_async(void **p, size_t bytes, cudaStream_t st) {
  DeviceState *d;
  esc_status s = device_state(&d);
  if (s != ESC_OK) return s;
  if (inject_alloc_failure()) return fail(ESC_ENOMEM, "device scratch allocation: injected failure (esc_debug_fail_allocs)");
  cudaError_t e = cudaMallocFromPoolAsync(p, bytes, d->pool, st);
  if (e != cudaSuccess) return fail(ESC_ENOMEM, std::string("device scratch allocation: ") + cudaGetErrorString(e));
  return ESC_OK;
}

// shape: the block shape (kScanShapes) of the instance that runs the launch.
esc_status launch_scan(const Launch &L, int shape, cudaStream_t st) {
  DeviceState *d;
  esc_status s = device_state(&d);
  if (s != ESC_OK) return s;
  if (L.total_units == 0) return ESC_OK;
  const uint32_t cap = (uint32_t)(d->sms * d->blocks_per_sm);
  const uint32_t grid = std::min<uint32_t>(cap, L.total_units);
  launch_scan_shape(shape, grid, L, st);
  ESC_CK(cudaGetLastError());
  return ESC_OK;
}

// Second pass of compaction: the write kernel, one block per compaction unit.
esc_status launch_write(const Launch &L, uint32_t unit_blocks, cudaStream_t st) {
  if (unit_blocks == 0) return ESC_OK;
  write_kernel<<<unit_blocks, kWriteThreads, kWriteSmem, st>>>(L);
  ESC_CK(cudaGetLastError());
  return ESC_OK;
}

// Compaction scratch of one query: unit totals and look-back words (both
// zeroed before the scan), then the selection bitmap (the scan writes every
// word before the write kernel reads it).
size_t select_zeroed_bytes(const Query &q) { return ((size_t)q.nwunits * 16 + 255) & ~(size_t)255; }
size_t select_other_bytes(const Query &q) {
  const size_t groups = (size_t)q.ntiles * q.gmax;
  return (groups * 32 + 255) & ~(size_t)255;
}
void select_bind(Query &q, uint8_t *zeroed, uint8_t *other) {
  q.unit_total = reinterpret_cast<unsigned long long *>(zeroed);
  q.unit_status = q.unit_total + q.nwunits;
  q.bitmap = reinterpret_cast<uint32_t *>(other);
}

// Validates a (table, pred, rows) call and fills the per-call query.
esc_status prepare_query(const esc_table *t, const esc_pred *p, const esc_rows *rows, int mode, Query *q) {
  if (!t || !p) return fail(ESC_EINVAL, "table and predicate are required");
  DeviceState *d;
  esc_status ds = device_state(&d);
  if (ds != ESC_OK) return ds;
  if (p->table != t) return fail(ESC_EINVAL, "predicate was compiled against another table");
  std::memset(q, 0, sizeof *q);
  fill_query_program(p, q);
  q->nrows = (uint32_t)t->nrows;
  q->mode = mode;
  if (mode == MODE_SELECT) {
    if (!rows) return fail(ESC_EINVAL, "rows is NULL");
    if (rows->capacity > 0 && !rows->row_ids) return fail(ESC_EINVAL, "rows->row_ids is NULL");
    if (q->nproj > 0 && rows->capacity > 0 && !rows->proj) return fail(ESC_EINVAL, "rows->proj is NULL");
    q->out_ids = rows->row_ids;
    q->capacity = rows->capacity;
    for (int i = 0; i < q->nproj; ++i) {
      q->out_proj[i] = rows->capacity ? rows->proj[i] : nullptr;
      if (rows->capacity && !q->out_proj[i]) return fail(ESC_EINVAL, "a projected output pointer is NULL");
    }
  }
  layout_stage(*q, d->sms, p->tuning);
  return ESC_OK;
}

}  // namespace esc

using namespace esc;

namespace {

struct SingleScratch {
  ScratchHdr hdr;
  unsigned long long count;
  unsigned int tiles_left;
  unsigned int pad;
};

// Enqueues one sub-query.  dev_count: where the count goes (null: scratch).
esc_status run_single(const esc_table *t, const esc_pred *p, esc_rows *rows, int mode, uint32_t *bitmap,
                      unsigned long long *dev_count, cudaStream_t st, SingleScratch **scratch_out) {
  Launch L;
  std::memset(&L, 0, sizeof L);
  esc_status s = prepare_query(t, p, rows, mode, &L.q0);
  if (s != ESC_OK) return s;
  L.q0.bitmap = bitmap;
  L.nq = 1;
  L.total_units = L.q0.nunits;
  // scratch: header + count, then (compaction) unit totals and look-back
  // words (zeroed with the header), then the selection bitmap
  const size_t head = (sizeof(SingleScratch) + 255) & ~(size_t)255;
  const size_t zeroed = mode == MODE_SELECT ? select_zeroed_bytes(L.q0) : 0;
  const size_t other = mode == MODE_SELECT ? select_other_bytes(L.q0) : 0;
  void *mem = nullptr;
  if ((s = alloc_async(&mem, head + zeroed + other, st)) != ESC_OK) return s;
  // The caller's count word: a scan stores the final count there itself (the
  // counting goes to the zeroed scratch); the constant kernel, and a launch
  // without work, count into the word, which is then zeroed first.
  uint32_t cval = 0;
  const bool constant = program_constant(L.q0, &cval);
  const bool direct = dev_count && !constant && L.total_units > 0;
  cudaError_t e = cudaMemsetAsync(mem, 0, head + zeroed, st);
  if (e == cudaSuccess && dev_count && !direct) e = cudaMemsetAsync(dev_count, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) {
    cudaFreeAsync(mem, st);
    return fail(ESC_ECUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
  }
  uint8_t *base = static_cast<uint8_t *>(mem);
  SingleScratch *sc = static_cast<SingleScratch *>(mem);
  L.hdr = &sc->hdr;
  L.q0.count = dev_count && !direct ? dev_count : &sc->count;
  L.count_out = direct ? dev_count : nullptr;
  if (mode == MODE_SELECT) select_bind(L.q0, base + head, base + head + zeroed);
  if (constant) {
    s = launch_const(L, cval, st);
  } else {
    s = launch_scan(L, query_shape(L.q0, p->tuning), st);
    if (s == ESC_OK && mode == MODE_SELECT) s = launch_write(L, L.q0.nwunits, st);
  }
  if (s != ESC_OK) {
    cudaFreeAsync(mem, st);
    return s;
  }
  *scratch_out = sc;
  return ESC_OK;
}

// Reads the count and the device status back, synchronises, frees scratch.
esc_status finish_single(SingleScratch *sc, uint64_t *count, cudaStream_t st) {
  SingleScratch h;
  cudaError_t e1 = cudaMemcpyAsync(&h, sc, sizeof h, cudaMemcpyDeviceToHost, st);
  cudaError_t e2 = cudaFreeAsync(sc, st);
  cudaError_t e3 = cudaStreamSynchronize(st);
  if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
    cudaError_t e = e1 != cudaSuccess ? e1 : e2 != cudaSuccess ? e2 : e3;
    return fail(ESC_ECUDA, std::string("sub-query readback: ") + cudaGetErrorString(e));
  }
  if (h.hdr.status != 0) return device_status(h.hdr, "sub-query");
  if (count) *count = h.count;
  return ESC_OK;
}

}  // namespace

extern "C" {

esc_status esc_selectivity(const esc_table *t, const esc_pred *p, uint64_t *count, esc_rows *rows, void *stream) {
  ESC_RANGE("esc_selectivity");
  if (!count) return fail(ESC_EINVAL, "esc_selectivity: count is NULL");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  SingleScratch *sc = nullptr;
  esc_status s = run_single(t, p, rows, rows ? MODE_SELECT : MODE_COUNT, nullptr, nullptr, st, &sc);
  if (s != ESC_OK) return s;
  uint64_t c = 0;
  if ((s = finish_single(sc, &c, st)) != ESC_OK) return s;
  *count = c;
  if (rows) {
    rows->written = std::min<uint64_t>(c, rows->capacity);
    if (c > rows->capacity) return fail(ESC_ETRUNC, "esc_selectivity: more qualifying rows than capacity");
  }
  clear_error();
  return ESC_OK;
}

esc_status esc_selectivity_async(const esc_table *t, const esc_pred *p, uint64_t *dev_count, esc_rows *rows,
                                 void *stream) {
  ESC_RANGE("esc_selectivity_async");
  if (!dev_count) return fail(ESC_EINVAL, "esc_selectivity_async: dev_count is NULL");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  SingleScratch *sc = nullptr;
  esc_status s = run_single(t, p, rows, rows ? MODE_SELECT : MODE_COUNT, nullptr,
                            reinterpret_cast<unsigned long long *>(dev_count), st, &sc);
  if (s != ESC_OK) return s;
  cudaError_t e = cudaFreeAsync(sc, st);
  if (e != cudaSuccess) return fail(ESC_ECUDA, std::string("cudaFreeAsync: ") + cudaGetErrorString(e));
  clear_error();
  return ESC_OK;
}

esc_status esc_bitmap_build(const esc_table *dim, const esc_pred *p, uint32_t *dev_bitmap, uint64_t *count,
                            void *stream) {
  ESC_RANGE("esc_bitmap_build");
  if (!dim) return fail(ESC_EINVAL, "esc_bitmap_build: dim is NULL");
  if (!dev_bitmap && dim->nrows > 0) return fail(ESC_EINVAL, "esc_bitmap_build: dev_bitmap is NULL");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  SingleScratch *sc = nullptr;
  esc_status s = run_single(dim, p, nullptr, MODE_BITMAP, dev_bitmap, nullptr, st, &sc);
  if (s != ESC_OK) return s;
  uint64_t c = 0;
  if ((s = finish_single(sc, &c, st)) != ESC_OK) return s;
  if (count) *count = c;
  clear_error();
  return ESC_OK;
}

// ------------------------------------------------------------------ batches
}  // extern "C"

struct esc_batch {
  int32_t n = 0;
  int32_t nwaves = 1;               // scan (+ write) launches, one header each at the start of scratch
  int device = 0;
  void *dev_mem = nullptr;          // queries + scratch, owned
  Query *queries = nullptr;         // device
  uint8_t *scratch = nullptr;       // device: hdr, counts, done, countdowns, unit words
  size_t scratch_bytes = 0;
  unsigned long long *counts = nullptr;
  unsigned long long *done = nullptr;
  unsigned int *tiles_left = nullptr;
  unsigned int *tiles_init = nullptr;  // device copy of each query's countdown start
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

void batch_free(esc_batch *b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->dev_mem) cudaFree(b->dev_mem);
  delete b;
}

constexpr int kMaxWaves = 16;

// Work of a sub-query, for ordering a batch and grouping it into waves: the
// bytes its scan reads (0 for a program folded to a constant).
uint64_t query_work(const Query &q) {
  if (q.is_const) return 0;
  uint64_t bpr = 0;
  for (int i = 0; i < q.nref; ++i) bpr += q.ref_w[i];
  return (uint64_t)q.nrows * std::max<uint64_t>(bpr, 1);
}

// A prepared batch: the sub-queries sorted by work (smallest first) and cut
// into `waves` consecutive groups whose work doubles from one to the next
// (the last holds about half of it); each wave is one persistent scan launch
// and, when it materialises, one write launch.  Counts, completion times and
// countdowns stay indexed in the caller's order.
esc_status batch_prepare(const esc_table *const *tables, const esc_pred *const *preds, int32_t n,
                         const esc_rows *rows, int32_t waves, esc_batch **out) {
  if (!out) return fail(ESC_EINVAL, "esc_batch_prepare: out is NULL");
  *out = nullptr;
  if (n < 1 || !tables || !preds) return fail(ESC_EINVAL, "esc_batch_prepare: need n >= 1 tables and predicates");
  if (waves < 1 || waves > kMaxWaves) return fail(ESC_EINVAL, "esc_batch_prepare: waves must be 1..16");
  DeviceState *d;
  esc_status s = device_state(&d);
  if (s != ESC_OK) return s;
  std::vector<Query> qin((size_t)n);
  for (int i = 0; i < n; ++i) {
    const esc_rows *r = rows ? &rows[i] : nullptr;
    const bool compact = r && (r->capacity > 0 || r->row_ids != nullptr);
    if ((s = prepare_query(tables[i], preds[i], compact ? r : nullptr, compact ? MODE_SELECT : MODE_COUNT,
                           &qin[i])) != ESC_OK)
      return s;
    layout_write_units(qin[i], 0);  // one write grid for all queries: full-size units
    mark_constant(qin[i]);
  }
  // smallest work first (stable: equal work keeps the caller's order)
  std::vector<int> ord((size_t)n);
  for (int i = 0; i < n; ++i) ord[i] = i;
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return query_work(qin[a]) < query_work(qin[b]); });
  std::vector<Query> qs((size_t)n);
  uint64_t total_work = 0;
  for (int k = 0; k < n; ++k) {
    qs[k] = qin[ord[k]];
    total_work += query_work(qs[k]);
  }
  // wave k ends once the work so far reaches total / 2^(waves-1-k)
  std::vector<int> wend;
  {
    uint64_t acc = 0;
    int k = 0;
    for (int w = 0; w < waves; ++w) {
      const uint64_t target = w + 1 == waves ? ~0ull : total_work >> (waves - 1 - w);
      while (k < n && (acc < target || w + 1 == waves)) acc += query_work(qs[k++]);
      if (k > (wend.empty() ? 0 : wend.back())) wend.push_back(k);
    }
    if (wend.empty() || wend.back() != n) wend.push_back(n);
  }
  const int nw = (int)wend.size();
  std::vector<uint32_t> cidx;
  std::vector<uint32_t> w_units((size_t)nw, 0), w_wunits((size_t)nw, 0);
  std::vector<int> w_shape((size_t)nw, 0);
  uint64_t zeroed = 0, other = 0;
  for (int w = 0, k0 = 0; w < nw; k0 = wend[w++]) {
    uint64_t units = 0, wunits = 0;
    for (int k = k0; k < wend[w]; ++k) {
      Query &q = qs[k];
      if (q.is_const) cidx.push_back((uint32_t)k);
      q.unit_base = (uint32_t)units;
      q.wunit_base = (uint32_t)wunits;
      units += q.nunits;
      if (q.mode == MODE_SELECT) {
        wunits += q.nwunits;
        zeroed += select_zeroed_bytes(q);
        other += select_other_bytes(q);
      }
      if (units >= (1ull << 31)) return fail(ESC_EINVAL, "esc_batch_prepare: too many work units in one batch");
    }
    w_units[w] = (uint32_t)units;
    w_wunits[w] = (uint32_t)wunits;
    w_shape[w] = launch_shape(&qs[k0], wend[w] - k0);
  }
  esc_batch *b = new (std::nothrow) esc_batch;
  if (!b) return fail(ESC_ENOMEM, "esc_batch_prepare: out of host memory");
  b->n = n;
  b->nwaves = nw;
  cudaGetDevice(&b->device);
  // device memory: queries (sorted) + constant indices | zeroed every run:
  // one header per wave, counts, done times, countdowns (caller's order),
  // unit totals + look-back words | countdown initial values | selection
  // bitmaps
  const size_t q_span = (sizeof(Query) * (size_t)n + 4 * (size_t)n + 255) & ~(size_t)255;
  const size_t hdr_bytes = 256 * (size_t)nw;
  const size_t cnt_bytes = ((size_t)n * 8 + 255) & ~(size_t)255;
  const size_t left_bytes = ((size_t)n * 4 + 255) & ~(size_t)255;
  b->scratch_bytes = hdr_bytes + 2 * cnt_bytes + left_bytes + (size_t)zeroed;
  const size_t total = q_span + b->scratch_bytes + left_bytes + (size_t)other;
  cudaError_t e = inject_alloc_failure() ? cudaErrorMemoryAllocation : cudaMalloc(&b->dev_mem, total);
  if (e != cudaSuccess) {
    batch_free(b);
    return fail(ESC_ENOMEM, std::string("esc_batch_prepare: cudaMalloc: ") + cudaGetErrorString(e));
  }
  uint8_t *base = static_cast<uint8_t *>(b->dev_mem);
  b->queries = reinterpret_cast<Query *>(base);
  b->scratch = base + q_span;
  b->counts = reinterpret_cast<unsigned long long *>(b->scratch + hdr_bytes);
  b->done = reinterpret_cast<unsigned long long *>(b->scratch + hdr_bytes + cnt_bytes);
  b->tiles_left = reinterpret_cast<unsigned int *>(b->scratch + hdr_bytes + 2 * cnt_bytes);
  uint8_t *zp = b->scratch + hdr_bytes + 2 * cnt_bytes + left_bytes;
  b->tiles_init = reinterpret_cast<unsigned int *>(b->scratch + b->scratch_bytes);
  uint8_t *op = b->scratch + b->scratch_bytes + left_bytes;
  std::vector<unsigned int> init((size_t)n);
  for (int k = 0; k < n; ++k) {
    Query &q = qs[k];
    const int i = ord[k];
    int w = 0;
    while (k >= wend[w]) ++w;
    q.count = &b->counts[i];
    q.done_ns = &b->done[i];
    q.tiles_left = &b->tiles_left[i];
    if (q.is_const) {
      init[i] = kConstBlocks;                         // counted down by the constant kernel
    } else if (q.mode == MODE_SELECT) {
      select_bind(q, zp, op);
      zp += select_zeroed_bytes(q);
      op += select_other_bytes(q);
      init[i] = q.nwunits;                            // counted down by the write kernel
    } else {
      init[i] = q.ntiles * (unsigned)kScanShapes[w_shape[w]].consumers;  // counted down by the scan kernel
    }
  }
  if ((uintptr_t)op > (uintptr_t)base + total) {
    batch_free(b);
    return fail(ESC_EINVAL, "esc_batch_prepare: internal layout error");
  }
  uint32_t *dev_cidx = reinterpret_cast<uint32_t *>(base + sizeof(Query) * (size_t)n);
  e = cudaMemcpy(b->queries, qs.data(), sizeof(Query) * (size_t)n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !cidx.empty())
    e = cudaMemcpy(dev_cidx, cidx.data(), 4 * cidx.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->tiles_init, init.data(), (size_t)n * 4, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    batch_free(b);
    return fail(ESC_ECUDA, std::string("esc_batch_prepare: cudaMemcpy: ") + cudaGetErrorString(e));
  }
  // Capture reset + constant kernel + (scan + write) per wave into a graph
  // once; runs replay it.
  cudaStream_t cs;
  e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    batch_free(b);
    return fail(ESC_ECUDA, std::string("esc_batch_prepare: cudaStreamCreate: ") + cudaGetErrorString(e));
  }
  e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  esc_status ls = ESC_OK;
  if (e == cudaSuccess) {
    cudaMemsetAsync(b->scratch, 0, b->scratch_bytes, cs);
    cudaMemcpyAsync(b->tiles_left, b->tiles_init, (size_t)n * 4, cudaMemcpyDeviceToDevice, cs);
    if (!cidx.empty()) ls = launch_const_batch(b->queries, dev_cidx, (uint32_t)cidx.size(), cs);
    for (int w = 0, k0 = 0; w < nw && ls == ESC_OK; k0 = wend[w++]) {
      Launch L;
      std::memset(&L, 0, sizeof L);
      L.queries = b->queries + k0;
      L.nq = wend[w] - k0;
      L.total_units = w_units[w];
      L.hdr = reinterpret_cast<ScratchHdr *>(b->scratch + 256 * (size_t)w);
      ls = launch_scan(L, w_shape[w], cs);
      if (ls == ESC_OK) ls = launch_write(L, w_wunits[w], cs);
    }
    e = cudaStreamEndCapture(cs, &b->graph);
  }
  if (e == cudaSuccess && ls == ESC_OK) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
  cudaStreamDestroy(cs);
  if (e != cudaSuccess || ls != ESC_OK) {
    batch_free(b);
    if (ls != ESC_OK) return ls;
    return fail(ESC_ECUDA, std::string("esc_batch_prepare: graph capture: ") + cudaGetErrorString(e));
  }
  *out = b;
  clear_error();
  return ESC_OK;
}


}  // namespace

extern "C" {

esc_status esc_batch_prepare(const esc_table *const *tables, const esc_pred *const *preds, int32_t n,
                             const esc_rows *rows, esc_batch **out) {
  return batch_prepare(tables, preds, n, rows, 1, out);
}

esc_status esc_batch_prepare_waves(const esc_table *const *tables, const esc_pred *const *preds, int32_t n,
                                   const esc_rows *rows, int32_t waves, esc_batch **out) {
  ESC_RANGE("esc_batch_prepare_waves");
  return batch_prepare(tables, preds, n, rows, waves, out);
}

esc_status esc_batch_run(esc_batch *b, uint64_t *dev_counts, uint64_t *dev_done_ns, void *stream) {
  ESC_RANGE("esc_batch_run");
  if (!b) return fail(ESC_EINVAL, "esc_batch_run: batch is NULL");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  ESC_CK(cudaGraphLaunch(b->exec, st));
  if (dev_counts) ESC_CK(cudaMemcpyAsync(dev_counts, b->counts, (size_t)b->n * 8, cudaMemcpyDeviceToDevice, st));
  if (dev_done_ns) ESC_CK(cudaMemcpyAsync(dev_done_ns, b->done, (size_t)b->n * 8, cudaMemcpyDeviceToDevice, st));
  clear_error();
  return ESC_OK;
}

esc_status esc_batch_destroy(esc_batch *b) {
  if (b) cudaDeviceSynchronize();
  batch_free(b);
  return ESC_OK;
}

esc_status esc_selectivity_batch(const esc_table *const *tables, const esc_pred *const *preds, int32_t n,
                                 uint64_t *counts, esc_rows *rows, void *stream) {
  if (!counts) return fail(ESC_EINVAL, "esc_selectivity_batch: counts is NULL");
  esc_batch *b = nullptr;
  esc_status s = esc_batch_prepare(tables, preds, n, rows, &b);
  if (s != ESC_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  s = esc_batch_run(b, nullptr, nullptr, st);
  std::vector<uint8_t> hb(256 * (size_t)b->nwaves);
  if (s == ESC_OK) {
    cudaError_t e = cudaMemcpyAsync(counts, b->counts, (size_t)n * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hb.data(), b->scratch, hb.size(), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) s = fail(ESC_ECUDA, std::string("esc_selectivity_batch: ") + cudaGetErrorString(e));
  }
  const int nw = b->nwaves;
  batch_free(b);
  if (s != ESC_OK) return s;
  for (int w = 0; w < nw; ++w) {
    ScratchHdr h;
    std::memcpy(&h, hb.data() + 256 * (size_t)w, sizeof h);
    if (h.status != 0) return device_status(h, "esc_selectivity_batch");
  }
  bool trunc = false;
  if (rows)
    for (int i = 0; i < n; ++i) {
      if (rows[i].capacity > 0 || rows[i].row_ids) {
        rows[i].written = std::min<uint64_t>(counts[i], rows[i].capacity);
        trunc = trunc || counts[i] > rows[i].capacity;
      }
    }
  if (trunc) return fail(ESC_ETRUNC, "esc_selectivity_batch: some sub-query had more rows than capacity");
  clear_error();
  return ESC_OK;
}

esc_status esc_selectivity_batch_async(const esc_table *const *tables, const esc_pred *const *preds, int32_t n,
                                       const esc_rows *rows, uint64_t *dev_counts, uint64_t *dev_done_ns,
                                       void *stream) {
  ESC_RANGE("esc_selectivity_batch_async");
  if (n < 1 || !tables || !preds || !dev_counts)
    return fail(ESC_EINVAL, "esc_selectivity_batch_async: need n >= 1 tables, predicates and dev_counts");
  std::vector<Query> qs((size_t)n);
  std::vector<uint32_t> cidx;
  uint64_t units = 0, wunits = 0, zeroed = 0, other = 0;
  esc_status s;
  for (int i = 0; i < n; ++i) {
    const esc_rows *r = rows ? &rows[i] : nullptr;
    const bool compact = r && (r->capacity > 0 || r->row_ids != nullptr);
    if ((s = prepare_query(tables[i], preds[i], compact ? r : nullptr, compact ? MODE_SELECT : MODE_COUNT,
                           &qs[i])) != ESC_OK)
      return s;
    layout_write_units(qs[i], 0);  // one write grid for all queries: full-size units
    mark_constant(qs[i]);
    if (qs[i].is_const) cidx.push_back((uint32_t)i);
    qs[i].unit_base = (uint32_t)units;
    qs[i].wunit_base = (uint32_t)wunits;
    units += qs[i].nunits;
    if (compact) {
      wunits += qs[i].nwunits;
      zeroed += select_zeroed_bytes(qs[i]);
      other += select_other_bytes(qs[i]);
    }
    if (units >= (1ull << 31)) return fail(ESC_EINVAL, "esc_selectivity_batch_async: too many work units");
  }
  // device block: queries | zeroed: header, counts, done, countdowns, unit words | bitmaps, group data
  const size_t q_span = (sizeof(Query) * (size_t)n + 4 * (size_t)n + 255) & ~(size_t)255;  // queries + cidx
  const size_t cnt_bytes = ((size_t)n * 8 + 255) & ~(size_t)255;
  const size_t left_bytes = ((size_t)n * 4 + 255) & ~(size_t)255;
  const size_t zbytes = 256 + 2 * cnt_bytes + left_bytes + (size_t)zeroed;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  void *mem = nullptr;
  if ((s = alloc_async(&mem, q_span + zbytes + (size_t)other, st)) != ESC_OK) return s;
  uint8_t *base = static_cast<uint8_t *>(mem);
  uint8_t *z = base + q_span;
  unsigned long long *counts = reinterpret_cast<unsigned long long *>(z + 256);
  unsigned long long *done = reinterpret_cast<unsigned long long *>(z + 256 + cnt_bytes);
  unsigned int *left = reinterpret_cast<unsigned int *>(z + 256 + 2 * cnt_bytes);
  uint8_t *zp = z + 256 + 2 * cnt_bytes + left_bytes;
  uint8_t *op = z + zbytes;
  std::vector<unsigned int> init((size_t)n);
  const int shape = launch_shape(qs.data(), n);
  for (int i = 0; i < n; ++i) {
    qs[i].count = &counts[i];
    qs[i].done_ns = dev_done_ns ? &done[i] : nullptr;
    qs[i].tiles_left = &left[i];
    if (qs[i].is_const) {
      init[i] = kConstBlocks;
    } else if (qs[i].mode == MODE_SELECT) {
      select_bind(qs[i], zp, op);
      zp += select_zeroed_bytes(qs[i]);
      op += select_other_bytes(qs[i]);
      init[i] = qs[i].nwunits;
    } else {
      init[i] = qs[i].ntiles * (unsigned)kScanShapes[shape].consumers;
    }
  }
  uint32_t *dev_cidx = reinterpret_cast<uint32_t *>(base + sizeof(Query) * (size_t)n);
  cudaError_t e = cudaMemsetAsync(z, 0, zbytes, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(base, qs.data(), sizeof(Query) * (size_t)n, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && !cidx.empty())
    e = cudaMemcpyAsync(dev_cidx, cidx.data(), 4 * cidx.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && dev_done_ns)
    e = cudaMemcpyAsync(left, init.data(), (size_t)n * 4, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) {
    cudaFreeAsync(mem, st);
    return fail(ESC_ECUDA, std::string("esc_selectivity_batch_async: ") + cudaGetErrorString(e));
  }
  Launch L;
  std::memset(&L, 0, sizeof L);
  L.queries = reinterpret_cast<const Query *>(base);
  L.nq = n;
  L.total_units = (uint32_t)units;
  L.hdr = reinterpret_cast<ScratchHdr *>(z);
  s = cidx.empty() ? ESC_OK : launch_const_batch(L.queries, dev_cidx, (uint32_t)cidx.size(), st);
  if (s == ESC_OK) s = launch_scan(L, shape, st);
  if (s == ESC_OK) s = launch_write(L, (uint32_t)wunits, st);
  if (s == ESC_OK) {
    e = cudaMemcpyAsync(dev_counts, counts, (size_t)n * 8, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && dev_done_ns)
      e = cudaMemcpyAsync(dev_done_ns, done, (size_t)n * 8, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) s = fail(ESC_ECUDA, std::string("esc_selectivity_batch_async: ") + cudaGetErrorString(e));
  }
  cudaFreeAsync(mem, st);
  if (s == ESC_OK) clear_error();
  return s;
}

// One shared scan: `n` count-only predicates of table t whose read columns
// (union `ucols`, table column indices) fit one stage layout.
static esc_status run_shared_group(const esc_table *t, const esc_pred *const *preds, int32_t n,
                                   const std::vector<int32_t> &ucols, uint64_t *dev_counts, cudaStream_t st) {
  DeviceState *d;
  esc_status s = device_state(&d);
  if (s != ESC_OK) return s;
  Launch L;
  std::memset(&L, 0, sizeof L);
  Query &Y = L.q0;
  Y.nrows = (uint32_t)t->nrows;
  Y.mode = MODE_COUNT;
  Y.nref = (int32_t)ucols.size();
  for (size_t k = 0; k < ucols.size(); ++k) {
    Y.ref_w[k] = (uint8_t)dtype_width(t->dtypes[ucols[k]]);
    Y.ref_ptr[k] = static_cast<const uint8_t *>(t->data[ucols[k]]);
  }
  layout_stage(Y, d->sms, kDefaultTuning);
  std::vector<Query> qs((size_t)n);
  for (int k = 0; k < n; ++k) {
    if ((s = prepare_query(t, preds[k], nullptr, MODE_COUNT, &qs[k])) != ESC_OK) return s;
    auto uslot = [&](int local) {
      const int32_t col = preds[k]->ref_cols[local];
      return (int)(std::find(ucols.begin(), ucols.end(), col) - ucols.begin());
    };
    for (int pc = 0; pc < qs[k].ninstr; ++pc) {  // stage offsets into the union layout
      Instr &I = qs[k].code[pc];
      if (I.op == OP_RANGE || I.op == OP_IN || I.op == OP_INSET || I.op == OP_UDF)
        I.soff = (uint16_t)Y.stage_off[uslot(I.ref)];
      if (I.op == OP_UDF) I.soff2 = (uint16_t)Y.stage_off[uslot(I.ref2)];
    }
  }
  const size_t head = 256;
  const size_t cnt_bytes = ((size_t)n * 8 + 255) & ~(size_t)255;
  const size_t q_bytes = sizeof(Query) * (size_t)n;
  void *mem = nullptr;
  if ((s = alloc_async(&mem, head + cnt_bytes + q_bytes, st)) != ESC_OK) return s;
  uint8_t *base = static_cast<uint8_t *>(mem);
  unsigned long long *counts = reinterpret_cast<unsigned long long *>(base + head);
  Query *dq = reinterpret_cast<Query *>(base + head + cnt_bytes);
  for (int k = 0; k < n; ++k) qs[k].count = &counts[k];
  cudaError_t e = cudaMemsetAsync(base, 0, head + cnt_bytes, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dq, qs.data(), q_bytes, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && Y.nunits > 0) {
    L.queries = dq;
    L.nq = n;
    L.total_units = Y.nunits;
    L.hdr = reinterpret_cast<ScratchHdr *>(base);
    const uint32_t grid = std::min<uint32_t>((uint32_t)(d->sms * d->blocks_per_sm), Y.nunits);
    shared_kernel<<<grid, kThreads, SharedSmem::total, st>>>(L);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(dev_counts, counts, (size_t)n * 8, cudaMemcpyDeviceToDevice, st);
  cudaFreeAsync(mem, st);
  if (e != cudaSuccess) return fail(ESC_ECUDA, std::string("esc_selectivity_shared_async: ") + cudaGetErrorString(e));
  return ESC_OK;
}

esc_status esc_selectivity_shared_async(const esc_table *t, const esc_pred *const *preds, int32_t n,
                                        uint64_t *dev_counts, void *stream) {
  ESC_RANGE("esc_selectivity_shared_async");
  if (!t || !preds || n < 1 || !dev_counts)
    return fail(ESC_EINVAL, "esc_selectivity_shared_async: need a table, n >= 1 predicates and dev_counts");
  for (int i = 0; i < n; ++i)
    if (!preds[i] || preds[i]->table != t)
      return fail(ESC_EINVAL, "esc_selectivity_shared_async: every predicate must be compiled against the table");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // greedy groups: the union of read columns fits the stage layout
  int i = 0;
  while (i < n) {
    std::vector<int32_t> ucols;
    int j = i;
    for (; j < n && j - i < kSharedMaxQueries; ++j) {
      std::vector<int32_t> add;
      for (int32_t c : preds[j]->ref_cols)
        if (std::find(ucols.begin(), ucols.end(), c) == ucols.end()) add.push_back(c);
      if (ucols.size() + add.size() > (size_t)kMaxRef) break;
      ucols.insert(ucols.end(), add.begin(), add.end());
    }
    esc_status s = run_shared_group(t, preds + i, j - i, ucols, dev_counts + i, st);
    if (s != ESC_OK) return s;
    i = j;
  }
  clear_error();
  return ESC_OK;
}

esc_status esc_timestamp(uint64_t *dev_ns, void *stream) {
  if (!dev_ns) return fail(ESC_EINVAL, "esc_timestamp: dev_ns is NULL");
  timestamp_kernel<<<1, 1, 0, static_cast<cudaStream_t>(stream)>>>(reinterpret_cast<unsigned long long *>(dev_ns));
  ESC_CK(cudaGetLastError());
  return ESC_OK;
}

esc_status esc_selftest_wait_timeout(uint64_t limit_ns, void *stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  void *mem = nullptr;
  esc_status s = alloc_async(&mem, 64, st);
  if (s != ESC_OK) return s;
  ESC_CK(cudaMemsetAsync(mem, 0, 64, st));
  ScratchHdr *hdr = static_cast<ScratchHdr *>(mem);
  const unsigned *flag = reinterpret_cast<const unsigned *>(static_cast<uint8_t *>(mem) + 32);
  wait_selftest_kernel<<<1, 32, 0, st>>>(flag, hdr, limit_ns);
  ESC_CK(cudaGetLastError());
  ScratchHdr h;
  ESC_CK(cudaMemcpyAsync(&h, hdr, sizeof h, cudaMemcpyDeviceToHost, st));
  ESC_CK(cudaFreeAsync(mem, st));
  ESC_CK(cudaStreamSynchronize(st));
  if (h.status != 0) return fail((esc_status)h.status, "the bounded wait gave up (expected)");
  clear_error();
  return ESC_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ allocation-free variant
// esc_selectivity_noalloc: the same sub-query for callers that must not
// allocate device memory.  Its scratch (launch header, count, unit words,
// selection bitmap) is one array in this library's device
// image, sized kNoAllocScratchBytes; the CUDA driver reserves it on every
// device where the library's kernels are loaded, until the process exits.

namespace {
constexpr size_t kNoAllocScratchBytes = (size_t)12 << 20;  // 12 MiB
}  // namespace

static __device__ __align__(256) uint8_t g_noalloc_scratch[kNoAllocScratchBytes];

namespace {

struct NoAllocDevice {
  bool ready = false;
  int sms = 0;
  int blocks_per_sm = 0;
  uint8_t *scratch = nullptr;  // device address of g_noalloc_scratch on this device
};
std::mutex g_noalloc_mu;
NoAllocDevice g_noalloc[64];

struct NoAllocHead {
  ScratchHdr hdr;
  unsigned long long count;
  unsigned long long pad;
};

// One-time set-up per device, on the current device: kernel attributes and
// the device address of the scratch array (host code cannot use the array's
// name as a device pointer).  Allocates nothing.
esc_status noalloc_device(NoAllocDevice **out) {
  int dev = 0;
  ESC_CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(ESC_EINVAL, "esc_selectivity_noalloc: device index out of range");
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  NoAllocDevice &d = g_noalloc[dev];
  if (!d.ready) {
    ESC_CK(cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev));
    esc_status cs = configure_kernels(&d.blocks_per_sm);
    if (cs != ESC_OK) return cs;
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr)
      return fail(ESC_ECUDA, std::string("esc_selectivity_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    d.scratch = static_cast<uint8_t *>(p);
    d.ready = true;
  }
  *out = &d;
  return ESC_OK;
}

}  // namespace

extern "C" esc_status esc_selectivity_noalloc(const esc_table *t, const esc_pred *p, uint64_t *count,
                                              esc_rows *rows, void *stream) {
  ESC_RANGE("esc_selectivity_noalloc");
  if (!count) return fail(ESC_EINVAL, "esc_selectivity_noalloc: count is NULL");
  if (!t || !p) return fail(ESC_EINVAL, "esc_selectivity_noalloc: table and predicate are required");
  if (p->table != t) return fail(ESC_EINVAL, "esc_selectivity_noalloc: predicate was compiled against another table");
  NoAllocDevice *d;
  esc_status s = noalloc_device(&d);
  if (s != ESC_OK) return s;
  const int mode = rows ? MODE_SELECT : MODE_COUNT;
  Launch L;
  std::memset(&L, 0, sizeof L);
  Query &q = L.q0;
  fill_query_program(p, &q);
  q.nrows = (uint32_t)t->nrows;
  q.mode = mode;
  if (rows) {
    if (rows->capacity > 0 && !rows->row_ids) return fail(ESC_EINVAL, "esc_selectivity_noalloc: rows->row_ids is NULL");
    if (q.nproj > 0 && rows->capacity > 0 && !rows->proj)
      return fail(ESC_EINVAL, "esc_selectivity_noalloc: rows->proj is NULL");
    q.out_ids = rows->row_ids;
    q.capacity = rows->capacity;
    for (int i = 0; i < q.nproj; ++i) {
      q.out_proj[i] = rows->capacity ? rows->proj[i] : nullptr;
      if (rows->capacity && !q.out_proj[i])
        return fail(ESC_EINVAL, "esc_selectivity_noalloc: a projected output pointer is NULL");
    }
  }
  layout_stage(q, d->sms, p->tuning);
  L.nq = 1;
  L.total_units = q.nunits;
  const size_t head = (sizeof(NoAllocHead) + 255) & ~(size_t)255;
  const size_t zeroed = mode == MODE_SELECT ? select_zeroed_bytes(q) : 0;
  const size_t other = mode == MODE_SELECT ? select_other_bytes(q) : 0;
  if (head + zeroed + other > kNoAllocScratchBytes)
    return fail(ESC_EINVAL, "esc_selectivity_noalloc: materialising this table needs " +
                                std::to_string(head + zeroed + other) +
                                " bytes of scratch, more than the built-in 12 MiB; use esc_selectivity");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // the array keeps the previous call's contents: clear what must start at zero
  ESC_CK(cudaMemsetAsync(d->scratch, 0, head + zeroed, st));
  NoAllocHead *h = reinterpret_cast<NoAllocHead *>(d->scratch);
  L.hdr = &h->hdr;
  q.count = &h->count;
  if (mode == MODE_SELECT) select_bind(q, d->scratch + head, d->scratch + head + zeroed);
  uint32_t cval = 0;
  if (program_constant(q, &cval)) {
    // launched here rather than through launch_const, which would set up the
    // library's memory pool on first use
    const uint64_t work = (mode == MODE_SELECT && cval) ? std::min<uint64_t>(q.nrows, q.capacity) : 0;
    const uint32_t grid =
        (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)d->sms * 8, (work + 255) / 256));
    const_kernel<<<grid, 256, 0, st>>>(L, cval);
    ESC_CK(cudaGetLastError());
  } else if (L.total_units > 0) {
    const uint32_t grid = std::min<uint32_t>((uint32_t)(d->sms * d->blocks_per_sm), L.total_units);
    launch_scan_shape(query_shape(q, p->tuning), grid, L, st);
    ESC_CK(cudaGetLastError());
    if (mode == MODE_SELECT) {
      write_kernel<<<q.nwunits, kWriteThreads, kWriteSmem, st>>>(L);
      ESC_CK(cudaGetLastError());
    }
  }
  NoAllocHead back;
  ESC_CK(cudaMemcpyAsync(&back, h, sizeof back, cudaMemcpyDeviceToHost, st));
  ESC_CK(cudaStreamSynchronize(st));
  if (back.hdr.status != 0) return device_status(back.hdr, "esc_selectivity_noalloc");
  *count = back.count;
  if (rows) {
    rows->written = std::min<uint64_t>(back.count, rows->capacity);
    if (back.count > rows->capacity)
      return fail(ESC_ETRUNC, "esc_selectivity_noalloc: more qualifying rows than capacity");
  }
  clear_error();
  return ESC_OK;
}
