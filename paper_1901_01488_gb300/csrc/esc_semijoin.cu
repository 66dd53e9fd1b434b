// Exact semi-join cardinalities over dense keys: the COUNT(*) foreign-key
// join queries of the paper's overhead experiments (Sec. 3.1: lineitem joined
// with a filtered orders / part / supplier table) generalised to a star
// schema.  One pass over the fact table's foreign-key columns:
//   m(i) = sum_d [0 <= fk_d[i] < D_d and bitmap_d bit fk_d[i]] << d,
//   h[v] = |{ i : m(i) = v }|          (2^ndims bins)
// and on the host, for every dimension subset S,
//   count(S) = sum over v that contain S of h[v]   (superset sum).
//
// Kernel shape: persistent grid, each thread streams 16 rows per step with
// 16-byte non-allocating loads of every FK column (4 rows per load), probes
// bitmaps that fit in shared memory there and the others through the L1/L2
// read-only path, and counts the 16 bins in two 64-bit registers of eight
// 8-bit counters each (flushed before they can overflow).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>

#include "esc_internal.h"

namespace esc {

constexpr int kSjThreads = 512;
constexpr int kSjMaxDims = 4;
constexpr uint32_t kSjSmemBitmapBytes = 160 * 1024;

struct SjParams {
  const int32_t *fk[kSjMaxDims];
  const uint32_t *bitmap[kSjMaxDims];
  uint32_t dim_rows[kSjMaxDims];
  uint32_t smem_off[kSjMaxDims];   // word offset in shared memory, or ~0u: read from global
  uint32_t words[kSjMaxDims];
  int32_t ndims;
  uint32_t nrows;
  unsigned long long *hist;        // 16 bins, zeroed
};

__device__ __forceinline__ int4 ld_stream(const int32_t *p) {
  int4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.s32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p));
  return v;
}

template <int ND>
__device__ __forceinline__ uint32_t probe(const SjParams &P, const uint32_t *sbm, const int32_t (&k)[ND]) {
  uint32_t m = 0;
#pragma unroll
  for (int d = 0; d < ND; ++d) {
    const uint32_t key = (uint32_t)k[d];
    uint32_t bit = 0;
    if (key < P.dim_rows[d]) {  // negative keys wrap to large unsigned values
      const uint32_t w = P.smem_off[d] != ~0u ? sbm[P.smem_off[d] + (key >> 5)] : __ldg(&P.bitmap[d][key >> 5]);
      bit = (w >> (key & 31u)) & 1u;
    }
    m |= bit << d;
  }
  return m;
}

__device__ __forceinline__ void bump(uint64_t &lo, uint64_t &hi, uint32_t m) {
  const uint64_t inc = 1ull << (8u * (m & 7u));
  if (m & 8u) hi += inc; else lo += inc;
}

__device__ __forceinline__ void flush(uint64_t &lo, uint64_t &hi, uint32_t (&c)[16]) {
#pragma unroll
  for (int v = 0; v < 8; ++v) {
    c[v] += (uint32_t)((lo >> (8 * v)) & 0xffu);
    c[v + 8] += (uint32_t)((hi >> (8 * v)) & 0xffu);
  }
  lo = hi = 0;
}

template <int ND>
__global__ void __launch_bounds__(kSjThreads, 1) semijoin_kernel(const __grid_constant__ SjParams P) {
  extern __shared__ __align__(16) uint32_t sbm[];
  __shared__ unsigned long long bins[16];
  for (int d = 0; d < ND; ++d) {
    if (P.smem_off[d] == ~0u) continue;
    for (uint32_t w = threadIdx.x; w < P.words[d]; w += blockDim.x) sbm[P.smem_off[d] + w] = P.bitmap[d][w];
  }
  if (threadIdx.x < 16) bins[threadIdx.x] = 0;
  __syncthreads();

  uint32_t c[16];
#pragma unroll
  for (int v = 0; v < 16; ++v) c[v] = 0;
  uint64_t lo = 0, hi = 0;
  uint32_t pending = 0;

  const uint32_t nchunks = P.nrows / 16u;  // 16 rows per thread step
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t ch = blockIdx.x * blockDim.x + threadIdx.x; ch < nchunks; ch += stride) {
    int4 v[ND][4];
#pragma unroll
    for (int d = 0; d < ND; ++d)
#pragma unroll
      for (int q = 0; q < 4; ++q) v[d][q] = ld_stream(P.fk[d] + (size_t)ch * 16 + 4 * q);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int32_t k0[ND], k1[ND], k2[ND], k3[ND];
#pragma unroll
      for (int d = 0; d < ND; ++d) {
        k0[d] = v[d][q].x;
        k1[d] = v[d][q].y;
        k2[d] = v[d][q].z;
        k3[d] = v[d][q].w;
      }
      bump(lo, hi, probe<ND>(P, sbm, k0));
      bump(lo, hi, probe<ND>(P, sbm, k1));
      bump(lo, hi, probe<ND>(P, sbm, k2));
      bump(lo, hi, probe<ND>(P, sbm, k3));
    }
    pending += 16;
    if (pending >= 240) {  // 8-bit counters: flush before 255
      flush(lo, hi, c);
      pending = 0;
    }
  }
  // ragged tail: rows nchunks*16 .. nrows-1, one per thread of block 0
  if (blockIdx.x == 0) {
    const uint32_t r = nchunks * 16u + threadIdx.x;
    if (r < P.nrows) {
      int32_t k[ND];
#pragma unroll
      for (int d = 0; d < ND; ++d) k[d] = P.fk[d][r];
      bump(lo, hi, probe<ND>(P, sbm, k));
    }
  }
  flush(lo, hi, c);
#pragma unroll
  for (int v = 0; v < 16; ++v) {
    uint32_t x = c[v];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0 && x) atomicAdd(&bins[v], (unsigned long long)x);
  }
  __syncthreads();
  if (threadIdx.x < 16 && bins[threadIdx.x]) atomicAdd(&P.hist[threadIdx.x], bins[threadIdx.x]);
}

template <int ND>
cudaError_t launch_semijoin(const SjParams &P, size_t smem, int grid, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(semijoin_kernel<ND>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  semijoin_kernel<ND><<<grid, kSjThreads, smem, st>>>(P);
  return cudaGetLastError();
}

}  // namespace esc

using namespace esc;

extern "C" esc_status esc_semijoin_counts(const esc_table *fact, const char *const *fk_cols, int32_t ndims,
                                          const uint32_t *const *dev_bitmaps, const uint64_t *dim_rows,
                                          uint64_t *subset_counts, void *stream) {
  if (!fact || !fk_cols || !dev_bitmaps || !dim_rows || !subset_counts)
    return fail(ESC_EINVAL, "esc_semijoin_counts: NULL argument");
  if (ndims < 1 || ndims > kSjMaxDims) return fail(ESC_EINVAL, "esc_semijoin_counts: ndims must be 1..4");
  SjParams P;
  std::memset(&P, 0, sizeof P);
  P.ndims = ndims;
  P.nrows = (uint32_t)fact->nrows;
  uint32_t smem_words = 0;
  for (int d = 0; d < ndims; ++d) {
    if (!fk_cols[d]) return fail(ESC_EINVAL, "esc_semijoin_counts: NULL column name");
    int c = -1;
    for (size_t i = 0; i < fact->names.size(); ++i)
      if (fact->names[i] == fk_cols[d]) c = (int)i;
    if (c < 0) return fail(ESC_EINVAL, std::string("esc_semijoin_counts: unknown column ") + fk_cols[d]);
    if (fact->dtypes[c] != ESC_I32) return fail(ESC_ETYPE, "esc_semijoin_counts: foreign keys must be i32");
    for (int e = 0; e < d; ++e)
      if (P.fk[e] == fact->data[c]) return fail(ESC_EINVAL, "esc_semijoin_counts: repeated foreign-key column");
    if (dim_rows[d] >= (1ull << 32)) return fail(ESC_EINVAL, "esc_semijoin_counts: dimension too large");
    if (dim_rows[d] > 0 && !dev_bitmaps[d]) return fail(ESC_EINVAL, "esc_semijoin_counts: NULL bitmap");
    P.fk[d] = static_cast<const int32_t *>(fact->data[c]);
    P.bitmap[d] = dev_bitmaps[d];
    P.dim_rows[d] = (uint32_t)dim_rows[d];
    P.words[d] = (uint32_t)((dim_rows[d] + 31) / 32);
    P.smem_off[d] = ~0u;
  }
  // smallest bitmaps first into shared memory
  int order[kSjMaxDims] = {0, 1, 2, 3};
  std::sort(order, order + ndims, [&](int a, int b) { return P.words[a] < P.words[b]; });
  for (int i = 0; i < ndims; ++i) {
    const int d = order[i];
    if ((uint64_t)(smem_words + P.words[d]) * 4 <= kSjSmemBitmapBytes) {
      P.smem_off[d] = smem_words;
      smem_words += (P.words[d] + 3) & ~3u;
    }
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  void *mem = nullptr;
  cudaError_t e = cudaMallocAsync(&mem, 16 * 8, st);
  if (e != cudaSuccess) return fail(ESC_ENOMEM, std::string("esc_semijoin_counts: ") + cudaGetErrorString(e));
  e = cudaMemsetAsync(mem, 0, 16 * 8, st);
  P.hist = static_cast<unsigned long long *>(mem);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = (size_t)smem_words * 4;
  const int per_sm = smem <= 100 * 1024 ? 2 : 1;
  const uint32_t chunks = P.nrows / 16u;
  const int grid = std::max(1, std::min<int>(sms * per_sm, (int)((chunks + kSjThreads - 1) / kSjThreads)));
  if (e == cudaSuccess) {
    switch (ndims) {
      case 1: e = launch_semijoin<1>(P, smem, grid, st); break;
      case 2: e = launch_semijoin<2>(P, smem, grid, st); break;
      case 3: e = launch_semijoin<3>(P, smem, grid, st); break;
      default: e = launch_semijoin<4>(P, smem, grid, st); break;
    }
  }
  unsigned long long h[16];
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, mem, sizeof h, cudaMemcpyDeviceToHost, st);
  cudaFreeAsync(mem, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(ESC_ECUDA, std::string("esc_semijoin_counts: ") + cudaGetErrorString(e));
  const uint32_t nsub = 1u << ndims;
  for (uint32_t S = 0; S < nsub; ++S) {
    uint64_t sum = 0;
    for (uint32_t v = 0; v < 16; ++v)
      if ((v & S) == S && v < nsub) sum += h[v];
    subset_counts[S] = sum;
  }
  clear_error();
  return ESC_OK;
}
