// Exact semi-join cardinalities over dense keys: the COUNT(*) foreign-key
// join queries of the paper's overhead experiments (Sec. 3.1: lineitem joined
// with a filtered orders / part / supplier table) generalised to a star
// schema.  One pass over the fact table's foreign-key columns:
//   m(i) = sum_d [0 <= fk_d[i] < D_d and bitmap_d bit fk_d[i]] << d,
//   h[v] = |{ i : m(i) = v }|          (2^ndims bins)
// and on the host, for every dimension subset S,
//   count(S) = sum over v that contain S of h[v]   (superset sum).
//
// Kernel shape: persistent grid of one block of 512 threads per SM (shared
// memory sized to the bitmaps it holds, the rest of the SM's on-chip memory
// left to L1; up to 128 registers a thread); each thread streams 8 rows per
// step with 16-byte non-allocating loads of every FK column (4 rows per
// load).  The kernel is specialised on how many bitmaps sit in shared memory
// (dimensions are ordered smallest bitmap first, so the shared ones come
// first): each probe is then a fixed sequence -- clamp the word index, load,
// shift, mask with the bounds test.  The 16 bins are 8-bit
// counters in two 64-bit registers, added into shared per-block bins (warp
// reductions) before they can overflow.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>

#include "esc_internal.h"

namespace esc {

constexpr int kSjThreads = 512;
constexpr int kSjMaxDims = 4;
constexpr uint32_t kSjSmemBitmapBytes = 96 * 1024;  // shared copies of the smaller bitmaps

struct SjParams {
  const int32_t *fk[kSjMaxDims];       // in probe order
  const uint32_t *bitmap[kSjMaxDims];
  uint32_t dim_rows[kSjMaxDims];
  uint32_t smem_off[kSjMaxDims];       // word offset in shared memory (the first NS dimensions)
  uint32_t words[kSjMaxDims];
  int32_t ndims;
  uint32_t nrows;
  unsigned long long *hist;            // 16 bins, zeroed
  ScratchHdr *hdr;                     // launch header (zeroed): the checked build's findings
  uint32_t smem_words;                 // shared-memory words the launch has (checked build)
};

__device__ __forceinline__ int4 ld_stream(const int32_t *p) {
  int4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.s32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p));
  return v;
}

// Bit `key` of a bitmap of `rows` bits, 0 when key is out of range (negative
// keys wrap to large unsigned values).  A shared-memory copy ends with a zero
// word at index `wlast` and has the bits past `rows` cleared, so clamping the
// word index is the whole bounds test there; a bitmap read in place is
// tested explicitly.
__device__ __forceinline__ uint32_t test_bit(const uint32_t *bm, uint32_t key, uint32_t rows, uint32_t wlast,
                                             bool shared) {
  if (shared) return (bm[min(key >> 5, wlast)] >> (key & 31u)) & 1u;
  const uint32_t w = __ldg(&bm[min(key >> 5, wlast)]);
  return key < rows ? (w >> (key & 31u)) & 1u : 0u;
}

// The same, in the checked build: the word index is tested against the
// bitmap's words (in shared memory: its copy and the zero word).
__device__ __forceinline__ uint32_t test_bit_checked(const uint32_t *bm, uint32_t key, uint32_t rows, uint32_t wlast,
                                                     bool shared, uint32_t words, ScratchHdr *hdr) {
  const uint32_t wi = min(key >> 5, wlast);
  if (!ESC_INB(hdr, wi < (shared ? words + 1 : words), 32, wi)) return 0u;
  return test_bit(bm, key, rows, wlast, shared);
}

__device__ __forceinline__ void bump(uint64_t &lo, uint64_t &hi, uint32_t m) {
  const uint64_t inc = 1ull << (8u * (m & 7u));
  if (m & 8u) hi += inc; else lo += inc;
}

// Adds this warp's byte counters into the block's bins.
__device__ __forceinline__ void flush(uint64_t &lo, uint64_t &hi, unsigned int *bins) {
#pragma unroll
  for (int v = 0; v < 8; ++v) {
    const uint32_t a = __reduce_add_sync(0xffffffffu, (uint32_t)((lo >> (8 * v)) & 0xffu));
    const uint32_t b = __reduce_add_sync(0xffffffffu, (uint32_t)((hi >> (8 * v)) & 0xffu));
    if ((threadIdx.x & 31) == 0) {
      if (a) atomicAdd(&bins[v], a);
      if (b) atomicAdd(&bins[v + 8], b);
    }
  }
  lo = hi = 0;
}

template <int ND, int NS>
__device__ __forceinline__ uint32_t probe_row(const SjParams &P, const uint32_t *const (&bm)[ND],
                                              const uint32_t (&wmax)[ND], const int32_t (&k)[ND]) {
  uint32_t m = 0;
#pragma unroll
  for (int d = 0; d < ND; ++d) {
#ifdef ESC_CHECKED
    m |= test_bit_checked(bm[d], (uint32_t)k[d], P.dim_rows[d], wmax[d], d < NS, P.words[d], P.hdr) << d;
#else
    m |= test_bit(bm[d], (uint32_t)k[d], P.dim_rows[d], wmax[d], d < NS) << d;
#endif
  }
  return m;
}

template <int ND, int NS>
__global__ void __launch_bounds__(kSjThreads, 1) semijoin_kernel(const __grid_constant__ SjParams P) {
  extern __shared__ __align__(16) uint32_t sbm[];
  __shared__ unsigned int bins[16];
#pragma unroll
  for (int d = 0; d < NS; ++d) {
    // the words (bits past the last row cleared) and a zero word
    const uint32_t tail = P.dim_rows[d] & 31u;
    for (uint32_t w = threadIdx.x; w <= P.words[d]; w += blockDim.x) {
      uint32_t x = w < P.words[d] ? P.bitmap[d][w] : 0u;
      if (w + 1 == P.words[d] && tail) x &= (1u << tail) - 1u;
      if (ESC_INB(P.hdr, P.smem_off[d] + w < P.smem_words, 31, P.smem_off[d] + w)) sbm[P.smem_off[d] + w] = x;
    }
  }
  if (threadIdx.x < 16) bins[threadIdx.x] = 0;
  __syncthreads();
  const uint32_t *bm[ND];
  uint32_t wmax[ND];
#pragma unroll
  for (int d = 0; d < ND; ++d) {
    bm[d] = d < NS ? sbm + P.smem_off[d] : P.bitmap[d];
    wmax[d] = d < NS ? P.words[d] : P.words[d] - 1u;  // shared: the zero word; global: words >= 1
  }

  uint64_t lo = 0, hi = 0;
  uint32_t pending = 0;
  const uint32_t nchunks = P.nrows / 8u;  // 8 rows per thread step
  const uint32_t stride = gridDim.x * blockDim.x;
  // warp-uniform trip count (the flush is warp-collective); lanes past the end idle
  for (uint32_t wb = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); wb < nchunks; wb += stride) {
    const uint32_t ch = wb + (threadIdx.x & 31u);
    if (ch < nchunks && ESC_INB(P.hdr, (uint64_t)ch * 8 + 8 <= P.nrows, 30, ch)) {
    int4 v[ND][2];
#pragma unroll
    for (int d = 0; d < ND; ++d)
#pragma unroll
      for (int q = 0; q < 2; ++q) v[d][q] = ld_stream(P.fk[d] + (size_t)ch * 8 + 4 * q);
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      int32_t k0[ND], k1[ND], k2[ND], k3[ND];
#pragma unroll
      for (int d = 0; d < ND; ++d) {
        k0[d] = v[d][q].x;
        k1[d] = v[d][q].y;
        k2[d] = v[d][q].z;
        k3[d] = v[d][q].w;
      }
      bump(lo, hi, probe_row<ND, NS>(P, bm, wmax, k0));
      bump(lo, hi, probe_row<ND, NS>(P, bm, wmax, k1));
      bump(lo, hi, probe_row<ND, NS>(P, bm, wmax, k2));
      bump(lo, hi, probe_row<ND, NS>(P, bm, wmax, k3));
    }
    }
    pending += 8;
    if (pending >= 248) {  // 8-bit counters: flush before any can pass 255
      flush(lo, hi, bins);
      pending = 0;
    }
  }
  // ragged tail: rows nchunks*8 .. nrows-1, one per thread of block 0
  if (blockIdx.x == 0) {
    const uint32_t r = nchunks * 8u + threadIdx.x;
    if (r < P.nrows) {
      int32_t k[ND];
#pragma unroll
      for (int d = 0; d < ND; ++d) k[d] = P.fk[d][r];
      bump(lo, hi, probe_row<ND, NS>(P, bm, wmax, k));
    }
  }
  flush(lo, hi, bins);
  __syncthreads();
  if (threadIdx.x < 16 && bins[threadIdx.x]) atomicAdd(&P.hist[threadIdx.x], (unsigned long long)bins[threadIdx.x]);
}

template <int ND, int NS>
cudaError_t launch_semijoin(const SjParams &P, size_t smem, int grid, cudaStream_t st) {
  static std::once_flag once[64];
  static cudaError_t attr[64];
  int dev = 0;
  cudaGetDevice(&dev);
  std::call_once(once[dev & 63], [&] {
    attr[dev & 63] = cudaFuncSetAttribute(semijoin_kernel<ND, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)kSjSmemBitmapBytes);
    // as much L1 as the launch leaves: a bitmap probed in place (too large for
    // shared memory) is then mostly served from L1 (its hot words: Zipf keys)
    if (attr[dev & 63] == cudaSuccess)
      attr[dev & 63] = cudaFuncSetAttribute(semijoin_kernel<ND, NS>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                            (int)cudaSharedmemCarveoutMaxL1);
  });
  if (attr[dev & 63] != cudaSuccess) return attr[dev & 63];
  semijoin_kernel<ND, NS><<<grid, kSjThreads, smem, st>>>(P);
  return cudaGetLastError();
}

template <int ND>
cudaError_t launch_nd(const SjParams &P, int ns, size_t smem, int grid, cudaStream_t st) {
  switch (ns) {
    case 0: return launch_semijoin<ND, 0>(P, smem, grid, st);
    case 1: return launch_semijoin<ND, (ND >= 1 ? 1 : 0)>(P, smem, grid, st);
    case 2: return launch_semijoin<ND, (ND >= 2 ? 2 : 0)>(P, smem, grid, st);
    case 3: return launch_semijoin<ND, (ND >= 3 ? 3 : 0)>(P, smem, grid, st);
    default: return launch_semijoin<ND, ND>(P, smem, grid, st);
  }
}

// Stream-ordered allocation from the library's device pool (esc_scan.cu).
esc_status alloc_async(void **p, size_t bytes, cudaStream_t st);

}  // namespace esc

using namespace esc;

extern "C" esc_status esc_semijoin_counts(const esc_table *fact, const char *const *fk_cols, int32_t ndims,
                                          const uint32_t *const *dev_bitmaps, const uint64_t *dim_rows,
                                          uint64_t *subset_counts, void *stream) {
  ESC_RANGE("esc_semijoin_counts");
  if (!fact || !fk_cols || !dev_bitmaps || !dim_rows || !subset_counts)
    return fail(ESC_EINVAL, "esc_semijoin_counts: NULL argument");
  if (ndims < 1 || ndims > kSjMaxDims) return fail(ESC_EINVAL, "esc_semijoin_counts: ndims must be 1..4");
  SjParams P;
  std::memset(&P, 0, sizeof P);
  P.ndims = ndims;
  P.nrows = (uint32_t)fact->nrows;
  const int32_t *fk[kSjMaxDims];
  uint32_t words[kSjMaxDims];
  for (int d = 0; d < ndims; ++d) {
    if (!fk_cols[d]) return fail(ESC_EINVAL, "esc_semijoin_counts: NULL column name");
    int c = -1;
    for (size_t i = 0; i < fact->names.size(); ++i)
      if (fact->names[i] == fk_cols[d]) c = (int)i;
    if (c < 0) return fail(ESC_EINVAL, std::string("esc_semijoin_counts: unknown column ") + fk_cols[d]);
    if (fact->dtypes[c] != ESC_I32) return fail(ESC_ETYPE, "esc_semijoin_counts: foreign keys must be i32");
    for (int e = 0; e < d; ++e)
      if (fk[e] == fact->data[c]) return fail(ESC_EINVAL, "esc_semijoin_counts: repeated foreign-key column");
    if (dim_rows[d] >= (1ull << 32)) return fail(ESC_EINVAL, "esc_semijoin_counts: dimension too large");
    if (dim_rows[d] > 0 && !dev_bitmaps[d]) return fail(ESC_EINVAL, "esc_semijoin_counts: NULL bitmap");
    fk[d] = static_cast<const int32_t *>(fact->data[c]);
    words[d] = (uint32_t)((dim_rows[d] + 31) / 32);
  }
  // probe order: smallest bitmap first; a prefix of them goes to shared memory
  int order[kSjMaxDims] = {0, 1, 2, 3};
  std::stable_sort(order, order + ndims, [&](int a, int b) { return words[a] < words[b]; });
  uint32_t smem_words = 0;
  int ns = 0;
  for (int i = 0; i < ndims; ++i) {
    const int d = order[i];
    P.fk[i] = fk[d];
    P.bitmap[i] = dev_bitmaps[d];
    P.dim_rows[i] = (uint32_t)dim_rows[d];
    P.words[i] = words[d];
    P.smem_off[i] = ~0u;
    // shared copy: the words and a zero word (an empty dimension is that word alone)
    if (ns == i && (uint64_t)(smem_words + words[d] + 1) * 4 <= kSjSmemBitmapBytes) {
      P.smem_off[i] = smem_words;
      smem_words += (words[d] + 1 + 3) & ~3u;
      ++ns;
    }
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  void *mem = nullptr;
  // the library's device pool (memory stays reserved between calls): 16
  // bins, then the launch header
  if (esc_status as = alloc_async(&mem, 16 * 8 + sizeof(ScratchHdr), st); as != ESC_OK) return as;
  cudaError_t e = cudaMemsetAsync(mem, 0, 16 * 8 + sizeof(ScratchHdr), st);
  P.hist = static_cast<unsigned long long *>(mem);
  P.hdr = reinterpret_cast<ScratchHdr *>(static_cast<uint8_t *>(mem) + 16 * 8);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = (size_t)std::max<uint32_t>(smem_words, 4) * 4;
  P.smem_words = (uint32_t)(smem / 4);
  const uint32_t chunks = P.nrows / 8u;
  const int grid = std::max(1, std::min<int>(sms, (int)((chunks + kSjThreads - 1) / kSjThreads)));
  if (e == cudaSuccess) {
    switch (ndims) {
      case 1: e = launch_nd<1>(P, ns, smem, grid, st); break;
      case 2: e = launch_nd<2>(P, ns, smem, grid, st); break;
      case 3: e = launch_nd<3>(P, ns, smem, grid, st); break;
      default: e = launch_nd<4>(P, ns, smem, grid, st); break;
    }
  }
  struct {
    unsigned long long h[16];
    ScratchHdr hdr;
  } back;
  unsigned long long *h = back.h;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&back, mem, sizeof back, cudaMemcpyDeviceToHost, st);
  cudaFreeAsync(mem, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(ESC_ECUDA, std::string("esc_semijoin_counts: ") + cudaGetErrorString(e));
  if (back.hdr.status != 0) return device_status(back.hdr, "esc_semijoin_counts");
  // bins are in probe order (bit i = dimension order[i]): back to the caller's bits
  const uint32_t nsub = 1u << ndims;
  uint64_t hc[16] = {0};
  for (uint32_t v = 0; v < nsub; ++v) {
    uint32_t vc = 0;
    for (int i = 0; i < ndims; ++i) vc |= ((v >> i) & 1u) << order[i];
    hc[vc] += h[v];
  }
  for (uint32_t S = 0; S < nsub; ++S) {
    uint64_t sum = 0;
    for (uint32_t v = 0; v < nsub; ++v)
      if ((v & S) == S) sum += hc[v];
    subset_counts[S] = sum;
  }
  clear_error();
  return ESC_OK;
}
