// Internal layout shared by the host compiler (esc_host.cpp) and the CUDA
// kernels (esc_scan.cu, esc_semijoin.cu).  Not part of the public ABI.
#pragma once
#include <stdint.h>
#include <string>
#include <vector>

#include "../../include/esc.h"
#include <nvtx3/nvToolsExt.h>

#ifdef __CUDACC__
#define ESC_HD __host__ __device__
#else
#define ESC_HD
#endif

namespace esc {

constexpr int kMaxInstr = 64;   // program length
constexpr int kMaxRef = 16;     // distinct columns a predicate reads
constexpr int kMaxProj = 16;    // projected columns
constexpr int kMaxPool = 128;   // int64 constants (IN lists, udf divisors)
constexpr int kMaxIn = 16;      // values in one IN list
constexpr int kMaxDepth = 8;    // evaluation stack: 8 masks of 8 bits in one u64
constexpr int kV = 8;           // rows per lane per group
constexpr int kGroup = 256;     // rows per warp group (32 lanes x 8 rows)
constexpr int kMaxTileRows = 32768;
constexpr int kMaxUnitRows = 65536;   // rows per scan work unit at most, and per compaction unit at most

// Block shapes of the scan kernel, one compiled instance each: consumer
// warps per CTA, 256-row groups each warp evaluates per decoded instruction
// (8 rows per lane per group), and whether the instance has the udf path
// (whose registers limit how many warps fit).
struct ScanShape {
  int consumers;
  int groups;
  bool udf;
};
constexpr ScanShape kScanShapes[] = {{15, 2, true}, {19, 2, false}, {19, 1, true}, {23, 1, false}, {15, 4, false}};
constexpr int kNumScanShapes = 5;
// Automatic choice, from per-predicate timings of the four shapes on a
// 60M-row table: programs reading more than kWideBytes bytes per row run
// faster with one group per pass and more warps (their many loads and
// tests need latency hiding more than fewer decodes); narrower ones with two
// groups per pass; a udf needs an instance with the udf path.
constexpr uint32_t kWideBytes = 20;
inline int auto_scan_shape(bool has_udf, bool wide) { return has_udf ? (wide ? 2 : 0) : (wide ? 3 : 1); }
// The shape a tuning asks for (consumer_warps, rows_per_pass), for a program
// with or without a udf reading `read_bytes` bytes per row: its index, the
// automatic one for (0, 0), or -1 when no compiled shape matches.
inline int scan_shape_for(uint32_t consumer_warps, uint32_t rows_per_pass, bool has_udf, uint32_t read_bytes) {
  if (consumer_warps == 0 && rows_per_pass == 0) return auto_scan_shape(has_udf, read_bytes > kWideBytes);
  for (int i = 0; i < kNumScanShapes; ++i)
    if ((uint32_t)kScanShapes[i].consumers == consumer_warps && 8u * (uint32_t)kScanShapes[i].groups == rows_per_pass &&
        (kScanShapes[i].udf || !has_udf))
      return i;
  return -1;
}

// Lane l of a warp owns, in a 256-row group, the rows
//   64*j + 2*l + i   for j in 0..3, i in 0..1;
// its 8-bit mask has bit 2*j + i for that row.  Each of the 4 loads per
// column then reads 2 consecutive elements per lane, i.e. 32 lanes read one
// contiguous run of 64 elements: conflict-free shared-memory access for
// every element width.

enum Op : uint8_t {
  OP_RANGE = 0,   // push  lo <= col <= hi
  OP_IN = 1,      // push  col in pool[off .. off+n)
  OP_UDF = 2,     // push  lo <= (col*col2) mod m <= hi   (m, magic at pool[off..off+4))
  OP_AND = 3,     // pop b, pop a, push a & b
  OP_OR = 4,      // pop b, pop a, push a | b
  OP_NOT = 5,     // top = ~top
  OP_TRUE = 6,    // push all-ones
  OP_FALSE = 7,   // push zero
  OP_INSET = 8,   // push  col in a 256-bit set of values 0..255 (8 words at pool[off..off+4))
  OP_JZ = 9,      // if the top is zero for every row the warp holds, jump to `off` (an AND's result is known)
  OP_JNZ = 10,    // if the top is all-ones for every row the warp holds, jump to `off` (an OR's result is known)
};

struct Instr {
  uint8_t op;
  uint8_t dtype;    // esc_dtype of the (first) operand column
  uint8_t dtype2;   // udf: esc_dtype of the second operand column
  uint8_t ref;      // stage slot of the (first) operand column
  uint8_t ref2;     // udf: stage slot of the second operand column
  uint8_t pad0;
  uint16_t n;       // IN: number of values
  uint16_t off;     // IN / UDF: first pool entry
  uint16_t soff;    // byte offset of the operand column's slice in a stage (set at launch)
  uint16_t soff2;   // same for the udf's second column
  uint16_t pad1;
  int64_t lo;       // inclusive range, already clamped to the operand's domain
  int64_t hi;
};
static_assert(sizeof(Instr) == 32, "Instr layout");

// MODE_COUNT: exact count.  MODE_BITMAP: count + caller's dense-key bitmap.
// MODE_SELECT: first pass of ordered compaction: count + selection bitmap and
// per-unit totals in scratch; the write kernel then materialises the rows.
enum Mode : int32_t { MODE_COUNT = 0, MODE_SELECT = 1, MODE_BITMAP = 2 };

// One sub-query as the scan kernel sees it.  Built on the host per call (or
// per prepared batch); read-only on the device.
struct Query {
  int32_t ninstr;
  int32_t nref;
  int32_t nproj;
  int32_t mode;
  uint32_t nrows;
  uint32_t tile_rows;     // rows staged per tile, a multiple of kGroup
  uint32_t ntiles;
  uint32_t unit_tiles;    // tiles per work unit (one ticket, one look-back)
  uint32_t nunits;
  uint32_t unit_base;     // first global ticket of this query
  uint32_t gmax;          // groups per full tile (tile_rows / kGroup)
  uint32_t wunit_base;    // first block of this query in the write kernel (compaction only)
  uint32_t stage_off[kMaxRef];    // byte offset of each read column in a stage
  uint8_t ref_w[kMaxRef];         // element width of each read column
  uint8_t proj_w[kMaxProj];
  int8_t proj_ref[kMaxProj];      // stage slot of the projected column (informational), or -1
  uint32_t is_const;      // the program reads no column: no work units, answered by the constant kernel
  uint32_t const_value;   // its value (0 or 1) when is_const
  uint32_t nwunits;       // compaction units (write-kernel blocks, unit totals), wunit_groups groups each
  uint32_t unit_big;      // work units 0..unit_big-1 hold unit_tiles tiles, the later ones one tile
  uint32_t wunit_groups;  // groups per compaction unit (1..kMaxUnitRows / kGroup)
  uint32_t wunit_recip;   // ceil(2^32 / wunit_groups), 0 for one group: group -> unit by a multiply-high
  uint32_t pad2[2];
  const uint8_t *ref_ptr[kMaxRef];
  const uint8_t *proj_ptr[kMaxProj];
  void *out_proj[kMaxProj];
  uint32_t *out_ids;
  uint32_t *bitmap;               // MODE_BITMAP: caller's bitmap; MODE_SELECT: selection bitmap scratch
  uint64_t capacity;
  unsigned long long *count;      // exact count accumulates here (zeroed before launch)
  unsigned long long *unit_total; // MODE_SELECT: qualifying rows per unit (zeroed)
  unsigned long long *unit_status;// write kernel's decoupled look-back words, one per unit (zeroed)
  unsigned int *tiles_left;       // completion countdown (set before launch; see the kernels)
  unsigned long long *done_ns;    // %globaltimer when the last tile finished (may be null)
  Instr code[kMaxInstr];
  int64_t pool[kMaxPool];
};
static_assert(sizeof(Query) % 16 == 0, "Query is copied with 16-byte vectors");

// Per-launch header in device scratch memory (zeroed before launch).
struct ScratchHdr {
  unsigned int ticket;   // next global tile ticket
  unsigned int status;   // esc_status raised on the device (0 = OK)
  unsigned int abort;    // set together with status; everyone stops working
  unsigned int site;     // checked build: where the first out-of-range index was found
  unsigned long long value;  // checked build: that index
  unsigned int warps_done;   // consumer warps of the scan that have finished (see Launch::count_out)
  unsigned int pad;
};
static_assert(sizeof(ScratchHdr) == 32, "ScratchHdr layout");

#ifdef __CUDACC__
// Checked build (-DESC_CHECKED, libesc_checked.so; the stand-in for a memory
// checker): ESC_INB(hdr, cond, site, value) is false when an index a kernel
// is about to use is out of range.  The first such event of a launch records
// ESC_EBOUNDS, the site number and the index in the launch header and makes
// the launch wind down; the access itself is skipped.  In the release build
// every check is `true` and compiles away.
#ifdef ESC_CHECKED
__device__ __forceinline__ bool inb(bool ok, ScratchHdr *hdr, uint32_t site, uint64_t value) {
  if (!ok && atomicCAS(&hdr->status, 0u, (unsigned)ESC_EBOUNDS) == 0u) {
    hdr->site = site;
    hdr->value = value;
    __threadfence();
    atomicExch(&hdr->abort, 1u);
  }
  return ok;
}
#define ESC_INB(hdr, cond, site, value) esc::inb((cond), (hdr), (site), (uint64_t)(value))
#else
#define ESC_INB(hdr, cond, site, value) true
#endif
#endif

}  // namespace esc

// ------------------------------------------------------------------ host side
struct esc_table {
  uint64_t nrows;
  std::vector<std::string> names;
  std::vector<int32_t> dtypes;
  std::vector<const void *> data;
};

struct esc_pred {
  const esc_table *table;
  esc_tuning tuning{32768u, 512u, 8, 0, 0};
  std::string text;
  int32_t ninstr = 0;
  std::vector<int32_t> ref_cols;    // table column index of each stage slot
  std::vector<int32_t> proj_cols;   // table column index of each projected column
  std::vector<int32_t> proj_ref;    // stage slot of each projected column or -1
  std::vector<esc::Instr> code;
  std::vector<int64_t> pool;
  int32_t depth = 0;
};

namespace esc {
int dtype_width(int32_t dt);
esc_status fail(esc_status s, const std::string &msg);
void clear_error();
// The status a launch's header reports, as an error with its message
// (ESC_EBOUNDS: the site and the index the checked build recorded).
esc_status device_status(const ScratchHdr &h, const char *where);
// Test hook: true when a device allocation of the library is to fail
// (esc_debug_fail_allocs counts them down).
bool inject_alloc_failure();
// A named range on the calling host thread for timeline tools (NVTX; with
// no tool attached a push or pop is a call through a no-op pointer).  Every
// public entry point that launches GPU work opens one.
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};
#define ESC_RANGE(name) ::esc::NvtxRange esc_nvtx_range_(name)
// Defaults of esc_tuning.
constexpr esc_tuning kDefaultTuning{32768u, 512u, 8, 0, 0};
// Fills the static part of a Query (program, read columns, projection) for a pred.
void fill_query_program(const esc_pred *p, Query *q);
// Granlund-Montgomery unsigned magic for divisor d (Fig. 4.1 of their paper).
void udiv_magic(uint64_t d, uint64_t *mult, int32_t *sh1, int32_t *sh2);
}  // namespace esc
