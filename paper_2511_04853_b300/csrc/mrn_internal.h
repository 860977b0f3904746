// Internal declarations shared by the library's host and device sources.
#pragma once

#include <cstddef>
#include <cstdint>
#include <memory>
#include <tuple>
#include <string>
#include <vector>

#include "../../include/mrn.h"
#include "mrn_plan.h"

struct mrn_schema_node;

// One flattened column of a compiled schema.  In field-major layouts a
// column lives in a storage column: its own, or, for the columns of an
// interleaved array property, the array's one storage column of E-element
// rows (`sub` = byte offset of the column's element in a row, `es` = bytes
// between consecutive records' elements, E * size).
struct MrnColumn {
  uint32_t size;
  uint32_t aos_off;
  int32_t dtype;
  std::string name;
  uint32_t es = 0;
  uint32_t sub = 0;
  uint32_t store = 0;
};

// One field-major storage column: element bytes and alignment.
struct MrnStore {
  uint32_t es;
  uint32_t align;
};

struct mrn_schema {
  // ---- builder state
  bool finalized = false;
  std::vector<std::unique_ptr<mrn_schema_node>> roots;
  std::vector<mrn_schema_node*> open_groups;
  // ---- compiled state (valid once finalized)
  std::vector<MrnColumn> cols;
  std::vector<MrnStore> stores;  // field-major storage columns
  bool interleaved = false;      // some array property is stored interleaved
  uint32_t stride = 0;
  uint32_t align = 1;
  bool has_jagged = false;
  uint32_t len_off = 0, begin_off = 0, off_size = 0;
  std::unique_ptr<mrn_schema> child;
  uint64_t hash = 0;
};

namespace mrn {

inline uint64_t align_up(uint64_t x, uint64_t a) { return (x + a - 1) / a * a; }

uint32_t dtype_size(int dtype);

// ---- layout rules (the library's own implementation)
uint64_t aosoa_block_bytes(const mrn_schema* s, uint32_t B);
uint64_t aosoa_col_start(const mrn_schema* s, uint32_t B, uint32_t c);
// Start of column c (child: the jagged child's column c) inside a
// single-block field-major view: its storage region plus its element offset.
uint64_t fm_col_start(const mrn_schema* s, int kind, uint32_t B, uint64_t n, uint64_t m, bool child, uint32_t c,
                      uint64_t m2 = 0);
// Regions of a single-block field-major view of either kind (SoA: data
// storage columns, offsets, then the child level; jagged AoSoA(B): blocks,
// offsets, then the child level), each 128-byte aligned.  The child level
// is the child schema's single-block SoA for (m, m2): child storage columns
// and, for a nested jagged member, the children's offsets and the
// grandchild storage columns.  m2 counts grandchildren (0 unless nested).
uint32_t parent_regions(const mrn_schema* s, int kind);
uint32_t fm_region_count(const mrn_schema* s, int kind);
uint64_t fm_region_bytes(const mrn_schema* s, int kind, uint32_t B, uint64_t n, uint64_t m, uint32_t r,
                         uint64_t m2 = 0);
uint64_t fm_region_start(const mrn_schema* s, int kind, uint32_t B, uint64_t n, uint64_t m, uint32_t r,
                         uint64_t m2 = 0);
uint64_t fm_total_bytes(const mrn_schema* s, int kind, uint32_t B, uint64_t n, uint64_t m, uint64_t m2 = 0);
uint64_t soa_total_bytes(const mrn_schema* s, uint64_t n, uint64_t m);
uint64_t base_bytes(const mrn_schema* s, const mrn_layout& l, uint64_t n, uint64_t m, uint64_t m2 = 0);
// A schema whose jagged member's children have a jagged member of their own.
inline bool is_nested(const mrn_schema* s) { return s->has_jagged && s->child->has_jagged; }
// Nested member of a single-block field-major view: the children's offsets
// (m + 1 entries) and grandchild column g.
uint64_t fm_child_offsets_start(const mrn_schema* s, int kind, uint32_t B, uint64_t n, uint64_t m, uint64_t m2);
uint64_t fm_gchild_col_start(const mrn_schema* s, int kind, uint32_t B, uint64_t n, uint64_t m, uint64_t m2,
                             uint32_t g);

// ---- device status word and scratch helpers (mrn_kernels.cu)
// Stream-ordered scratch for one call, from the library's own pool on the
// stream's device (it keeps reserved between calls the most its calls have
// held at once: at least 256 MiB, at most 1/64 of the device's memory or
// 4 GiB); freed in stream order with scratch_free.  MRN_ENOMEM on failure.
int scratch_alloc(void** p, size_t bytes, void* stream);
void scratch_free(void* p, void* stream);
// Returns device dev's pool memory that no call holds (mrn_scratch_release).
int scratch_release(int dev);
int device_sm_count();
int read_and_clear_status(void* stream, uint32_t* bits);
int status_from_bits(uint32_t bits);

// ---- plan building (mrn_api.cpp)
uint64_t tune_key(uint64_t hash, const mrn_layout& a, const mrn_layout& b);
// Builds the conversion plan of a validated non-jagged view pair.
int build_plan(const mrn_view& src, const mrn_view& dst, ConvPlan* p);
// Recomputes the shared-memory tile geometry of a plan for stages of
// `stage_bytes` (tg.tma = 0 when the plan cannot be staged).
void plan_tiles(const mrn_schema* s, ConvPlan* p, uint32_t stage_bytes);
// A validated non-jagged pair converted by the direct kernel only (plain
// loads and stores: mapped host memory on one side).
int convert_direct(const mrn_view& src, const mrn_view& dst, void* stream);
// Builds the plan of a validated jagged view pair.
int build_jagged_plan(const mrn_view& src, const mrn_view& dst, JagPlan* jp);
// Parents a jagged AoS -> field-major conversion covers: n, or n rounded up
// to whole AoSoA blocks (the slots after n are written as zero).
inline uint64_t jagged_tile_records(const JagPlan& jp) {
  return jp.parent.n_fm_pad > jp.parent.n ? jp.parent.n_fm_pad : jp.parent.n;
}
// The children of a jagged SoA -> AoS plan as a plain conversion of the
// child schema (child row j -> pool record j, j < m_src), with tiles.
int jagged_children_plan(const mrn_schema* s, const JagPlan& jp, ConvPlan* out);
// Zero-fill plans of a destination view's bytes that no value fills: the
// holes inside every AoSoA block, and the bytes between the regions of a
// single-block field-major view.  Returns how many plans (0..2) it wrote.
int gap_plans_of(const mrn_view& dst, GapPlan g[2]);
// Zeroes those bytes of a device view.
int zero_dst_gaps(const mrn_view& dst, void* stream);
// True when a field-major view keeps its offsets and child columns inside
// view.base (single block); its offsets pointer.
bool fm_single_block(const mrn_view& v);
char* fm_offsets(const mrn_view& v);
// A nested jagged member between AoS and a single-block field-major side,
// level by level (mrn_nested.cpp).
int convert_nested(const mrn_view& src, const mrn_view& dst, void* stream);
// Host-side validation of a device view pair; fills *is_jagged.
int validate_pair(const mrn_view* src, const mrn_view* dst, bool need_device, bool* is_jagged);

// ---- kernel launchers (mrn_kernels.cu); all asynchronous on `stream`
struct LaunchShape {
  uint32_t threads = 256;    // direct kernel: threads per CTA
  uint32_t ctas_per_sm = 0;  // 0: fill the SM (occupancy)
  uint32_t tile_records = 0; // direct kernel: records per tile (0: default)
  uint32_t generic = 0;      // 1: direct kernel even when the plan can be staged
};
// With `cond` (staged plans only) the launch does nothing when *cond != 0.
int launch_convert(const ConvPlan& p, void* stream, const LaunchShape* shape, const unsigned int* cond = nullptr);
// The stage table of a staged plan (header and column descriptors).
void fill_stage_rec(const ConvPlan& p, StageRec* out);
int launch_zero_gaps(const GapPlan& g, void* stream);
// Jagged conversions.  `scratch` (AoS->SoA only) must hold
// jagged_scratch_bytes(n, tile) bytes for the launch's tile size; it is
// cleared on `stream` first.  `small`: tiles of MRN_JAG_SMALL_TILE parents
// (single conversions of few tiles) instead of MRN_JAG_TILE.
uint64_t jagged_scratch_bytes(uint64_t n, uint32_t tile = MRN_JAG_TILE);
int launch_jagged_a2s(JagPlan& jp, void* scratch, void* stream, bool small = false);
// The same conversion split (JAG_SPLIT): the scan (group bases, offsets[n],
// the check that the pool is canonical), the parents' data columns and
// offsets as one staged conversion, the pool's records as one staged
// conversion `pool` of the child schema into the child rows when it is
// canonical, and a pass in which the tiles gather their children when it is
// not.  With `local` (jagged_local_ok holds), the local form instead
// (JAG_LOCAL): no scan, the parents' begins written as offsets with the
// pool's checks, the pool conversion when they passed, and otherwise the
// whole conversion again, fused.  jp.parent and `pool` must be staged;
// n > 0; `scratch` holds jagged_split_scratch_bytes(n) bytes.
uint64_t jagged_split_scratch_bytes(uint64_t n, size_t* group_at = nullptr);
int launch_jagged_a2s_split(JagPlan& jp, const ConvPlan& pool, void* scratch, void* stream, bool local);
int launch_jagged_s2a(const JagPlan& jp, void* stream);
// The column scan (ColScan) of one jagged level: `scratch` holds
// col_scan_scratch_bytes(cs.n) bytes (counter, pool word at +128, the local
// form's word at +192, chunk words), cleared on `stream` first.  Sets
// cs.noncanon.  With `local` (the largest offset, pool_n, fits the offset
// type), the local form first (k_col_local: the begins as offsets and the
// neighbours' checks), the scan then running only where a check failed.
// Then its gathering form (returns at once for a canonical pool unless
// `force`): `P` converts the pool's records into the level's columns,
// `capacity` rows there.
uint64_t col_scan_scratch_bytes(uint64_t n);
int launch_col_scan(ColScan& cs, void* scratch, void* stream, bool local);
int launch_col_gather(const ColScan& cs, const ConvPlan& P, uint64_t capacity, bool force, void* stream);
// The child pool of a jagged AoS -> field-major plan as a plain conversion of
// the child schema (pool record j -> child row j, j < pool_n), with tiles.
int jagged_pool_plan(const mrn_schema* s, const JagPlan& jp, ConvPlan* out);
// True when a jagged AoS -> field-major plan can run split (split runs are
// enabled, the pool fits the destination's child capacity and its
// conversion can be staged); fills *pool and gives jp->parent its staged
// tiles where it can have them.
bool jagged_split_ok(const mrn_schema* s, JagPlan* jp, ConvPlan* pool);
// A batch job may run split (JAG_LOCAL: offsets from the begins, the pool
// checked locally): its largest offset, offset_base + pool_n, fits the
// offset type.
bool jagged_local_ok(const JagPlan& jp);
// mrn_debug_set key 7: children from which a nested AoS -> field-major
// conversion splits its parent level (negative: never).
long long nested_split_children();
int launch_jagged_count(const ConvPlan& parent, uint64_t* dev_total, void* stream);
// Parents' {length, begin} columns from a field-major side's offsets.
int launch_len_begin(const char* offsets, uint32_t off_size, uint64_t n, unsigned int* len,
                     unsigned long long* beg, void* stream);
// A plain schema whose AoS record is byte for byte the parent record of the
// jagged schema s (its data fields and the "length" u32 and "begin" u64 of
// the jagged member, in offset order); field k of it is data column src[k]
// of s, or the length (-1) or the begin (-2).  nullptr when natural
// alignment cannot reproduce the record.  Cached per schema structure.
struct FlatParent {
  std::unique_ptr<mrn_schema> schema;
  std::vector<int> src;
};
const FlatParent* flat_parent_schema(const mrn_schema* s);

// Moves of byte ranges inside device memory whose source and destination
// may overlap (disjoint ones become plain copies); with elem (4 or 8) the
// range holds unsigned integers and delta is added to each.  Ranges must not
// overlap one another.
struct MoveRange {
  const char* src;
  char* dst;
  uint64_t bytes;
  uint32_t elem;
  long long delta;
};
int launch_moves(const MoveRange* r, size_t n, void* stream);
// count unsigned integers of elem bytes at dst = the one at `from`.
int launch_fill_from(char* dst, const char* from, uint64_t count, uint32_t elem, void* stream);

// Persistent launch of a batch (mrn_batch.cpp owns the device tables);
// max_chunk caps the consecutive tiles a CTA takes at once.
int launch_batch(const BatchJob* jobs, const unsigned long long* first_tile, unsigned int njobs,
                 unsigned long long total_tiles, unsigned int* counter,
                 unsigned int ctas_per_sm, unsigned int max_chunk, void* stream,
                 const unsigned int* conds = nullptr);
// The jagged AoS -> field-major jobs of a batch (their own tile numbering,
// tile_job[t] = job of tile t), one CTA per tile.
int launch_batch_jag(const BatchJob* jobs, const unsigned int* tile_job, unsigned long long total,
                     unsigned int* counter, unsigned long long* states, void* stream);
// The fall-back pass of the batch's split jagged jobs (flags[j] != 0: job j
// of `jobs` is converted whole again, fused; nothing runs unless *any !=
// 0); max_tiles: the most fused tiles of one job.
int launch_batch_jag_rest(const BatchJob* jobs, unsigned int njobs, unsigned long long max_tiles,
                          const unsigned int* flags, const unsigned int* any, void* stream);
int batch_occupancy();

// Cached launch shape for a plan (autotuner), or the default.
LaunchShape tuned_shape(const ConvPlan& p);

}  // namespace mrn

namespace mrn {
void store_tuned_shape(uint64_t key, const LaunchShape& s);
void clear_tuned_shapes();
}  // namespace mrn
