// Plain-old-data conversion plans: built on the host from a schema and two
// views, passed to kernels by value (kernel parameters live in the constant
// bank) or stored in a device job table for the batched launch.
#pragma once

#include <cstdint>

#define MRN_MAX_COLS 64   // flattened data columns per schema (and per child)
#define MRN_MAX_GAPS 160  // zero-fill ranges of one destination
#define MRN_JAG_GAPS 8    // zero-fill ranges a jagged tile 0 takes over
#define MRN_NO_SHIFT 0xffffffffu

enum MrnKind : int32_t { K_AOS = 0, K_SOA = 1, K_AOSOA = 2 };
enum MrnDir : uint32_t { DIR_AOS_FM = 0, DIR_FM_AOS = 1, DIR_FM_FM = 2 };

// Field-major side (SoA or AoSoA) or record-major side (AoS) of a plan.
struct SidePlan {
  int32_t kind;
  uint32_t block;        // AoSoA B
  uint32_t block_shift;  // log2(B) when B is a power of two, else MRN_NO_SHIFT
  uint32_t reserved;
  uint64_t block_bytes;  // AoSoA bytes per block
  char* base;            // AoS records / AoSoA blocks
  // SoA: start of column c.  AoSoA: base + start of column c inside a block.
  char* col[MRN_MAX_COLS];
};

// One entry of the AoS record, in increasing offset order.
struct ColPlan {
  uint16_t size;     // 1, 2, 4 or 8
  int16_t fm;        // field-major column index, or FM_JLEN / FM_JBEGIN
  uint32_t aos_off;  // byte offset in the AoS record
};
#define FM_JLEN (-1)    // the jagged member's uint32 length
#define FM_JBEGIN (-2)  // the jagged member's uint64 begin

// Shared-memory tile geometry of a conversion that is staged with TMA bulk
// copies: tiles of T records; a side's tile is one contiguous range (AoS:
// T*stride bytes; AoSoA: T/B whole blocks) or, for SoA, one range per column
// packed in column order (column c at off[c] inside the tile).
#define MRN_BATCH_STAGE_BYTES 12288u  // stage of the warp-specialized pipeline
#define MRN_COL_SUB (1u << 30)
struct TileGeom {
  uint32_t tma;        // 1: full tiles go through the TMA pipeline
  uint32_t T;          // records per tile (multiple of G)
  uint32_t G;          // staging granule: lcm(32, each AoSoA B)
  uint32_t src_bytes;  // bytes of a source tile
  uint32_t dst_bytes;  // bytes of a destination tile
  uint32_t pad;        // 1: the AoS record has padding bytes (zeroed first)
  uint32_t nsize;      // columns of 8, 4, 2 and 1 bytes: n8 | n4 << 8 | n2 << 16 | n1 << 24
  // AoS destination each of whose padding bytes some field can be stored
  // wide enough to cover: nwide > 0 such fields, stored 2^w bytes wide (w
  // in col bits 28-29), zero-extended, come last in `worder`, after the
  // others in size-class order (counts in wnsize); with that table the
  // record needs no zeroing pass.  Single conversions use it; a batch's
  // stage tables keep `order`.
  uint32_t nwide, wnsize;
  // 1: the schema stores an array property interleaved (an N x E array):
  // a field-major tile holds that property's rows, column c of it at
  // off[c] + slot * es_c, and descriptor word 3 carries es_c (the
  // instance k_convert_ws<false, false, true>; batches take such jobs on
  // the direct path)
  uint32_t inter;
  uint32_t src_off[MRN_MAX_COLS];  // SoA: column offset in the tile; AoSoA: column start in a block
  uint32_t dst_off[MRN_MAX_COLS];
  // per data column: AoS offset | log2(size) << 24 | w << 28, and
  // MRN_COL_SUB for the elements after the first of an interleaved row
  // (copied with that row's bulk copy)
  uint32_t col[MRN_MAX_COLS];
  uint8_t order[MRN_MAX_COLS];     // data columns by decreasing size (stable)
  uint8_t worder[MRN_MAX_COLS];
};

// The fields of a plan the staged transform reads, copied into shared memory
// next to the column descriptors.  Each side of a tile is described by one
// row geometry, whatever its layout: record r lies in row block
// r >> shift (r / block when shift is MRN_NO_SHIFT) at byte bb * row block,
// slot r - block * row block.  AoS: block 1, shift 0, bb = stride (every
// record its own row, slot 0); SoA: shift 31 (one row, slot r); AoSoA(B):
// block B, bb = block bytes.
struct TileHdr {
  uint32_t ncols, stride, vec, pad, T, nsize;
  uint32_t sblock, sshift, sbb;  // source row geometry
  uint32_t dblock, dshift, dbb;  // destination row geometry
  // 1, 2 or 4: an AoS <-> SoA pair of that many 4-byte columns, the AoS
  // record being exactly those words in column order (records move as one
  // vector); 0x102: the AoS record is two 2-byte columns in order (one
  // 4-byte word); 0 otherwise
  uint32_t packed;
  // AoS destination: the last nwide descriptors are fields stored wider
  // than they are, over the padding that follows them (see TileGeom)
  uint32_t nwide;
};

// What the consumers of a staged tile read: the header and one descriptor
// per column in size-class order {log2 size, source offset, destination
// offset, log2 store size of a widened field (else unused)}.  A batch job
// carries its own, built on the host, and the loader brings
// it into a stage's table with one bulk copy beside the tile's data.
struct alignas(16) StageRec {
  TileHdr h;
  uint32_t pad[2];
  uint32_t d[MRN_MAX_COLS][4];
};

struct ConvPlan {
  uint64_t n;          // records
  uint64_t n_fm_pad;   // records written on the destination (AoSoA: N rounded up to B)
  uint32_t dir;        // MrnDir
  uint32_t naos;       // entries of aos_cols
  uint32_t ncols;      // field-major (data) columns
  uint32_t stride;     // AoS stride
  uint32_t aos_words;  // ceil(stride / 4)
  uint32_t vec;        // AoS access width in bytes (1, 2, 4, 8, 16)
  uint64_t tune_key;   // (schema, layout pair) key of the launch-shape cache
  ColPlan aos_cols[MRN_MAX_COLS + 2];
  uint8_t fm_size[MRN_MAX_COLS];
  uint16_t fm_es[MRN_MAX_COLS];  // field-major bytes between records' elements (size, or E * size interleaved)
  SidePlan src, dst;
  TileGeom tg;
};

// Jagged AoS <-> SoA conversion: the parents' plan (data columns plus the
// {length, begin} descriptor) and the children's plan (pool <-> child
// columns), with the offsets column and the look-back scratch.
struct JagPlan {
  ConvPlan parent;
  ConvPlan child;
  char* offsets;             // SoA offsets column (N+1 entries)
  uint32_t off_size;         // 4 or 8
  uint32_t len_off;          // AoS -> SoA: byte offset of the length in a parent record
  uint64_t offset_base;      // added to every offset written (AoS -> SoA)
  uint64_t pool_n;           // AoS -> SoA: child records in the source pool
  uint64_t capacity;         // AoS -> SoA: child capacity of the destination
  uint64_t m_src;            // SoA -> AoS: child values in the source
  uint64_t ntiles;           // AoS -> SoA: tiles of MRN_JAG_TILE parents
  unsigned long long* tile_state;  // ntiles words: flag (2 bits) | value
  unsigned int* tile_counter;      // dynamic tile id
  unsigned long long timeout_ns;   // bound of each look-back wait
  long long skip_publish_tile;     // fault injection: tile that never publishes (-1: none)
  unsigned long long* total_out;   // optional: receives the number of children
  // Single conversions: the few bytes between the regions of a single-block
  // destination, zeroed by tile 0 of the AoS -> SoA kernel (no extra launch)
  char* gap_base;
  uint32_t ngaps;
  uint32_t gap_len[MRN_JAG_GAPS];
  uint64_t gap_off[MRN_JAG_GAPS];
  // AoS -> field-major runs fused (JAG_FUSED: the tiles above scan, convert
  // the parents and gather their own children) or split (JAG_SPLIT):
  //  - k_jag_scan sums the lengths in chunks of MRN_SCAN_CHUNK parents
  //    (decoupled look-back over chunk_state), writes the children before
  //    each 32-parent group to group_base, offsets[n], and sets *noncanon
  //    (and *any_noncanon) unless the pool is canonical: every parent's
  //    children at its own offset, and no other records in the pool;
  //  - the parents' data columns and offsets are a staged conversion job
  //    (JOB_JAG_PARENTS), and a canonical pool is one more (pool record j
  //    -> child row j);
  //  - otherwise the fall-back pass gathers the children (tiles in mode
  //    JAG_CHILDREN, their bases read from the finished offsets).
  // or, in batches, split by a local check (JAG_LOCAL), with no scan: a
  // pool is canonical exactly when begin[0] = 0, begin[i] + length[i] =
  // begin[i+1] and begin[n-1] + length[n-1] = pool_n, each a comparison of
  // neighbours, and its offsets are then offset_base + the begins:
  //  - the parents job (JOB_JAG_PARENTS, in the batch's first persistent
  //    launch) writes those offsets and makes the checks; a failed one
  //    sets *noncanon and *any_noncanon;
  //  - the pool job runs in the second persistent launch, skipped when
  //    *noncanon;
  //  - otherwise the fall-back pass runs the whole job fused (look-back
  //    words tile_state, tiles ticketed from *tile_counter), rewriting the
  //    parents, offsets and children.
  uint32_t mode;
  uint32_t begin_off;               // byte offset of the begin in a parent record
  unsigned int* noncanon;
  unsigned int* any_noncanon;
  unsigned long long* group_base;   // ceil(n / 32) words
  unsigned long long* chunk_state;  // the scan's look-back words, one per chunk
  uint64_t chunk_begin;             // batches: the job's first chunk in the scan's numbering
  uint64_t nchunks;
};
// The scan of a jagged level whose lengths and begins are two columns (the
// child level of a nested member, its descriptors gathered by level 0):
// writes the level's offsets (count + 1 entries, starting at 0) and sets
// *noncanon unless the pool is canonical for them.
struct ColScan {
  const unsigned int* len;        // lengths
  const unsigned long long* beg;  // begins into the pool
  uint64_t n;                     // entries of len / beg; the count is at most n
  const unsigned long long* count;  // the count, in device memory (nullptr: n)
  uint64_t pool_n;                // records in the pool
  char* offsets;
  uint32_t off_size;              // 4 or 8
  uint32_t reserved;
  unsigned long long* state;      // one look-back word per chunk of MRN_SCAN_CHUNK
  unsigned int* counter;          // dynamic chunk id
  unsigned int* noncanon;
  unsigned long long timeout_ns;
  long long skip_publish_tile;
  // The local form (k_col_local before the scan): its word "some check
  // failed", and the scan's condition (nullptr: the scan always runs; else
  // only when *only_if != 0)
  unsigned int* local_bad;
  const unsigned int* only_if;
};

#define JAG_FUSED 0u
#define JAG_SPLIT 1u
#define JAG_CHILDREN 2u
#define JAG_LOCAL 3u
#define MRN_SCAN_CHUNK 8192u  // parents per chunk of the split scan (256 groups of 32)

// Zero-fill of the alignment holes of a destination: for each of `nblocks`
// blocks of `block_bytes`, the byte ranges [off[k], off[k] + len[k]).
struct GapPlan {
  char* base;
  uint64_t nblocks;
  uint64_t block_bytes;
  uint32_t ngaps;
  uint32_t reserved;
  uint64_t off[MRN_MAX_GAPS];
  uint32_t len[MRN_MAX_GAPS];
};

// Tiles of a staged conversion of n source records (nrec records written:
// n, or n rounded up to whole AoSoA blocks): the full tiles of T records,
// then a staged tile of the largest multiple of G inside the partial last
// tile, then one direct tile of the records left (fewer than G, plus any
// AoSoA padding slots).
struct StagedTiles {
  uint64_t nfull;  // full tiles
  uint64_t rs;     // records of the partial staged tile (0: none)
  uint64_t d0;     // first record of the direct tile (== nrec: none)
};
#ifdef __CUDACC__
__host__ __device__
#endif
inline StagedTiles staged_tiles(uint64_t n, uint64_t nrec, uint32_t T, uint32_t G) {
  StagedTiles s;
  s.nfull = n / T;
  s.rs = (n - s.nfull * T) / G * G;
  s.d0 = s.nfull * T + s.rs;
  return s;
}
#ifdef __CUDACC__
__host__ __device__
#endif
inline uint64_t staged_tile_count(uint64_t n, uint64_t nrec, uint32_t T, uint32_t G) {
  const StagedTiles s = staged_tiles(n, nrec, T, G);
  return s.nfull + (s.rs ? 1 : 0) + (nrec > s.d0 ? 1 : 0);
}

#ifndef MRN_JAG_TILE
#define MRN_JAG_TILE 1024    // parents per tile of the jagged scan
#endif
#ifndef MRN_JAG_THREADS
#define MRN_JAG_THREADS 512  // threads per jagged tile (MRN_JAG_TILE / MRN_JAG_THREADS parents each)
#endif
#ifndef MRN_JAG_CTAS
#define MRN_JAG_CTAS 3       // resident jagged CTAs per SM the kernels are compiled for
#endif
#define MRN_JAG_WARPS (MRN_JAG_THREADS / 32)
#define MRN_JAG_SMALL_TILE 256     // parents per tile of small single conversions
#define MRN_JAG_SMALL_THREADS 256
#define MRN_JAG_CHILD_GROUP 128  // child records per warp group of a jagged SoA -> AoS conversion

// One job of a batched launch: a plain conversion (plan in jp.parent), a
// jagged conversion, the parents of a split jagged conversion (a conversion
// of jp.parent that also writes the offsets from jp.group_base), or the
// zero-fill of a destination's alignment holes, and its slice of the
// batch's global tile sequence.
enum MrnJobKind : uint32_t { JOB_CONVERT = 0, JOB_JAG_A2S = 1, JOB_JAG_S2A = 2, JOB_ZERO = 3, JOB_JAG_PARENTS = 4 };
struct BatchJob {
  uint32_t kind;
  uint32_t tile_records;        // JOB_CONVERT: records per tile (multiple of 256)
  uint64_t tile_begin;          // first tile of this job in the batch
  uint64_t ntiles;
  uint64_t parent_groups;       // JOB_JAG_S2A: 32-record groups of parents
  // JOB_CONVERT: 0, or 1 + the index of the jagged job whose pool this job
  // converts; its tiles are skipped when that job's pool is not canonical
  uint32_t cond;
  // host side: 1 + the index of the split jagged job this job belongs to
  // (its pool or its parents), else 0
  uint32_t jag_link;
  union {
    JagPlan jp;                 // JOB_CONVERT uses jp.parent
    GapPlan gp;                 // JOB_ZERO
  };
  StageRec stage;               // JOB_CONVERT with staged tiles: jp.parent's stage table
};
