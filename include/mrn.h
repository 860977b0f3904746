/*
 * mrn.h — C ABI of the B300 (sm_103a) layout-conversion library.
 *
 * The library converts collections of records between memory layouts, as
 * described by "Marionette: Data Structure Description and Management for
 * Heterogeneous Computing" (arXiv 2511.04853):
 *
 *   - a record schema is a list of properties (Sec. V): per-item properties,
 *     fixed-extent array properties, sub-groups and one jagged vector
 *     property;
 *   - a collection is stored in a layout (Sec. IV, Sec. VI-B): array of
 *     structures (AoS), structure of arrays (SoA) or blocks of B records
 *     (AoSoA(B)), in a memory context (Sec. VI-A: host, pinned host, device);
 *   - a transfer between two layouts copies every property of every object
 *     (Sec. VI-B "Transferring data between layouts"); between memory
 *     contexts it is fused with the copy (Sec. VI-A, memcopy_with_context).
 *
 * Conventions for every call:
 *   - Every function returns an int status (MRN_OK = 0, else an MRN_E* code)
 *     unless documented otherwise.  No C++ exception crosses this boundary.
 *   - Pointers are plain host or device addresses.  The caller owns every
 *     data buffer; the library owns schemas, its scratch and staging memory,
 *     batches and servers.
 *   - Device work is ordered on the caller's stream (`mrn_stream` is a
 *     cudaStream_t; NULL is the legacy default stream) and is asynchronous
 *     unless documented otherwise.  Errors found on the host are returned at
 *     once; errors found by a kernel (offset overflow, bad child indices, a
 *     destination that is too small, a wait that timed out) are recorded in
 *     a per-device status word, returned and cleared by mrn_sync().
 *   - Only the current CUDA device is used; device views must name it.
 *   - Source and destination buffers must not overlap.
 */
#ifndef MRN_H
#define MRN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status codes */
#define MRN_OK 0
#define MRN_EINVAL 1       /* bad schema, view or argument                    */
#define MRN_ESIZE 2        /* a destination (or child capacity) is too small  */
#define MRN_EALIGN 3       /* a column is not aligned to its element size     */
#define MRN_EOVERFLOW 4    /* a prefix sum does not fit the offset type       */
#define MRN_ENOMEM 5       /* allocation failed / request exceeds a budget    */
#define MRN_ETIMEOUT 6     /* a bounded device or host wait expired           */
#define MRN_ECUDA 7        /* a CUDA runtime call failed                      */
#define MRN_EBUSY 8        /* not finished yet (server poll)                  */
#define MRN_ENOTFOUND 9    /* unknown ticket                                  */
#define MRN_EUNSUPPORTED 10 /* valid request this build does not implement    */

/* Human-readable name of a status code (static string, never NULL). */
const char* mrn_status_str(int status);
/* Library version, major*10000 + minor*100 + patch. */
int mrn_version(void);

/* ------------------------------------------------------------------ schema */
/* Element types of a property.  MRN_BOOL is one byte, copied verbatim. */
typedef enum mrn_dtype {
  MRN_U8 = 0, MRN_I8 = 1, MRN_U16 = 2, MRN_I16 = 3, MRN_U32 = 4, MRN_I32 = 5,
  MRN_U64 = 6, MRN_I64 = 7, MRN_F32 = 8, MRN_F64 = 9, MRN_BOOL = 10
} mrn_dtype;

typedef struct mrn_schema mrn_schema; /* opaque, library-owned */

/* Creates an empty, unfinalized schema.  *out receives the handle. */
int mrn_schema_create(mrn_schema** out);

/* Appends a per-item property (extent 1) or an array property of `extent`
 * elements (Sec. V, "per-item property", "array property").  An array of
 * extent E is stored as E separate columns in SoA/AoSoA layouts and as a C
 * array inside the AoS record.  `name` is copied (max 63 bytes). */
int mrn_schema_add_field(mrn_schema* s, const char* name, int dtype, uint32_t extent);

/* Appends an array property of `extent` elements stored interleaved: in
 * SoA its E elements per record form ONE column of N rows of E elements
 * (record i's element k at byte (i * extent + k) * size of the column), the
 * array property's single-array interface (Sec. V); in an AoSoA(B) block
 * the array is a B x extent member; the AoS record is the same as for
 * mrn_schema_add_field.  The array still flattens to `extent` columns
 * (mrn_schema_column reports fm_stride = extent * size); a per-column SoA
 * view passes, for column k of the array, the address of element k of the
 * first row.  extent * size <= 65535.  Conversions between any layouts run
 * on the device (mrn_convert, batches); transfers, servers, collections and
 * jagged child schemas with such a property return MRN_EUNSUPPORTED. */
int mrn_schema_add_field_interleaved(mrn_schema* s, const char* name, int dtype, uint32_t extent);

/* Opens / closes a sub-group property (Sec. V, "sub-group property"): its
 * members are stored as separate columns, as if declared at the top level;
 * in the AoS record the group is a nested struct (aligned to its widest
 * member, size rounded up to that alignment).  Groups may nest. */
int mrn_schema_begin_group(mrn_schema* s, const char* name);
int mrn_schema_end_group(mrn_schema* s);

/* Appends a jagged vector property (Sec. V, "jagged vector property"): a
 * per-object vector of child records described by the finalized schema
 * `child` (copied; the caller keeps ownership of `child`).  `offset_dtype`
 * is MRN_U32 or MRN_U64, the type of the prefix sum of the sizes.
 *   AoS side: the member is stored as {uint32 length; uint64 begin} at its
 *     position in the record; `begin` indexes a separate pool of child
 *     records (view.child_pool, child AoS layout).
 *   SoA side: an offsets column of N+1 entries (offsets[0] = 0 unless an
 *     offset base is given, offsets[N] = number of children) and one column
 *     per flattened child property, holding all children contiguously.
 * At most one jagged property per schema.  The child may itself have one
 * jagged property (nesting once, Sec. V: the children are a collection
 * described by properties) whose own child is not jagged:
 *   AoS side: the children's {length, begin} index a second pool
 *     (view.grandchild_pool, view.n_grandchildren records);
 *   field-major side (single block only, view.base): after the parents'
 *     offsets, the child level is laid out as the child schema's
 *     single-block SoA for (n_children, n_grandchildren): child columns,
 *     the children's offsets (n_children + 1), the grandchild columns.
 *   Nested members convert between AoS and SoA / AoSoA(B) with
 *   mrn_convert, asynchronously like any conversion (too few child or
 *   grandchild slots record MRN_ESIZE, reported by mrn_sync).  Other calls
 *   return MRN_EUNSUPPORTED for them.
 * Returns MRN_EINVAL for deeper nesting or two jagged properties;
 * MRN_EUNSUPPORTED for a child with an interleaved array property. */
int mrn_schema_add_jagged(mrn_schema* s, const char* name, int offset_dtype,
                          const mrn_schema* child);

/* Compiles the schema (flattening, AoS offsets, column tables).  After this
 * the schema is immutable and may be shared between threads. */
int mrn_schema_finalize(mrn_schema* s);

/* Frees a schema.  Views that point to it must not be used afterwards. */
void mrn_schema_destroy(mrn_schema* s);

typedef struct mrn_schema_info {
  uint32_t n_columns;      /* flattened data columns (jagged member excluded) */
  uint32_t aos_stride;     /* bytes per AoS record                           */
  uint32_t aos_align;      /* alignment of the AoS record                    */
  int32_t has_jagged;      /* 1 if the schema has a jagged property          */
  uint32_t jag_length_offset; /* AoS offset of the jagged uint32 length      */
  uint32_t jag_begin_offset;  /* AoS offset of the jagged uint64 begin       */
  uint32_t offset_size;    /* 4 or 8 (jagged), else 0                        */
  uint32_t child_columns;  /* flattened child columns (jagged), else 0       */
  uint32_t child_stride;   /* bytes per child AoS record (jagged), else 0    */
  uint32_t reserved;
  uint64_t hash;           /* structural hash (sizes, offsets, nesting)      */
} mrn_schema_info;

typedef struct mrn_column_info {
  uint32_t size;        /* element bytes: 1, 2, 4 or 8                       */
  uint32_t aos_offset;  /* byte offset inside the AoS record                 */
  int32_t dtype;        /* mrn_dtype                                         */
  uint32_t fm_stride;   /* bytes between consecutive records' elements in
                           SoA / AoSoA: size, or extent * size for a column
                           of an interleaved array property                 */
  char name[128];       /* dotted path, "[k]" suffix for array elements      */
} mrn_column_info;

/* Information about a finalized schema. */
int mrn_schema_info_get(const mrn_schema* s, mrn_schema_info* out);
/* Column c (0 <= c < n_columns) of a finalized schema; `child` = 1 selects
 * the jagged child's columns. */
int mrn_schema_column(const mrn_schema* s, int child, uint32_t c, mrn_column_info* out);
/* AoS stride and the AoS offsets of the n_columns data columns (up to cap). */
int mrn_schema_aos_layout(const mrn_schema* s, size_t* stride, size_t* offsets, size_t cap);

/* ------------------------------------------------------------------ layout */
typedef enum mrn_layout_kind { MRN_AOS = 0, MRN_SOA = 1, MRN_AOSOA = 2 } mrn_layout_kind;
typedef enum mrn_memctx {
  MRN_MEM_HOST = 0,        /* pageable host memory                           */
  MRN_MEM_HOST_PINNED = 1, /* page-locked host memory (cudaHostAlloc)        */
  MRN_MEM_DEVICE = 2       /* device global memory of `device`               */
} mrn_memctx;

/* kind + block size B (AoSoA only; B >= 1, ignored otherwise).
 *   AoS:      record i at base + i*aos_stride.
 *   SoA:      column c is a contiguous array; either view.columns[c], or, if
 *             view.columns is NULL, the single-block ("DynamicStruct",
 *             Sec. VI-B) arrangement inside view.base: regions in order
 *             [data columns][offsets][child columns], each region starting at
 *             a multiple of 128 bytes from base, sized for N records / N+1
 *             offsets / M children.
 *   AoSoA(B): block b at base + b*block_bytes is the C struct
 *             { T_0 c0[B]; T_1 c1[B]; ... } of the flattened columns; record
 *             i is slot i%B of block i/B.  For a jagged schema the blocks
 *             hold the parent columns and are followed, inside view.base,
 *             by the offsets (N+1) and the child columns (M each), each
 *             region starting at a multiple of 128 bytes (view.offsets /
 *             view.child_columns may point elsewhere instead), as the
 *             paper's size tags and global properties allow for any
 *             layout (Sec. V, Sec. VI-B).
 * In every destination, bytes no property writes (AoS padding, alignment
 * holes, unused AoSoA slots of the last block) are written as zero. */
typedef struct mrn_layout {
  int32_t kind;
  uint32_t block;
} mrn_layout;

typedef struct mrn_view {
  const mrn_schema* schema;
  mrn_layout layout;
  int32_t mem;            /* mrn_memctx                                       */
  int32_t device;         /* CUDA ordinal for MRN_MEM_DEVICE                  */
  uint64_t n_records;     /* N, size tag of the objects                       */
  uint64_t n_children;    /* M, size tag of the jagged values: the number of
                             child records (source) or the child capacity
                             (destination)                                    */
  void* base;             /* AoS records / AoSoA blocks / single-block SoA    */
  void* const* columns;   /* SoA: optional n_columns column pointers          */
  void* offsets;          /* SoA jagged: optional offsets column (N+1)        */
  void* const* child_columns; /* SoA jagged: optional child column pointers   */
  void* child_pool;       /* AoS jagged: child records (child AoS layout)     */
  uint64_t offset_base;   /* SoA jagged destination: added to every offset
                             (shards of one collection); 0 otherwise          */
  /* Nested jagged member (the children have a jagged member of their own):
   * the second level's size tag and, on the AoS side, the pool of the
   * children's child records that their {length, begin} index. */
  uint64_t n_grandchildren; /* M2: grandchildren (source) / capacity (dst)  */
  void* grandchild_pool;    /* AoS side: grandchild records                  */
} mrn_view;

/* Bytes needed for view.base of a collection of n records / m children in
 * `layout` (AoS: records only; the child pool is mrn_child_pool_bytes). */
int mrn_required_bytes(const mrn_schema* s, mrn_layout layout, uint64_t n, uint64_t m, size_t* out);
/* Bytes of an AoS child pool of m child records. */
int mrn_child_pool_bytes(const mrn_schema* s, uint64_t m, size_t* out);
/* For a nested jagged member: view.base bytes with m2 grandchildren, the
 * bytes of an AoS pool of m2 grandchild records, and the start of item r
 * of a single-block field-major view (SoA: data column r < n_columns, the
 * offsets at n_columns, then the child level's items counted the same way:
 * child columns, the children's offsets, grandchild columns; AoSoA(B):
 * blocks at 0, offsets at 1, then the child level's items). */
int mrn_required_bytes_nested(const mrn_schema* s, mrn_layout layout, uint64_t n, uint64_t m, uint64_t m2,
                              size_t* out);
int mrn_grandchild_pool_bytes(const mrn_schema* s, uint64_t m2, size_t* out);
int mrn_region_offset_nested(const mrn_schema* s, mrn_layout layout, uint64_t n, uint64_t m, uint64_t m2,
                             uint32_t r, size_t* out);
/* Start of region r inside a single-block SoA of n records / m children:
 * r < n_columns: data column r; r == n_columns: offsets; then child columns.
 * Each stored column starts at a multiple of 128 bytes; the columns of an
 * interleaved array share one stored N x extent array and column k of it
 * starts at element k of its first row. */
int mrn_soa_region_offset(const mrn_schema* s, uint64_t n, uint64_t m, uint32_t r, size_t* out);
/* Start of region r inside view.base for either field-major layout: SoA as
 * mrn_soa_region_offset; jagged AoSoA(B): r == 0 the blocks, r == 1 the
 * offsets, r >= 2 child column r - 2.  Other layouts: MRN_EINVAL. */
int mrn_region_offset(const mrn_schema* s, mrn_layout layout, uint64_t n, uint64_t m, uint32_t r,
                      size_t* out);
/* AoSoA(B): bytes per block, and the start of column c inside a block. */
int mrn_aosoa_block_bytes(const mrn_schema* s, uint32_t B, size_t* out);
int mrn_aosoa_column_offset(const mrn_schema* s, uint32_t B, uint32_t c, size_t* out);

/* --------------------------------------------------------------- convert */
/* Converts src into dst, both MRN_MEM_DEVICE on the current device, same
 * schema and n_records.  Any pair of AoS / SoA / AoSoA(B) layouts for a
 * schema without a jagged property.  For a jagged schema, AoS to or from
 * either field-major layout (SoA, AoSoA(B); "SoA" below means either), and
 * one field-major layout to another (the parents change layout; offsets
 * and child values are copied as they are, dst.n_children >= src's):
 *   AoS -> SoA: offsets = offset_base + exclusive prefix sum of the lengths
 *     (N+1 entries), child values gathered from child_pool[begin + k] in
 *     object order.  dst.n_children is the child capacity; children beyond it
 *     are not written and MRN_ESIZE is recorded.  Sum of lengths larger than
 *     the offset type records MRN_EOVERFLOW; begin + length beyond
 *     src.n_children records MRN_EINVAL (the bad children are not read).
 *   SoA -> AoS: length = offsets[i+1] - offsets[i], begin = offsets[i]; the
 *     src.n_children child values are written to pool slots 0..M-1
 *     (dst.n_children must be >= src.n_children, else MRN_ESIZE).
 * Asynchronous on `stream`.  The CUDA path is the only path: without a
 * device the call returns MRN_ECUDA. */
int mrn_convert(const mrn_view* src, const mrn_view* dst, void* stream);

/* Waits for `stream` and returns the first error a kernel recorded since the
 * previous mrn_sync on this device (then clears it), else MRN_OK.  When
 * several were recorded the order is ETIMEOUT, EOVERFLOW, EINVAL, ESIZE. */
int mrn_sync(void* stream);
/* As mrn_sync, but returns every recorded code: bit k of *bits = code k. */
int mrn_sync_bits(void* stream, uint32_t* bits);

/* Device scratch.  The calls that need scratch (jagged and nested
 * conversions, large staged conversions, batches' look-back words) take it
 * in stream order from a memory pool the library owns on each device.
 * Between calls the pool keeps reserved the most its calls have held at
 * once, so that a repeated call does not map its scratch again: at least
 * 256 MiB, at most 1/64 of the device's memory or 4 GiB, whichever is less
 * (a 2,097,152-parent nested conversion holds about 0.5 GB).  This call
 * returns the pool's memory that no call holds to the device and resets
 * the amount kept to 256 MiB.  MRN_OK (also when the library has no pool
 * on `device` yet), MRN_EINVAL for a device index outside 0..63,
 * MRN_ECUDA when CUDA refuses.  Scratch still in use by queued work stays
 * reserved until it is freed. */
int mrn_scratch_release(int device);

/* The jagged AoS -> SoA conversion of mrn_convert, without any device
 * allocation by the library.  The paper has no counterpart: this exists for
 * callers that cannot let a library allocate device memory (an application
 * whose own pool owns the whole GPU, a process at the edge of device memory,
 * a latency-critical loop that cannot take an allocator call).
 * Semantics and outputs are those of mrn_convert for a jagged schema with an
 * AoS source and a SoA destination; any other pair returns MRN_EINVAL.
 * The scan's scratch is a fixed 256 KiB array inside the library, present on
 * every device that loads the library until the process exits; it holds at
 * most 33,521,664 parents per call, larger n_records returns MRN_ESIZE before
 * anything is launched.  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) with that device current; make that
 * first call before any stream capture.  `stream` must belong to the
 * current device (else MRN_EINVAL), since the address is that device's.  All calls share the array and each
 * clears it on its stream before use, so calls that overlap on the GPU
 * (different streams, no ordering between them) race and must not be
 * issued. */
int mrn_convert_jagged_noalloc(const mrn_view* src, const mrn_view* dst, void* stream);

/* Sum of the jagged lengths of an AoS device view (the number of child
 * values an AoS -> SoA conversion writes).  Synchronous; *m receives it. */
int mrn_jagged_count(const mrn_view* src, uint64_t* m, void* stream);

/* Test and fault-injection settings (host side; they take effect for
 * conversions planned afterwards):
 *   key 1: index of a jagged tile (in a split single conversion: a scan
 *          chunk of 8,192 parents) that never publishes its sum (-1: none),
 *          so that its successors' bounded waits expire and record
 *          MRN_ETIMEOUT;
 *   key 2: bound of each look-back wait in nanoseconds (default 2e9);
 *   key 3: 1 = single conversions use the direct kernel (vector loads and
 *          stores per lane) even where the TMA-staged kernel applies;
 *   key 4: parents from which a single jagged AoS -> SoA / AoSoA conversion
 *          runs split (default: never, the fused kernel is as fast or faster
 *          for one collection at every size measured): the parents as one
 *          staged conversion that writes their begins as offsets and checks
 *          that the pool is canonical (its records exactly the children, in
 *          parent order: each begin the previous begin plus its length), the
 *          pool as one staged conversion of the child schema when it is, and
 *          otherwise the whole conversion again with the fused kernel.
 *          Batches split every jagged AoS job whose pool fits the
 *          destination's child capacity and whose offsets fit their type,
 *          in their own form (see mrn_batch_create).  A negative value
 *          turns split runs off (single conversions and batches);
 *   key 5: parents up to which a single fused jagged AoS -> SoA / AoSoA
 *          conversion uses tiles of 256 parents instead of 1,024 (default
 *          250,000; -1: never);
 *   key 6: 1 = split single conversions take the scan form instead: a scan
 *          of the lengths in chunks of 8,192 parents (offsets' bases and the
 *          pool's check) before the parents and the pool, and a pass that
 *          gathers the children when the pool is not canonical (the form
 *          also taken where offset_base + the pool's size overflows the
 *          offset type);
 *   key 7: children from which a nested AoS -> field-major conversion runs
 *          its parent level split in the local form (default 262,144; -1:
 *          never): the parents with their begins as offsets and the child
 *          pool's check, then the child pool as one staged conversion of the
 *          child record (its {length, begin} included), and the fused
 *          kernel again only for a pool that is not canonical. */
int mrn_debug_set(int key, long long value);

/* ------------------------------------------------------- transfer+convert */
typedef struct mrn_transfer_opts {
  size_t chunk_bytes; /* source bytes per chunk (0: 4 MiB); rounded to records
                         (and to whole blocks for AoSoA)                      */
  int32_t n_slots;    /* staging slots in flight (0: 4, max 16)               */
  int32_t flags;      /* MRN_TRANSFER_* bits (0: chunked staging)             */
} mrn_transfer_opts;

/* Zero-copy: no staging; the conversion kernel reads (host -> device) or
 * writes (device -> host) the pinned host buffers directly over the host
 * link, through their mapped device addresses.  Needs MRN_MEM_HOST_PINNED
 * memory that the driver maps (cudaHostGetDevicePointer; otherwise
 * MRN_EUNSUPPORTED); jagged schemas return MRN_EUNSUPPORTED.  An
 * alternative to the chunked pipeline for the paper's memcopy with extra
 * arguments (Sec. VI-A). */
#define MRN_TRANSFER_ZERO_COPY 1

/* Converts between a host view (MRN_MEM_HOST or MRN_MEM_HOST_PINNED) and a
 * device view, in either direction (the analogue of a copy between
 * collections in different memory contexts, Sec. VI-A/VI-B).  The source is
 * split into chunks of whole records; host->device chunks are copied into
 * device staging slots with cudaMemcpyAsync on a copy stream and converted
 * from staging into their final place on a compute stream, so copies and
 * conversions of different chunks overlap; device->host is the mirror
 * (convert into staging, then copy out).  Equal layouts skip staging.
 * Jagged schemas: the whole source is staged, then converted.
 * Ordered after prior work on `stream`; later work on `stream` waits for
 * it.  Each device has one pipeline per direction: calls in the same
 * direction write their destinations in call order (a call's first copies
 * may overlap the previous call's last conversions, through staging slots
 * the two do not share), and a host->device and a device->host call issued
 * on different streams overlap (both directions of the host link).
 * Pageable host memory works but serialises the copies.  With
 * MRN_TRANSFER_ZERO_COPY in opts->flags the kernel moves the data over the
 * host link itself (see above), on `stream`. */
int mrn_transfer_convert(const mrn_view* src, const mrn_view* dst,
                         const mrn_transfer_opts* opts, void* stream);

/* ---------------------------------------------------------------- batching */
typedef struct mrn_job {
  const mrn_view* src; /* device view */
  const mrn_view* dst; /* device view */
} mrn_job;

typedef struct mrn_batch mrn_batch; /* opaque */

/* Prepares many independent conversions (any schemas, any supported layout
 * pairs, jagged AoS<->SoA included) to run in one persistent kernel launch:
 * a device job table, a prefix over the jobs' tiles, per-job tile sizes
 * from the autotuner cache.  A jagged AoS -> field-major job runs split
 * where it can (see mrn_debug_set, key 4) and needs no scan: a pool is
 * canonical (its records exactly the children, in parent order) when every
 * parent's begin is the previous parent's begin plus its length (the first
 * 0, the last parent's end the pool's size), and its offsets are then the
 * begins.  The persistent launch converts the parents, writing the begins
 * as offsets and checking those equalities; a second persistent launch
 * converts the child pools (each a plain conversion, skipped unless its
 * check passed); a last launch converts the jobs whose pools were not
 * canonical whole again with the fused kernel (it returns at once when
 * every pool was).  Jagged jobs that cannot run split (a pool larger than
 * the destination's child capacity, or offsets beyond their type) run in
 * one more launch before the persistent one, one CTA per tile of 1,024
 * parents that scans, converts and gathers.  With use_graph = 1 the launch sequence (scratch reset +
 * the launches) is captured once into a CUDA graph and each mrn_batch_launch
 * replays it.  The views' buffers must stay valid while the batch is used.
 * Copies the job descriptions; `jobs` may be freed. */
int mrn_batch_create(const mrn_job* jobs, size_t n_jobs, int use_graph, mrn_batch** out);
/* Runs every job of the batch on `stream`. */
int mrn_batch_launch(mrn_batch* b, void* stream);
/* As mrn_batch_launch, and records three caller-created CUDA events
 * (cudaEvent_t, passed as void*) on `stream`: ev_begin before the batch's
 * work, ev_mid after the scratch reset and the fused jagged launch, ev_end
 * after the two persistent launches and the fall-back pass.
 * With use_graph = 1 the events are record nodes of a second graph of the
 * same work, captured at the first call and pointed at the given events at
 * each call (three distinct events, else MRN_EINVAL; the events of earlier
 * calls may have been destroyed since); a batch without jobs of one kind
 * records two events back to back.  For measuring each kernel of a replay; no counterpart in the
 * paper (the batched form is not the paper's). */
int mrn_batch_launch_timed(mrn_batch* b, void* stream, void* ev_begin, void* ev_mid, void* ev_end);
/* Baseline: runs the same jobs with one mrn_convert launch per job. */
int mrn_batch_launch_per_job(mrn_batch* b, void* stream);
/* Points job j at new buffers of the same schemas, layouts and sizes (the
 * job table is rewritten; the graph is reused). */
int mrn_batch_update(mrn_batch* b, size_t j, const mrn_view* src, const mrn_view* dst);
void mrn_batch_destroy(mrn_batch* b);

typedef struct mrn_batch_tune_result {
  uint32_t max_chunk;   /* consecutive tiles a CTA takes at once (1..16)     */
  uint32_t ctas_per_sm; /* resident CTAs per SM of the grid (0: occupancy)   */
  double ms;            /* device time of one launch with the winner         */
  double default_ms;    /* device time of one launch with the defaults       */
  double worst_ms;      /* device time of the slowest shape tried            */
  uint32_t candidates;  /* shapes timed                                      */
  uint32_t reserved;
} mrn_batch_tune_result;

/* Autotunes the launch shape of this batch on its own jobs: times launches
 * on `stream` for every chunk size in {1, 2, 4, 8, 16} and CTAs per SM in
 * {occupancy, 2}, times the fastest against the default twice more
 * (alternately), keeps it only when it is at least 1% faster (the graph is
 * re-captured) and reports the shape kept.  The jobs' destinations are
 * written by the trial launches. */
int mrn_batch_tune(mrn_batch* b, void* stream, mrn_batch_tune_result* out);

typedef struct mrn_tune_result {
  uint32_t threads;       /* threads per CTA                                  */
  uint32_t ctas_per_sm;   /* resident CTAs per SM of the grid (0: occupancy)  */
  uint32_t tile_records;  /* records per tile                                 */
  uint32_t staged;        /* 1: tiles staged through shared memory by TMA
                             bulk copies; 0: direct vector loads and stores  */
  double gbps;            /* algorithmic GB/s of the winner                   */
  double default_gbps;    /* algorithmic GB/s of the default configuration    */
} mrn_tune_result;

/* Times candidate launch shapes for converting n_hint records of `s` from
 * `src` to `dst` layouts on scratch device buffers: the TMA-staged kernel
 * (when buffers and tile fit) at two grid sizes, and the direct kernel over
 * threads per CTA, CTAs per SM and records per tile.  The fastest is timed
 * against the default three more times (alternately) and kept only when it
 * is at least 3% faster.  Caches the shape kept for this (schema hash,
 * layout pair); later conversions and batches use it.  Synchronous.  `out`
 * may be NULL. */
int mrn_autotune(const mrn_schema* s, mrn_layout src, mrn_layout dst, uint64_t n_hint,
                 mrn_tune_result* out);
/* Forgets every cached tuning result. */
int mrn_autotune_clear(void);

/* ------------------------------------------------------------------ server */
typedef struct mrn_server mrn_server; /* opaque, internally synchronised */

typedef struct mrn_server_opts {
  size_t hbm_budget_bytes; /* device memory the server may hold at once       */
  int32_t max_slots;       /* requests on the device at once (0: 8)           */
  int32_t reserved;
  size_t chunk_bytes;      /* transfer chunk (0: 4 MiB)                       */
} mrn_server_opts;

typedef struct mrn_server_stats {
  uint64_t submitted, admitted, completed, rejected, failed;
  uint64_t bytes_in, bytes_out;  /* source / destination bytes of completed   */
  double p50_ms, p99_ms, max_ms, mean_ms; /* latency, arrival -> completion   */
  double busy_s;                 /* wall time from first arrival to last done */
  uint64_t peak_device_bytes;    /* high-water mark of admitted footprints    */
} mrn_server_stats;

/* Starts a conversion server on the current device: a host thread admits
 * requests in arrival order as slots and budget allow (continuous batching:
 * new requests join while others are on the device), runs each on its own
 * stream pair, and records latency from submission to completion. */
int mrn_server_create(const mrn_server_opts* opts, mrn_server** out);
/* Queues one conversion.  At least one side must be a host view; device
 * sides must be on the current device.  A request whose device footprint
 * (staging plus device intermediates) exceeds the whole budget is rejected
 * at once with MRN_ENOMEM.  *ticket identifies the request.  The views'
 * buffers must stay valid until the request completes. */
int mrn_server_submit(mrn_server* sv, const mrn_view* src, const mrn_view* dst, uint64_t* ticket);
/* Non-blocking: *done = 1 and *status = the request's status when finished. */
int mrn_server_poll(mrn_server* sv, uint64_t ticket, int* done, int* status);
/* Blocks until the request finished or timeout_ns passed (MRN_ETIMEOUT). */
int mrn_server_wait(mrn_server* sv, uint64_t ticket, uint64_t timeout_ns, int* status);
/* As mrn_server_wait, and *latency_ms receives this request's latency
 * (submission -> completion of its work, as the statistics count it), so
 * that callers can split latency by request size or kind. */
int mrn_server_wait_latency(mrn_server* sv, uint64_t ticket, uint64_t timeout_ns, int* status,
                            double* latency_ms);
int mrn_server_stats_get(mrn_server* sv, mrn_server_stats* out);
/* Drains outstanding requests, stops the thread, frees device memory. */
void mrn_server_destroy(mrn_server* sv);

/* ---------------------------------------------------- overlapping moves */
/* Moves `bytes` bytes from src to dst inside one memory context, where the
 * two ranges may overlap (the partially overlapping memcopy of Sec. VI-A,
 * used to open or close a gap for insertion and deletion): afterwards dst
 * holds what src held before.  MRN_MEM_DEVICE: both ranges on the current
 * device, asynchronous on `stream`, one kernel that reads each chunk before
 * any chunk overlapping it is written (each wait bounded; MRN_ETIMEOUT is
 * recorded if one expires).  MRN_MEM_HOST / MRN_MEM_HOST_PINNED: a host
 * memmove once `stream` is idle. */
int mrn_memmove(void* dst, const void* src, uint64_t bytes, int mem, void* stream);

/* ------------------------------------------------------------ collections */
/* A library-owned collection (Sec. VI-A memory contexts, Sec. VI-B layout
 * holders): one schema, one layout and one memory context, storage for
 * `capacity` objects (and, for a jagged schema, `child_capacity` child
 * values), and the current sizes n <= capacity and m <= child_capacity.
 * Storage per layout:
 *   AoS: capacity records (jagged: plus a child pool of child_capacity child
 *        records; the parents' {length, begin} index into it);
 *   SoA: one block laid out as the single-block SoA for (capacity,
 *        child_capacity) -- data columns, offsets, child columns;
 *   AoSoA(B): ceil(capacity / B) blocks (jagged: then offsets and child
 *        columns, as the single-block jagged AoSoA for the capacities).
 * Every field-major jagged collection keeps offsets[0] == 0 and
 * m == offsets[n].  Objects a resize adds are all-zero (jagged: no
 * children).  Unused AoSoA slots of the last block stay zero.
 * Memory contexts: MRN_MEM_DEVICE (device `device`; moves and fills run
 * in kernels on `stream`), MRN_MEM_HOST_PINNED and MRN_MEM_HOST (moves and
 * fills on the host once `stream` is idle; conversions into them go
 * through mrn_transfer_convert, which needs MRN_MEM_HOST_PINNED).
 * A collection is not internally synchronised. */
typedef struct mrn_collection mrn_collection; /* opaque */

int mrn_collection_create(const mrn_schema* s, mrn_layout layout, int mem, int device, uint64_t capacity,
                          uint64_t child_capacity, mrn_collection** out);
void mrn_collection_destroy(mrn_collection* c);
/* A view of the current contents (n objects, m children).  Its pointer
 * arrays belong to the collection and stay valid until the next call that
 * reallocates (reserve, a growing resize / insert / assign, shrink_to_fit,
 * set_context) or destroy. */
int mrn_collection_view(const mrn_collection* c, mrn_view* out);
int mrn_collection_sizes(const mrn_collection* c, uint64_t* n, uint64_t* m, uint64_t* capacity,
                         uint64_t* child_capacity);
/* Grows the capacities (never shrinks them): new storage in the same
 * context, the contents copied over, the old storage freed. */
int mrn_collection_reserve(mrn_collection* c, uint64_t capacity, uint64_t child_capacity, void* stream);
/* Sets n.  Growing appends all-zero objects (capacity doubled as needed);
 * shrinking drops the last objects (jagged: and their children). */
int mrn_collection_resize(mrn_collection* c, uint64_t n, void* stream);
int mrn_collection_clear(mrn_collection* c, void* stream);
/* Reallocates to capacity n and child capacity m. */
int mrn_collection_shrink_to_fit(mrn_collection* c, void* stream);
/* Removes objects [first, first + count) (jagged: with their children; the
 * later offsets drop by the children removed).  AoS and SoA collections,
 * and jagged AoS (the children stay in the pool, unreferenced); AoSoA:
 * MRN_EUNSUPPORTED.  A field-major jagged erase waits for `stream` to read
 * two offsets. */
int mrn_collection_erase(mrn_collection* c, uint64_t first, uint64_t count, void* stream);
/* Inserts the objects of `src` (same schema; any layout, any context
 * mrn_convert or mrn_transfer_convert accepts against this collection's)
 * before object `pos`: the tail moves up, then src is converted into the
 * gap.  AoS and SoA collections, and jagged SoA; other layouts:
 * MRN_EUNSUPPORTED.  A jagged insert waits for `stream` (offsets, and the
 * child count of an AoS source). */
int mrn_collection_insert(mrn_collection* c, uint64_t pos, const mrn_view* src, void* stream);
/* Replaces the contents with those of `src` (same schema, any layout),
 * converted into this collection's layout (copy assignment between
 * layouts, Sec. VI-B). */
int mrn_collection_assign(mrn_collection* c, const mrn_view* src, void* stream);
/* Moves the collection to another memory context (update of the memory
 * context information, Sec. VI-A): new storage there with the same
 * capacities and layout, the contents copied, the old storage freed. */
int mrn_collection_set_context(mrn_collection* c, int mem, int device, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* MRN_H */
