/*
 * Plain, slow CPU oracle for schema-driven layout conversion.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline / reference legs may load this library.  It
 * shares no code, header or table with the CUDA library.
 *
 * What it computes is the plain definition of the paper's default transfer
 * between layouts (Sec. VI-B, Defining Layouts), which moves the data of
 * each property in turn: for every object and every property, copy the
 * property's bytes from its source address to its destination address.
 * Layout rules:
 *
 *  - Schema lowering.  Sub-group members are stored as if declared at the
 *    top level (Sec. V, sub-group property); an array property of extent E
 *    is E separate per-index columns (Sec. V, array property: one array
 *    per element index), or, declared interleaved, one field-major column of
 *    E-element rows (the property's other interface, a single N x E array:
 *    record i's element k at row i, position k); a jagged
 *    vector property keeps a prefix sum of the sizes as a global property
 *    and all values as one contiguous vector (Sec. V, jagged vector
 *    property).
 *  - AoS record: natural C alignment, a sub-group laid out as a nested
 *    struct (aligned to its widest member, size rounded up to it).  The
 *    jagged member is the pair {uint32 length, uint64 begin} at the member's
 *    position, `begin` an element index into a separate child-record pool.
 *  - SoA, single block ("DynamicStruct", Sec. VI-B): columns in flattened
 *    order, each starting at a multiple of 128 bytes; for a jagged schema
 *    the offsets column (N+1 entries) and the child columns (M entries
 *    each) follow.
 *  - AoSoA(B) (Sec. IV: memory allocated in fixed-size blocks of records):
 *    each block is the C struct { T_0 c0[B]; T_1 c1[B]; ... } of the
 *    flattened columns (an interleaved array of extent E: T a[B][E]); for
 *    a jagged schema the blocks are followed, in the
 *    same buffer, by the offsets column and the child columns (each region
 *    128-byte aligned, as in the single-block SoA).
 *  - A jagged member may nest once: its child records may hold a jagged
 *    member of their own (Sec. V: the children are themselves a collection
 *    described by properties).  AoS: the children's {length, begin} index a
 *    second pool of grandchild records.  Field-major: the child level is
 *    laid out as a single-block SoA of the child schema (child columns, the
 *    children's offsets, m + 1 entries, the grandchild columns), after the
 *    parents' offsets.
 *  - Every destination byte that no property writes is 0.
 *
 * Field-major storage: every flattened column is stored on its own (its
 * own SoA region, its own B-element array in an AoSoA block) except the
 * columns of one interleaved array, which share one storage column whose
 * element is the whole E-element row; column k of the array is then at
 * byte k * size of each row, and consecutive records' elements are E * size
 * bytes apart.
 *
 * Parity unpinned: the 128-byte SoA column alignment, the AoSoA in-block
 * arrangement, the regions of a jagged AoSoA side, the placement of a
 * nested member's child level and the AoS jagged descriptor are readings
 * (the paper fixes no bytes for them); they are checked by round trips and
 * special cases only.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ESIZE 2
#define ORC_EOVERFLOW 4

#define ORC_AOS 0
#define ORC_SOA 1
#define ORC_AOSOA 2

#define TK_FIELD 1
#define TK_GROUP 2
#define TK_END 3
#define TK_JAGGED 4
#define TK_IFIELD 5 /* interleaved array property: size, extent */

#define ORC_MAXCOLS 1024

typedef struct orc_schema {
  int ncols;
  uint32_t col_size[ORC_MAXCOLS];
  uint64_t col_aos_off[ORC_MAXCOLS];
  /* field-major storage of each column: its storage column, its byte offset
   * inside a storage element, and the bytes between consecutive records'
   * elements (the storage element's size) */
  int col_store[ORC_MAXCOLS];
  uint32_t col_sub[ORC_MAXCOLS];
  uint32_t col_es[ORC_MAXCOLS];
  int nstore;
  uint32_t store_es[ORC_MAXCOLS];   /* storage element bytes */
  uint32_t store_align[ORC_MAXCOLS]; /* alignment of a storage element */
  uint64_t stride;
  uint64_t align;
  int has_jagged;
  uint64_t len_off;   /* AoS offset of the uint32 length */
  uint64_t begin_off; /* AoS offset of the uint64 begin */
  uint32_t off_size;  /* 4 or 8 */
  struct orc_schema* child;
} orc_schema;

typedef struct orc_side {
  int32_t kind;
  uint32_t block;
  uint8_t* base;        /* AoS records / AoSoA blocks / SoA single block */
  uint8_t** cols;       /* SoA per-column pointers, or NULL */
  uint8_t* offsets;     /* SoA offsets column, or NULL (inside base) */
  uint8_t** child_cols; /* SoA child columns, or NULL (inside base) */
  uint8_t* pool;        /* AoS child-record pool */
  uint64_t n;           /* records */
  uint64_t m;           /* children (capacity when destination) */
  uint8_t* gpool;       /* nested jagged, AoS: the children's own child pool */
  uint64_t m2;          /* nested jagged: grandchildren (capacity when destination) */
  uint8_t* child_offsets; /* nested jagged, SoA: the children's offsets, or NULL (inside base) */
  uint8_t** gchild_cols;  /* nested jagged, SoA: grandchild columns, or NULL (inside base) */
} orc_side;

static uint64_t align_up(uint64_t x, uint64_t a) { return (x + a - 1) / a * a; }

static void free_schema(orc_schema* s) {
  if (!s) return;
  free_schema(s->child);
  free(s);
}

/* Lays out members until TK_END (nested) or the end of the tokens.
 * Column offsets are written relative to the start of this (sub)struct. */
/* `level` is 0 for the collection's own records, 1 for a jagged member's
 * children, 2 for the children's children (a jagged member nests at most
 * once). */
static int layout_members(orc_schema* s, const int32_t* tk, int ntk, int* pos,
                          int nested, int level, uint64_t* size_out,
                          uint64_t* align_out) {
  uint64_t cur = 0, al = 1;
  int closed = 0;
  while (*pos < ntk) {
    int op = tk[*pos];
    if (op == TK_END) {
      if (nested <= 0) return ORC_EINVAL;
      (*pos)++;
      closed = 1;
      break;
    } else if (op == TK_FIELD || op == TK_IFIELD) {
      if (*pos + 2 >= ntk) return ORC_EINVAL;
      uint32_t size = (uint32_t)tk[*pos + 1];
      int32_t extent = tk[*pos + 2];
      int inter = op == TK_IFIELD;
      *pos += 3;
      if (!(size == 1 || size == 2 || size == 4 || size == 8) || extent < 1)
        return ORC_EINVAL;
      uint64_t off = align_up(cur, size);
      for (int k = 0; k < extent; k++) {
        if (s->ncols >= ORC_MAXCOLS || s->nstore >= ORC_MAXCOLS) return ORC_EINVAL;
        s->col_size[s->ncols] = size;
        s->col_aos_off[s->ncols] = off + (uint64_t)k * size;
        if (!inter || k == 0) {
          s->store_es[s->nstore] = inter ? size * (uint32_t)extent : size;
          s->store_align[s->nstore] = size;
          s->nstore++;
        }
        s->col_store[s->ncols] = s->nstore - 1;
        s->col_sub[s->ncols] = inter ? (uint32_t)k * size : 0;
        s->col_es[s->ncols] = s->store_es[s->nstore - 1];
        s->ncols++;
      }
      cur = off + (uint64_t)extent * size;
      if (size > al) al = size;
    } else if (op == TK_GROUP) {
      (*pos)++;
      int first = s->ncols;
      int had_jag = s->has_jagged;
      uint64_t gsize, galign;
      int rc = layout_members(s, tk, ntk, pos, 1, level, &gsize, &galign);
      if (rc) return rc;
      uint64_t goff = align_up(cur, galign);
      for (int c = first; c < s->ncols; c++) s->col_aos_off[c] += goff;
      if (s->has_jagged && !had_jag) {
        s->len_off += goff;
        s->begin_off += goff;
      }
      cur = goff + gsize;
      if (galign > al) al = galign;
    } else if (op == TK_JAGGED) {
      if (*pos + 2 >= ntk || s->has_jagged || level >= 2) return ORC_EINVAL;
      uint32_t osz = (uint32_t)tk[*pos + 1];
      int nchild = tk[*pos + 2];
      *pos += 3;
      if (!(osz == 4 || osz == 8) || nchild < 1 || *pos + nchild > ntk)
        return ORC_EINVAL;
      orc_schema* ch = (orc_schema*)calloc(1, sizeof(orc_schema));
      if (!ch) return ORC_EINVAL;
      int cpos = 0;
      uint64_t csize, calign;
      int rc = layout_members(ch, tk + *pos, nchild, &cpos, 0, level + 1, &csize, &calign);
      if (rc || ch->ncols == 0) {
        free_schema(ch);
        return ORC_EINVAL;
      }
      ch->stride = csize;
      ch->align = calign;
      *pos += nchild;
      s->has_jagged = 1;
      s->off_size = osz;
      s->child = ch;
      s->len_off = align_up(cur, 4);
      cur = s->len_off + 4;
      s->begin_off = align_up(cur, 8);
      cur = s->begin_off + 8;
      if (al < 8) al = 8;
    } else {
      return ORC_EINVAL;
    }
  }
  if (nested > 0 && !closed) return ORC_EINVAL;
  *size_out = align_up(cur, al);
  *align_out = al;
  return ORC_OK;
}

orc_schema* orc_schema_new(const int32_t* tokens, int ntokens, int* status) {
  orc_schema* s = (orc_schema*)calloc(1, sizeof(orc_schema));
  int pos = 0;
  uint64_t size, al;
  int rc = s ? layout_members(s, tokens, ntokens, &pos, 0, 0, &size, &al) : ORC_EINVAL;
  if (rc == ORC_OK && s->ncols == 0 && !s->has_jagged) rc = ORC_EINVAL;
  if (rc) {
    free_schema(s);
    if (status) *status = rc;
    return NULL;
  }
  s->stride = size;
  s->align = al;
  if (status) *status = ORC_OK;
  return s;
}

void orc_schema_free(orc_schema* s) { free_schema(s); }
int orc_ncols(const orc_schema* s) { return s->ncols; }
uint32_t orc_col_size(const orc_schema* s, int c) { return s->col_size[c]; }
uint64_t orc_col_aos_off(const orc_schema* s, int c) { return s->col_aos_off[c]; }
uint64_t orc_stride(const orc_schema* s) { return s->stride; }
int orc_has_jagged(const orc_schema* s) { return s->has_jagged; }
uint64_t orc_len_off(const orc_schema* s) { return s->len_off; }
uint64_t orc_begin_off(const orc_schema* s) { return s->begin_off; }
uint32_t orc_off_size(const orc_schema* s) { return s->off_size; }
const orc_schema* orc_child(const orc_schema* s) { return s->child; }

/* ---- layout address rules ---- */

/* AoSoA(B): start of storage column q inside a block (C struct of
 * B-element arrays of storage elements). */
static uint64_t aosoa_store_start(const orc_schema* s, uint32_t B, int q) {
  uint64_t end = 0, start = 0;
  for (int k = 0; k <= q; k++) {
    start = align_up(end, s->store_align[k]);
    end = start + (uint64_t)B * s->store_es[k];
  }
  return start;
}

/* Start of column c's first element inside a block. */
uint64_t orc_aosoa_col_start(const orc_schema* s, uint32_t B, int c) {
  return aosoa_store_start(s, B, s->col_store[c]) + s->col_sub[c];
}

uint64_t orc_aosoa_block_bytes(const orc_schema* s, uint32_t B) {
  uint64_t end = 0, al = 1;
  for (int k = 0; k < s->nstore; k++) {
    end = align_up(end, s->store_align[k]) + (uint64_t)B * s->store_es[k];
    if (s->store_align[k] > al) al = s->store_align[k];
  }
  return align_up(end, al);
}

/* Single-block field-major sides.  SoA: region q of the block, in order:
 * the data storage columns 0..nstore-1, then (jagged) the offsets column,
 * then the child level as a single-block SoA of the child schema (its data
 * storage columns, and for a nested jagged member its own offsets and the
 * grandchildren's storage columns).  AoSoA(B) of a jagged schema: the
 * parent blocks, then the offsets column, then the child level.  Each
 * region starts at a multiple of 128 bytes.  Counts: n records, m
 * children, m2 grandchildren. */
static int parent_regions(const orc_schema* s, int kind) { return kind == ORC_AOSOA ? 1 : s->nstore; }

static uint64_t fm_region_bytes(const orc_schema* s, int kind, uint32_t B, uint64_t n, uint64_t m, uint64_t m2,
                                int q) {
  int P = parent_regions(s, kind);
  if (q < P) {
    if (kind == ORC_AOSOA) return (B ? (n + B - 1) / B : 0) * orc_aosoa_block_bytes(s, B);
    return n * s->store_es[q];
  }
  if (q == P) return (n + 1) * s->off_size;
  return fm_region_bytes(s->child, ORC_SOA, 0, m, m2, 0, q - P - 1);
}

static int fm_nregions(const orc_schema* s, int kind) {
  return parent_regions(s, kind) + (s->has_jagged ? 1 + fm_nregions(s->child, ORC_SOA) : 0);
}

static uint64_t region_start(const orc_schema* s, int kind, uint32_t B, uint64_t n, uint64_t m, uint64_t m2,
                             int q) {
  uint64_t start = 0, end = 0;
  for (int k = 0; k <= q; k++) {
    start = align_up(end, 128);
    end = start + fm_region_bytes(s, kind, B, n, m, m2, k);
  }
  return start;
}

/* Region and byte offset of item r of a single-block field-major side, r
 * counted by columns: SoA: data column r (r < ncols), the offsets (r ==
 * ncols), then item r - ncols - 1 of the child level counted the same way
 * (child columns, its offsets, grandchild columns); jagged AoSoA(B): the
 * blocks (r == 0), the offsets (r == 1), child-level item r - 2.  A column
 * of an interleaved array starts at its element inside the first row. */
static void item_region(const orc_schema* s, int kind, int r, int* q, uint64_t* sub) {
  int P = parent_regions(s, kind);
  int Pc = kind == ORC_AOSOA ? 1 : s->ncols;
  if (r < Pc) {
    *q = kind == ORC_AOSOA ? 0 : s->col_store[r];
    *sub = kind == ORC_AOSOA ? 0 : s->col_sub[r];
  } else if (r == Pc) {
    *q = P;
    *sub = 0;
  } else {
    item_region(s->child, ORC_SOA, r - Pc - 1, q, sub);
    *q += P + 1;
  }
}

uint64_t orc_fm_region_start(const orc_schema* s, int kind, uint32_t B, uint64_t n, uint64_t m, uint64_t m2, int r) {
  int q;
  uint64_t sub;
  item_region(s, kind, r, &q, &sub);
  return region_start(s, kind, B, n, m, m2, q) + sub;
}

uint64_t orc_soa_region_start(const orc_schema* s, uint64_t n, uint64_t m, uint64_t m2, int r) {
  return orc_fm_region_start(s, ORC_SOA, 0, n, m, m2, r);
}

static uint64_t fm_bytes(const orc_schema* s, int kind, uint32_t B, uint64_t n, uint64_t m, uint64_t m2) {
  int nr = fm_nregions(s, kind);
  uint64_t end = region_start(s, kind, B, n, m, m2, nr - 1) + fm_region_bytes(s, kind, B, n, m, m2, nr - 1);
  return align_up(end, 128);
}

uint64_t orc_soa_bytes(const orc_schema* s, uint64_t n, uint64_t m, uint64_t m2) {
  return fm_bytes(s, ORC_SOA, 0, n, m, m2);
}

/* Bytes of the `base` buffer of a side. */
uint64_t orc_base_bytes(const orc_schema* s, int kind, uint32_t B, uint64_t n, uint64_t m, uint64_t m2) {
  if (kind == ORC_AOS) return n * s->stride;
  if (kind == ORC_SOA) return orc_soa_bytes(s, n, m, m2);
  if (kind == ORC_AOSOA) {
    if (s->has_jagged) return fm_bytes(s, ORC_AOSOA, B, n, m, m2);
    return (B ? (n + B - 1) / B : 0) * orc_aosoa_block_bytes(s, B);
  }
  return 0;
}

int orc_col_es(const orc_schema* s, int c) { return (int)s->col_es[c]; }
int orc_col_sub(const orc_schema* s, int c) { return (int)s->col_sub[c]; }
int orc_col_store(const orc_schema* s, int c) { return s->col_store[c]; }
int orc_nstore(const orc_schema* s) { return s->nstore; }

/* Address of record i's element of column c (SoA per-column pointers: the
 * pointer of each column, an interleaved array's columns pointing at their
 * element of the first row). */
static uint8_t* col_addr(const orc_schema* s, const orc_side* v, int c, uint64_t i) {
  uint64_t es = s->col_es[c];
  switch (v->kind) {
    case ORC_AOS:
      return v->base + i * s->stride + s->col_aos_off[c];
    case ORC_SOA:
      if (v->cols) return v->cols[c] + i * es;
      return v->base + orc_soa_region_start(s, v->n, v->m, v->m2, c) + i * es;
    default:
      return v->base + (i / v->block) * orc_aosoa_block_bytes(s, v->block) +
             orc_aosoa_col_start(s, v->block, c) + (i % v->block) * es;
  }
}

/* Item index of the offsets of a field-major side (see item_region). */
static int offsets_item(const orc_schema* s, int kind) { return kind == ORC_AOSOA ? 1 : s->ncols; }

static uint8_t* offsets_ptr(const orc_schema* s, const orc_side* v) {
  if (v->offsets) return v->offsets;
  return v->base + orc_fm_region_start(s, v->kind, v->block, v->n, v->m, v->m2, offsets_item(s, v->kind));
}

/* Child column cc of a field-major side (element j at + j * es). */
static uint8_t* child_col_ptr(const orc_schema* s, const orc_side* v, int cc) {
  if (v->child_cols) return v->child_cols[cc];
  return v->base + orc_fm_region_start(s, v->kind, v->block, v->n, v->m, v->m2, offsets_item(s, v->kind) + 1 + cc);
}

/* Nested jagged member of a field-major side (single block): the
 * children's offsets (m + 1 entries) and grandchild column g. */
static uint8_t* child_offsets_ptr(const orc_schema* s, const orc_side* v) {
  if (v->child_offsets) return v->child_offsets;
  return v->base + orc_fm_region_start(s, v->kind, v->block, v->n, v->m, v->m2,
                                       offsets_item(s, v->kind) + 1 + s->child->ncols);
}

static uint8_t* gchild_col_ptr(const orc_schema* s, const orc_side* v, int g) {
  if (v->gchild_cols) return v->gchild_cols[g];
  return v->base + orc_fm_region_start(s, v->kind, v->block, v->n, v->m, v->m2,
                                       offsets_item(s, v->kind) + 2 + s->child->ncols + g);
}

static uint64_t rd(const uint8_t* p, uint32_t size) {
  uint64_t x = 0;
  memcpy(&x, p, size); /* little-endian host */
  return x;
}

static void wr(uint8_t* p, uint64_t x, uint32_t size) { memcpy(p, &x, size); }

static int valid_side(const orc_side* v) {
  if (v->kind == ORC_AOSOA) return v->block >= 1;
  return v->kind == ORC_AOS || v->kind == ORC_SOA;
}

/* Sets every byte of the destination to zero (step "zero the non-data
 * bytes"; data bytes are overwritten afterwards). */
static void zero_side(const orc_schema* s, const orc_side* d) {
  if (d->kind == ORC_SOA && d->cols) {
    for (int c = 0; c < s->ncols; c++)
      if (s->col_sub[c] == 0) memset(d->cols[c], 0, d->n * s->col_es[c]);
    if (s->has_jagged) {
      memset(offsets_ptr(s, d), 0, (d->n + 1) * s->off_size);
      for (int cc = 0; cc < s->child->ncols; cc++)
        if (s->child->col_sub[cc] == 0) memset(child_col_ptr(s, d, cc), 0, d->m * s->child->col_es[cc]);
      if (s->child->has_jagged) {
        const orc_schema* gc = s->child->child;
        memset(child_offsets_ptr(s, d), 0, (d->m + 1) * s->child->off_size);
        for (int g = 0; g < gc->ncols; g++)
          if (gc->col_sub[g] == 0) memset(gchild_col_ptr(s, d, g), 0, d->m2 * gc->col_es[g]);
      }
    }
    return;
  }
  memset(d->base, 0, orc_base_bytes(s, d->kind, d->block, d->n, d->m, d->m2));
  if (d->kind != ORC_AOS && s->has_jagged) {
    if (d->offsets) memset(d->offsets, 0, (d->n + 1) * s->off_size);
    if (d->child_cols)
      for (int cc = 0; cc < s->child->ncols; cc++)
        if (s->child->col_sub[cc] == 0) memset(d->child_cols[cc], 0, d->m * s->child->col_es[cc]);
    if (s->child->has_jagged) {
      const orc_schema* gc = s->child->child;
      if (d->child_offsets) memset(d->child_offsets, 0, (d->m + 1) * s->child->off_size);
      if (d->gchild_cols)
        for (int g = 0; g < gc->ncols; g++)
          if (gc->col_sub[g] == 0) memset(d->gchild_cols[g], 0, d->m2 * gc->col_es[g]);
    }
  }
  if (d->kind == ORC_AOS && s->has_jagged && d->pool)
    memset(d->pool, 0, d->m * s->child->stride);
  if (d->kind == ORC_AOS && s->has_jagged && s->child->has_jagged && d->gpool)
    memset(d->gpool, 0, d->m2 * s->child->child->stride);
}

/* A nested jagged member (the children have a jagged member of their
 * own): an AoS side needs the second pool when it has children. */
static int nested_ok(const orc_schema* s, const orc_side* v) {
  if (!s->has_jagged || !s->child->has_jagged || v->kind != ORC_AOS) return 1;
  return v->m == 0 || (v->pool != NULL && (v->m2 == 0 || v->gpool != NULL));
}

/* Converts one collection from `src` to `dst` (same schema, same N).
 * For a jagged schema the AoS side is converted to or from a field-major
 * side (SoA or AoSoA(B)), or one field-major side to another; *m_out
 * receives the number of child values written. */
int orc_convert(const orc_schema* s, const orc_side* src, orc_side* dst, uint64_t* m_out) {
  if (!valid_side(src) || !valid_side(dst) || src->n != dst->n) return ORC_EINVAL;
  if (!nested_ok(s, src) || !nested_ok(s, dst)) return ORC_EINVAL;
  const int nest = s->has_jagged && s->child->has_jagged;
  uint64_t n = src->n;
  if (m_out) *m_out = 0;
  if (s->has_jagged) {
    int a2s = src->kind == ORC_AOS && dst->kind != ORC_AOS;
    int s2a = src->kind != ORC_AOS && dst->kind == ORC_AOS;
    int f2f = src->kind != ORC_AOS && dst->kind != ORC_AOS;
    if (!a2s && !s2a && !f2f) return ORC_EINVAL;
    if (a2s) {
      /* Prefix sum of the sizes, checked against the offset type (Sec. V,
       * jagged vector property: the prefix type may be narrower than the
       * collection's size type). */
      uint64_t total = 0;
      uint64_t lim = s->off_size == 4 ? 0xffffffffull : ~0ull;
      for (uint64_t i = 0; i < n; i++) {
        const uint8_t* rec = src->base + i * s->stride;
        uint64_t len = rd(rec + s->len_off, 4);
        uint64_t beg = rd(rec + s->begin_off, 8);
        if (beg > src->m || len > src->m - beg) return ORC_EINVAL;
        if (len > lim - total) return ORC_EOVERFLOW;
        total += len;
      }
      if (total > dst->m) return ORC_ESIZE;
      if (nest) {
        /* the same checks one level down, over the children reached */
        const orc_schema* ch = s->child;
        uint64_t total1 = 0, lim1 = ch->off_size == 4 ? 0xffffffffull : ~0ull;
        for (uint64_t i = 0; i < n; i++) {
          const uint8_t* rec = src->base + i * s->stride;
          uint64_t len = rd(rec + s->len_off, 4), beg = rd(rec + s->begin_off, 8);
          for (uint64_t k = 0; k < len; k++) {
            const uint8_t* c = src->pool + (beg + k) * ch->stride;
            uint64_t len1 = rd(c + ch->len_off, 4), beg1 = rd(c + ch->begin_off, 8);
            if (beg1 > src->m2 || len1 > src->m2 - beg1) return ORC_EINVAL;
            if (len1 > lim1 - total1) return ORC_EOVERFLOW;
            total1 += len1;
          }
        }
        if (total1 > dst->m2) return ORC_ESIZE;
      }
    } else {
      const uint8_t* off = offsets_ptr(s, src);
      for (uint64_t i = 0; i < n; i++) {
        uint64_t a = rd(off + i * s->off_size, s->off_size);
        uint64_t b = rd(off + (i + 1) * s->off_size, s->off_size);
        if (b < a || b - a > 0xffffffffull) return ORC_EINVAL;
      }
      if (n > 0 && rd(off + n * s->off_size, s->off_size) > src->m) return ORC_EINVAL;
      if (dst->m < src->m) return ORC_ESIZE;
      if (nest) {
        const orc_schema* ch = s->child;
        const uint8_t* off1 = child_offsets_ptr(s, src);
        for (uint64_t j = 0; j < src->m; j++) {
          uint64_t a = rd(off1 + j * ch->off_size, ch->off_size);
          uint64_t b = rd(off1 + (j + 1) * ch->off_size, ch->off_size);
          if (b < a || b - a > 0xffffffffull) return ORC_EINVAL;
        }
        if (src->m > 0 && rd(off1 + src->m * ch->off_size, ch->off_size) > src->m2) return ORC_EINVAL;
        if (dst->m2 < src->m2) return ORC_ESIZE;
      }
    }
  }

  zero_side(s, dst);

  /* The default transfer: every property of every object, one by one. */
  for (uint64_t i = 0; i < n; i++)
    for (int c = 0; c < s->ncols; c++)
      memcpy(col_addr(s, dst, c, i), col_addr(s, src, c, i), s->col_size[c]);

  if (!s->has_jagged) return ORC_OK;
  const orc_schema* ch = s->child;
  if (src->kind != ORC_AOS && dst->kind != ORC_AOS) {
    /* Field-major to field-major: the offsets and the child values keep
     * their order; only the parents change layout. */
    memcpy(offsets_ptr(s, dst), offsets_ptr(s, src), (n + 1) * s->off_size);
    for (int cc = 0; cc < ch->ncols; cc++)
      if (ch->col_sub[cc] == 0)
        memcpy(child_col_ptr(s, dst, cc), child_col_ptr(s, src, cc), src->m * ch->col_es[cc]);
    if (nest) {
      const orc_schema* gc = ch->child;
      memcpy(child_offsets_ptr(s, dst), child_offsets_ptr(s, src), (src->m + 1) * ch->off_size);
      for (int g = 0; g < gc->ncols; g++)
        if (gc->col_sub[g] == 0) memcpy(gchild_col_ptr(s, dst, g), gchild_col_ptr(s, src, g), src->m2 * gc->col_es[g]);
    }
    if (m_out) *m_out = src->m;
    return ORC_OK;
  }
  if (src->kind == ORC_AOS) {
    uint8_t* off = offsets_ptr(s, dst);
    uint64_t run = 0;
    wr(off, 0, s->off_size);
    for (uint64_t i = 0; i < n; i++) {
      const uint8_t* rec = src->base + i * s->stride;
      uint64_t len = rd(rec + s->len_off, 4);
      uint64_t beg = rd(rec + s->begin_off, 8);
      for (uint64_t k = 0; k < len; k++)
        for (int cc = 0; cc < ch->ncols; cc++)
          memcpy(child_col_ptr(s, dst, cc) + (run + k) * ch->col_es[cc],
                 src->pool + (beg + k) * ch->stride + ch->col_aos_off[cc], ch->col_size[cc]);
      run += len;
      wr(off + (i + 1) * s->off_size, run, s->off_size);
    }
    if (m_out) *m_out = run;
    if (nest) {
      /* The children's own jagged member, one level down: child j (in
       * parent order) gets offsets1[j+1] = offsets1[j] + its length, and its
       * grandchildren are copied, property by property, after the previous
       * child's. */
      const orc_schema* gc = ch->child;
      uint8_t* off1 = child_offsets_ptr(s, dst);
      uint64_t j = 0, run1 = 0;
      wr(off1, 0, ch->off_size);
      for (uint64_t i = 0; i < n; i++) {
        const uint8_t* rec = src->base + i * s->stride;
        uint64_t len = rd(rec + s->len_off, 4), beg = rd(rec + s->begin_off, 8);
        for (uint64_t k = 0; k < len; k++) {
          const uint8_t* c = src->pool + (beg + k) * ch->stride;
          uint64_t len1 = rd(c + ch->len_off, 4), beg1 = rd(c + ch->begin_off, 8);
          for (uint64_t q = 0; q < len1; q++)
            for (int g = 0; g < gc->ncols; g++)
              memcpy(gchild_col_ptr(s, dst, g) + (run1 + q) * gc->col_es[g],
                     src->gpool + (beg1 + q) * gc->stride + gc->col_aos_off[g], gc->col_size[g]);
          run1 += len1;
          j++;
          wr(off1 + j * ch->off_size, run1, ch->off_size);
        }
      }
    }
  } else {
    const uint8_t* off = offsets_ptr(s, src);
    for (uint64_t i = 0; i < n; i++) {
      uint8_t* rec = dst->base + i * s->stride;
      uint64_t a = rd(off + i * s->off_size, s->off_size);
      uint64_t b = rd(off + (i + 1) * s->off_size, s->off_size);
      wr(rec + s->len_off, b - a, 4);
      wr(rec + s->begin_off, a, 8);
    }
    /* Child values are written contiguously, slot j <- value j. */
    for (uint64_t j = 0; j < src->m; j++)
      for (int cc = 0; cc < ch->ncols; cc++)
        memcpy(dst->pool + j * ch->stride + ch->col_aos_off[cc],
               child_col_ptr(s, src, cc) + j * ch->col_es[cc], ch->col_size[cc]);
    if (nest) {
      /* one level down: child j's {length, begin} from the children's
       * offsets, the grandchildren contiguously into the second pool */
      const orc_schema* gc = ch->child;
      const uint8_t* off1 = child_offsets_ptr(s, src);
      for (uint64_t j = 0; j < src->m; j++) {
        uint8_t* c = dst->pool + j * ch->stride;
        uint64_t a = rd(off1 + j * ch->off_size, ch->off_size);
        uint64_t b = rd(off1 + (j + 1) * ch->off_size, ch->off_size);
        wr(c + ch->len_off, b - a, 4);
        wr(c + ch->begin_off, a, 8);
      }
      for (uint64_t k = 0; k < src->m2; k++)
        for (int g = 0; g < gc->ncols; g++)
          memcpy(dst->gpool + k * gc->stride + gc->col_aos_off[g],
                 gchild_col_ptr(s, src, g) + k * gc->col_es[g], gc->col_size[g]);
    }
    if (m_out) *m_out = src->m;
  }
  return ORC_OK;
}
