// C ABI entry points for device conversions: view validation, plan
// building, kernel dispatch, device status.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <climits>
#include <cstring>
#include <mutex>

#include "mrn_internal.h"

namespace mrn {

// Fault-injection and bounded-wait settings of the jagged look-back, set
// through mrn_debug_set.
std::atomic<long long> g_skip_publish_tile{-1};
std::atomic<unsigned long long> g_timeout_ns{2000000000ull};
// When set, conversions use the direct kernel even when they could be staged.
std::atomic<int> g_force_direct{0};
// Parents from which a single jagged AoS -> field-major conversion runs
// split (scan, parents, pool conversion, fall-back pass); by default never:
// measured at 100,000 to 4,194,304 parents, its four launches lose to the
// fused kernel (4,194,304: 308 against 267 us).  Batches split their
// jagged jobs (in one persistent launch the pools stream at the copy
// rate) unless the value is negative.
std::atomic<long long> g_split_parents{LLONG_MAX};
// Parents up to which a single fused jagged AoS -> field-major conversion
// takes tiles of MRN_JAG_SMALL_TILE parents (more CTAs for few parents).
std::atomic<long long> g_small_tile_parents{250000};
// 1: split single conversions take the scan form (JAG_SPLIT) even where the
// local check (JAG_LOCAL) applies.
std::atomic<int> g_split_scan{0};
// Children from which a nested AoS -> field-major conversion runs its
// parent level split in the local form (the child pool one staged
// conversion of the child record's flat schema); negative: never.
std::atomic<long long> g_nested_split_children{1 << 18};

namespace {

bool is_pow2(uint64_t x) { return x && !(x & (x - 1)); }

uint32_t log2u(uint64_t x) {
  uint32_t k = 0;
  while ((1ull << k) < x) ++k;
  return k;
}

uint32_t lowbit(uint64_t x) { return x ? (uint32_t)(x & (~x + 1)) : 1u << 30; }

int current_device() {
  int d = -1;
  if (cudaGetDevice(&d) != cudaSuccess) return -1;
  return d;
}

bool on_device(const mrn_view& v) { return v.mem == MRN_MEM_DEVICE; }

// Fills the field-major column pointers of a SoA / AoSoA side.
int fm_side(const mrn_schema* s, const mrn_view& v, bool child, SidePlan* sp) {
  const mrn_schema* t = child ? s->child.get() : s;
  const uint32_t nc = (uint32_t)t->cols.size();
  std::memset(sp, 0, sizeof(*sp));
  sp->kind = child ? K_SOA : v.layout.kind;  // child values are columns in either layout
  sp->block_shift = MRN_NO_SHIFT;
  if (v.layout.kind == MRN_SOA || child) {
    void* const* cols = child ? v.child_columns : v.columns;
    for (uint32_t c = 0; c < nc; ++c) {
      char* p;
      if (cols) {
        p = static_cast<char*>(cols[c]);
        // the columns of an interleaved array are elements of one row
        if (t->cols[c].sub && p != sp->col[c - 1] + t->cols[c - 1].size) return MRN_EINVAL;
      } else {
        if (!v.base) return MRN_EINVAL;
        p = static_cast<char*>(v.base) +
            fm_col_start(s, v.layout.kind, v.layout.block, v.n_records, v.n_children, child, c, v.n_grandchildren);
      }
      if (!p && (child ? v.n_children : v.n_records) > 0) return MRN_EINVAL;
      if (reinterpret_cast<uintptr_t>(p) % t->cols[c].size) return MRN_EALIGN;
      sp->col[c] = p;
    }
    return MRN_OK;
  }
  // AoSoA
  const uint32_t B = v.layout.block;
  sp->block = B;
  sp->block_bytes = aosoa_block_bytes(t, B);
  if (is_pow2(B)) sp->block_shift = log2u(B);
  sp->base = static_cast<char*>(v.base);
  if (!sp->base && v.n_records > 0) return MRN_EINVAL;
  if (reinterpret_cast<uintptr_t>(sp->base) % 8) return MRN_EALIGN;
  for (uint32_t c = 0; c < nc; ++c) sp->col[c] = sp->base + aosoa_col_start(t, B, c);
  return MRN_OK;
}

// AoS entries of a schema level, sorted by offset; the jagged descriptor is
// included for the parent level.
void aos_entries(const mrn_schema* t, bool with_jag, ConvPlan* p) {
  uint32_t k = 0;
  for (uint32_t c = 0; c < t->cols.size(); ++c)
    p->aos_cols[k++] = ColPlan{(uint16_t)t->cols[c].size, (int16_t)c, t->cols[c].aos_off};
  if (with_jag && t->has_jagged) {
    p->aos_cols[k++] = ColPlan{4, (int16_t)FM_JLEN, t->len_off};
    p->aos_cols[k++] = ColPlan{8, (int16_t)FM_JBEGIN, t->begin_off};
  }
  std::stable_sort(p->aos_cols, p->aos_cols + k,
                   [](const ColPlan& a, const ColPlan& b) { return a.aos_off < b.aos_off; });
  p->naos = k;
  p->ncols = (uint32_t)t->cols.size();
  for (uint32_t c = 0; c < t->cols.size(); ++c) {
    p->fm_size[c] = (uint8_t)t->cols[c].size;
    p->fm_es[c] = (uint16_t)t->cols[c].es;
  }
  p->stride = t->stride;
  p->aos_words = (t->stride + 3) / 4;
}

uint32_t aos_vec(uint32_t stride, const void* base) {
  return std::min<uint32_t>(16, std::min(lowbit(stride), lowbit(reinterpret_cast<uintptr_t>(base))));
}

// Plan of one schema level between two views (child = the jagged children).
int level_plan(const mrn_schema* s, const mrn_view& src, const mrn_view& dst, bool child, uint64_t n,
               ConvPlan* p) {
  std::memset(p, 0, sizeof(*p));
  const mrn_schema* t = child ? s->child.get() : s;
  if (t->cols.size() > MRN_MAX_COLS) return MRN_EUNSUPPORTED;
  aos_entries(t, !child, p);
  p->n = n;
  p->n_fm_pad = n;
  const bool sa = src.layout.kind == MRN_AOS, da = dst.layout.kind == MRN_AOS;
  int rc;
  if (sa && !da) {
    p->dir = DIR_AOS_FM;
    p->src.kind = K_AOS;
    p->src.base = static_cast<char*>(child ? src.child_pool : src.base);
    if ((rc = fm_side(s, dst, child, &p->dst))) return rc;
    p->vec = aos_vec(p->stride, p->src.base);
  } else if (!sa && da) {
    p->dir = DIR_FM_AOS;
    p->dst.kind = K_AOS;
    p->dst.base = static_cast<char*>(child ? dst.child_pool : dst.base);
    if ((rc = fm_side(s, src, child, &p->src))) return rc;
    p->vec = aos_vec(p->stride, p->dst.base);
  } else if (!sa && !da) {
    p->dir = DIR_FM_FM;
    if ((rc = fm_side(s, src, child, &p->src))) return rc;
    if ((rc = fm_side(s, dst, child, &p->dst))) return rc;
    p->vec = 1;
  } else {
    return MRN_EINVAL;  // AoS -> AoS is a plain copy, handled by the caller
  }
  if (!child && dst.layout.kind == MRN_AOSOA) {
    const uint64_t B = dst.layout.block;
    p->n_fm_pad = (n + B - 1) / B * B;
  }
  if ((p->dir == DIR_AOS_FM && !p->src.base && n) || (p->dir == DIR_FM_AOS && !p->dst.base && n))
    return MRN_EINVAL;
  return MRN_OK;
}

// Zero-fill plans of a destination (see gap_plans_of).
int gap_plans(const mrn_schema* s, const mrn_view& dst, GapPlan g[2]) {
  int np = 0;
  if (dst.layout.kind == MRN_AOSOA && dst.base) {  // holes inside every block
    GapPlan& h = g[np];
    std::memset(&h, 0, sizeof(h));
    const uint32_t B = dst.layout.block;
    uint64_t prev_end = 0;
    auto add = [&](uint64_t a, uint64_t b) {
      if (b > a && h.ngaps < MRN_MAX_GAPS) {
        h.off[h.ngaps] = a;
        h.len[h.ngaps] = (uint32_t)(b - a);
        h.ngaps++;
      }
    };
    for (uint32_t c = 0; c < s->cols.size(); ++c) {
      if (s->cols[c].sub) continue;  // inside its interleaved array's rows
      const uint64_t st = aosoa_col_start(s, B, c);
      add(prev_end, st);
      prev_end = st + (uint64_t)B * s->cols[c].es;
    }
    add(prev_end, aosoa_block_bytes(s, B));
    h.base = static_cast<char*>(dst.base);
    h.block_bytes = aosoa_block_bytes(s, B);
    h.nblocks = (dst.n_records + B - 1) / B;
    if (h.ngaps && h.nblocks) ++np;
  }
  const bool fm = dst.layout.kind == MRN_SOA || (dst.layout.kind == MRN_AOSOA && s->has_jagged);
  if (fm && fm_single_block(dst)) {  // bytes between the regions of one block
    GapPlan& h = g[np];
    std::memset(&h, 0, sizeof(h));
    const int kind = dst.layout.kind;
    const uint32_t B = dst.layout.block;
    const uint64_t n = dst.n_records, m = dst.n_children, m2 = dst.n_grandchildren;
    uint64_t prev_end = 0;
    auto add = [&](uint64_t a, uint64_t b) {
      if (b > a && h.ngaps < MRN_MAX_GAPS) {
        h.off[h.ngaps] = a;
        h.len[h.ngaps] = (uint32_t)(b - a);
        h.ngaps++;
      }
    };
    for (uint32_t r = 0; r < fm_region_count(s, kind); ++r) {
      const uint64_t st = fm_region_start(s, kind, B, n, m, r, m2);
      add(prev_end, st);
      prev_end = st + fm_region_bytes(s, kind, B, n, m, r, m2);
    }
    add(prev_end, fm_total_bytes(s, kind, B, n, m, m2));
    h.base = static_cast<char*>(dst.base);
    h.nblocks = 1;
    h.block_bytes = 0;
    if (h.ngaps) ++np;
  }
  return np;
}

}  // namespace

bool fm_single_block(const mrn_view& v) {
  if (!v.base) return false;
  if (v.layout.kind == MRN_SOA && v.columns) return false;
  if (v.schema->has_jagged && (v.offsets || v.child_columns)) return false;
  return true;
}

char* fm_offsets(const mrn_view& v) {
  if (v.offsets) return static_cast<char*>(v.offsets);
  if (!v.base) return nullptr;
  const mrn_schema* s = v.schema;
  return static_cast<char*>(v.base) + fm_region_start(s, v.layout.kind, v.layout.block, v.n_records,
                                                      v.n_children, parent_regions(s, v.layout.kind));
}

int gap_plans_of(const mrn_view& dst, GapPlan g[2]) { return gap_plans(dst.schema, dst, g); }

int zero_dst_gaps(const mrn_view& dst, void* stream) {
  GapPlan g[2];
  const int np = gap_plans(dst.schema, dst, g);
  for (int i = 0; i < np; ++i) {
    const int rc = launch_zero_gaps(g[i], stream);
    if (rc) return rc;
  }
  return MRN_OK;
}

int validate_pair(const mrn_view* src, const mrn_view* dst, bool need_device, bool* is_jagged) {
  if (!src || !dst || !src->schema || !dst->schema) return MRN_EINVAL;
  const mrn_schema* s = src->schema;
  if (!s->finalized || !dst->schema->finalized || s->hash != dst->schema->hash) return MRN_EINVAL;
  if (src->n_records != dst->n_records) return MRN_EINVAL;
  for (const mrn_view* v : {src, dst}) {
    if (v->layout.kind < MRN_AOS || v->layout.kind > MRN_AOSOA) return MRN_EINVAL;
    if (v->layout.kind == MRN_AOSOA && v->layout.block < 1) return MRN_EINVAL;
    if (v->mem < MRN_MEM_HOST || v->mem > MRN_MEM_DEVICE) return MRN_EINVAL;
  }
  if (need_device) {
    const int dev = current_device();
    if (dev < 0) return MRN_ECUDA;
    if (!on_device(*src) || !on_device(*dst) || src->device != dev || dst->device != dev)
      return MRN_EINVAL;
  }
  *is_jagged = s->has_jagged;
  if (s->cols.size() > MRN_MAX_COLS) return MRN_EUNSUPPORTED;
  if (s->has_jagged) {
    if (s->child->cols.size() > MRN_MAX_COLS) return MRN_EUNSUPPORTED;
    // nothing to convert between equal layouts
    if (src->layout.kind == dst->layout.kind &&
        (src->layout.kind != MRN_AOSOA || src->layout.block == dst->layout.block))
      return MRN_EUNSUPPORTED;
  }
  return MRN_OK;
}

uint64_t tune_key(uint64_t hash, const mrn_layout& a, const mrn_layout& b) {
  uint64_t h = hash ^ 0x9e3779b97f4a7c15ull;
  for (uint64_t v : {(uint64_t)a.kind, (uint64_t)a.block, (uint64_t)b.kind, (uint64_t)b.block}) {
    h ^= v + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
  }
  return h;
}

namespace {

uint64_t gcd_u64(uint64_t a, uint64_t b) {
  while (b) {
    const uint64_t t = a % b;
    a = b;
    b = t;
  }
  return a;
}

bool aligned16(const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15) == 0; }

// Bytes of one tile of T records of a side in shared memory (and, for SoA /
// AoSoA, each column's offset in the tile / start in a block).
uint64_t tile_bytes(const mrn_schema* s, const SidePlan& sp, uint32_t T, uint32_t* off) {
  if (sp.kind == K_AOS) return (uint64_t)T * s->stride;
  if (sp.kind == K_AOSOA) {
    if (off)
      for (uint32_t c = 0; c < s->cols.size(); ++c) off[c] = (uint32_t)aosoa_col_start(s, sp.block, c);
    return (uint64_t)(T / sp.block) * sp.block_bytes;
  }
  // SoA: one range of T elements per storage column, in column order (an
  // interleaved array's T rows once, its columns at their sub-offsets)
  uint64_t pos = 0, row_at = 0;
  for (uint32_t c = 0; c < s->cols.size(); ++c) {
    const MrnColumn& q = s->cols[c];
    if (q.sub == 0) {
      row_at = pos;
      pos += (uint64_t)T * q.es;
    }
    if (off) off[c] = (uint32_t)(row_at + q.sub);
  }
  return pos;
}

// An AoSoA block without alignment holes or tail padding: a staged tile then
// covers every byte of its blocks with column elements.
bool aosoa_hole_free(const mrn_schema* s, uint32_t B) {
  uint64_t pos = 0;
  for (uint32_t c = 0; c < s->cols.size(); ++c) {
    if (s->cols[c].sub) continue;  // inside its interleaved array's rows
    if (aosoa_col_start(s, B, c) != pos) return false;
    pos += (uint64_t)B * s->cols[c].es;
  }
  return pos == aosoa_block_bytes(s, B);
}

bool side_stageable(const mrn_schema* s, const SidePlan& sp, bool is_dst) {
  if (sp.kind == K_AOS) return aligned16(sp.base);
  if (sp.kind == K_AOSOA)
    return aligned16(sp.base) && sp.block_bytes % 16 == 0 && (!is_dst || aosoa_hole_free(s, sp.block));
  for (uint32_t c = 0; c < s->cols.size(); ++c)
    if (s->cols[c].sub == 0 && !aligned16(sp.col[c])) return false;
  return true;
}

// An AoS destination record with padding is zeroed before its fields are
// written.  Where every padding byte lies within the widest store a field
// preceding it can make (aligned within the record, at most 8 bytes and
// the record's own alignment in a tile row), the field is stored that wide
// instead, its value zero-extended, and the zeroing pass is dropped.  The
// widened fields go to the end of a second descriptor order, outside the
// size classes.  Leaves nwide = 0 when some padding byte is not covered.
void widen_into_padding(const mrn_schema* s, TileGeom* g) {
  const uint32_t S = s->stride, nc = (uint32_t)s->cols.size();
  if (S > 256) return;
  bool field[256] = {}, covered[256] = {};
  for (uint32_t c = 0; c < nc; ++c)
    for (uint32_t b = 0; b < s->cols[c].size; ++b) field[s->cols[c].aos_off + b] = covered[s->cols[c].aos_off + b] = true;
  const uint32_t amax = std::min<uint32_t>(8, lowbit(S));
  uint32_t wide[MRN_MAX_COLS] = {};
  for (uint32_t c = 0; c < nc; ++c) {
    const uint32_t off = s->cols[c].aos_off, sz = s->cols[c].size;
    for (uint32_t w = amax; w > sz; w >>= 1) {
      if (off % w || off + w > S) continue;
      bool pad_only = true;
      for (uint32_t b = off + sz; b < off + w; ++b) pad_only = pad_only && !field[b];
      if (!pad_only) continue;
      wide[c] = w == 8 ? 3 : w == 4 ? 2 : 1;
      for (uint32_t b = off + sz; b < off + w; ++b) covered[b] = true;
      break;
    }
  }
  for (uint32_t b = 0; b < S; ++b)
    if (!covered[b]) return;
  uint8_t order[MRN_MAX_COLS];
  uint32_t k = 0, nwide = 0, nsize = 0;
  for (uint32_t i = 0; i < nc; ++i) {
    const uint32_t c = g->order[i];
    if (wide[c]) continue;
    order[k++] = (uint8_t)c;
    nsize += 1u << (8 * (3 - ((g->col[c] >> 24) & 3u)));
  }
  for (uint32_t i = 0; i < nc; ++i) {
    const uint32_t c = g->order[i];
    if (!wide[c]) continue;
    order[k++] = (uint8_t)c;
    g->col[c] |= wide[c] << 28;
    ++nwide;
  }
  std::memcpy(g->worder, order, nc);
  g->wnsize = nsize;
  g->nwide = nwide;
}

// Chooses the shared-memory tile of a plan: the largest T, a multiple of 32
// and of every AoSoA block size, whose source and destination tiles each fit
// one stage buffer.  Leaves tg.tma = 0 when the plan cannot be staged (an
// unaligned buffer or block, or a record too wide for a stage).
void tile_geometry(const mrn_schema* s, ConvPlan* p, uint32_t stage_bytes) {
  TileGeom& g = p->tg;
  std::memset(&g, 0, sizeof(g));
  if (!side_stageable(s, p->src, false) || !side_stageable(s, p->dst, true)) return;
  if (s->stride >= (1u << 24)) return;
  uint64_t q = 32;
  for (const SidePlan* sp : {&p->src, &p->dst})
    if (sp->kind == K_AOSOA) q = q / gcd_u64(q, sp->block) * sp->block;
  uint32_t T = 0;
  for (uint64_t cand = q; cand <= 4096; cand += q) {
    if (tile_bytes(s, p->src, (uint32_t)cand, nullptr) > stage_bytes ||
        tile_bytes(s, p->dst, (uint32_t)cand, nullptr) > stage_bytes)
      break;
    T = (uint32_t)cand;
  }
  if (T == 0) return;
  g.T = T;
  g.G = (uint32_t)q;
  g.src_bytes = (uint32_t)tile_bytes(s, p->src, T, g.src_off);
  g.dst_bytes = (uint32_t)tile_bytes(s, p->dst, T, g.dst_off);
  uint32_t used = 0, k = 0;
  for (uint32_t c = 0; c < s->cols.size(); ++c) {
    const uint32_t sz = s->cols[c].size;
    const uint32_t lsz = sz == 1 ? 0 : sz == 2 ? 1 : sz == 4 ? 2 : 3;
    g.col[c] = s->cols[c].aos_off | (lsz << 24) | (s->cols[c].sub ? MRN_COL_SUB : 0u);
    used += sz;
  }
  g.inter = s->interleaved ? 1u : 0u;
  // the transform walks the columns one size class at a time
  for (uint32_t lsz = 4; lsz-- > 0;) {
    uint32_t cnt = 0;
    for (uint32_t c = 0; c < s->cols.size(); ++c)
      if (((g.col[c] >> 24) & 3u) == lsz) {
        g.order[k++] = (uint8_t)c;
        ++cnt;
      }
    g.nsize |= cnt << (8 * (3 - lsz));
  }
  g.pad = used != s->stride;
  if (g.pad && p->dst.kind == K_AOS && !s->has_jagged) widen_into_padding(s, &g);
  g.tma = 1;
}

}  // namespace

void plan_tiles(const mrn_schema* s, ConvPlan* p, uint32_t stage_bytes) { tile_geometry(s, p, stage_bytes); }

int build_plan(const mrn_view& src, const mrn_view& dst, ConvPlan* p) {
  int rc = level_plan(src.schema, src, dst, false, src.n_records, p);
  if (!rc) tile_geometry(src.schema, p, MRN_BATCH_STAGE_BYTES);
  mrn_layout a = src.layout, b = dst.layout;
  if (a.kind != MRN_AOSOA) a.block = 0;
  if (b.kind != MRN_AOSOA) b.block = 0;
  p->tune_key = tune_key(src.schema->hash, a, b);
  return rc;
}

int jagged_children_plan(const mrn_schema* s, const JagPlan& jp, ConvPlan* out) {
  *out = jp.child;
  out->n = out->n_fm_pad = jp.m_src;
  tile_geometry(s->child.get(), out, MRN_BATCH_STAGE_BYTES);
  return MRN_OK;
}

int jagged_pool_plan(const mrn_schema* s, const JagPlan& jp, ConvPlan* out) {
  *out = jp.child;
  out->n = out->n_fm_pad = jp.pool_n;
  tile_geometry(s->child.get(), out, MRN_BATCH_STAGE_BYTES);
  return MRN_OK;
}

bool jagged_split_ok(const mrn_schema* s, JagPlan* jp, ConvPlan* pool) {
  if (g_split_parents.load() < 0 || jp->parent.n == 0 || jp->pool_n == 0 || jp->pool_n > jp->capacity) return false;
  if (jagged_pool_plan(s, *jp, pool) != MRN_OK || !pool->tg.tma) return false;
  tile_geometry(s, &jp->parent, MRN_BATCH_STAGE_BYTES);
  // a staged tile's groups: at most three per consumer warp; parents with
  // an interleaved array stay on the direct path (the parents instance has
  // no interleaved transform)
  if (jp->parent.tg.tma && (jp->parent.tg.T > 768 || jp->parent.tg.inter)) jp->parent.tg.tma = 0;
  return true;
}

long long nested_split_children() { return g_nested_split_children.load(); }

bool jagged_local_ok(const JagPlan& jp) {
  // the largest offset written, offset_base + pool_n, fits the offset type
  return jp.off_size == 8 || (jp.offset_base <= 0xffffffffull && jp.pool_n <= 0xffffffffull - jp.offset_base);
}

int build_jagged_plan(const mrn_view& src, const mrn_view& dst, JagPlan* jp) {
  const mrn_schema* s = src.schema;
  std::memset(jp, 0, sizeof(*jp));
  const bool a2s = src.layout.kind == MRN_AOS;
  const mrn_view& soa = a2s ? dst : src;
  const uint64_t m = a2s ? dst.n_children : src.n_children;
  int rc = level_plan(s, src, dst, false, src.n_records, &jp->parent);
  if (rc) return rc;
  rc = level_plan(s, src, dst, true, m, &jp->child);
  if (rc) return rc;
  jp->off_size = s->off_size;
  jp->len_off = s->len_off;
  jp->begin_off = s->begin_off;
  char* offs = fm_offsets(soa);
  if (!offs) return MRN_EINVAL;
  if (reinterpret_cast<uintptr_t>(offs) % s->off_size) return MRN_EALIGN;
  jp->offsets = offs;
  jp->skip_publish_tile = g_skip_publish_tile.load();
  jp->timeout_ns = g_timeout_ns.load();
  if (a2s) {
    jp->pool_n = src.n_children;
    jp->capacity = dst.n_children;
    jp->offset_base = dst.offset_base;
    if (src.n_children > 0 && !src.child_pool) return MRN_EINVAL;
  } else {
    jp->m_src = src.n_children;
    if (dst.n_children < src.n_children) return MRN_ESIZE;
    if (src.n_children > 0 && !dst.child_pool) return MRN_EINVAL;
  }
  return MRN_OK;
}

// A jagged collection from one field-major layout to another: the parents
// change layout (a plain conversion of the parent columns); the offsets
// and the child values keep their order and are copied as they are.
int convert_jagged_fm(const mrn_view& src, const mrn_view& dst, void* stream) {
  const mrn_schema* s = src.schema;
  if (dst.n_children < src.n_children) return MRN_ESIZE;
  ConvPlan p;
  int rc = build_plan(src, dst, &p);
  if (rc) return rc;
  if ((rc = launch_convert(p, stream, nullptr))) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const uint64_t n = src.n_records, m = src.n_children;
  char* so = fm_offsets(src);
  char* dof = fm_offsets(dst);
  if (!so || !dof) return MRN_EINVAL;
  if (cudaMemcpyAsync(dof, so, (n + 1) * s->off_size, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return MRN_ECUDA;
  SidePlan a, b;
  if ((rc = fm_side(s, src, true, &a)) || (rc = fm_side(s, dst, true, &b))) return rc;
  for (uint32_t c = 0; c < s->child->cols.size() && m; ++c)
    if (cudaMemcpyAsync(b.col[c], a.col[c], m * s->child->cols[c].size, cudaMemcpyDeviceToDevice, st) !=
        cudaSuccess)
      return MRN_ECUDA;
  return zero_dst_gaps(dst, stream);
}

// A non-jagged conversion on the direct kernel only (plain loads and stores,
// no bulk copies), for views in mapped host memory.
int convert_direct(const mrn_view& src, const mrn_view& dst, void* stream) {
  ConvPlan p;
  int rc = build_plan(src, dst, &p);
  if (rc) return rc;
  LaunchShape sh;
  sh.generic = 1;
  if ((rc = launch_convert(p, stream, &sh))) return rc;
  return zero_dst_gaps(dst, stream);
}
}  // namespace mrn

using namespace mrn;

namespace {
// One non-blocking side stream per device, for work that runs beside the
// caller's stream inside one call (joined back before the call returns).
cudaStream_t side_stream() {
  static std::mutex mu;
  static cudaStream_t streams[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(mu);
  if (!streams[dev] && cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    streams[dev] = nullptr;
  }
  return streams[dev];
}
}  // namespace

extern "C" {

const char* mrn_status_str(int st) {
  switch (st) {
    case MRN_OK: return "MRN_OK";
    case MRN_EINVAL: return "MRN_EINVAL";
    case MRN_ESIZE: return "MRN_ESIZE";
    case MRN_EALIGN: return "MRN_EALIGN";
    case MRN_EOVERFLOW: return "MRN_EOVERFLOW";
    case MRN_ENOMEM: return "MRN_ENOMEM";
    case MRN_ETIMEOUT: return "MRN_ETIMEOUT";
    case MRN_ECUDA: return "MRN_ECUDA";
    case MRN_EBUSY: return "MRN_EBUSY";
    case MRN_ENOTFOUND: return "MRN_ENOTFOUND";
    case MRN_EUNSUPPORTED: return "MRN_EUNSUPPORTED";
    default: return "MRN_UNKNOWN";
  }
}

int mrn_version(void) { return 10000; }

int mrn_convert(const mrn_view* src, const mrn_view* dst, void* stream) {
  bool jag = false;
  int rc = validate_pair(src, dst, true, &jag);
  if (rc) return rc;
  const mrn_schema* s = src->schema;
  if (is_nested(s)) return convert_nested(*src, *dst, stream);
  if (jag && src->layout.kind != MRN_AOS && dst->layout.kind != MRN_AOS)
    return convert_jagged_fm(*src, *dst, stream);
  if (jag) {
    JagPlan jp;
    if ((rc = build_jagged_plan(*src, *dst, &jp))) return rc;
    if (src->layout.kind == MRN_AOS) {
      cudaStream_t st = static_cast<cudaStream_t>(stream);
      void* scratch = nullptr;
      // a single-block destination's few gaps are zeroed by the kernel's
      // tile 0 instead of a launch of their own
      GapPlan g[2];
      const int np = src->n_records > 0 ? gap_plans_of(*dst, g) : -1;
      const bool fold = np == 0 || (np == 1 && g[0].nblocks == 1 && g[0].ngaps <= MRN_JAG_GAPS);
      if (fold && np == 1) {
        jp.gap_base = g[0].base;
        jp.ngaps = g[0].ngaps;
        for (uint32_t k = 0; k < g[0].ngaps; ++k) {
          jp.gap_off[k] = g[0].off[k];
          jp.gap_len[k] = g[0].len[k];
        }
      }
      // Large collections run split: their children become one staged
      // conversion of the pool when the pool turns out canonical.
      ConvPlan pool;
      const long long lim = g_split_parents.load();
      const bool split = lim >= 0 && src->n_records >= (uint64_t)lim && jagged_split_ok(s, &jp, &pool) &&
                         jp.parent.tg.tma;
      const bool small = !split && (long long)src->n_records <= g_small_tile_parents.load();
      if (src->n_records > 0) {
        const uint64_t sb =
            split ? jagged_split_scratch_bytes(src->n_records)
                  : jagged_scratch_bytes(jagged_tile_records(jp), small ? MRN_JAG_SMALL_TILE : MRN_JAG_TILE);
        if (scratch_alloc(&scratch, sb, st) != MRN_OK) return MRN_ENOMEM;
      }
      rc = split ? launch_jagged_a2s_split(jp, pool, scratch, stream, !g_split_scan.load() && jagged_local_ok(jp))
                 : launch_jagged_a2s(jp, scratch, stream, small);
      scratch_free(scratch, st);
      if (rc) return rc;
      if (fold) return MRN_OK;
    } else {
      // The children are stored contiguously on both sides (Sec. V, jagged
      // vector property): child row j -> pool record j is a plain SoA -> AoS
      // conversion of the child schema; the kernel builds only the parents.
      // The parents (a latency-bound kernel over few bytes) run on a side
      // stream beside the children's bandwidth-bound conversion.
      ConvPlan kids;
      if ((rc = jagged_children_plan(s, jp, &kids))) return rc;
      jp.m_src = 0;
      cudaStream_t st = static_cast<cudaStream_t>(stream);
      // Large SoA parents whose record a plain schema reproduces: their
      // {length, begin} become two scratch columns, and the parents one
      // plain staged SoA -> AoS conversion of that schema, then the
      // children's (small collections keep the two launches below).
      const FlatParent* fp =
          src->layout.kind == MRN_SOA && src->n_records >= (1u << 18) ? flat_parent_schema(s) : nullptr;
      if (fp) {
        const uint64_t n = src->n_records;
        char* scratch = nullptr;
        const uint64_t beg_at = align_up(4 * n, 256);
        if (scratch_alloc(reinterpret_cast<void**>(&scratch), beg_at + 8 * n, st) != MRN_OK) return MRN_ENOMEM;
        // The parents (a small conversion) go first, on a side stream, and
        // the children's conversion right after on the caller's: its CTAs
        // take the SMs as the parents' finish, so the two launches overlap
        // instead of draining one before the other fills.
        cudaStream_t side = side_stream();
        cudaEvent_t fork = nullptr, join = nullptr;
        const bool par = side && cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) == cudaSuccess &&
                         cudaEventCreateWithFlags(&join, cudaEventDisableTiming) == cudaSuccess &&
                         cudaEventRecord(fork, st) == cudaSuccess && cudaStreamWaitEvent(side, fork, 0) == cudaSuccess;
        if (!par) cudaGetLastError();
        cudaStream_t ps_stream = par ? side : st;
        rc = launch_len_begin(jp.offsets, jp.off_size, n, reinterpret_cast<unsigned int*>(scratch),
                              reinterpret_cast<unsigned long long*>(scratch + beg_at), ps_stream);
        std::vector<void*> cols(fp->src.size());
        for (size_t k = 0; k < cols.size(); ++k)
          cols[k] = fp->src[k] >= 0 ? jp.parent.src.col[fp->src[k]] : fp->src[k] == -1 ? scratch : scratch + beg_at;
        mrn_view ps = *src, pd = *dst;
        ps.schema = pd.schema = fp->schema.get();
        ps.columns = cols.data();
        ps.offsets = nullptr;
        ps.child_columns = nullptr;
        ps.n_children = pd.n_children = ps.n_grandchildren = pd.n_grandchildren = 0;
        pd.child_pool = pd.grandchild_pool = nullptr;
        if (!rc) rc = mrn_convert(&ps, &pd, ps_stream);
        if (!rc) rc = launch_convert(kids, stream, nullptr);
        if (par && (cudaEventRecord(join, side) != cudaSuccess || cudaStreamWaitEvent(st, join, 0) != cudaSuccess) &&
            !rc)
          rc = MRN_ECUDA;
        if (fork) cudaEventDestroy(fork);
        if (join) cudaEventDestroy(join);
        scratch_free(scratch, st);
        if (rc) return rc;
        return zero_dst_gaps(*dst, stream);
      }
      cudaStream_t side = side_stream();
      cudaEvent_t fork = nullptr, join = nullptr;
      const bool split = side && cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) == cudaSuccess &&
                         cudaEventCreateWithFlags(&join, cudaEventDisableTiming) == cudaSuccess &&
                         cudaEventRecord(fork, st) == cudaSuccess && cudaStreamWaitEvent(side, fork, 0) == cudaSuccess;
      if (!split) cudaGetLastError();
      rc = launch_jagged_s2a(jp, split ? side : st);
      if (split && cudaEventRecord(join, side) != cudaSuccess && !rc) rc = MRN_ECUDA;
      if (!rc) rc = launch_convert(kids, stream, nullptr);
      if (split && cudaStreamWaitEvent(st, join, 0) != cudaSuccess && !rc) rc = MRN_ECUDA;
      if (fork) cudaEventDestroy(fork);
      if (join) cudaEventDestroy(join);
      if (rc) return rc;
    }
    return zero_dst_gaps(*dst, stream);
  }
  if (src->layout.kind == MRN_AOS && dst->layout.kind == MRN_AOS) {
    const size_t bytes = (size_t)src->n_records * s->stride;
    if (bytes && (!src->base || !dst->base)) return MRN_EINVAL;
    if (!bytes) return MRN_OK;
    return cudaMemcpyAsync(dst->base, src->base, bytes, cudaMemcpyDeviceToDevice,
                           static_cast<cudaStream_t>(stream)) == cudaSuccess
               ? MRN_OK
               : MRN_ECUDA;
  }
  ConvPlan p;
  if ((rc = build_plan(*src, *dst, &p))) return rc;
  LaunchShape sh = tuned_shape(p);
  if (g_force_direct.load()) sh.generic = 1;
  if ((rc = launch_convert(p, stream, &sh))) return rc;
  return zero_dst_gaps(*dst, stream);
}

int mrn_sync(void* stream) {
  uint32_t bits = 0;
  int rc = read_and_clear_status(stream, &bits);
  if (rc) return rc;
  return status_from_bits(bits);
}

int mrn_scratch_release(int device) { return mrn::scratch_release(device); }

int mrn_sync_bits(void* stream, uint32_t* bits) {
  if (!bits) return MRN_EINVAL;
  return read_and_clear_status(stream, bits);
}

int mrn_jagged_count(const mrn_view* src, uint64_t* m, void* stream) {
  if (!src || !m || !src->schema || !src->schema->finalized || !src->schema->has_jagged ||
      src->layout.kind != MRN_AOS || src->mem != MRN_MEM_DEVICE)
    return MRN_EINVAL;
  if (src->device != current_device()) return MRN_EINVAL;
  *m = 0;
  if (src->n_records == 0) return MRN_OK;
  if (!src->base) return MRN_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  ConvPlan p;
  std::memset(&p, 0, sizeof(p));
  aos_entries(src->schema, true, &p);
  p.n = src->n_records;
  p.src.base = static_cast<char*>(src->base);
  uint64_t* d = nullptr;
  if (scratch_alloc(reinterpret_cast<void**>(&d), sizeof(uint64_t), st) != MRN_OK) return MRN_ENOMEM;
  int rc = MRN_OK;
  if (cudaMemsetAsync(d, 0, sizeof(uint64_t), st) != cudaSuccess) rc = MRN_ECUDA;
  if (!rc) rc = launch_jagged_count(p, d, stream);
  uint64_t h = 0;
  if (!rc && cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess) rc = MRN_ECUDA;
  scratch_free(d, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) rc = MRN_ECUDA;
  if (!rc) *m = h;
  return rc;
}

int mrn_debug_set(int key, long long value) {
  switch (key) {
    case 1: g_skip_publish_tile.store(value); return MRN_OK;
    case 2:
      if (value <= 0) return MRN_EINVAL;
      g_timeout_ns.store((unsigned long long)value);
      return MRN_OK;
    case 3: g_force_direct.store(value ? 1 : 0); return MRN_OK;
    case 4: g_split_parents.store(value < 0 ? -1 : value); return MRN_OK;
    case 5: g_small_tile_parents.store(value); return MRN_OK;
    case 6: g_split_scan.store(value ? 1 : 0); return MRN_OK;
    case 7: g_nested_split_children.store(value < 0 ? -1 : value); return MRN_OK;
    default: return MRN_EINVAL;
  }
}

}  // extern "C"
