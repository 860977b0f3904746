// Nested jagged members: a jagged member whose child records hold a jagged
// member of their own (Sec. V: the children are themselves a collection
// described by properties; one nesting level).  The conversion runs level by
// level with the library's own jagged kernels:
//
//   field-major -> AoS: the child level is an ordinary jagged SoA -> AoS
//     conversion of the child schema (child columns + the children's
//     offsets + grandchild columns -> child records with their {length,
//     begin} + the grandchild pool), then the parents' records are built
//     from their offsets;
//   AoS -> field-major: the parents' tile scan gathers each child's data
//     columns into the child level and its {length, begin} into two scratch
//     columns; the children's offsets are their begins when the grandchild
//     pool is canonical (checked child against child), else a scan of those
//     columns writes them; the pool is then converted as one staged
//     conversion when canonical and gathered child by child otherwise, all
//     on the device (the children's count never returns to the host).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "mrn_internal.h"

namespace mrn {

namespace {

// A finalized schema built through the C API, destroyed with the object.
struct OwnedSchema {
  mrn_schema* s = nullptr;
  ~OwnedSchema() { mrn_schema_destroy(s); }
};

mrn_view device_view(const mrn_schema* s, int kind, int device, uint64_t n, uint64_t m) {
  mrn_view v;
  std::memset(&v, 0, sizeof(v));
  v.schema = s;
  v.layout.kind = kind;
  v.layout.block = 0;
  v.mem = MRN_MEM_DEVICE;
  v.device = device;
  v.n_records = n;
  v.n_children = m;
  return v;
}

}  // namespace

int convert_nested(const mrn_view& src, const mrn_view& dst, void* stream) {
  const mrn_schema* s = src.schema;
  const mrn_schema* ch = s->child.get();
  const bool a2s = src.layout.kind == MRN_AOS, s2a = dst.layout.kind == MRN_AOS;
  if (a2s == s2a) return MRN_EUNSUPPORTED;  // field-major to field-major
  const mrn_view& fm = a2s ? dst : src;
  const mrn_view& aos = a2s ? src : dst;
  if (!fm.base || !fm_single_block(fm)) return MRN_EUNSUPPORTED;  // single-block field-major side
  if (aos.n_children > 0 && !aos.child_pool) return MRN_EINVAL;
  if (aos.n_grandchildren > 0 && !aos.grandchild_pool) return MRN_EINVAL;
  const int kind = fm.layout.kind;
  const uint32_t B = fm.layout.block;
  const uint64_t n = fm.n_records, m = fm.n_children, m2 = fm.n_grandchildren;
  char* base = static_cast<char*>(fm.base);
  // The field-major side's child level, as per-column pointers.
  std::vector<void*> kcols(ch->cols.size()), gcols(ch->child->cols.size());
  for (uint32_t c = 0; c < kcols.size(); ++c) kcols[c] = base + fm_col_start(s, kind, B, n, m, true, c, m2);
  for (uint32_t g = 0; g < gcols.size(); ++g) gcols[g] = base + fm_gchild_col_start(s, kind, B, n, m, m2, g);
  char* off1 = base + fm_child_offsets_start(s, kind, B, n, m, m2);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int rc;

  if (s2a) {
    if (dst.n_children < src.n_children || dst.n_grandchildren < src.n_grandchildren) return MRN_ESIZE;
    // child level: child columns + offsets + grandchild columns -> child
    // records (with their descriptors) + grandchild pool
    mrn_view ks = device_view(ch, MRN_SOA, src.device, src.n_children, src.n_grandchildren);
    ks.base = off1;
    ks.columns = kcols.data();
    ks.offsets = off1;
    ks.child_columns = gcols.data();
    mrn_view kd = device_view(ch, MRN_AOS, dst.device, src.n_children, dst.n_grandchildren);
    kd.base = dst.child_pool;
    kd.child_pool = dst.grandchild_pool;
    if ((rc = mrn_convert(&ks, &kd, stream))) return rc;
    // parents: records with {length, begin} from their offsets
    JagPlan jp;
    if ((rc = build_jagged_plan(src, dst, &jp))) return rc;
    jp.m_src = 0;
    return launch_jagged_s2a(jp, stream);
  }

  // AoS -> field-major.  Level 0 gathers the children's descriptors into
  // scratch columns beside their data columns.
  JagPlan jp;
  if ((rc = build_jagged_plan(src, dst, &jp))) return rc;
  ConvPlan& C = jp.child;
  const uint32_t nc = (uint32_t)ch->cols.size();
  if (nc + 2 > MRN_MAX_COLS) return MRN_EUNSUPPORTED;
  const uint64_t mcap = dst.n_children;
  // (the look-back words of level 0, fused or the split's fall-back)
  const uint64_t lb_bytes = align_up(jagged_scratch_bytes(std::max<uint64_t>(1, jagged_tile_records(jp))), 256);
  const uint64_t len_at = lb_bytes, beg_at = align_up(len_at + 4 * mcap, 256),
                 tot_at = align_up(beg_at + 8 * mcap, 256);
  char* scratch = nullptr;
  char* cscratch = nullptr;
  if (scratch_alloc(reinterpret_cast<void**>(&scratch), tot_at + 256, st) != MRN_OK) return MRN_ENOMEM;
  auto done = [&](int r) {
    scratch_free(cscratch, st);
    scratch_free(scratch, st);
    return r;
  };
  C.aos_cols[C.naos++] = ColPlan{4, (int16_t)nc, ch->len_off};
  C.aos_cols[C.naos++] = ColPlan{8, (int16_t)(nc + 1), ch->begin_off};
  std::stable_sort(C.aos_cols, C.aos_cols + C.naos,
                   [](const ColPlan& a, const ColPlan& b) { return a.aos_off < b.aos_off; });
  C.dst.col[nc] = scratch + len_at;
  C.dst.col[nc + 1] = scratch + beg_at;
  C.fm_size[nc] = 4;
  C.fm_es[nc] = 4;
  C.fm_size[nc + 1] = 8;
  C.fm_es[nc + 1] = 8;
  unsigned long long* d_total = reinterpret_cast<unsigned long long*>(scratch + tot_at);
  jp.total_out = d_total;
  if (cudaMemsetAsync(d_total, 0, sizeof(unsigned long long), st) != cudaSuccess) return done(MRN_ECUDA);
  // Many children: level 0 split in the local form (the parents with their
  // begins as offsets and the pool's check, then the child pool as one
  // staged conversion of the child record's flat schema, its {length,
  // begin} into the scratch columns, and the fused tiles again only for a
  // pool that is not canonical).  The parents need staged tiles of at most
  // 768 records and the pool's records a flat schema.
  const long long split_from = nested_split_children();
  bool split0 = false;
  ConvPlan pool0;
  const FlatParent* fc = split_from >= 0 && src.n_children >= (uint64_t)split_from && src.n_records > 0 &&
                                 src.n_children > 0 && src.n_children <= mcap && jagged_local_ok(jp)
                             ? flat_parent_schema(ch)
                             : nullptr;
  std::vector<void*> pcols;
  if (fc) {
    pcols.resize(fc->src.size());
    for (size_t k = 0; k < pcols.size(); ++k)
      pcols[k] = fc->src[k] >= 0 ? kcols[fc->src[k]] : fc->src[k] == -1 ? scratch + len_at : scratch + beg_at;
    mrn_view ps = device_view(fc->schema.get(), MRN_AOS, src.device, src.n_children, 0);
    ps.base = src.child_pool;
    mrn_view pd = device_view(fc->schema.get(), MRN_SOA, dst.device, src.n_children, 0);
    pd.base = scratch + len_at;  // not read: the columns are given
    pd.columns = pcols.data();
    if (build_plan(ps, pd, &pool0) == MRN_OK && pool0.tg.tma) {
      plan_tiles(s, &jp.parent, MRN_BATCH_STAGE_BYTES);
      split0 = jp.parent.tg.tma && jp.parent.tg.T <= 768 && !jp.parent.tg.inter;
    }
  }
  if ((rc = split0 ? launch_jagged_a2s_split(jp, pool0, scratch, stream, true) : launch_jagged_a2s(jp, scratch, stream)))
    return done(rc);

  // Level 1, without a return to the host: the children's count M stays in
  // device memory (a count above the capacity is recorded by level 0 as
  // MRN_ESIZE, and level 1 then covers the capacity).  The children's
  // offsets are their begins where the grandchild pool is canonical (the
  // grandchildren exactly its records, in child order: each begin the
  // previous begin plus its length), which a pass over the two gathered
  // columns checks; where a check fails, a scan of the columns writes the
  // offsets instead.  A canonical pool is then one staged conversion of
  // the grandchild schema, and otherwise a gathering pass copies each
  // child's grandchildren to its rows (all decided on the device).
  OwnedSchema desc;
  if (mrn_schema_create(&desc.s) ||
      mrn_schema_add_jagged(desc.s, "v", ch->off_size == 4 ? MRN_U32 : MRN_U64, ch->child.get()) ||
      mrn_schema_finalize(desc.s))
    return done(MRN_ENOMEM);
  mrn_view ds = device_view(desc.s, MRN_AOS, src.device, mcap, src.n_grandchildren);
  ds.base = scratch + len_at;  // not read: the plans need a non-null base
  ds.child_pool = src.grandchild_pool;
  mrn_view dd = device_view(desc.s, MRN_SOA, dst.device, mcap, dst.n_grandchildren);
  dd.base = off1;
  dd.offsets = off1;
  dd.child_columns = gcols.data();
  JagPlan jp1;
  ConvPlan pool;
  if ((rc = build_jagged_plan(ds, dd, &jp1)) || (rc = jagged_pool_plan(desc.s, jp1, &pool))) return done(rc);
  const bool staged_pool = pool.tg.tma && src.n_grandchildren <= dst.n_grandchildren;
  if (scratch_alloc(reinterpret_cast<void**>(&cscratch), col_scan_scratch_bytes(mcap), st) != MRN_OK)
    return done(MRN_ENOMEM);
  ColScan cs;
  std::memset(&cs, 0, sizeof(cs));
  cs.len = reinterpret_cast<const unsigned int*>(scratch + len_at);
  cs.beg = reinterpret_cast<const unsigned long long*>(scratch + beg_at);
  cs.n = mcap;
  cs.count = d_total;
  cs.pool_n = src.n_grandchildren;
  cs.offsets = off1;
  cs.off_size = ch->off_size;
  cs.timeout_ns = jp1.timeout_ns;
  cs.skip_publish_tile = jp1.skip_publish_tile;
  const bool local = cs.off_size == 8 || cs.pool_n <= 0xffffffffull;
  if ((rc = launch_col_scan(cs, cscratch, stream, local))) return done(rc);
  if (staged_pool && (rc = launch_convert(pool, stream, nullptr, cs.noncanon))) return done(rc);
  if ((rc = launch_col_gather(cs, jp1.child, dst.n_grandchildren, !staged_pool, stream))) return done(rc);
  if ((rc = zero_dst_gaps(dst, stream))) return done(rc);
  return done(MRN_OK);
}

}  // namespace mrn
