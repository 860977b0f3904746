// Schema builder and compiler: lowers a property description (Sec. V) to
// flattened columns with AoS offsets, and implements the layout rules.
#include <algorithm>
#include <cstdio>
#include <mutex>
#include <map>
#include <cstring>
#include <new>

#include "mrn_internal.h"

struct mrn_schema_node {
  enum Kind { FIELD, GROUP, JAGGED } kind;
  std::string name;
  int dtype = 0;
  uint32_t extent = 1;
  bool interleaved = false;  // FIELD: one field-major N x extent array
  int offset_dtype = 0;
  std::vector<std::unique_ptr<mrn_schema_node>> members;  // GROUP
  std::unique_ptr<mrn_schema> child;                      // JAGGED (finalized copy)
};

namespace mrn {

uint32_t dtype_size(int dtype) {
  switch (dtype) {
    case MRN_U8: case MRN_I8: case MRN_BOOL: return 1;
    case MRN_U16: case MRN_I16: return 2;
    case MRN_U32: case MRN_I32: case MRN_F32: return 4;
    case MRN_U64: case MRN_I64: case MRN_F64: return 8;
    default: return 0;
  }
}

namespace {

uint64_t fnv(uint64_t h, uint64_t v) {
  for (int i = 0; i < 8; ++i) {
    h ^= (v >> (8 * i)) & 0xff;
    h *= 1099511628211ull;
  }
  return h;
}

// Lays out the members of one struct level (C rules: each member at the
// next multiple of its alignment; a group is a nested struct).  Column
// offsets are relative to the struct start.  Returns false on error.
bool lay_out(const std::vector<std::unique_ptr<mrn_schema_node>>& members, const std::string& prefix,
             mrn_schema* s, uint64_t* size, uint64_t* align) {
  uint64_t cur = 0, al = 1;
  for (const auto& m : members) {
    if (m->kind == mrn_schema_node::FIELD) {
      const uint32_t sz = dtype_size(m->dtype);
      const uint64_t off = align_up(cur, sz);
      for (uint32_t k = 0; k < m->extent; ++k) {
        MrnColumn c;
        c.size = sz;
        c.aos_off = (uint32_t)(off + (uint64_t)k * sz);
        c.dtype = m->dtype;
        c.name = prefix + m->name;
        if (m->extent > 1) c.name += "[" + std::to_string(k) + "]";
        if (!m->interleaved || k == 0) s->stores.push_back(MrnStore{m->interleaved ? sz * m->extent : sz, sz});
        c.store = (uint32_t)s->stores.size() - 1;
        c.es = s->stores.back().es;
        c.sub = m->interleaved ? k * sz : 0;
        s->cols.push_back(c);
      }
      if (m->interleaved && m->extent > 1) s->interleaved = true;
      cur = off + (uint64_t)m->extent * sz;
      al = std::max<uint64_t>(al, sz);
    } else if (m->kind == mrn_schema_node::GROUP) {
      const size_t first = s->cols.size();
      const bool had = s->has_jagged;
      uint64_t gs = 0, ga = 1;
      if (!lay_out(m->members, prefix + m->name + ".", s, &gs, &ga)) return false;
      const uint64_t goff = align_up(cur, ga);
      for (size_t c = first; c < s->cols.size(); ++c) s->cols[c].aos_off += (uint32_t)goff;
      if (s->has_jagged && !had) {
        s->len_off += (uint32_t)goff;
        s->begin_off += (uint32_t)goff;
      }
      cur = goff + gs;
      al = std::max(al, ga);
    } else {
      if (s->has_jagged) return false;
      s->has_jagged = true;
      s->off_size = dtype_size(m->offset_dtype);
      s->len_off = (uint32_t)align_up(cur, 4);
      cur = s->len_off + 4;
      s->begin_off = (uint32_t)align_up(cur, 8);
      cur = s->begin_off + 8;
      al = std::max<uint64_t>(al, 8);
    }
    if (cur > 0xffffffffull) return false;
  }
  *size = align_up(cur, al);
  *align = al;
  return true;
}

mrn_schema_node* find_jagged(const std::vector<std::unique_ptr<mrn_schema_node>>& members) {
  for (const auto& m : members) {
    if (m->kind == mrn_schema_node::JAGGED) return m.get();
    if (m->kind == mrn_schema_node::GROUP)
      if (auto* j = find_jagged(m->members)) return j;
  }
  return nullptr;
}

std::unique_ptr<mrn_schema_node> clone_node(const mrn_schema_node& n);

std::unique_ptr<mrn_schema> clone_schema(const mrn_schema& s) {
  auto c = std::make_unique<mrn_schema>();
  for (const auto& r : s.roots) c->roots.push_back(clone_node(*r));
  c->finalized = s.finalized;
  c->cols = s.cols;
  c->stores = s.stores;
  c->interleaved = s.interleaved;
  c->stride = s.stride;
  c->align = s.align;
  c->has_jagged = s.has_jagged;
  c->len_off = s.len_off;
  c->begin_off = s.begin_off;
  c->off_size = s.off_size;
  if (s.child) c->child = clone_schema(*s.child);
  c->hash = s.hash;
  return c;
}

std::unique_ptr<mrn_schema_node> clone_node(const mrn_schema_node& n) {
  auto c = std::make_unique<mrn_schema_node>();
  c->kind = n.kind;
  c->name = n.name;
  c->dtype = n.dtype;
  c->extent = n.extent;
  c->interleaved = n.interleaved;
  c->offset_dtype = n.offset_dtype;
  for (const auto& m : n.members) c->members.push_back(clone_node(*m));
  if (n.child) c->child = clone_schema(*n.child);
  return c;
}

std::vector<std::unique_ptr<mrn_schema_node>>* current_list(mrn_schema* s) {
  return s->open_groups.empty() ? &s->roots : &s->open_groups.back()->members;
}

bool valid_name(const char* name) { return name && std::strlen(name) < 64; }

}  // namespace

namespace {
// Start of storage column q inside an AoSoA(B) block: the C struct of the
// storage columns' B-element arrays (an interleaved array: B rows of E).
uint64_t aosoa_store_start(const mrn_schema* s, uint32_t B, uint32_t q) {
  uint64_t end = 0, start = 0;
  for (uint32_t k = 0; k <= q; ++k) {
    start = align_up(end, s->stores[k].align);
    end = start + (uint64_t)B * s->stores[k].es;
  }
  return start;
}
}  // namespace

uint64_t aosoa_col_start(const mrn_schema* s, uint32_t B, uint32_t c) {
  return aosoa_store_start(s, B, s->cols[c].store) + s->cols[c].sub;
}

uint64_t aosoa_block_bytes(const mrn_schema* s, uint32_t B) {
  uint64_t end = 0, al = 1;
  for (const auto& q : s->stores) {
    end = align_up(end, q.align) + (uint64_t)B * q.es;
    al = std::max<uint64_t>(al, q.align);
  }
  return align_up(end, al);
}

// Regions of a single-block field-major view: SoA: the data storage
// columns, then (jagged) the offsets and the child storage columns; jagged
// AoSoA(B): the parent blocks, then the offsets and the child storage
// columns.
uint32_t parent_regions(const mrn_schema* s, int kind) {
  return kind == MRN_AOSOA ? 1u : (uint32_t)s->stores.size();
}
uint64_t fm_region_bytes(const mrn_schema* s, int kind, uint32_t B, uint64_t n, uint64_t m, uint32_t r,
                         uint64_t m2) {
  const uint32_t P = parent_regions(s, kind);
  if (r < P) return kind == MRN_AOSOA ? (n + B - 1) / B * aosoa_block_bytes(s, B) : n * s->stores[r].es;
  if (r == P) return (n + 1) * s->off_size;
  return fm_region_bytes(s->child.get(), MRN_SOA, 0, m, m2, r - P - 1, 0);
}

uint32_t fm_region_count(const mrn_schema* s, int kind) {
  return parent_regions(s, kind) + (s->has_jagged ? 1 + fm_region_count(s->child.get(), MRN_SOA) : 0);
}

uint64_t fm_region_start(const mrn_schema* s, int kind, uint32_t B, uint64_t n, uint64_t m, uint32_t r,
                         uint64_t m2) {
  uint64_t pos = 0;
  for (uint32_t k = 0; k < r; ++k) pos = align_up(pos + fm_region_bytes(s, kind, B, n, m, k, m2), 128);
  return pos;
}

uint64_t fm_child_offsets_start(const mrn_schema* s, int kind, uint32_t B, uint64_t n, uint64_t m, uint64_t m2) {
  return fm_region_start(s, kind, B, n, m, parent_regions(s, kind) + 1 + (uint32_t)s->child->stores.size(), m2);
}

uint64_t fm_gchild_col_start(const mrn_schema* s, int kind, uint32_t B, uint64_t n, uint64_t m, uint64_t m2,
                             uint32_t g) {
  const MrnColumn& gc = s->child->child->cols[g];
  return fm_region_start(s, kind, B, n, m, parent_regions(s, kind) + 2 + (uint32_t)s->child->stores.size() + gc.store,
                         m2) + gc.sub;
}

uint64_t soa_region_start(const mrn_schema* s, uint64_t n, uint64_t m, uint32_t r) {
  return fm_region_start(s, MRN_SOA, 0, n, m, r);
}

uint64_t fm_col_start(const mrn_schema* s, int kind, uint32_t B, uint64_t n, uint64_t m, bool child, uint32_t c,
                      uint64_t m2) {
  if (!child) return fm_region_start(s, kind, B, n, m, s->cols[c].store, m2) + s->cols[c].sub;
  const MrnColumn& cc = s->child->cols[c];
  return fm_region_start(s, kind, B, n, m, parent_regions(s, kind) + 1 + cc.store, m2) + cc.sub;
}

uint64_t fm_total_bytes(const mrn_schema* s, int kind, uint32_t B, uint64_t n, uint64_t m, uint64_t m2) {
  const uint32_t nr = fm_region_count(s, kind);
  return align_up(fm_region_start(s, kind, B, n, m, nr - 1, m2) + fm_region_bytes(s, kind, B, n, m, nr - 1, m2),
                  128);
}

uint64_t soa_total_bytes(const mrn_schema* s, uint64_t n, uint64_t m) { return fm_total_bytes(s, MRN_SOA, 0, n, m); }

uint64_t base_bytes(const mrn_schema* s, const mrn_layout& l, uint64_t n, uint64_t m, uint64_t m2) {
  switch (l.kind) {
    case MRN_AOS: return n * s->stride;
    case MRN_SOA: return fm_total_bytes(s, MRN_SOA, 0, n, m, m2);
    default:
      if (s->has_jagged) return fm_total_bytes(s, MRN_AOSOA, l.block, n, m, m2);
      return (n + l.block - 1) / l.block * aosoa_block_bytes(s, l.block);
  }
}

const FlatParent* flat_parent_schema(const mrn_schema* s) {
  static std::mutex mu;
  static std::map<uint64_t, std::unique_ptr<FlatParent>> cache;  // nullptr: not reproducible
  std::lock_guard<std::mutex> lk(mu);
  auto it = cache.find(s->hash);
  if (it != cache.end()) return it->second.get();
  std::unique_ptr<FlatParent> f;
  if (s->has_jagged && !s->interleaved && s->cols.size() + 2 <= MRN_MAX_COLS) {
    // every field of the record in offset order, the descriptor included
    struct Item {
      uint32_t off;
      int dtype;
      int src;
    };
    std::vector<Item> items;
    for (size_t c = 0; c < s->cols.size(); ++c) items.push_back({s->cols[c].aos_off, s->cols[c].dtype, (int)c});
    items.push_back({s->len_off, MRN_U32, -1});
    items.push_back({s->begin_off, MRN_U64, -2});
    std::stable_sort(items.begin(), items.end(), [](const Item& a, const Item& b) { return a.off < b.off; });
    f = std::make_unique<FlatParent>();
    mrn_schema* raw = nullptr;
    bool ok = mrn_schema_create(&raw) == MRN_OK;
    f->schema.reset(raw);
    for (size_t i = 0; ok && i < items.size(); ++i) {
      char nm[16];
      std::snprintf(nm, sizeof(nm), "f%zu", i);
      ok = mrn_schema_add_field(raw, nm, items[i].dtype, 1) == MRN_OK;
      f->src.push_back(items[i].src);
    }
    ok = ok && mrn_schema_finalize(raw) == MRN_OK;
    // usable only when the flat record is the parent record, byte for byte
    ok = ok && raw->stride == s->stride && raw->cols.size() == items.size();
    for (size_t i = 0; ok && i < items.size(); ++i) ok = raw->cols[i].aos_off == items[i].off;
    if (!ok) f.reset();
  }
  const FlatParent* r = f.get();
  cache.emplace(s->hash, std::move(f));
  return r;
}

}  // namespace mrn

using namespace mrn;

extern "C" {

int mrn_schema_create(mrn_schema** out) {
  if (!out) return MRN_EINVAL;
  *out = new (std::nothrow) mrn_schema();
  return *out ? MRN_OK : MRN_ENOMEM;
}

void mrn_schema_destroy(mrn_schema* s) { delete s; }

int mrn_schema_add_field(mrn_schema* s, const char* name, int dtype, uint32_t extent) {
  if (!s || s->finalized || !valid_name(name) || dtype_size(dtype) == 0 || extent < 1 ||
      extent > 4096)
    return MRN_EINVAL;
  auto n = std::make_unique<mrn_schema_node>();
  n->kind = mrn_schema_node::FIELD;
  n->name = name;
  n->dtype = dtype;
  n->extent = extent;
  current_list(s)->push_back(std::move(n));
  return MRN_OK;
}

int mrn_schema_add_field_interleaved(mrn_schema* s, const char* name, int dtype, uint32_t extent) {
  if (!s || s->finalized || !valid_name(name) || dtype_size(dtype) == 0 || extent < 1 ||
      (uint64_t)extent * dtype_size(dtype) > 65535)
    return MRN_EINVAL;
  auto n = std::make_unique<mrn_schema_node>();
  n->kind = mrn_schema_node::FIELD;
  n->name = name;
  n->dtype = dtype;
  n->extent = extent;
  n->interleaved = true;
  current_list(s)->push_back(std::move(n));
  return MRN_OK;
}

int mrn_schema_begin_group(mrn_schema* s, const char* name) {
  if (!s || s->finalized || !valid_name(name) || s->open_groups.size() >= 32) return MRN_EINVAL;
  auto n = std::make_unique<mrn_schema_node>();
  n->kind = mrn_schema_node::GROUP;
  n->name = name;
  mrn_schema_node* raw = n.get();
  current_list(s)->push_back(std::move(n));
  s->open_groups.push_back(raw);
  return MRN_OK;
}

int mrn_schema_end_group(mrn_schema* s) {
  if (!s || s->finalized || s->open_groups.empty()) return MRN_EINVAL;
  s->open_groups.pop_back();
  return MRN_OK;
}

int mrn_schema_add_jagged(mrn_schema* s, const char* name, int offset_dtype, const mrn_schema* child) {
  if (!s || s->finalized || !valid_name(name) || !child || !child->finalized || is_nested(child) ||
      child->cols.empty() || (offset_dtype != MRN_U32 && offset_dtype != MRN_U64) ||
      find_jagged(s->roots))
    return MRN_EINVAL;
  if (child->interleaved) return MRN_EUNSUPPORTED;  // child columns are stored one by one
  auto n = std::make_unique<mrn_schema_node>();
  n->kind = mrn_schema_node::JAGGED;
  n->name = name;
  n->offset_dtype = offset_dtype;
  n->child = clone_schema(*child);
  current_list(s)->push_back(std::move(n));
  return MRN_OK;
}

int mrn_schema_finalize(mrn_schema* s) {
  if (!s || s->finalized || !s->open_groups.empty()) return MRN_EINVAL;
  s->cols.clear();
  s->stores.clear();
  s->interleaved = false;
  s->has_jagged = false;
  uint64_t size = 0, al = 1;
  if (!lay_out(s->roots, "", s, &size, &al)) return MRN_EINVAL;
  if (s->cols.empty() && !s->has_jagged) return MRN_EINVAL;
  s->stride = (uint32_t)size;
  s->align = (uint32_t)al;
  if (s->has_jagged) s->child = clone_schema(*find_jagged(s->roots)->child);
  uint64_t h = 1469598103934665603ull;
  h = fnv(h, s->stride);
  h = fnv(h, s->cols.size());
  for (const auto& c : s->cols) h = fnv(fnv(fnv(fnv(h, c.size), c.aos_off), c.es), c.sub);
  if (s->has_jagged) {
    h = fnv(fnv(fnv(h, s->len_off), s->begin_off), s->off_size);
    h = fnv(h, s->child->hash);
  }
  s->hash = h;
  s->finalized = true;
  return MRN_OK;
}

int mrn_schema_info_get(const mrn_schema* s, mrn_schema_info* out) {
  if (!s || !s->finalized || !out) return MRN_EINVAL;
  std::memset(out, 0, sizeof(*out));
  out->n_columns = (uint32_t)s->cols.size();
  out->aos_stride = s->stride;
  out->aos_align = s->align;
  out->has_jagged = s->has_jagged ? 1 : 0;
  if (s->has_jagged) {
    out->jag_length_offset = s->len_off;
    out->jag_begin_offset = s->begin_off;
    out->offset_size = s->off_size;
    out->child_columns = (uint32_t)s->child->cols.size();
    out->child_stride = s->child->stride;
  }
  out->hash = s->hash;
  return MRN_OK;
}

int mrn_schema_column(const mrn_schema* s, int child, uint32_t c, mrn_column_info* out) {
  if (!s || !s->finalized || !out) return MRN_EINVAL;
  const mrn_schema* t = child ? s->child.get() : s;
  if (!t || c >= t->cols.size()) return MRN_EINVAL;
  std::memset(out, 0, sizeof(*out));
  out->size = t->cols[c].size;
  out->aos_offset = t->cols[c].aos_off;
  out->fm_stride = t->cols[c].es;
  out->dtype = t->cols[c].dtype;
  std::strncpy(out->name, t->cols[c].name.c_str(), sizeof(out->name) - 1);
  return MRN_OK;
}

int mrn_schema_aos_layout(const mrn_schema* s, size_t* stride, size_t* offsets, size_t cap) {
  if (!s || !s->finalized) return MRN_EINVAL;
  if (stride) *stride = s->stride;
  if (offsets)
    for (size_t c = 0; c < s->cols.size() && c < cap; ++c) offsets[c] = s->cols[c].aos_off;
  return MRN_OK;
}

int mrn_required_bytes(const mrn_schema* s, mrn_layout l, uint64_t n, uint64_t m, size_t* out) {
  if (!s || !s->finalized || !out || l.kind < MRN_AOS || l.kind > MRN_AOSOA ||
      (l.kind == MRN_AOSOA && l.block < 1))
    return MRN_EINVAL;
  *out = (size_t)base_bytes(s, l, n, m);
  return MRN_OK;
}

int mrn_required_bytes_nested(const mrn_schema* s, mrn_layout l, uint64_t n, uint64_t m, uint64_t m2,
                              size_t* out) {
  if (!s || !s->finalized || !out || l.kind < MRN_AOS || l.kind > MRN_AOSOA ||
      (l.kind == MRN_AOSOA && l.block < 1))
    return MRN_EINVAL;
  *out = (size_t)base_bytes(s, l, n, m, m2);
  return MRN_OK;
}

int mrn_grandchild_pool_bytes(const mrn_schema* s, uint64_t m2, size_t* out) {
  if (!s || !s->finalized || !is_nested(s) || !out) return MRN_EINVAL;
  *out = (size_t)(m2 * s->child->child->stride);
  return MRN_OK;
}

int mrn_region_offset_nested(const mrn_schema* s, mrn_layout l, uint64_t n, uint64_t m, uint64_t m2, uint32_t r,
                             size_t* out) {
  if (!s || !s->finalized || !out || !s->has_jagged || (l.kind != MRN_SOA && l.kind != MRN_AOSOA) ||
      (l.kind == MRN_AOSOA && l.block < 1))
    return MRN_EINVAL;
  const int kind = l.kind;
  const uint32_t B = l.kind == MRN_AOSOA ? l.block : 0;
  const uint32_t pc = kind == MRN_AOSOA ? 1u : (uint32_t)s->cols.size();  // items before the offsets
  const mrn_schema* ch = s->child.get();
  const uint32_t kc = (uint32_t)ch->cols.size();
  if (r < pc)
    *out = (size_t)(kind == MRN_AOSOA ? 0 : fm_col_start(s, kind, B, n, m, false, r, m2));
  else if (r == pc)
    *out = (size_t)fm_region_start(s, kind, B, n, m, parent_regions(s, kind), m2);
  else if (r - pc - 1 < kc)
    *out = (size_t)fm_col_start(s, kind, B, n, m, true, r - pc - 1, m2);
  else if (is_nested(s) && r - pc - 1 == kc)
    *out = (size_t)fm_child_offsets_start(s, kind, B, n, m, m2);
  else if (is_nested(s) && r - pc - 2 - kc < ch->child->cols.size())
    *out = (size_t)fm_gchild_col_start(s, kind, B, n, m, m2, r - pc - 2 - kc);
  else
    return MRN_EINVAL;
  return MRN_OK;
}

int mrn_child_pool_bytes(const mrn_schema* s, uint64_t m, size_t* out) {
  if (!s || !s->finalized || !s->has_jagged || !out) return MRN_EINVAL;
  *out = (size_t)(m * s->child->stride);
  return MRN_OK;
}

int mrn_soa_region_offset(const mrn_schema* s, uint64_t n, uint64_t m, uint32_t r, size_t* out) {
  if (!s || !s->finalized || !out) return MRN_EINVAL;
  const uint32_t nc = (uint32_t)s->cols.size();
  const uint32_t nk = s->has_jagged ? (uint32_t)s->child->cols.size() : 0;
  if (r < nc)
    *out = (size_t)fm_col_start(s, MRN_SOA, 0, n, m, false, r);
  else if (s->has_jagged && r == nc)
    *out = (size_t)fm_region_start(s, MRN_SOA, 0, n, m, parent_regions(s, MRN_SOA));
  else if (s->has_jagged && r <= nc + nk)
    *out = (size_t)fm_col_start(s, MRN_SOA, 0, n, m, true, r - nc - 1);
  else
    return MRN_EINVAL;
  return MRN_OK;
}

int mrn_region_offset(const mrn_schema* s, mrn_layout l, uint64_t n, uint64_t m, uint32_t r, size_t* out) {
  if (!s || !s->finalized || !out) return MRN_EINVAL;
  if (l.kind == MRN_SOA) return mrn_soa_region_offset(s, n, m, r, out);
  if (l.kind != MRN_AOSOA || l.block < 1 || !s->has_jagged || r >= 2 + s->child->cols.size())
    return MRN_EINVAL;
  *out = (size_t)(r < 2 ? fm_region_start(s, MRN_AOSOA, l.block, n, m, r)
                        : fm_col_start(s, MRN_AOSOA, l.block, n, m, true, r - 2));
  return MRN_OK;
}

int mrn_aosoa_block_bytes(const mrn_schema* s, uint32_t B, size_t* out) {
  if (!s || !s->finalized || !out || B < 1) return MRN_EINVAL;
  *out = (size_t)aosoa_block_bytes(s, B);
  return MRN_OK;
}

int mrn_aosoa_column_offset(const mrn_schema* s, uint32_t B, uint32_t c, size_t* out) {
  if (!s || !s->finalized || !out || B < 1 || c >= s->cols.size()) return MRN_EINVAL;
  *out = (size_t)aosoa_col_start(s, B, c);
  return MRN_OK;
}

}  // extern "C"
