// Library-owned collections and their size-changing operations (Sec. VI-A
// memory contexts and the partially overlapping memcopy; Sec. VI-B layout
// holders: resize, reserve, clear, shrink_to_fit, insert, erase).  The
// overlapping move they are built on runs in k_move.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "mrn_internal.h"

namespace mrn {
namespace {

int cuda_rc(cudaError_t e) {
  if (e == cudaSuccess) return MRN_OK;
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? MRN_ENOMEM : MRN_ECUDA;
}

bool is_host(int mem) { return mem == MRN_MEM_HOST || mem == MRN_MEM_HOST_PINNED; }

// Host work on a collection waits for `st` first (earlier GPU work may
// still read or write the memory); without a GPU there is nothing to wait
// for.
int host_wait(cudaStream_t st) {
  static const int ngpu = [] {
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess) {
      cudaGetLastError();
      n = 0;
    }
    return n;
  }();
  if (ngpu == 0) return MRN_OK;
  return cudaStreamSynchronize(st) == cudaSuccess ? MRN_OK : MRN_ECUDA;
}

template <typename T>
void add_delta(char* p, uint64_t count, long long delta) {
  T* q = reinterpret_cast<T*>(p);
  for (uint64_t i = 0; i < count; ++i) q[i] = (T)(q[i] + (T)delta);
}

int host_moves(const std::vector<MoveRange>& moves, cudaStream_t st) {
  if (host_wait(st)) return MRN_ECUDA;
  for (const MoveRange& m : moves) {
    if (m.bytes == 0) continue;
    if (m.src != m.dst) std::memmove(m.dst, m.src, m.bytes);
    if (m.elem == 8) add_delta<unsigned long long>(m.dst, m.bytes / 8, m.delta);
    if (m.elem == 4) add_delta<unsigned int>(m.dst, m.bytes / 4, m.delta);
  }
  return MRN_OK;
}

int run_moves(int mem, const std::vector<MoveRange>& moves, cudaStream_t st) {
  return is_host(mem) ? host_moves(moves, st) : launch_moves(moves.data(), moves.size(), st);
}

}  // namespace
}  // namespace mrn

extern "C" int mrn_memmove(void* dst, const void* src, uint64_t bytes, int mem, void* stream) {
  using namespace mrn;
  if (bytes == 0) return MRN_OK;
  if (!dst || !src || (mem != MRN_MEM_DEVICE && !is_host(mem))) return MRN_EINVAL;
  std::vector<MoveRange> mv{{static_cast<const char*>(src), static_cast<char*>(dst), bytes, 0u, 0}};
  return run_moves(mem, mv, static_cast<cudaStream_t>(stream));
}

// ------------------------------------------------------------ collections

struct mrn_collection {
  const mrn_schema* s = nullptr;
  mrn_layout layout{};
  int mem = MRN_MEM_DEVICE;
  int device = 0;
  uint64_t n = 0, m = 0, cap = 0, ccap = 0;
  // storage
  char* base = nullptr;  // records / blocks / single block
  char* pool = nullptr;  // AoS jagged: child records
  // derived pointers (views point into these arrays)
  std::vector<void*> cols, kids;
  char* offsets = nullptr;
};

namespace mrn {
namespace {

bool jagged(const mrn_collection* c) { return c->s->has_jagged; }
uint32_t off_size(const mrn_collection* c) { return c->s->off_size; }

// The storage of a collection for given capacities, in a memory context.
struct Storage {
  char* base = nullptr;
  char* pool = nullptr;
  std::vector<void*> cols, kids;
  char* offsets = nullptr;
};

int ctx_alloc(int mem, int device, size_t bytes, char** out) {
  *out = nullptr;
  if (bytes == 0) bytes = 16;
  bytes = (size_t)align_up(bytes, 256);
  if (mem == MRN_MEM_HOST) {
    *out = static_cast<char*>(std::aligned_alloc(256, bytes));
    return *out ? MRN_OK : MRN_ENOMEM;
  }
  int prev = 0;
  cudaGetDevice(&prev);
  if (mem == MRN_MEM_DEVICE && device != prev && cudaSetDevice(device) != cudaSuccess) return MRN_EINVAL;
  void* p = nullptr;
  const cudaError_t e = mem == MRN_MEM_DEVICE ? cudaMalloc(&p, bytes) : cudaHostAlloc(&p, bytes, cudaHostAllocMapped);
  if (mem == MRN_MEM_DEVICE && device != prev) cudaSetDevice(prev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return MRN_ENOMEM;
  }
  *out = static_cast<char*>(p);
  return MRN_OK;
}

void ctx_free(int mem, char* p) {
  if (!p) return;
  if (mem == MRN_MEM_HOST)
    std::free(p);
  else if (mem == MRN_MEM_DEVICE)
    cudaFree(p);
  else
    cudaFreeHost(p);
}

void free_storage(int mem, Storage* st) {
  ctx_free(mem, st->base);
  ctx_free(mem, st->pool);
  *st = Storage{};
}

int make_storage(const mrn_schema* s, const mrn_layout& l, int mem, int device, uint64_t cap, uint64_t ccap,
                 Storage* out) {
  Storage st;
  int rc = ctx_alloc(mem, device, base_bytes(s, l, cap, ccap), &st.base);
  if (rc == MRN_OK && l.kind == MRN_AOS && s->has_jagged)
    rc = ctx_alloc(mem, device, ccap * s->child->stride, &st.pool);
  if (rc) {
    free_storage(mem, &st);
    return rc;
  }
  if (l.kind == MRN_SOA) {
    for (uint32_t c = 0; c < s->cols.size(); ++c)
      st.cols.push_back(st.base + fm_region_start(s, MRN_SOA, 0, cap, ccap, c));
  }
  if (l.kind != MRN_AOS && s->has_jagged) {
    const uint32_t r0 = parent_regions(s, l.kind);
    st.offsets = st.base + fm_region_start(s, l.kind, l.block, cap, ccap, r0);
    for (uint32_t j = 0; j < s->child->cols.size(); ++j)
      st.kids.push_back(st.base + fm_region_start(s, l.kind, l.block, cap, ccap, r0 + 1 + j));
  }
  *out = std::move(st);
  return MRN_OK;
}

Storage storage_of(mrn_collection* c) {
  Storage st;
  st.base = c->base;
  st.pool = c->pool;
  st.cols = c->cols;
  st.kids = c->kids;
  st.offsets = c->offsets;
  return st;
}

void adopt(mrn_collection* c, Storage&& st, uint64_t cap, uint64_t ccap) {
  c->base = st.base;
  c->pool = st.pool;
  c->cols = std::move(st.cols);
  c->kids = std::move(st.kids);
  c->offsets = st.offsets;
  c->cap = cap;
  c->ccap = ccap;
}

uint64_t blocks_of(uint64_t n, uint32_t B) { return (n + B - 1) / B; }

// The regions holding n objects / m children of a storage, as (pointer,
// bytes) pairs in a fixed order, so that two storages of the same schema and
// layout pair up region by region.
std::vector<std::pair<char*, uint64_t>> regions(const mrn_collection* c, const Storage& st, uint64_t n, uint64_t m) {
  const mrn_schema* s = c->s;
  std::vector<std::pair<char*, uint64_t>> r;
  switch (c->layout.kind) {
    case MRN_AOS:
      r.push_back({st.base, n * s->stride});
      if (s->has_jagged) r.push_back({st.pool, m * s->child->stride});
      return r;
    case MRN_SOA:
      for (uint32_t k = 0; k < s->cols.size(); ++k) r.push_back({static_cast<char*>(st.cols[k]), n * s->cols[k].size});
      break;
    default:
      r.push_back({st.base, blocks_of(n, c->layout.block) * aosoa_block_bytes(s, c->layout.block)});
  }
  if (s->has_jagged) {
    r.push_back({st.offsets, (n + 1) * s->off_size});
    for (uint32_t k = 0; k < s->child->cols.size(); ++k)
      r.push_back({static_cast<char*>(st.kids[k]), m * s->child->cols[k].size});
  }
  return r;
}

int copy_kind(int to, int from, cudaMemcpyKind* k) {
  const bool dh = is_host(to), sh = is_host(from);
  *k = dh ? (sh ? cudaMemcpyHostToHost : cudaMemcpyDeviceToHost) : (sh ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice);
  return MRN_OK;
}

// Copies the contents (n objects, m children) of one storage into another of
// the same schema and layout, possibly in another memory context.
int copy_contents(mrn_collection* c, const Storage& to, int to_mem, const Storage& from, int from_mem, cudaStream_t st) {
  const auto a = regions(c, to, c->n, c->m), b = regions(c, from, c->n, c->m);
  if (is_host(to_mem) && is_host(from_mem)) {
    if (host_wait(st)) return MRN_ECUDA;
    for (size_t i = 0; i < a.size(); ++i)
      if (a[i].second) std::memcpy(a[i].first, b[i].first, a[i].second);
    return MRN_OK;
  }
  cudaMemcpyKind kind;
  copy_kind(to_mem, from_mem, &kind);
  for (size_t i = 0; i < a.size(); ++i)
    if (a[i].second) {
      const int rc = cuda_rc(cudaMemcpyAsync(a[i].first, b[i].first, a[i].second, kind, st));
      if (rc) return rc;
    }
  // the old storage is freed right after: host copies must have finished
  if (is_host(from_mem) || is_host(to_mem)) return cuda_rc(cudaStreamSynchronize(st));
  return MRN_OK;
}

int fill_zero(const mrn_collection* c, char* p, uint64_t bytes, cudaStream_t st);

int reallocate(mrn_collection* c, int mem, int device, uint64_t cap, uint64_t ccap, cudaStream_t st) {
  Storage fresh;
  int rc = make_storage(c->s, c->layout, mem, device, cap, ccap, &fresh);
  if (rc) return rc;
  Storage old = storage_of(c);
  if ((rc = copy_contents(c, fresh, mem, old, c->mem, st))) {
    free_storage(mem, &fresh);
    return rc;
  }
  // device storage is freed once the copies out of it are done
  if (!is_host(c->mem) && cudaStreamSynchronize(st) != cudaSuccess) rc = MRN_ECUDA;
  free_storage(c->mem, &old);
  adopt(c, std::move(fresh), cap, ccap);
  c->mem = mem;
  c->device = device;
  // AoSoA: the blocks past the copied ones start zeroed (unused slots)
  if (!rc && c->layout.kind == MRN_AOSOA) {
    const uint32_t B = c->layout.block;
    const uint64_t bb = aosoa_block_bytes(c->s, B), b0 = blocks_of(c->n, B);
    rc = fill_zero(c, c->base + b0 * bb, (blocks_of(cap, B) - b0) * bb, st);
  }
  return rc;
}

int fill_zero(const mrn_collection* c, char* p, uint64_t bytes, cudaStream_t st) {
  if (bytes == 0) return MRN_OK;
  if (is_host(c->mem)) {
    if (host_wait(st)) return MRN_ECUDA;
    std::memset(p, 0, bytes);
    return MRN_OK;
  }
  return cuda_rc(cudaMemsetAsync(p, 0, bytes, st));
}

// offsets[a .. b] = offsets[from]
int fill_offsets(const mrn_collection* c, uint64_t a, uint64_t b, uint64_t from, cudaStream_t st) {
  if (b < a) return MRN_OK;
  const uint32_t os = off_size(c);
  char* dst = c->offsets + a * os;
  const char* src = c->offsets + from * os;
  const uint64_t count = b - a + 1;
  if (is_host(c->mem)) {
    if (host_wait(st)) return MRN_ECUDA;
    for (uint64_t i = 0; i < count; ++i) std::memcpy(dst + i * os, src, os);
    return MRN_OK;
  }
  return launch_fill_from(dst, src, count, os, st);
}

int read_offset(const mrn_collection* c, uint64_t i, uint64_t* out, cudaStream_t st) {
  const uint32_t os = off_size(c);
  unsigned long long v = 0;
  if (is_host(c->mem)) {
    if (host_wait(st)) return MRN_ECUDA;
    std::memcpy(&v, c->offsets + i * os, os);
  } else {
    if (cudaMemcpyAsync(&v, c->offsets + i * os, os, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return MRN_ECUDA;
  }
  *out = v;
  return MRN_OK;
}

// Zeroes the objects [a, b) of the collection (jagged AoS: their records,
// i.e. zero lengths).  AoSoA: whole slots, block by block.
int zero_objects(const mrn_collection* c, uint64_t a, uint64_t b, cudaStream_t st) {
  if (b <= a) return MRN_OK;
  const mrn_schema* s = c->s;
  int rc = MRN_OK;
  switch (c->layout.kind) {
    case MRN_AOS: return fill_zero(c, c->base + a * s->stride, (b - a) * s->stride, st);
    case MRN_SOA:
      for (uint32_t k = 0; k < s->cols.size() && !rc; ++k)
        rc = fill_zero(c, static_cast<char*>(c->cols[k]) + a * s->cols[k].size, (b - a) * s->cols[k].size, st);
      return rc;
    default: {
      const uint32_t B = c->layout.block;
      const uint64_t bb = aosoa_block_bytes(s, B);
      // a partial first block, column by column; then whole blocks
      uint64_t r = a;
      if (r % B) {
        const uint64_t blk = r / B, e = std::min<uint64_t>(b, (blk + 1) * B);
        for (uint32_t k = 0; k < s->cols.size() && !rc; ++k) {
          const uint64_t sz = s->cols[k].size;
          rc = fill_zero(c, c->base + blk * bb + aosoa_col_start(s, B, k) + (r % B) * sz, (e - r) * sz, st);
        }
        r = e;
      }
      if (!rc && r < b) rc = fill_zero(c, c->base + (r / B) * bb, (blocks_of(b, B) - r / B) * bb, st);
      return rc;
    }
  }
}

int check_mem(int mem) {
  return mem == MRN_MEM_DEVICE || mem == MRN_MEM_HOST_PINNED || mem == MRN_MEM_HOST ? MRN_OK : MRN_EINVAL;
}

int grow_to(mrn_collection* c, uint64_t need, uint64_t cneed, cudaStream_t st) {
  if (need <= c->cap && cneed <= c->ccap) return MRN_OK;
  const uint64_t cap = need > c->cap ? std::max(need, 2 * c->cap) : c->cap;
  const uint64_t ccap = cneed > c->ccap ? std::max(cneed, 2 * c->ccap) : c->ccap;
  return reallocate(c, c->mem, c->device, cap, ccap, st);
}

// The view of objects [pos, pos + k) of a (field-major or AoS) collection,
// with `kids` child slots from child index `kid0` (SoA jagged).
mrn_view sub_view(mrn_collection* c, uint64_t pos, uint64_t k, uint64_t kid0, uint64_t kids,
                  std::vector<void*>* colp, std::vector<void*>* kidp) {
  const mrn_schema* s = c->s;
  mrn_view v{};
  v.schema = s;
  v.layout = c->layout;
  v.mem = c->mem;
  v.device = c->device;
  v.n_records = k;
  if (c->layout.kind == MRN_AOS) {
    v.base = c->base + pos * s->stride;
    return v;
  }
  colp->clear();
  for (uint32_t j = 0; j < s->cols.size(); ++j)
    colp->push_back(static_cast<char*>(c->cols[j]) + pos * s->cols[j].size);
  v.base = c->base;
  v.columns = colp->data();
  if (s->has_jagged) {
    kidp->clear();
    for (uint32_t j = 0; j < s->child->cols.size(); ++j)
      kidp->push_back(static_cast<char*>(c->kids[j]) + kid0 * s->child->cols[j].size);
    v.offsets = c->offsets + pos * s->off_size;
    v.child_columns = kidp->data();
    v.n_children = kids;
    v.offset_base = kid0;
  }
  return v;
}

// Region r of a field-major view (parents, offsets, child columns; SoA
// parents are one region per column): its own pointer, else its place in
// the single block.
char* fm_region(const mrn_view& v, uint32_t r) {
  const mrn_schema* s = v.schema;
  const uint32_t P = parent_regions(s, v.layout.kind);
  if (r < P && v.layout.kind == MRN_SOA && v.columns) return static_cast<char*>(v.columns[r]);
  if (r < P && v.layout.kind == MRN_AOSOA) return static_cast<char*>(v.base);
  if (r == P && v.offsets) return static_cast<char*>(v.offsets);
  if (r > P && v.child_columns) return static_cast<char*>(v.child_columns[r - P - 1]);
  return static_cast<char*>(v.base) +
         fm_region_start(s, v.layout.kind, v.layout.block, v.n_records, v.n_children, r);
}

// A jagged source already in the destination's field-major layout (the
// conversions take no equal-layout jagged pair): region by region copies;
// the offsets come over as they are.
int copy_same_fm(const mrn_view& src, const mrn_view& dst, cudaStream_t st) {
  const mrn_schema* s = src.schema;
  if (is_host(src.mem) || is_host(dst.mem)) return MRN_EUNSUPPORTED;
  const uint64_t n = src.n_records, m = src.n_children;
  const uint32_t P = parent_regions(s, src.layout.kind);
  const uint32_t R = fm_region_count(s, src.layout.kind);
  for (uint32_t r = 0; r < R; ++r) {
    uint64_t bytes;
    if (r < P)
      bytes = src.layout.kind == MRN_SOA ? n * s->cols[r].size
                                         : blocks_of(n, src.layout.block) * aosoa_block_bytes(s, src.layout.block);
    else if (r == P)
      bytes = (n + 1) * s->off_size;
    else
      bytes = m * s->child->cols[r - P - 1].size;
    if (bytes == 0) continue;
    const int rc = cuda_rc(cudaMemcpyAsync(fm_region(dst, r), fm_region(src, r), bytes, cudaMemcpyDeviceToDevice, st));
    if (rc) return rc;
  }
  return MRN_OK;
}

// offsets[pos .. pos + k] += first - offsets[pos] (offsets a field-major
// source brought as they were).
int rebase_offsets(mrn_collection* c, uint64_t pos, uint64_t k, uint64_t first, cudaStream_t st) {
  uint64_t s0 = 0;
  int rc = read_offset(c, pos, &s0, st);
  if (rc || s0 == first) return rc;
  const uint32_t os = off_size(c);
  char* p = c->offsets + pos * os;
  std::vector<MoveRange> fix{{p, p, (k + 1) * os, os, (long long)(first - s0)}};
  return run_moves(c->mem, fix, st);
}

// Converts src into dst through whichever entry point takes the pair.
int convert_any(const mrn_view& src, const mrn_view& dst, cudaStream_t st) {
  const bool sh = is_host(src.mem), dh = is_host(dst.mem);
  if (src.schema->has_jagged && src.layout.kind != MRN_AOS && src.layout.kind == dst.layout.kind &&
      (src.layout.kind != MRN_AOSOA || src.layout.block == dst.layout.block))
    return copy_same_fm(src, dst, st);
  if (!sh && !dh) return mrn_convert(&src, &dst, st);
  if (sh != dh) return mrn_transfer_convert(&src, &dst, nullptr, st);
  return MRN_EUNSUPPORTED;
}

// Children a source view brings (jagged schemas).
int source_children(const mrn_view& src, uint64_t* m, cudaStream_t st) {
  *m = 0;
  if (!src.schema->has_jagged) return MRN_OK;
  if (src.layout.kind != MRN_AOS) {
    *m = src.n_children;
    return MRN_OK;
  }
  if (is_host(src.mem)) return MRN_EUNSUPPORTED;
  int rc = mrn_jagged_count(&src, m, st);
  if (rc == MRN_OK) rc = mrn_sync(st);
  return rc;
}

}  // namespace
}  // namespace mrn

using namespace mrn;

extern "C" {

int mrn_collection_create(const mrn_schema* s, mrn_layout layout, int mem, int device, uint64_t capacity,
                          uint64_t child_capacity, mrn_collection** out) {
  if (!out) return MRN_EINVAL;
  *out = nullptr;
  if (!s || !s->finalized || check_mem(mem)) return MRN_EINVAL;
  if (layout.kind != MRN_AOS && layout.kind != MRN_SOA && layout.kind != MRN_AOSOA) return MRN_EINVAL;
  if (layout.kind == MRN_AOSOA && layout.block == 0) return MRN_EINVAL;
  if (s->interleaved || is_nested(s)) return MRN_EUNSUPPORTED;  // storage moves are per stored column
  mrn_collection* c = new (std::nothrow) mrn_collection;
  if (!c) return MRN_ENOMEM;
  c->s = s;
  c->layout = layout;
  if (layout.kind != MRN_AOSOA) c->layout.block = 0;
  c->mem = mem;
  c->device = device;
  Storage st;
  int rc = make_storage(s, c->layout, mem, device, capacity, s->has_jagged ? child_capacity : 0, &st);
  if (rc) {
    delete c;
    return rc;
  }
  adopt(c, std::move(st), capacity, s->has_jagged ? child_capacity : 0);
  // offsets[0] = 0; AoSoA blocks start zeroed (unused slots stay zero)
  if (jagged(c) && c->layout.kind != MRN_AOS) rc = fill_zero(c, c->offsets, off_size(c), nullptr);
  if (!rc && c->layout.kind == MRN_AOSOA)
    rc = fill_zero(c, c->base, blocks_of(capacity, c->layout.block) * aosoa_block_bytes(s, c->layout.block), nullptr);
  if (!rc && !is_host(mem)) rc = cuda_rc(cudaStreamSynchronize(nullptr));
  if (rc) {
    mrn_collection_destroy(c);
    return rc;
  }
  *out = c;
  return MRN_OK;
}

void mrn_collection_destroy(mrn_collection* c) {
  if (!c) return;
  Storage st = storage_of(c);
  if (!is_host(c->mem)) cudaDeviceSynchronize();
  free_storage(c->mem, &st);
  delete c;
}

int mrn_collection_view(const mrn_collection* c, mrn_view* out) {
  if (!c || !out) return MRN_EINVAL;
  mrn_view v{};
  v.schema = c->s;
  v.layout = c->layout;
  v.mem = c->mem;
  v.device = c->device;
  v.n_records = c->n;
  v.base = c->base;
  if (c->layout.kind == MRN_SOA) v.columns = c->cols.data();
  if (jagged(c)) {
    v.n_children = c->m;
    if (c->layout.kind == MRN_AOS) {
      v.child_pool = c->pool;
    } else {
      v.offsets = c->offsets;
      v.child_columns = c->kids.data();
    }
  }
  *out = v;
  return MRN_OK;
}

int mrn_collection_sizes(const mrn_collection* c, uint64_t* n, uint64_t* m, uint64_t* capacity,
                         uint64_t* child_capacity) {
  if (!c) return MRN_EINVAL;
  if (n) *n = c->n;
  if (m) *m = c->m;
  if (capacity) *capacity = c->cap;
  if (child_capacity) *child_capacity = c->ccap;
  return MRN_OK;
}

int mrn_collection_reserve(mrn_collection* c, uint64_t capacity, uint64_t child_capacity, void* stream) {
  if (!c) return MRN_EINVAL;
  if (!jagged(c)) child_capacity = 0;
  const uint64_t cap = std::max(capacity, c->cap), ccap = std::max(child_capacity, c->ccap);
  if (cap == c->cap && ccap == c->ccap) return MRN_OK;
  return reallocate(c, c->mem, c->device, cap, ccap, static_cast<cudaStream_t>(stream));
}

int mrn_collection_resize(mrn_collection* c, uint64_t n, void* stream) {
  if (!c) return MRN_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int rc = MRN_OK;
  if (n > c->n) {
    if ((rc = grow_to(c, n, c->m, st))) return rc;
    if (c->layout.kind == MRN_AOSOA) {
      // slots past n in the last block are already zero; later blocks too
      // (created or reserved zeroed, and zeroed again on shrinking)
    } else if ((rc = zero_objects(c, c->n, n, st))) {
      return rc;
    }
    if (jagged(c) && c->layout.kind != MRN_AOS && (rc = fill_offsets(c, c->n + 1, n, c->n, st))) return rc;
  } else if (n < c->n) {
    if (c->layout.kind == MRN_AOSOA && (rc = zero_objects(c, n, c->n, st))) return rc;
    if (jagged(c) && c->layout.kind != MRN_AOS) {
      uint64_t mn = 0;
      if ((rc = read_offset(c, n, &mn, st))) return rc;
      c->m = mn;
    }
  }
  c->n = n;
  return MRN_OK;
}

int mrn_collection_clear(mrn_collection* c, void* stream) { return mrn_collection_resize(c, 0, stream); }

int mrn_collection_shrink_to_fit(mrn_collection* c, void* stream) {
  if (!c) return MRN_EINVAL;
  if (c->cap == c->n && c->ccap == c->m) return MRN_OK;
  return reallocate(c, c->mem, c->device, c->n, c->m, static_cast<cudaStream_t>(stream));
}

int mrn_collection_erase(mrn_collection* c, uint64_t first, uint64_t count, void* stream) {
  if (!c) return MRN_EINVAL;
  if (first > c->n || count > c->n - first) return MRN_EINVAL;
  if (count == 0) return MRN_OK;
  if (c->layout.kind == MRN_AOSOA) return MRN_EUNSUPPORTED;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const mrn_schema* s = c->s;
  const uint64_t tail = c->n - first - count;
  std::vector<MoveRange> mv;
  uint64_t removed = 0;
  if (c->layout.kind == MRN_AOS) {
    mv.push_back({c->base + (first + count) * s->stride, c->base + first * s->stride, tail * s->stride, 0u, 0});
  } else {
    for (uint32_t k = 0; k < s->cols.size(); ++k) {
      char* col = static_cast<char*>(c->cols[k]);
      const uint64_t sz = s->cols[k].size;
      mv.push_back({col + (first + count) * sz, col + first * sz, tail * sz, 0u, 0});
    }
    if (jagged(c)) {
      uint64_t a = 0, b = 0;
      int rc = read_offset(c, first, &a, st);
      if (!rc) rc = read_offset(c, first + count, &b, st);
      if (rc) return rc;
      removed = b - a;
      const uint32_t os = off_size(c);
      mv.push_back({c->offsets + (first + count) * os, c->offsets + first * os, (tail + 1) * os, os,
                    -(long long)removed});
      for (uint32_t k = 0; k < s->child->cols.size(); ++k) {
        char* col = static_cast<char*>(c->kids[k]);
        const uint64_t sz = s->child->cols[k].size;
        mv.push_back({col + b * sz, col + a * sz, (c->m - b) * sz, 0u, 0});
      }
    }
  }
  const int rc = run_moves(c->mem, mv, st);
  if (rc) return rc;
  c->n -= count;
  if (c->layout.kind != MRN_AOS) c->m -= removed;
  return MRN_OK;
}

int mrn_collection_insert(mrn_collection* c, uint64_t pos, const mrn_view* src, void* stream) {
  if (!c || !src || src->schema != c->s) return MRN_EINVAL;
  if (pos > c->n) return MRN_EINVAL;
  if (c->layout.kind == MRN_AOSOA || (c->layout.kind == MRN_AOS && jagged(c))) return MRN_EUNSUPPORTED;
  const uint64_t k = src->n_records;
  if (k == 0) return MRN_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const mrn_schema* s = c->s;
  uint64_t km = 0;
  int rc = source_children(*src, &km, st);
  if (rc) return rc;
  if ((rc = grow_to(c, c->n + k, c->m + km, st))) return rc;
  const uint64_t tail = c->n - pos;
  uint64_t a = 0;
  std::vector<MoveRange> mv;
  if (c->layout.kind == MRN_AOS) {
    mv.push_back({c->base + pos * s->stride, c->base + (pos + k) * s->stride, tail * s->stride, 0u, 0});
  } else {
    for (uint32_t j = 0; j < s->cols.size(); ++j) {
      char* col = static_cast<char*>(c->cols[j]);
      const uint64_t sz = s->cols[j].size;
      mv.push_back({col + pos * sz, col + (pos + k) * sz, tail * sz, 0u, 0});
    }
    if (jagged(c)) {
      if ((rc = read_offset(c, pos, &a, st))) return rc;
      const uint32_t os = off_size(c);
      // offsets[pos .. n] move up by k and grow by km (offsets[pos] is
      // rewritten by the conversion below with the same value)
      mv.push_back({c->offsets + pos * os, c->offsets + (pos + k) * os, (tail + 1) * os, os, (long long)km});
      for (uint32_t j = 0; j < s->child->cols.size(); ++j) {
        char* col = static_cast<char*>(c->kids[j]);
        const uint64_t sz = s->child->cols[j].size;
        mv.push_back({col + a * sz, col + (a + km) * sz, (c->m - a) * sz, 0u, 0});
      }
    }
  }
  if ((rc = run_moves(c->mem, mv, st))) return rc;
  std::vector<void*> colp, kidp;
  const mrn_view gap = sub_view(c, pos, k, a, km, &colp, &kidp);
  if ((rc = convert_any(*src, gap, st))) return rc;
  // a field-major jagged source brings its own offsets: rebase them
  if (jagged(c) && src->layout.kind != MRN_AOS && (rc = rebase_offsets(c, pos, k, a, st))) return rc;
  if (!is_host(c->mem) && (rc = mrn_sync(st))) return rc;
  c->n += k;
  if (c->layout.kind != MRN_AOS) c->m += km;
  return MRN_OK;
}

int mrn_collection_assign(mrn_collection* c, const mrn_view* src, void* stream) {
  if (!c || !src || src->schema != c->s) return MRN_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  uint64_t km = 0;
  int rc = source_children(*src, &km, st);
  if (rc) return rc;
  if ((rc = mrn_collection_clear(c, stream))) return rc;
  if ((rc = grow_to(c, src->n_records, km, st))) return rc;
  mrn_view dst{};
  mrn_collection_view(c, &dst);
  dst.n_records = src->n_records;
  if (jagged(c)) dst.n_children = c->layout.kind == MRN_AOS ? c->ccap : km;
  if ((rc = convert_any(*src, dst, st))) return rc;
  if (jagged(c) && c->layout.kind != MRN_AOS && src->layout.kind != MRN_AOS &&
      (rc = rebase_offsets(c, 0, src->n_records, 0, st)))
    return rc;
  if (!is_host(c->mem) && (rc = mrn_sync(st))) return rc;
  c->n = src->n_records;
  c->m = km;
  return MRN_OK;
}

int mrn_collection_set_context(mrn_collection* c, int mem, int device, void* stream) {
  if (!c || check_mem(mem)) return MRN_EINVAL;
  if (mem == c->mem && (mem != MRN_MEM_DEVICE || device == c->device)) return MRN_OK;
  return reallocate(c, mem, device, c->cap, c->ccap, static_cast<cudaStream_t>(stream));
}

}  // extern "C"
