// Transfer-and-convert between host and device views (the analogue of a
// copy between collections in different memory contexts, Sec. VI-A/VI-B):
// the source is cut into chunks of whole records; chunk k is copied with
// cudaMemcpyAsync on a copy stream into staging slot k % S and converted on
// a compute stream, so copies and conversions of different chunks overlap.
#include "mrn_transfer.h"

#include <algorithm>
#include <cstring>
#include <new>
#include <numeric>

namespace mrn {

namespace {

constexpr uint64_t kPartAlign = 256;

bool is_host(const mrn_view& v) { return v.mem == MRN_MEM_HOST || v.mem == MRN_MEM_HOST_PINNED; }

bool same_layout(const mrn_view& a, const mrn_view& b) {
  return a.layout.kind == b.layout.kind &&
         (a.layout.kind != MRN_AOSOA || a.layout.block == b.layout.block);
}

char* fm_part(const mrn_view& v, uint32_t region, void* const* cols, uint32_t idx) {
  if (cols) return static_cast<char*>(cols[idx]);
  return static_cast<char*>(v.base) +
         fm_region_start(v.schema, v.layout.kind, v.layout.block, v.n_records, v.n_children, region);
}

uint64_t gcd64(uint64_t a, uint64_t b) {
  while (b) {
    const uint64_t t = a % b;
    a = b;
    b = t;
  }
  return a;
}

uint64_t lcm64(uint64_t a, uint64_t b) { return a / gcd64(a, b) * b; }

}  // namespace

// A device view with the same structure as `like`, its parts packed into
// `stage` (each part 256-byte aligned).  Returns the bytes used.
uint64_t staged_view(const mrn_view& like, char* stage, mrn_view* out, std::vector<void*>& cols,
                     std::vector<void*>& ccols) {
  const mrn_schema* s = like.schema;
  *out = like;
  out->mem = MRN_MEM_DEVICE;
  int dev = 0;
  cudaGetDevice(&dev);
  out->device = dev;
  out->offset_base = like.offset_base;
  uint64_t pos = 0;
  auto take = [&](uint64_t bytes) {
    char* p = stage ? stage + pos : nullptr;
    pos += align_up(std::max<uint64_t>(bytes, 1), kPartAlign);
    return p;
  };
  const uint64_t n = like.n_records, m = like.n_children;
  out->columns = nullptr;
  out->child_columns = nullptr;
  out->offsets = nullptr;
  out->child_pool = nullptr;
  if (like.layout.kind == MRN_AOS) {
    out->base = take(n * s->stride);
    if (s->has_jagged) out->child_pool = take(m * s->child->stride);
  } else {
    if (like.layout.kind == MRN_AOSOA) {
      out->base = take((n + like.layout.block - 1) / like.layout.block * aosoa_block_bytes(s, like.layout.block));
    } else {
      cols.assign(s->cols.size(), nullptr);
      for (size_t c = 0; c < s->cols.size(); ++c) cols[c] = take(n * s->cols[c].size);
      out->columns = cols.data();
      out->base = cols.empty() ? nullptr : cols[0];
    }
    if (s->has_jagged) {
      out->offsets = take((n + 1) * s->off_size);
      ccols.assign(s->child->cols.size(), nullptr);
      for (size_t c = 0; c < s->child->cols.size(); ++c) ccols[c] = take(m * s->child->cols[c].size);
      out->child_columns = ccols.data();
    }
  }
  return pos;
}

namespace {

int copy_parts(const std::vector<ViewPart>& from, const std::vector<ViewPart>& to, cudaMemcpyKind kind,
               cudaStream_t s) {
  if (from.size() != to.size()) return MRN_EINVAL;
  for (size_t i = 0; i < from.size(); ++i) {
    const uint64_t b = std::min(from[i].bytes, to[i].bytes);
    if (!b) continue;
    if (!from[i].ptr || !to[i].ptr) return MRN_EINVAL;
    if (cudaMemcpyAsync(to[i].ptr, from[i].ptr, b, kind, s) != cudaSuccess) return MRN_ECUDA;
  }
  return MRN_OK;
}

}  // namespace

std::vector<ViewPart> view_parts(const mrn_view& v) {
  const mrn_schema* s = v.schema;
  const uint64_t n = v.n_records, m = v.n_children;
  std::vector<ViewPart> out;
  if (v.layout.kind == MRN_AOS) {
    out.push_back({static_cast<char*>(v.base), n * s->stride});
    if (s->has_jagged) out.push_back({static_cast<char*>(v.child_pool), m * s->child->stride});
  } else {
    uint32_t P;
    if (v.layout.kind == MRN_AOSOA) {
      const uint64_t B = v.layout.block;
      out.push_back({static_cast<char*>(v.base), (n + B - 1) / B * aosoa_block_bytes(s, (uint32_t)B)});
      P = 1;
    } else {
      P = (uint32_t)s->cols.size();
      for (uint32_t c = 0; c < P; ++c) out.push_back({fm_part(v, c, v.columns, c), n * s->cols[c].size});
    }
    if (s->has_jagged) {
      char* offs = v.offsets ? static_cast<char*>(v.offsets) : fm_part(v, P, nullptr, 0);
      out.push_back({offs, (n + 1) * s->off_size});
      for (uint32_t c = 0; c < s->child->cols.size(); ++c)
        out.push_back({fm_part(v, P + 1 + c, v.child_columns, c), m * s->child->cols[c].size});
    }
  }
  return out;
}

mrn_view sub_view(const mrn_view& v, uint64_t r0, uint64_t cnt, std::vector<void*>& cols) {
  const mrn_schema* s = v.schema;
  mrn_view o = v;
  o.n_records = cnt;
  if (v.layout.kind == MRN_AOS) {
    o.base = static_cast<char*>(v.base) + r0 * s->stride;
  } else if (v.layout.kind == MRN_AOSOA) {
    o.base = static_cast<char*>(v.base) + r0 / v.layout.block * aosoa_block_bytes(s, v.layout.block);
  } else {
    cols.assign(s->cols.size(), nullptr);
    for (uint32_t c = 0; c < s->cols.size(); ++c)
      cols[c] = fm_part(v, c, v.columns, c) + r0 * s->cols[c].size;
    o.columns = cols.data();
    o.base = cols.empty() ? nullptr : cols[0];
  }
  return o;
}

uint64_t record_bytes(const mrn_schema* s, const mrn_layout& l) {
  if (l.kind == MRN_AOS) return s->stride;
  if (l.kind == MRN_AOSOA) return (aosoa_block_bytes(s, l.block) + l.block - 1) / l.block;
  uint64_t b = 0;
  for (const auto& c : s->cols) b += c.size;
  return b;
}

TransferEngine::~TransferEngine() {
  if (!ready_) return;
  cudaStreamSynchronize(s_copy_);
  cudaStreamSynchronize(s_conv_);
  for (auto e : ev_copied_) cudaEventDestroy(e);
  for (auto e : ev_free_) cudaEventDestroy(e);
  cudaEventDestroy(ev_start_);
  cudaEventDestroy(ev_copy_done_);
  cudaEventDestroy(ev_done_);
  for (int h = 0; h < 2; ++h) {
    cudaEventDestroy(ev_whole_free_[h]);
    if (whole_[h]) cudaFree(whole_[h]);
  }
  cudaStreamDestroy(s_copy_);
  cudaStreamDestroy(s_conv_);
  if (staging_) cudaFree(staging_);
}

int TransferEngine::init() {
  if (ready_) return MRN_OK;
  if (cudaStreamCreateWithFlags(&s_copy_, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s_conv_, cudaStreamNonBlocking) != cudaSuccess)
    return MRN_ECUDA;
  const unsigned fl = cudaEventDisableTiming;
  ev_copied_.resize(16);
  ev_free_.resize(16);
  for (int i = 0; i < 16; ++i)
    if (cudaEventCreateWithFlags(&ev_copied_[i], fl) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev_free_[i], fl) != cudaSuccess)
      return MRN_ECUDA;
  if (cudaEventCreateWithFlags(&ev_start_, fl) != cudaSuccess ||
      cudaEventCreateWithFlags(&ev_copy_done_, fl) != cudaSuccess ||
      cudaEventCreateWithFlags(&ev_done_, fl) != cudaSuccess ||
      cudaEventCreateWithFlags(&ev_whole_free_[0], fl) != cudaSuccess ||
      cudaEventCreateWithFlags(&ev_whole_free_[1], fl) != cudaSuccess)
    return MRN_ECUDA;
  ready_ = true;
  return MRN_OK;
}

int TransferEngine::ensure_staging(uint64_t bytes) {
  if (bytes <= staging_bytes_) return MRN_OK;
  cudaStreamSynchronize(s_copy_);
  cudaStreamSynchronize(s_conv_);
  if (staging_) cudaFree(staging_);
  staging_ = nullptr;
  staging_bytes_ = 0;
  if (cudaMalloc(&staging_, bytes) != cudaSuccess) {
    staging_ = nullptr;
    cudaGetLastError();
    return MRN_ENOMEM;
  }
  staging_bytes_ = bytes;
  return MRN_OK;
}

int TransferEngine::ensure_whole(int h, uint64_t bytes) {
  if (bytes <= whole_bytes_[h]) return MRN_OK;
  cudaStreamSynchronize(s_copy_);
  cudaStreamSynchronize(s_conv_);
  if (whole_[h]) cudaFree(whole_[h]);
  whole_[h] = nullptr;
  whole_bytes_[h] = 0;
  if (cudaMalloc(&whole_[h], bytes) != cudaSuccess) {
    whole_[h] = nullptr;
    cudaGetLastError();
    return MRN_ENOMEM;
  }
  whole_bytes_[h] = bytes;
  return MRN_OK;
}

namespace {
// Records per chunk and staging bytes per slot.
void chunk_geometry(const mrn_view& src, const mrn_view& dst, uint64_t chunk_bytes, uint64_t* R,
                    uint64_t* slot_bytes) {
  const bool h2d = src.mem != MRN_MEM_DEVICE;
  const mrn_view& hv = h2d ? src : dst;  // host-side layout is the staged one
  uint64_t q = 32;
  if (src.layout.kind == MRN_AOSOA) q = lcm64(q, src.layout.block);
  if (dst.layout.kind == MRN_AOSOA) q = lcm64(q, dst.layout.block);
  const uint64_t rb = std::max<uint64_t>(1, record_bytes(hv.schema, hv.layout));
  uint64_t r = std::max<uint64_t>(1, chunk_bytes / rb);
  r = std::max<uint64_t>(q, r / q * q);
  r = std::min<uint64_t>(r, std::max<uint64_t>(q, (src.n_records + q - 1) / q * q));
  *R = r;
  mrn_view like = hv;
  like.n_records = r;
  mrn_view tmp;
  std::vector<void*> a, b;
  *slot_bytes = staged_view(like, nullptr, &tmp, a, b);
}
}  // namespace

uint64_t slot_stride(uint64_t chunk_bytes, uint64_t slot_bytes) {
  // a chunk's staged view exceeds chunk_bytes by at most one staging
  // granule of records and its regions' 128-byte alignment
  const uint64_t base = align_up(chunk_bytes, 4096) + (64ull << 10);
  return slot_bytes <= base ? base : align_up(slot_bytes, 4096);
}

uint64_t TransferEngine::staging_bytes(const mrn_view& src, const mrn_view& dst, uint64_t chunk_bytes,
                                       int n_slots) {
  const bool whole = src.schema->has_jagged;
  if (same_layout(src, dst)) return 0;
  if (whole) {
    const mrn_view& hv = src.mem != MRN_MEM_DEVICE ? src : dst;
    mrn_view like = hv, tmp;
    if (src.mem == MRN_MEM_DEVICE) like.n_children = src.n_children;
    std::vector<void*> a, b;
    return staged_view(like, nullptr, &tmp, a, b);
  }
  uint64_t R, slot;
  const uint64_t cb = chunk_bytes ? chunk_bytes : (4ull << 20);
  chunk_geometry(src, dst, cb, &R, &slot);
  return slot_stride(cb, slot) * (uint64_t)std::max(1, std::min(16, n_slots ? n_slots : 4));
}

namespace {
// Zeroes the alignment holes of a host single-block field-major destination
// (the bytes between and after its regions), on the calling thread.
void zero_host_soa_gaps(const mrn_view& dst) {
  const bool fm = dst.layout.kind == MRN_SOA || (dst.layout.kind == MRN_AOSOA && dst.schema->has_jagged);
  if (!fm || !fm_single_block(dst)) return;
  char* base = static_cast<char*>(dst.base);
  uint64_t prev = 0;
  for (const auto& p : view_parts(dst)) {
    const uint64_t st = p.ptr - base;
    if (st > prev) std::memset(base + prev, 0, st - prev);
    prev = st + p.bytes;
  }
  const uint64_t total = base_bytes(dst.schema, dst.layout, dst.n_records, dst.n_children);
  if (total > prev) std::memset(base + prev, 0, total - prev);
}
}  // namespace

int TransferEngine::run(const mrn_view& src, const mrn_view& dst, uint64_t chunk_bytes, int n_slots,
                        cudaStream_t user, char* arena, uint64_t arena_bytes) {
  int rc = init();
  if (rc) return rc;
  if (!chunk_bytes) chunk_bytes = 4ull << 20;
  n_slots = std::max(1, std::min(16, n_slots ? n_slots : 4));
  const bool equal = same_layout(src, dst);
  const bool chunked = !equal && !src.schema->has_jagged;
  // a whole source staged in one of the engine's two whole buffers
  const bool whole_own = !equal && !chunked && !arena;
  const uint64_t need = equal ? 0 : staging_bytes(src, dst, chunk_bytes, n_slots);
  char* stage = arena;
  int whole_h = -1;
  if (whole_own) {
    whole_h = next_whole_;
    if ((rc = ensure_whole(whole_h, need))) return rc;
    next_whole_ ^= 1;
    stage = whole_[whole_h];
  } else if (!equal) {
    if (!stage) {
      if ((rc = ensure_staging(need))) return rc;
      stage = staging_;
    } else if (arena_bytes < need) {
      return MRN_ENOMEM;
    }
  }
  uint64_t R = 0, slot_bytes = 0, stride = 0;
  if (chunked) {
    chunk_geometry(src, dst, chunk_bytes, &R, &slot_bytes);
    stride = slot_stride(chunk_bytes, slot_bytes);
  }
  // The staging memory and both internal streams are shared by every call
  // of this engine, whatever stream it came from.  A chunked call that
  // takes the same slots as the previous chunked call waits for each slot
  // it reuses (the slot events); a call that stages a whole source in one
  // of the engine's two whole buffers waits until that buffer is free.
  // Any other call (equal layouts, whose copies write the destination
  // directly, included) starts only after the previous call's copies and
  // conversions have all finished (ev_done_ is recorded once both streams
  // have joined).  Destinations are therefore written in call order:
  // conversions run in order on s_conv_ and copies to the host in order on
  // s_copy_.  Either way a call starts after the caller's earlier work, and
  // its own chunks overlap each other.
  const bool reuse = chunked && stage == pipe_stage_ && stride == pipe_stride_ && n_slots == pipe_slots_;
  if (whole_own) {
    if (cudaStreamWaitEvent(s_copy_, ev_whole_free_[whole_h], 0) != cudaSuccess ||
        cudaStreamWaitEvent(s_conv_, ev_whole_free_[whole_h], 0) != cudaSuccess)
      return MRN_ECUDA;
  } else if (!reuse) {
    if (cudaStreamWaitEvent(s_copy_, ev_done_, 0) != cudaSuccess ||
        cudaStreamWaitEvent(s_conv_, ev_done_, 0) != cudaSuccess)
      return MRN_ECUDA;
    next_slot_ = 0;
  }
  if (chunked) {
    pipe_stage_ = stage;
    pipe_stride_ = stride;
    pipe_slots_ = n_slots;
  } else if (!whole_own) {  // an arena's whole source or equal layouts: the slots start over
    pipe_stage_ = nullptr;
    pipe_slots_ = 0;
  }
  if (cudaEventRecord(ev_start_, user) != cudaSuccess) return MRN_ECUDA;
  cudaStreamWaitEvent(s_copy_, ev_start_, 0);
  cudaStreamWaitEvent(s_conv_, ev_start_, 0);
  const bool h2d = is_host(src);
  const cudaMemcpyKind kind = h2d ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost;
  // Every destination byte that no property writes is zero: the holes of a
  // single-block SoA destination are cleared here (host) or after the
  // copies (device).
  if (!h2d) zero_host_soa_gaps(dst);
  if (same_layout(src, dst)) {
    // Equal layouts: the storage is copied part by part.
    rc = copy_parts(view_parts(src), view_parts(dst), kind, s_copy_);
    if (!rc && h2d) rc = zero_dst_gaps(dst, s_copy_);
  } else {
    rc = src.schema->has_jagged ? run_whole(src, dst, user, stage, need)
                                : run_chunked(src, dst, R, stride, n_slots, stage);
    // the whole buffer is free once the stream that reads it last is past
    // this call (host -> device: the conversion; device -> host: the copy)
    if (whole_own && cudaEventRecord(ev_whole_free_[whole_h], is_host(src) ? s_conv_ : s_copy_) != cudaSuccess &&
        !rc)
      rc = MRN_ECUDA;
  }
  // Every return path after ev_start_ joins the two streams and orders the
  // caller's stream after them, so that work already queued by a call that
  // fails part way is finished before the caller's next work (and before a
  // caller that syncs its own stream frees the buffers).
  int jrc = MRN_OK;
  if (cudaEventRecord(ev_copy_done_, s_copy_) != cudaSuccess ||
      cudaStreamWaitEvent(s_conv_, ev_copy_done_, 0) != cudaSuccess ||
      cudaEventRecord(ev_done_, s_conv_) != cudaSuccess || cudaStreamWaitEvent(user, ev_done_, 0) != cudaSuccess)
    jrc = MRN_ECUDA;
  return rc ? rc : jrc;
}

int TransferEngine::run_whole(const mrn_view& src, const mrn_view& dst, cudaStream_t, char* stage,
                              uint64_t) {
  const bool h2d = is_host(src);
  std::vector<void*> a, b;
  mrn_view staged;
  int rc;
  if (h2d) {
    staged_view(src, stage, &staged, a, b);
    if ((rc = copy_parts(view_parts(src), view_parts(staged), cudaMemcpyHostToDevice, s_copy_))) return rc;
    cudaEventRecord(ev_copied_[0], s_copy_);
    cudaStreamWaitEvent(s_conv_, ev_copied_[0], 0);
    return mrn_convert(&staged, &dst, s_conv_);
  }
  mrn_view like = dst;
  like.n_children = dst.layout.kind == MRN_AOS ? src.n_children : dst.n_children;
  staged_view(like, stage, &staged, a, b);
  if ((rc = mrn_convert(&src, &staged, s_conv_))) return rc;
  cudaEventRecord(ev_copied_[0], s_conv_);
  cudaStreamWaitEvent(s_copy_, ev_copied_[0], 0);
  auto from = view_parts(staged), to = view_parts(dst);
  return copy_parts(from, to, cudaMemcpyDeviceToHost, s_copy_);
}

int TransferEngine::run_chunked(const mrn_view& src, const mrn_view& dst, uint64_t R, uint64_t slot_bytes,
                                int n_slots, char* stage) {
  const bool h2d = is_host(src);
  const mrn_view& hv = h2d ? src : dst;
  const mrn_view& dv = h2d ? dst : src;
  const uint64_t n = src.n_records;
  int rc;
  std::vector<void*> hc, dc, sc, sc2;
  for (uint64_t r0 = 0; r0 < n; r0 += R) {
    const uint64_t cnt = std::min(R, n - r0);
    const int slot = next_slot_;
    next_slot_ = (next_slot_ + 1) % n_slots;
    mrn_view hsub = sub_view(hv, r0, cnt, hc);
    mrn_view dsub = sub_view(dv, r0, cnt, dc);
    mrn_view like = hv;
    like.n_records = cnt;
    mrn_view staged;
    staged_view(like, stage + (uint64_t)slot * slot_bytes, &staged, sc, sc2);
    if (h2d) {
      cudaStreamWaitEvent(s_copy_, ev_free_[slot], 0);
      if ((rc = copy_parts(view_parts(hsub), view_parts(staged), cudaMemcpyHostToDevice, s_copy_))) return rc;
      cudaEventRecord(ev_copied_[slot], s_copy_);
      cudaStreamWaitEvent(s_conv_, ev_copied_[slot], 0);
      if ((rc = mrn_convert(&staged, &dsub, s_conv_))) return rc;
      cudaEventRecord(ev_free_[slot], s_conv_);
    } else {
      cudaStreamWaitEvent(s_conv_, ev_free_[slot], 0);
      if ((rc = mrn_convert(&dsub, &staged, s_conv_))) return rc;
      cudaEventRecord(ev_copied_[slot], s_conv_);
      cudaStreamWaitEvent(s_copy_, ev_copied_[slot], 0);
      if ((rc = copy_parts(view_parts(staged), view_parts(hsub), cudaMemcpyDeviceToHost, s_copy_))) return rc;
      cudaEventRecord(ev_free_[slot], s_copy_);
    }
  }
  // Device single-block SoA destination: zero its alignment holes once.
  if (h2d) return zero_dst_gaps(dst, s_conv_);
  return MRN_OK;
}

namespace {
// The same view with its host buffers replaced by their mapped device
// addresses (pinned memory the driver maps into the device's address
// space); `cols` holds the mapped SoA column pointers.
int map_host_view(const mrn_view& v, int dev, mrn_view* out, std::vector<void*>* cols) {
  auto map = [](void* h, void** d) -> int {
    if (!h) {
      *d = nullptr;
      return MRN_OK;
    }
    if (cudaHostGetDevicePointer(d, h, 0) != cudaSuccess) {
      cudaGetLastError();
      return MRN_EUNSUPPORTED;
    }
    return MRN_OK;
  };
  *out = v;
  out->mem = MRN_MEM_DEVICE;
  out->device = dev;
  int rc = map(v.base, &out->base);
  if (rc) return rc;
  if (v.columns) {
    const size_t nc = v.schema->cols.size();
    cols->assign(nc, nullptr);
    for (size_t c = 0; c < nc; ++c)
      if ((rc = map(v.columns[c], &(*cols)[c]))) return rc;
    out->columns = cols->data();
  }
  return MRN_OK;
}

// The default pipelines: one per device and direction, so that a
// host -> device and a device -> host transfer (issued on different
// streams) use both directions of the host link at once.
constexpr int kMaxDevices = 64;
std::mutex g_engine_mu[kMaxDevices][2];
TransferEngine* g_engine[kMaxDevices][2];
}  // namespace

}  // namespace mrn

using namespace mrn;

extern "C" int mrn_transfer_convert(const mrn_view* src, const mrn_view* dst, const mrn_transfer_opts* opts,
                                    void* stream) {
  bool jag = false;
  int rc = validate_pair(src, dst, false, &jag);
  if (rc) return rc;
  // staging and the chunk views keep each field-major column separate
  if (src->schema->interleaved || is_nested(src->schema)) return MRN_EUNSUPPORTED;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return MRN_ECUDA;
  const bool h2d = is_host(*src) && dst->mem == MRN_MEM_DEVICE && dst->device == dev;
  const bool d2h = src->mem == MRN_MEM_DEVICE && src->device == dev && is_host(*dst);
  if (!h2d && !d2h) return MRN_EINVAL;
  if (jag && dst->layout.kind == MRN_AOS && dst->n_children < src->n_children) return MRN_ESIZE;
  if (opts && (opts->flags & MRN_TRANSFER_ZERO_COPY)) {
    if (jag) return MRN_EUNSUPPORTED;
    const mrn_view& hv = h2d ? *src : *dst;
    if (hv.mem != MRN_MEM_HOST_PINNED) return MRN_EINVAL;
    if (same_layout(*src, *dst) || (src->layout.kind == MRN_AOS && dst->layout.kind == MRN_AOS))
      return MRN_EINVAL;  // nothing to convert: a plain copy
    std::vector<void*> cols;
    mrn_view mapped;
    if ((rc = map_host_view(hv, dev, &mapped, &cols))) return rc;
    if (!h2d) zero_host_soa_gaps(*dst);
    return convert_direct(h2d ? mapped : *src, h2d ? *dst : mapped, stream);
  }
  if (dev >= kMaxDevices) return MRN_EUNSUPPORTED;
  const int dir = h2d ? 0 : 1;
  std::lock_guard<std::mutex> lk(g_engine_mu[dev][dir]);
  TransferEngine*& e = g_engine[dev][dir];
  if (!e) e = new (std::nothrow) TransferEngine();
  if (!e) return MRN_ENOMEM;
  return e->run(*src, *dst, opts ? opts->chunk_bytes : 0, opts ? opts->n_slots : 0,
                static_cast<cudaStream_t>(stream));
}
