// Device routines of the conversion kernels (sm_103a).
//
// Mapping: one warp handles 32 consecutive records, one record per lane.
//  - Record-major side (AoS): each lane moves its own record with the widest
//    vector access the stride and base alignment allow (16 B for a 32-byte
//    record, 8 B for a 24-byte one); the 32 lanes together touch one
//    contiguous span of 32*stride bytes, whose sectors L1 reuses across the
//    lane's successive vector loads.
//  - Field-major side (SoA / AoSoA): for every column the 32 lanes access 32
//    consecutive elements, i.e. one contiguous 32*size byte segment per warp
//    instruction (a full 128-byte line for 4-byte fields).
//  - Between the two, each lane keeps its record as 32-bit words in a
//    lane-private shared-memory column (word k of lane l at k*33 + l, so a
//    warp's accesses to word k hit 32 distinct banks); fields are extracted
//    from / merged into those words by their byte offset, which the schema
//    only knows at run time.  Records longer than a window (W words: 64
//    bytes for the per-call kernels, 32 for the batch kernel, whose shared
//    memory is tighter) are processed window by window (a naturally aligned
//    field never straddles one).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "mrn_plan.h"

#define MRN_WIN_WORDS 16
#define MRN_TW_PITCH 33
#define MRN_TW_WORDS_PER_WARP (MRN_WIN_WORDS * MRN_TW_PITCH)
#define MRN_TW_WORDS(W) ((W) * MRN_TW_PITCH)

__device__ __forceinline__ uint32_t lowbits_mask(uint32_t size) {
  return size >= 4 ? 0xffffffffu : ((1u << (8 * size)) - 1u);
}

// A load through the read-only data path (global memory, G) or a plain
// load (shared memory).
template <bool G, class T>
__device__ __forceinline__ T ldx(const T* p) {
  if constexpr (G) return __ldg(p); else return *p;
}

// Address of element i of field-major column c, whose consecutive
// elements are `es` bytes apart (the element size, or E * size for a
// column of an interleaved array).
__device__ __forceinline__ char* fm_addr(const SidePlan& sp, int c, uint32_t es, uint64_t i) {
  char* col = sp.col[c];
  if (sp.kind == K_SOA) return col + i * es;
  uint64_t blk, slot;
  if (sp.block_shift != MRN_NO_SHIFT) {
    blk = i >> sp.block_shift;
    slot = i & (uint64_t)(sp.block - 1);
  } else {
    blk = i / sp.block;
    slot = i - blk * sp.block;
  }
  return col + blk * sp.block_bytes + slot * es;
}

template <bool G = true>
__device__ __forceinline__ uint64_t ld_elem(const char* a, uint32_t size) {
  switch (size) {
    case 1: return ldx<G>(reinterpret_cast<const unsigned char*>(a));
    case 2: return ldx<G>(reinterpret_cast<const unsigned short*>(a));
    case 4: return ldx<G>(reinterpret_cast<const unsigned int*>(a));
    default: return ldx<G>(reinterpret_cast<const unsigned long long*>(a));
  }
}

__device__ __forceinline__ void st_elem(char* a, uint32_t size, uint64_t v) {
  switch (size) {
    case 1: *reinterpret_cast<unsigned char*>(a) = (unsigned char)v; break;
    case 2: *reinterpret_cast<unsigned short*>(a) = (unsigned short)v; break;
    case 4: *reinterpret_cast<unsigned int*>(a) = (unsigned int)v; break;
    default: *reinterpret_cast<unsigned long long*>(a) = v; break;
  }
}

// Loads nbytes (<= 4W, a multiple of V) of a record window into w[0..W-1]
// with V-byte accesses; w must be zero on entry for V < 4.
template <int V, int W, bool G = true>
__device__ __forceinline__ void load_words(const char* p, uint32_t nbytes, uint32_t (&w)[W]) {
  if constexpr (V == 16) {
#pragma unroll
    for (int k = 0; k < W / 4; ++k)
      if (k * 16 < (int)nbytes) {
        uint4 v = ldx<G>(reinterpret_cast<const uint4*>(p) + k);
        w[4 * k] = v.x; w[4 * k + 1] = v.y; w[4 * k + 2] = v.z; w[4 * k + 3] = v.w;
      }
  } else if constexpr (V == 8) {
#pragma unroll
    for (int k = 0; k < W / 2; ++k)
      if (k * 8 < (int)nbytes) {
        uint2 v = ldx<G>(reinterpret_cast<const uint2*>(p) + k);
        w[2 * k] = v.x; w[2 * k + 1] = v.y;
      }
  } else if constexpr (V == 4) {
#pragma unroll
    for (int k = 0; k < W; ++k)
      if (k * 4 < (int)nbytes) w[k] = ldx<G>(reinterpret_cast<const unsigned int*>(p) + k);
  } else if constexpr (V == 2) {
#pragma unroll
    for (int k = 0; k < 2 * W; ++k)
      if (k * 2 < (int)nbytes)
        w[k >> 1] |= (uint32_t)ldx<G>(reinterpret_cast<const unsigned short*>(p) + k) << ((k & 1) * 16);
  } else {
#pragma unroll
    for (int k = 0; k < 4 * W; ++k)
      if (k < (int)nbytes)
        w[k >> 2] |= (uint32_t)ldx<G>(reinterpret_cast<const unsigned char*>(p) + k) << ((k & 3) * 8);
  }
}

// V == 0: the access width is chosen at run time from `vec` (a uniform
// branch per window), for kernels that serve many plans at once.
template <int V, int W, bool G = true>
__device__ __forceinline__ void load_any(const char* p, uint32_t nbytes, uint32_t (&w)[W], uint32_t vec) {
  if constexpr (V != 0) {
    load_words<V, W, G>(p, nbytes, w);
  } else {
    switch (vec) {
      case 16: load_words<16, W, G>(p, nbytes, w); break;
      case 8: load_words<8, W, G>(p, nbytes, w); break;
      case 4: load_words<4, W, G>(p, nbytes, w); break;
      case 2: load_words<2, W, G>(p, nbytes, w); break;
      default: load_words<1, W, G>(p, nbytes, w); break;
    }
  }
}

template <int V, int W>
__device__ __forceinline__ void store_words(char* p, uint32_t nbytes, const uint32_t (&w)[W]) {
  if constexpr (V == 16) {
#pragma unroll
    for (int k = 0; k < W / 4; ++k)
      if (k * 16 < (int)nbytes)
        reinterpret_cast<uint4*>(p)[k] = make_uint4(w[4 * k], w[4 * k + 1], w[4 * k + 2], w[4 * k + 3]);
  } else if constexpr (V == 8) {
#pragma unroll
    for (int k = 0; k < W / 2; ++k)
      if (k * 8 < (int)nbytes) reinterpret_cast<uint2*>(p)[k] = make_uint2(w[2 * k], w[2 * k + 1]);
  } else if constexpr (V == 4) {
#pragma unroll
    for (int k = 0; k < W; ++k)
      if (k * 4 < (int)nbytes) reinterpret_cast<unsigned int*>(p)[k] = w[k];
  } else if constexpr (V == 2) {
#pragma unroll
    for (int k = 0; k < 2 * W; ++k)
      if (k * 2 < (int)nbytes)
        reinterpret_cast<unsigned short*>(p)[k] = (unsigned short)(w[k >> 1] >> ((k & 1) * 16));
  } else {
#pragma unroll
    for (int k = 0; k < 4 * W; ++k)
      if (k < (int)nbytes)
        reinterpret_cast<unsigned char*>(p)[k] = (unsigned char)(w[k >> 2] >> ((k & 3) * 8));
  }
}

template <int V, int W>
__device__ __forceinline__ void store_any(char* p, uint32_t nbytes, const uint32_t (&w)[W], uint32_t vec) {
  if constexpr (V != 0) {
    store_words<V, W>(p, nbytes, w);
  } else {
    switch (vec) {
      case 16: store_words<16, W>(p, nbytes, w); break;
      case 8: store_words<8, W>(p, nbytes, w); break;
      case 4: store_words<4, W>(p, nbytes, w); break;
      case 2: store_words<2, W>(p, nbytes, w); break;
      default: store_words<1, W>(p, nbytes, w); break;
    }
  }
}

// AoS record -> field-major columns, one record per lane.
//   r      destination record index (field-major side)
//   ld_ok  the lane has a source record at `rec`
//   st_ok  the lane writes destination record r (zeros when !ld_ok)
// The jagged descriptor, if the plan has one, is returned in *jlen / *jbeg.
template <int V, int W = MRN_WIN_WORDS>
__device__ __forceinline__ void aos_to_fm_lane(const ConvPlan& p, uint64_t r, bool ld_ok, bool st_ok,
                                               const char* rec, uint32_t* tw, int lane,
                                               uint32_t* jlen, uint64_t* jbeg) {
  uint32_t ci = 0;
  const uint32_t naos = p.naos, stride = p.stride, aw = p.aos_words;
  for (uint32_t win = 0; win < aw; win += W) {
    uint32_t w[W];
#pragma unroll
    for (int k = 0; k < W; ++k) w[k] = 0;
    const uint32_t nb = min(4u * W, stride - win * 4);
    if (ld_ok) load_any<V, W>(rec + win * 4, nb, w, p.vec);
    const uint32_t nw = min((uint32_t)W, aw - win);
#pragma unroll
    for (int k = 0; k < W; ++k)
      if (k < (int)nw) tw[k * MRN_TW_PITCH + lane] = w[k];
    const uint32_t wend = (win + W) * 4;
    for (; ci < naos; ++ci) {
      const ColPlan cp = p.aos_cols[ci];
      if (cp.aos_off >= wend) break;
      const uint32_t wi = cp.aos_off / 4 - win;
      const uint32_t lo = tw[wi * MRN_TW_PITCH + lane];
      if (cp.fm >= 0) {
        if (st_ok) {
          char* d = fm_addr(p.dst, cp.fm, p.fm_es[cp.fm], r);
          const uint32_t sh = (cp.aos_off & 3) * 8;
          switch (cp.size) {
            case 1: *reinterpret_cast<unsigned char*>(d) = (unsigned char)(lo >> sh); break;
            case 2: *reinterpret_cast<unsigned short*>(d) = (unsigned short)(lo >> sh); break;
            case 4: *reinterpret_cast<unsigned int*>(d) = lo; break;
            default:
              *reinterpret_cast<uint2*>(d) = make_uint2(lo, tw[(wi + 1) * MRN_TW_PITCH + lane]);
              break;
          }
        }
      } else if (cp.fm == FM_JLEN) {
        *jlen = lo;
      } else {
        *jbeg = (uint64_t)lo | ((uint64_t)tw[(wi + 1) * MRN_TW_PITCH + lane] << 32);
      }
    }
  }
}

// Field-major columns -> AoS record, one record per lane; padding bytes are
// written as zero.  The jagged descriptor (if any) is taken from jlen/jbeg.
template <int V, int W = MRN_WIN_WORDS>
__device__ __forceinline__ void fm_to_aos_lane(const ConvPlan& p, uint64_t r, bool ok, char* rec,
                                               uint32_t* tw, int lane, uint32_t jlen, uint64_t jbeg) {
  uint32_t ci = 0;
  const uint32_t naos = p.naos, stride = p.stride, aw = p.aos_words;
  for (uint32_t win = 0; win < aw; win += W) {
    const uint32_t nw = min((uint32_t)W, aw - win);
#pragma unroll
    for (int k = 0; k < W; ++k)
      if (k < (int)nw) tw[k * MRN_TW_PITCH + lane] = 0;
    const uint32_t wend = (win + W) * 4;
    for (; ci < naos; ++ci) {
      const ColPlan cp = p.aos_cols[ci];
      if (cp.aos_off >= wend) break;
      const uint32_t wi = cp.aos_off / 4 - win;
      uint64_t v;
      if (cp.fm >= 0)
        v = ok ? ld_elem(fm_addr(p.src, cp.fm, p.fm_es[cp.fm], r), cp.size) : 0;
      else
        v = cp.fm == FM_JLEN ? (uint64_t)jlen : jbeg;
      uint32_t* t = tw + wi * MRN_TW_PITCH + lane;
      if (cp.size == 8) {
        t[0] = (uint32_t)v;
        t[MRN_TW_PITCH] = (uint32_t)(v >> 32);
      } else if (cp.size == 4) {
        t[0] = (uint32_t)v;
      } else {
        t[0] |= ((uint32_t)v & lowbits_mask(cp.size)) << ((cp.aos_off & 3) * 8);
      }
    }
    if (ok) {
      uint32_t w[W];
#pragma unroll
      for (int k = 0; k < W; ++k) w[k] = k < (int)nw ? tw[k * MRN_TW_PITCH + lane] : 0u;
      store_any<V, W>(rec + win * 4, min(4u * W, stride - win * 4), w, p.vec);
    }
  }
}

// fm_to_aos_lane with the loads of up to 8 consecutive columns of a window
// issued before any of them is used, so that a record costs one memory
// round trip per 8 columns instead of one per column (for kernels with
// registers to spare; the columns are in AoS order).
template <int V, int W = MRN_WIN_WORDS>
__device__ __forceinline__ void fm_to_aos_lane_ilp(const ConvPlan& p, uint64_t r, bool ok, char* rec,
                                                   uint32_t* tw, int lane, uint32_t jlen, uint64_t jbeg) {
  constexpr int NB = 8;
  uint32_t ci = 0;
  const uint32_t naos = p.naos, stride = p.stride, aw = p.aos_words;
  for (uint32_t win = 0; win < aw; win += W) {
    const uint32_t nw = min((uint32_t)W, aw - win);
#pragma unroll
    for (int k = 0; k < W; ++k)
      if (k < (int)nw) tw[k * MRN_TW_PITCH + lane] = 0;
    const uint32_t wend = (win + W) * 4;
    while (ci < naos && p.aos_cols[ci].aos_off < wend) {
      uint64_t v[NB];
      uint32_t cnt = 0;
#pragma unroll
      for (int k = 0; k < NB; ++k) {
        v[k] = 0;
        const uint32_t c = ci + k;
        if (c < naos && c == ci + cnt) {
          const ColPlan cp = p.aos_cols[c];
          if (cp.aos_off < wend) {
            if (cp.fm >= 0) {
              if (ok) v[k] = ld_elem(fm_addr(p.src, cp.fm, p.fm_es[cp.fm], r), cp.size);
            } else {
              v[k] = cp.fm == FM_JLEN ? (uint64_t)jlen : jbeg;
            }
            ++cnt;
          }
        }
      }
#pragma unroll
      for (int k = 0; k < NB; ++k) {
        if (k >= (int)cnt) break;
        const ColPlan cp = p.aos_cols[ci + k];
        uint32_t* t = tw + (cp.aos_off / 4 - win) * MRN_TW_PITCH + lane;
        if (cp.size == 8) {
          t[0] = (uint32_t)v[k];
          t[MRN_TW_PITCH] = (uint32_t)(v[k] >> 32);
        } else if (cp.size == 4) {
          t[0] = (uint32_t)v[k];
        } else {
          t[0] |= ((uint32_t)v[k] & lowbits_mask(cp.size)) << ((cp.aos_off & 3) * 8);
        }
      }
      ci += cnt;
    }
    if (ok) {
      uint32_t w[W];
#pragma unroll
      for (int k = 0; k < W; ++k) w[k] = k < (int)nw ? tw[k * MRN_TW_PITCH + lane] : 0u;
      store_any<V, W>(rec + win * 4, min(4u * W, stride - win * 4), w, p.vec);
    }
  }
}

// Field-major -> field-major (SoA <-> AoSoA(B), AoSoA(B) -> AoSoA(B')),
// one record per lane, column by column.
__device__ __forceinline__ void fm_to_fm_lane(const ConvPlan& p, uint64_t r, bool ld_ok, bool st_ok) {
  if (!st_ok) return;
  for (uint32_t c = 0; c < p.ncols; ++c) {
    const uint32_t sz = p.fm_size[c], es = p.fm_es[c];
    const uint64_t v = ld_ok ? ld_elem(fm_addr(p.src, c, es, r), sz) : 0;
    st_elem(fm_addr(p.dst, c, es, r), sz, v);
  }
}

// ---- ordered global memory access for the decoupled look-back
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// A word other CTAs update atomically, read where they update it (L2).
__device__ __forceinline__ unsigned int ld_relaxed_u32(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ uint32_t ld_acquire_u32(const unsigned int* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

#define MRN_TS_AGG (1ull << 62)
#define MRN_TS_PREFIX (2ull << 62)
#define MRN_TS_VALUE ((1ull << 62) - 1)

// ------------------------------------------------------- TMA bulk copies
// One-dimensional bulk copies between global and shared memory, completed
// on an mbarrier (loads) or a bulk group (stores).  Global and shared
// addresses are 16-byte aligned and sizes are multiples of 16.

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Waits for phase `parity` of an mbarrier, bounded by ~2 s of wall clock
// and an iteration count; false when the bound expired.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long deadline = global_ns() + 2000000000ull;
  for (uint32_t i = 0; i < (1u << 24); ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 63) == 63 && global_ns() > deadline) return false;
  }
  return false;
}

// Prefetch of a global range into L2 (bulk copy engine; address 16-byte
// aligned, size a multiple of 16: a range that is not is left out, a
// prefetch being only a hint).
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, uint32_t bytes) {
  if (((reinterpret_cast<uintptr_t>(src) | bytes) & 15u) != 0 || bytes == 0) return;
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst_smem, const void* src, uint32_t bytes,
                                         unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst_smem)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void bulk_s2g(void* dst, const void* src_smem, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src_smem)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }

// Waits until at most N bulk store groups still read shared memory.
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}

// Waits until every bulk store group has completed.
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Orders this thread's generic-proxy shared-memory writes before later
// async-proxy (bulk copy) accesses.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 32-bit shared-memory accesses (the staged kernels address tiles with
// shared-window offsets, not generic pointers).
__device__ __forceinline__ uint32_t lds8(uint32_t a) {
  uint32_t v;
  asm volatile("ld.shared.u8 %0, [%1];" : "=r"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ uint32_t lds16(uint32_t a) {
  uint32_t v;
  asm volatile("ld.shared.u16 %0, [%1];" : "=r"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ uint32_t lds32(uint32_t a) {
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ uint2 lds64(uint32_t a) {
  uint2 v;
  asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(a));
  return v;
}
__device__ __forceinline__ uint4 lds128(uint32_t a) {
  uint4 v;
  asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(a));
  return v;
}
__device__ __forceinline__ void sts8(uint32_t a, uint32_t v) {
  asm volatile("st.shared.u8 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void sts16(uint32_t a, uint32_t v) {
  asm volatile("st.shared.u16 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void sts32(uint32_t a, uint32_t v) {
  asm volatile("st.shared.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void sts64(uint32_t a, uint2 v) {
  asm volatile("st.shared.v2.u32 [%0], {%1, %2};" ::"r"(a), "r"(v.x), "r"(v.y) : "memory");
}
__device__ __forceinline__ void sts128(uint32_t a, uint4 v) {
  asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(a), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
               : "memory");
}
__device__ __forceinline__ void sts128_zero(uint32_t a) {
  asm volatile("st.shared.v4.u32 [%0], {%1, %1, %1, %1};" ::"r"(a), "r"(0u) : "memory");
}

// Row geometry of one side of a plan (see TileHdr).
__host__ __device__ __forceinline__ void tile_side_geometry(uint32_t kind, uint32_t block, uint32_t shift, uint64_t bb,
                                                            uint32_t stride, uint32_t* gb, uint32_t* gs,
                                                            uint32_t* gbb) {
  if (kind == K_AOS) {
    *gb = 1, *gs = 0, *gbb = stride;
  } else if (kind == K_SOA) {
    *gb = 1, *gs = 31, *gbb = 0;
  } else {
    *gb = block, *gs = shift, *gbb = (uint32_t)bb;
  }
}

// Lane view of record r of a tile side: the byte address of its row and
// its slot in the row.
__device__ __forceinline__ void tile_row(uint32_t block, uint32_t shift, uint32_t bb, uint32_t tile, uint32_t r,
                                         uint32_t* base, uint32_t* idx) {
  const uint32_t blk = shift != MRN_NO_SHIFT ? r >> shift : r / block;
  *idx = r - blk * block;
  *base = tile + blk * bb;
}

// Zeroes an AoS destination record whose padding bytes no column writes
// (h.pad is set only for such destinations).
__device__ __forceinline__ void zero_record(const TileHdr& h, uint32_t db) {
  if (h.pad) {
    const uint32_t S = h.stride, v = h.vec;
    if (v == 16) {
      for (uint32_t o = 0; o < S; o += 16) sts128_zero(db + o);
    } else if (v == 8) {
      for (uint32_t o = 0; o < S; o += 8) sts64(db + o, make_uint2(0, 0));
    } else if (v == 4) {
      for (uint32_t o = 0; o < S; o += 4) sts32(db + o, 0);
    } else if (v == 2) {
      for (uint32_t o = 0; o < S; o += 2) sts16(db + o, 0);
    } else {
      for (uint32_t o = 0; o < S; ++o) sts8(db + o, 0);
    }
  }
}

// Shared loads and stores of 2^L bytes.
template <int L>
__device__ __forceinline__ uint2 lds_l(uint32_t a) {
  if constexpr (L == 3) return lds64(a);
  if constexpr (L == 2) return make_uint2(lds32(a), 0u);
  if constexpr (L == 1) return make_uint2(lds16(a), 0u);
  return make_uint2(lds8(a), 0u);
}

template <int L>
__device__ __forceinline__ void sts_l(uint32_t a, uint2 v) {
  if constexpr (L == 3) sts64(a, v);
  if constexpr (L == 2) sts32(a, v.x);
  if constexpr (L == 1) sts16(a, v.x);
  if constexpr (L == 0) sts8(a, v.x);
}

// The columns [c0, c1) of the descriptor table, all of 2^L bytes, for the
// lane's records: row + column offset + (slot << L) on both sides, the
// loads of two columns of both records before their stores.
template <int L>
__device__ __forceinline__ void tile_class(uint32_t desc, uint32_t c0, uint32_t c1, uint32_t sb0, uint32_t si0,
                                           uint32_t sb1, uint32_t si1, uint32_t db0, uint32_t di0, uint32_t db1,
                                           uint32_t di1, bool two) {
  const uint32_t so0 = si0 << L, so1 = si1 << L, do0 = di0 << L, do1 = di1 << L;
  uint32_t c = c0;
  for (; c + 1 < c1; c += 2) {
    const uint4 d0 = lds128(desc + c * 16), d1 = lds128(desc + c * 16 + 16);
    const uint2 v00 = lds_l<L>(sb0 + d0.y + so0), v10 = lds_l<L>(sb0 + d1.y + so0);
    uint2 v01 = v00, v11 = v10;
    if (two) {
      v01 = lds_l<L>(sb1 + d0.y + so1);
      v11 = lds_l<L>(sb1 + d1.y + so1);
    }
    sts_l<L>(db0 + d0.z + do0, v00);
    sts_l<L>(db0 + d1.z + do0, v10);
    if (two) {
      sts_l<L>(db1 + d0.z + do1, v01);
      sts_l<L>(db1 + d1.z + do1, v11);
    }
  }
  if (c < c1) {
    const uint4 d0 = lds128(desc + c * 16);
    const uint2 v00 = lds_l<L>(sb0 + d0.y + so0);
    uint2 v01 = v00;
    if (two) v01 = lds_l<L>(sb1 + d0.y + so1);
    sts_l<L>(db0 + d0.z + do0, v00);
    if (two) sts_l<L>(db1 + d0.z + do1, v01);
  }
}

// The columns [c0, c1) of 2^L bytes of a plan with an interleaved array:
// on a field-major side column c of slot i lies at its offset + i * es_c
// (the low 16 bits of descriptor word 3; an interleaved array's row is
// es_c = E * 2^L bytes, any other column's es_c = 2^L), on an AoS side at
// its offset (slot 0).  Two columns' loads of both records before their
// stores, as tile_class.
template <int L>
__device__ __forceinline__ void tile_class_es(uint32_t desc, uint32_t c0, uint32_t c1, uint32_t sb0, uint32_t si0,
                                              uint32_t sb1, uint32_t si1, uint32_t db0, uint32_t di0, uint32_t db1,
                                              uint32_t di1, bool two) {
  uint32_t c = c0;
  for (; c + 1 < c1; c += 2) {
    const uint4 d0 = lds128(desc + c * 16), d1 = lds128(desc + c * 16 + 16);
    const uint2 v00 = lds_l<L>(sb0 + d0.y + si0 * (d0.w & 0xffffu)), v10 = lds_l<L>(sb0 + d1.y + si0 * (d1.w & 0xffffu));
    uint2 v01 = v00, v11 = v10;
    if (two) {
      v01 = lds_l<L>(sb1 + d0.y + si1 * (d0.w & 0xffffu));
      v11 = lds_l<L>(sb1 + d1.y + si1 * (d1.w & 0xffffu));
    }
    sts_l<L>(db0 + d0.z + di0 * (d0.w & 0xffffu), v00);
    sts_l<L>(db0 + d1.z + di0 * (d1.w & 0xffffu), v10);
    if (two) {
      sts_l<L>(db1 + d0.z + di1 * (d0.w & 0xffffu), v01);
      sts_l<L>(db1 + d1.z + di1 * (d1.w & 0xffffu), v11);
    }
  }
  if (c < c1) {
    const uint4 d0 = lds128(desc + c * 16);
    const uint2 v00 = lds_l<L>(sb0 + d0.y + si0 * (d0.w & 0xffffu));
    uint2 v01 = v00;
    if (two) v01 = lds_l<L>(sb1 + d0.y + si1 * (d0.w & 0xffffu));
    sts_l<L>(db0 + d0.z + di0 * (d0.w & 0xffffu), v00);
    if (two) sts_l<L>(db1 + d0.z + di1 * (d0.w & 0xffffu), v01);
  }
}

// The widened columns [c0, c1) of an AoS destination (see tile_convert):
// a field of 2^x bytes (x < 3, descriptor word x) is loaded as usual and
// stored, zero-extended, with 2^w bytes (word w), which also writes the
// padding that follows it in the record.
__device__ __forceinline__ uint2 lds_any(uint32_t a, uint32_t L) {
  if (L == 2) return make_uint2(lds32(a), 0u);
  if (L == 1) return make_uint2(lds16(a), 0u);
  return make_uint2(lds8(a), 0u);
}

__device__ __forceinline__ void sts_wide(uint32_t a, uint2 v, uint32_t w) {
  if (w == 3) sts64(a, v);
  else if (w == 2) sts32(a, v.x);
  else sts16(a, v.x);
}

__device__ __forceinline__ void tile_wide(uint32_t desc, uint32_t c0, uint32_t c1, uint32_t sb0, uint32_t si0,
                                          uint32_t sb1, uint32_t si1, uint32_t db0, uint32_t db1, bool two) {
  for (uint32_t c = c0; c < c1; ++c) {
    const uint4 d = lds128(desc + c * 16);
    const uint2 v0 = lds_any(sb0 + d.y + (si0 << d.x), d.x);
    uint2 v1 = v0;
    if (two) v1 = lds_any(sb1 + d.y + (si1 << d.x), d.x);
    sts_wide(db0 + d.z, v0, d.w);
    if (two) sts_wide(db1 + d.z, v1, d.w);
  }
}

// tile_wide for a plan with an interleaved array: the field-major source's
// slot offset is slot * es_c (word 3's low 16 bits), the store width 2^w
// (word 3's bits 16-17).
__device__ __forceinline__ void tile_wide_es(uint32_t desc, uint32_t c0, uint32_t c1, uint32_t sb0, uint32_t si0,
                                             uint32_t sb1, uint32_t si1, uint32_t db0, uint32_t db1, bool two) {
  for (uint32_t c = c0; c < c1; ++c) {
    const uint4 d = lds128(desc + c * 16);
    const uint32_t es = d.w & 0xffffu, w = d.w >> 16;
    const uint2 v0 = lds_any(sb0 + d.y + si0 * es, d.x);
    uint2 v1 = v0;
    if (two) v1 = lds_any(sb1 + d.y + si1 * es, d.x);
    sts_wide(db0 + d.z, v0, w);
    if (two) sts_wide(db1 + d.z, v1, w);
  }
}

// Staged tile transform: each lane converts records r0 and r1 (= r0 + 256,
// when `two`) of the tile.  Per column one shared load and one shared store
// per record, addressed from the column descriptor table `desc` (uint4
// {log2(size), source column offset, destination column offset, 0} per
// column, in shared memory, ordered by decreasing size with h.nsize giving
// the size classes; a column offset on an AoS side is the field's offset in
// the record) as row + column offset + (slot << log2(size)).  One body
// serves every pair of layouts, so tiles of different layout pairs running
// side by side share their instructions; each size class is a loop of its
// own, so no element access branches on its size.  With Wide, the last
// h.nwide descriptors are fields of an AoS destination stored wider than
// they are, over the padding after them; such records are not zeroed first.
// With Inter (a plan with an interleaved array), the slot's offset is slot
// times descriptor word 3's low 16 bits instead (tile_class_es; widened
// fields: tile_wide_es, the store width in bits 16-17).
// An AoS <-> SoA tile whose AoS record is W (1, 2 or 4) 4-byte words, the
// columns in order (h.packed): the record moves as one 4-, 8- or 16-byte
// vector on the AoS side, and word k to or from its SoA column.  Narrow
// records are bound by the per-column work of the general body.
template <int W>
__device__ __forceinline__ void tile_convert_packed(const TileHdr& h, uint32_t desc, uint32_t st, uint32_t dt,
                                                    uint32_t r0, bool two) {
  const bool a2s = h.sshift == 0;  // AoS source (a row per record)
  uint32_t off[W];
#pragma unroll
  for (int k = 0; k < W; ++k) {
    const uint4 d = lds128(desc + k * 16);
    off[k] = a2s ? d.z : d.y;  // the SoA side's column offset in the tile
  }
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    if (q == 1 && !two) break;
    const uint32_t r = r0 + 256 * q;
    if constexpr (W == 1) {  // one 4-byte column: the tile is copied word by word
      sts32(dt + (a2s ? off[0] : 0u) + r * 4, lds32(st + (a2s ? 0u : off[0]) + r * 4));
    } else if (a2s) {
      if constexpr (W == 2) {
        const uint2 v = lds64(st + r * 8);
        sts32(dt + off[0] + r * 4, v.x);
        sts32(dt + off[1] + r * 4, v.y);
      } else {
        const uint4 v = lds128(st + r * 16);
        sts32(dt + off[0] + r * 4, v.x);
        sts32(dt + off[1] + r * 4, v.y);
        sts32(dt + off[2] + r * 4, v.z);
        sts32(dt + off[3] + r * 4, v.w);
      }
    } else {
      if constexpr (W == 2) {
        sts64(dt + r * 8, make_uint2(lds32(st + off[0] + r * 4), lds32(st + off[1] + r * 4)));
      } else {
        sts128(dt + r * 16, make_uint4(lds32(st + off[0] + r * 4), lds32(st + off[1] + r * 4),
                                       lds32(st + off[2] + r * 4), lds32(st + off[3] + r * 4)));
      }
    }
  }
}

// An AoS <-> SoA tile whose AoS record is two 2-byte columns in order
// (h.packed == kPacked2x16): one 4-byte word per record on the AoS side,
// its halves to or from the two columns.
constexpr uint32_t kPacked2x16 = 0x102u;
__device__ __forceinline__ void tile_convert_2x16(const TileHdr& h, uint32_t desc, uint32_t st, uint32_t dt,
                                                  uint32_t r0, bool two) {
  const bool a2s = h.sshift == 0;
  const uint4 d0 = lds128(desc), d1 = lds128(desc + 16);
  const uint32_t o0 = a2s ? d0.z : d0.y, o1 = a2s ? d1.z : d1.y;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    if (q == 1 && !two) break;
    const uint32_t r = r0 + 256 * q;
    if (a2s) {
      const uint32_t v = lds32(st + r * 4);
      sts16(dt + o0 + r * 2, v & 0xffffu);
      sts16(dt + o1 + r * 2, v >> 16);
    } else {
      sts32(dt + r * 4, lds16(st + o0 + r * 2) | (lds16(st + o1 + r * 2) << 16));
    }
  }
}

template <bool Wide, bool Narrow, bool Inter>
__device__ __forceinline__ void tile_convert(const TileHdr& h, uint32_t desc, uint32_t st, uint32_t dt,
                                             uint32_t r0, bool two) {
  if constexpr (Inter) {  // plans with an interleaved array: no packed records
  } else if constexpr (Narrow) {
    if (h.packed) {
      if (h.packed == 4) return tile_convert_packed<4>(h, desc, st, dt, r0, two);
      if (h.packed == 2) return tile_convert_packed<2>(h, desc, st, dt, r0, two);
      if (h.packed == kPacked2x16) return tile_convert_2x16(h, desc, st, dt, r0, two);
      return tile_convert_packed<1>(h, desc, st, dt, r0, two);
    }
  } else {  // the batch instance: packed records of two or four words only
    if (h.packed == 2) return tile_convert_packed<2>(h, desc, st, dt, r0, two);
    if (h.packed == 4) return tile_convert_packed<4>(h, desc, st, dt, r0, two);
  }
  const uint32_t r1 = two ? r0 + 256 : r0;
  uint32_t sb0, si0, db0, di0, sb1, si1, db1, di1;
  tile_row(h.sblock, h.sshift, h.sbb, st, r0, &sb0, &si0);
  tile_row(h.dblock, h.dshift, h.dbb, dt, r0, &db0, &di0);
  tile_row(h.sblock, h.sshift, h.sbb, st, r1, &sb1, &si1);
  tile_row(h.dblock, h.dshift, h.dbb, dt, r1, &db1, &di1);
  zero_record(h, db0);
  if (two) zero_record(h, db1);
  const uint32_t e8 = h.nsize & 0xff, e4 = e8 + ((h.nsize >> 8) & 0xff), e2 = e4 + ((h.nsize >> 16) & 0xff);
  const uint32_t ew = Wide ? h.ncols - h.nwide : h.ncols;
  if constexpr (Inter) {
    tile_class_es<3>(desc, 0, e8, sb0, si0, sb1, si1, db0, di0, db1, di1, two);
    tile_class_es<2>(desc, e8, e4, sb0, si0, sb1, si1, db0, di0, db1, di1, two);
    tile_class_es<1>(desc, e4, e2, sb0, si0, sb1, si1, db0, di0, db1, di1, two);
    tile_class_es<0>(desc, e2, ew, sb0, si0, sb1, si1, db0, di0, db1, di1, two);
    if (Wide && ew < h.ncols) tile_wide_es(desc, ew, h.ncols, sb0, si0, sb1, si1, db0, db1, two);
    return;
  }
  tile_class<3>(desc, 0, e8, sb0, si0, sb1, si1, db0, di0, db1, di1, two);
  tile_class<2>(desc, e8, e4, sb0, si0, sb1, si1, db0, di0, db1, di1, two);
  tile_class<1>(desc, e4, e2, sb0, si0, sb1, si1, db0, di0, db1, di1, two);
  tile_class<0>(desc, e2, ew, sb0, si0, sb1, si1, db0, di0, db1, di1, two);
  if (Wide && ew < h.ncols) tile_wide(desc, ew, h.ncols, sb0, si0, sb1, si1, db0, db1, two);
}
