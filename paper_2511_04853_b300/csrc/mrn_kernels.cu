// Conversion kernels for sm_103a and their launchers.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "mrn_device.cuh"
#include "mrn_internal.h"

// Per-device status word: bit k set = a kernel found error code k.
__device__ unsigned int g_mrn_status_bits;

__device__ __forceinline__ void flag_error(int code) { atomicOr(&g_mrn_status_bits, 1u << code); }

// ------------------------------------------------------------- conversion

// Records [t0, t1) of a plan; the CTA's warps take 32-record groups in turn.
template <int V, int W = MRN_WIN_WORDS>
__device__ __forceinline__ void conv_range(const ConvPlan& p, uint64_t t0, uint64_t t1, uint32_t* tw,
                                           int lane, int warp, int nwarps) {
  const uint32_t dir = p.dir;
  const uint64_t nrec = dir == DIR_FM_AOS ? p.n : p.n_fm_pad;
  if (t1 > nrec) t1 = nrec;
  for (uint64_t g = t0 + (uint64_t)warp * 32; g < t1; g += (uint64_t)nwarps * 32) {
    const uint64_t r = g + lane;
    const bool ld_ok = r < p.n;
    const bool st_ok = r < nrec;
    if (dir == DIR_AOS_FM) {
      uint32_t jl = 0;
      uint64_t jb = 0;
      aos_to_fm_lane<V, W>(p, r, ld_ok, st_ok, p.src.base + r * p.stride, tw, lane, &jl, &jb);
    } else if (dir == DIR_FM_AOS) {
      fm_to_aos_lane<V, W>(p, r, ld_ok, p.dst.base + r * p.stride, tw, lane, 0u, 0ull);
    } else {
      fm_to_fm_lane(p, r, ld_ok, st_ok);
    }
  }
}

// One conversion: CTAs take tiles of `tile_records` records, grid-stride.
template <int V>
__global__ void __launch_bounds__(256) k_convert(const __grid_constant__ ConvPlan p, uint32_t tile_records) {
  extern __shared__ uint32_t smem[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  uint32_t* tw = smem + warp * MRN_TW_WORDS_PER_WARP;
  const uint64_t nrec = p.dir == DIR_FM_AOS ? p.n : p.n_fm_pad;
  const uint64_t ntiles = (nrec + tile_records - 1) / tile_records;
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x)
    conv_range<V>(p, t * tile_records, (t + 1) * tile_records, tw, lane, warp, nwarps);
}

// ------------------------------------------------- staged tile transform

// All threads: source tile -> destination tile in shared memory.  Wide:
// the tables may hold widened fields (k_convert_ws<true, false>, for single
// conversions that have them; no other instance carries the branch).
// Narrow: the instance takes the one-column and two-2-byte-column record
// paths (single conversions); the persistent batch kernel leaves them out
// (those records take the general body there) because their branches cost
// its other jobs about 1%.  Inter: plans with an interleaved array (single
// conversions; tile_class_es).
template <bool Wide, bool Narrow, bool Inter>
__device__ __forceinline__ void tma_transform(const TileHdr& h, uint32_t desc, const char* st, char* dt, uint32_t R,
                                              int lane, int warp) {
  const uint32_t s = smem_u32(st), d = smem_u32(dt);
  const TileHdr hh = h;
  if (Narrow && !Inter && hh.packed == 1) {
    // one 4-byte column: both tiles hold the same words (R, a multiple of
    // 32, records), copied 16 bytes per thread and step
    const uint4 dd = lds128(desc);
    const uint32_t so = hh.sshift == 0 ? 0u : dd.y, dof = hh.sshift == 0 ? dd.z : 0u;
    if (((so | dof) & 15u) == 0) {
      for (uint32_t i = (uint32_t)warp * 32 + lane; i < R / 4; i += 8 * 32) sts128(d + dof + 16 * i, lds128(s + so + 16 * i));
      return;
    }
  }
  for (uint32_t g = (uint32_t)warp * 32; g < R; g += 2 * 8 * 32)
    tile_convert<Wide, Narrow, Inter>(hh, desc, s, d, g + lane, g + 8 * 32 < R);
}

// Entry k of the staged-transform descriptor table: the k-th column in
// size-class order (see tile_convert); with `wide`, the order with the
// fields widened over an AoS destination's padding last.  Word 3 is the
// widened store's log2 size, or (Inter: a plan with an interleaved array)
// the column's field-major element stride with that log2 size in bits
// 16-17.  Inter is a template argument:
// as a run-time choice in the loader's stage-table fill it cost single
// points SoA -> AoS 3% and AoSoA(32) -> AoS 5%.
template <bool Inter>
__host__ __device__ __forceinline__ uint4 tile_desc(const ConvPlan& p, uint32_t k, bool wide = false) {
  const bool w = wide && p.dst.kind == K_AOS && p.tg.nwide;
  const uint32_t c = w ? p.tg.worder[k] : p.tg.order[k];
  const uint32_t col = p.tg.col[c], aos_off = col & 0xffffffu;
  return make_uint4((col >> 24) & 3u, p.src.kind == K_AOS ? aos_off : p.tg.src_off[c],
                    p.dst.kind == K_AOS ? aos_off : p.tg.dst_off[c],
                    Inter ? (uint32_t)p.fm_es[c] | (((col >> 28) & 3u) << 16) : (col >> 28) & 3u);
}

template <bool Inter>
__host__ __device__ __forceinline__ TileHdr tile_hdr(const ConvPlan& p, bool wide = false) {
  const bool w = wide && p.dst.kind == K_AOS && p.tg.nwide;
  TileHdr h;
  h.ncols = p.ncols;
  h.stride = p.stride;
  h.vec = p.vec;
  h.pad = p.dst.kind == K_AOS && !w ? p.tg.pad : 0u;
  h.T = p.tg.T;
  h.nsize = w ? p.tg.wnsize : p.tg.nsize;
  h.nwide = w ? p.tg.nwide : 0u;
  h.packed = 0;
  const uint32_t n4 = (p.tg.nsize >> 8) & 0xff;
  // (not for interleaved plans, whose SoA tiles hold rows, not columns:
  // only the Inter instances meet them)
  const bool rows = Inter && p.tg.inter;
  const bool pair =
      !rows && ((p.src.kind == K_AOS && p.dst.kind == K_SOA) || (p.src.kind == K_SOA && p.dst.kind == K_AOS));
  if (pair && p.tg.nsize == (n4 << 8) && (n4 == 1 || n4 == 2 || n4 == 4) && p.ncols == n4 && p.stride == 4 * n4) {
    bool in_order = true;
    for (uint32_t k = 0; k < n4; ++k) in_order = in_order && (p.tg.col[p.tg.order[k]] & 0xffffffu) == 4 * k;
    if (in_order) h.packed = n4;
  }
  // a 4-byte record of two 2-byte columns, in order
  if (pair && p.tg.nsize == (2u << 16) && p.ncols == 2 && p.stride == 4 && (p.tg.col[p.tg.order[0]] & 0xffffffu) == 0 &&
      (p.tg.col[p.tg.order[1]] & 0xffffffu) == 2)
    h.packed = kPacked2x16;
  tile_side_geometry(p.src.kind, p.src.block, p.src.block_shift, p.src.block_bytes, p.stride, &h.sblock, &h.sshift,
                     &h.sbb);
  tile_side_geometry(p.dst.kind, p.dst.block, p.dst.block_shift, p.dst.block_bytes, p.stride, &h.dblock, &h.dshift,
                     &h.dbb);
  return h;
}

__device__ __forceinline__ void zero_gap_item(const GapPlan& g, uint64_t t) {
  const uint64_t b = t / g.ngaps;
  const uint32_t k = (uint32_t)(t - b * g.ngaps);
  char* p = g.base + b * g.block_bytes + g.off[k];
  for (uint32_t i = 0; i < g.len[k]; ++i) p[i] = 0;
}

__global__ void k_zero_gaps(const __grid_constant__ GapPlan g) {
  const uint64_t total = g.nblocks * g.ngaps;
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (uint64_t)gridDim.x * blockDim.x)
    zero_gap_item(g, t);
}

// ------------------------------------------------------------------ jagged

__device__ __forceinline__ void write_offset(char* offs, uint32_t osz, uint64_t i, uint64_t v) {
  if (osz == 4)
    reinterpret_cast<unsigned int*>(offs)[i] = (unsigned int)v;
  else
    reinterpret_cast<unsigned long long*>(offs)[i] = v;
}

__device__ __forceinline__ uint64_t read_offset(const char* offs, uint32_t osz, uint64_t i) {
  if (osz == 4) return __ldg(reinterpret_cast<const unsigned int*>(offs) + i);
  return __ldg(reinterpret_cast<const unsigned long long*>(offs) + i);
}

// The shapes of a fused jagged tile: parents per tile and threads per CTA.
// JagBig (1,024 parents, 512 threads) serves every launch but the small
// single conversions, which take JagSmall (256 parents, 256 threads): a
// collection of 100,000 parents then has 391 tiles to spread over the
// SMs instead of 98.
template <int TILE, int THREADS>
struct JagCfg {
  static constexpr int kTile = TILE, kThreads = THREADS, kWarps = THREADS / 32;
  static_assert(TILE % THREADS == 0, "whole parents per thread");
};
using JagBig = JagCfg<MRN_JAG_TILE, MRN_JAG_THREADS>;
using JagSmall = JagCfg<MRN_JAG_SMALL_TILE, MRN_JAG_SMALL_THREADS>;

// Shared state of a jagged tile: per-parent arrays (JagShared), written only
// after every warp has finished its parent conversion, and small per-warp
// values (JagWarp).
template <class Cfg>
struct JagSharedT {
  unsigned long long excl[Cfg::kTile + 1];
  unsigned long long beg[Cfg::kTile];
};
template <class Cfg>
struct JagWarpT {
  unsigned long long warp[Cfg::kWarps];
  unsigned long long kmin[Cfg::kWarps], kmax[Cfg::kWarps];  // per warp: min / max of begin - exclusive offset
  unsigned long long base;
  unsigned long long lsum[Cfg::kWarps];  // per warp: sum of its lengths (early aggregate)
};
using JagShared = JagSharedT<JagBig>;
using JagWarp = JagWarpT<JagBig>;

// Loads and stores of one column element of S bytes.
template <int S>
__device__ __forceinline__ unsigned long long ld_sized(const char* p) {
  if constexpr (S == 8) return __ldg(reinterpret_cast<const unsigned long long*>(p));
  if constexpr (S == 4) return __ldg(reinterpret_cast<const unsigned int*>(p));
  if constexpr (S == 2) return __ldg(reinterpret_cast<const unsigned short*>(p));
  return __ldg(reinterpret_cast<const unsigned char*>(p));
}

template <int S>
__device__ __forceinline__ void st_sized(char* p, unsigned long long v) {
  if constexpr (S == 8) *reinterpret_cast<unsigned long long*>(p) = v;
  if constexpr (S == 4) *reinterpret_cast<unsigned int*>(p) = (unsigned int)v;
  if constexpr (S == 2) *reinterpret_cast<unsigned short*>(p) = (unsigned short)v;
  if constexpr (S == 1) *reinterpret_cast<unsigned char*>(p) = (unsigned char)v;
}

// A record of at most 16 bytes held as two little-endian 64-bit halves,
// moved with the widest access its alignment `vec` allows.  A field never
// straddles the halves (natural alignment).
__device__ __forceinline__ void load_small(const char* p, uint32_t stride, uint32_t vec, uint64_t* lo,
                                           uint64_t* hi) {
  uint64_t a = 0, b = 0;
  if (vec >= 8) {
    a = __ldg(reinterpret_cast<const unsigned long long*>(p));
    if (stride > 8) b = __ldg(reinterpret_cast<const unsigned long long*>(p + 8));
  } else if (vec == 4) {
#pragma unroll
    for (uint32_t k = 0; k < 4; ++k)
      if (4 * k < stride) {
        const uint64_t w = __ldg(reinterpret_cast<const unsigned int*>(p + 4 * k));
        if (k < 2) a |= w << (32 * k); else b |= w << (32 * (k - 2));
      }
  } else {
#pragma unroll
    for (uint32_t k = 0; k < 16; ++k)
      if (k < stride) {
        const uint64_t w = __ldg(reinterpret_cast<const unsigned char*>(p + k));
        if (k < 8) a |= w << (8 * k); else b |= w << (8 * (k - 8));
      }
  }
  *lo = a;
  *hi = b;
}

__device__ __forceinline__ void store_small(char* p, uint32_t stride, uint32_t vec, uint64_t lo, uint64_t hi) {
  if (vec >= 8) {
    *reinterpret_cast<unsigned long long*>(p) = lo;
    if (stride > 8) *reinterpret_cast<unsigned long long*>(p + 8) = hi;
  } else if (vec == 4) {
#pragma unroll
    for (uint32_t k = 0; k < 4; ++k)
      if (4 * k < stride)
        *reinterpret_cast<unsigned int*>(p + 4 * k) = (unsigned int)(k < 2 ? lo >> (32 * k) : hi >> (32 * (k - 2)));
  } else {
#pragma unroll
    for (uint32_t k = 0; k < 16; ++k)
      if (k < stride)
        *reinterpret_cast<unsigned char*>(p + k) = (unsigned char)(k < 8 ? lo >> (8 * k) : hi >> (8 * (k - 8)));
  }
}

__device__ __forceinline__ uint64_t small_field(uint64_t lo, uint64_t hi, uint32_t off, uint32_t size) {
  const uint64_t v = off < 8 ? lo >> (8 * off) : hi >> (8 * (off - 8));
  return size == 8 ? v : v & ((1ull << (8 * size)) - 1);
}

template <int S>
__device__ __forceinline__ void st_col(char* col, uint64_t i, uint64_t v) {
  st_sized<S>(col + i * S, v);
}

constexpr int kJagSlots = MRN_JAG_CHILD_GROUP / 32;  // child slots per lane per pass

// One child column of Z bytes for the S slots of a lane: all loads, then
// all stores (zeros where the slot has no valid source).
template <int Z, int S>
__device__ __forceinline__ void child_column(const char* src, uint32_t stride, char* col, const uint64_t* si,
                                             const uint64_t* di, uint32_t ld_ok, uint32_t st_ok) {
  unsigned long long v[S];
#pragma unroll
  for (int u = 0; u < S; ++u) v[u] = (ld_ok >> u) & 1 ? ld_sized<Z>(src + si[u] * stride) : 0ull;
#pragma unroll
  for (int u = 0; u < S; ++u)
    if ((st_ok >> u) & 1) st_col<Z>(col, di[u], v[u]);
}

// The children of a jagged tile: slot j (0 <= j < agg) is child
// j - excl[p] of the last parent p with excl[p] <= j; it moves from pool
// record beg[p] + j - excl[p] to row base + j of every child column (the
// destination of a jagged conversion is always SoA).  Each lane moves
// kJagSlots slots per pass: records of at most 16 bytes are loaded whole
// and split in registers, wider ones column by column.  When the tile's
// children form one run of the pool (Run: beg[p] - excl[p] is the same `key`
// for every parent with children), the parent lookup is skipped.
template <bool Run, class Cfg, int S = kJagSlots>
__device__ __forceinline__ void jagged_children(const JagPlan& jp, const JagSharedT<Cfg>& sh, unsigned long long agg,
                                                unsigned long long base, unsigned long long key, int lane,
                                                int warp) {
  const ConvPlan& C = jp.child;
  const uint32_t nc = C.naos, stride = C.stride, vec = C.vec;
  const char* pool = C.src.base;
  constexpr unsigned long long kPass = 32 * S;
  for (unsigned long long j0 = (unsigned long long)warp * kPass; j0 < agg; j0 += Cfg::kWarps * kPass) {
    uint64_t si[S], di[S];
    uint32_t ld_ok = 0, st_ok = 0;
#pragma unroll
    for (int u = 0; u < S; ++u) {
      const unsigned long long j = j0 + u * 32 + lane;
      const bool cok = j < agg;
      bool good = cok;
      si[u] = key + j;
      if (!Run && cok) {
        int lo = 0, hi = Cfg::kTile;
        while (hi - lo > 1) {
          const int mid = (lo + hi) >> 1;
          if (sh.excl[mid] <= j) lo = mid; else hi = mid;
        }
        const unsigned long long pb = sh.beg[lo];
        good = pb != ~0ull;
        si[u] = pb + (j - sh.excl[lo]);
      }
      di[u] = base + j;
      const bool sok = cok && di[u] < jp.capacity;
      if (cok && !sok) flag_error(MRN_ESIZE);
      st_ok |= (uint32_t)sok << u;
      ld_ok |= (uint32_t)(sok && good) << u;
    }
    if (!st_ok) continue;
    if (stride <= 16) {
      uint64_t rl[S], rh[S];
#pragma unroll
      for (int u = 0; u < S; ++u) {
        rl[u] = rh[u] = 0;
        if ((ld_ok >> u) & 1) load_small(pool + si[u] * stride, stride, vec, &rl[u], &rh[u]);
      }
      for (uint32_t ci = 0; ci < nc; ++ci) {
        const ColPlan cp = C.aos_cols[ci];
        char* col = C.dst.col[cp.fm];
#pragma unroll
        for (int u = 0; u < S; ++u) {
          if (!((st_ok >> u) & 1)) continue;
          const uint64_t v = small_field(rl[u], rh[u], cp.aos_off, cp.size);
          switch (cp.size) {
            case 8: st_col<8>(col, di[u], v); break;
            case 4: st_col<4>(col, di[u], v); break;
            case 2: st_col<2>(col, di[u], v); break;
            default: st_col<1>(col, di[u], v); break;
          }
        }
      }
      continue;
    }
    for (uint32_t ci = 0; ci < nc; ++ci) {
      const ColPlan cp = C.aos_cols[ci];
      const char* src = pool + cp.aos_off;
      char* col = C.dst.col[cp.fm];
      switch (cp.size) {
        case 8: child_column<8, S>(src, stride, col, si, di, ld_ok, st_ok); break;
        case 4: child_column<4, S>(src, stride, col, si, di, ld_ok, st_ok); break;
        case 2: child_column<2, S>(src, stride, col, si, di, ld_ok, st_ok); break;
        default: child_column<1, S>(src, stride, col, si, di, ld_ok, st_ok); break;
      }
    }
  }
}

// The children of a jagged tile that form one run of the pool, for child
// records of at most 8 bytes: slot j moves pool record key + j to row
// base + j; each lane holds S records (one 64-bit word each) in flight.
template <int S, class Cfg>
__device__ __forceinline__ void jagged_run_small(const JagPlan& jp, unsigned long long agg, unsigned long long base,
                                                 unsigned long long key, int lane, int warp) {
  const ConvPlan& C = jp.child;
  const uint32_t nc = C.naos, stride = C.stride, vec = C.vec;
  const char* pool = C.src.base;
  constexpr unsigned long long kPass = 32 * S;
  for (unsigned long long j0 = (unsigned long long)warp * kPass; j0 < agg; j0 += Cfg::kWarps * kPass) {
    uint64_t rec[S];
    uint32_t ok = 0;
#pragma unroll
    for (int u = 0; u < S; ++u) {
      const unsigned long long j = j0 + u * 32 + lane;
      const bool cok = j < agg;
      const bool sok = cok && base + j < jp.capacity;
      if (cok && !sok) flag_error(MRN_ESIZE);
      ok |= (uint32_t)sok << u;
      uint64_t hi;
      rec[u] = 0;
      if (sok) load_small(pool + (key + j) * stride, stride, vec, &rec[u], &hi);
    }
    if (!ok) continue;
    for (uint32_t ci = 0; ci < nc; ++ci) {
      const ColPlan cp = C.aos_cols[ci];
      char* col = C.dst.col[cp.fm];
#pragma unroll
      for (int u = 0; u < S; ++u) {
        if (!((ok >> u) & 1)) continue;
        const unsigned long long row = base + j0 + u * 32 + lane;
        const uint64_t v = small_field(rec[u], 0, cp.aos_off, cp.size);
        switch (cp.size) {
          case 8: st_col<8>(col, row, v); break;
          case 4: st_col<4>(col, row, v); break;
          case 2: st_col<2>(col, row, v); break;
          default: st_col<1>(col, row, v); break;
        }
      }
    }
  }
}

// Children of a jagged SoA -> AoS conversion, records [j0, j0 + 32 *
// kJagSlots) of one warp: records of at most 16 bytes are assembled in
// registers from the child columns and stored whole; wider ones go through
// the lane-word path.
template <int VC, int W = MRN_WIN_WORDS>
__device__ __forceinline__ void jagged_s2a_children(const JagPlan& jp, uint64_t j0, uint32_t* tw, int lane) {
  const ConvPlan& C = jp.child;
  const uint32_t stride = C.stride;
  if (stride > 16) {
#pragma unroll 1
    for (int u = 0; u < kJagSlots; ++u) {
      const uint64_t j = j0 + u * 32 + lane;
      fm_to_aos_lane<VC, W>(C, j, j < jp.m_src, C.dst.base + j * stride, tw, lane, 0u, 0ull);
    }
    return;
  }
  const uint32_t nc = C.naos, vec = C.vec;
  uint64_t rl[kJagSlots], rh[kJagSlots];
#pragma unroll
  for (int u = 0; u < kJagSlots; ++u) rl[u] = rh[u] = 0;
  for (uint32_t ci = 0; ci < nc; ++ci) {
    const ColPlan cp = C.aos_cols[ci];
    const char* col = C.src.col[cp.fm];
    const uint32_t sh = 8 * (cp.aos_off & 7);
#pragma unroll
    for (int u = 0; u < kJagSlots; ++u) {
      const uint64_t j = j0 + u * 32 + lane;
      if (j >= jp.m_src) continue;
      uint64_t v;
      switch (cp.size) {
        case 8: v = ld_sized<8>(col + j * 8); break;
        case 4: v = ld_sized<4>(col + j * 4); break;
        case 2: v = ld_sized<2>(col + j * 2); break;
        default: v = ld_sized<1>(col + j); break;
      }
      if (cp.aos_off < 8) rl[u] |= v << sh; else rh[u] |= v << sh;
    }
  }
#pragma unroll
  for (int u = 0; u < kJagSlots; ++u) {
    const uint64_t j = j0 + u * 32 + lane;
    if (j < jp.m_src) store_small(C.dst.base + j * stride, stride, vec, rl[u], rh[u]);
  }
}

// Child count of all tiles before `tile`, by a decoupled look-back over the
// published tile words st[] (warp-wide: 32 predecessors per step; each wait
// bounded by jp.timeout_ns and an iteration count).  Run by one whole warp;
// every lane returns the sum.
__device__ __forceinline__ unsigned long long jagged_lookback(unsigned long long timeout_ns, uint64_t tile,
                                                              const unsigned long long* st, int lane) {
  unsigned long long prefix = 0;
  long long j = (long long)tile - 1;  // highest tile not yet accumulated
  // One deadline for the whole warp (lanes may arrive at different times,
  // e.g. after lane 0 alone stored to shared memory), and one decision when
  // it expires: a lane that left the loop alone would leave the others in
  // a warp-wide ballot it never reaches.
  const unsigned long long deadline = __shfl_sync(0xffffffffu, global_ns() + timeout_ns, 0);
  unsigned int spins = 0;
  while (j >= 0) {
    const long long jj = j - lane;
    const unsigned long long v = jj >= 0 ? ld_acquire_u64(&st[jj]) : MRN_TS_PREFIX;
    const unsigned long long fl = v & ~MRN_TS_VALUE;
    const unsigned int pref = __ballot_sync(0xffffffffu, fl == MRN_TS_PREFIX);
    const unsigned int zero = __ballot_sync(0xffffffffu, fl == 0);
    const unsigned int upto = pref ? ((pref & (0u - pref)) << 1) - 1u : 0xffffffffu;  // lanes to sum
    if (zero & upto) {
      if (__any_sync(0xffffffffu, global_ns() > deadline || ++spins > (1u << 24))) {
        if (lane == 0) flag_error(MRN_ETIMEOUT);
        break;
      }
      __nanosleep(64);
      continue;
    }
    unsigned long long x = ((upto >> lane) & 1u) ? (v & MRN_TS_VALUE) : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    prefix += x;
    if (pref) break;
    j -= 32;
  }
  return prefix;
}

// One tile of MRN_JAG_TILE (1,024) parents of a jagged AoS -> SoA conversion
// (512 threads, two parents each): converts the parents, scans their
// lengths, obtains the tile's child base by a decoupled look-back over the
// predecessors' published sums in `st`, writes the offsets and gathers the
// tile's children, load-balanced over the tile's threads.  Each tile
// publishes its own sum before its look-back, and tiles are handed out in
// increasing order, so every predecessor a look-back waits for is already
// running.
template <int VP, int VC, class Cfg = JagBig>
__device__ __forceinline__ void jagged_a2s_tile(const JagPlan& jp, uint64_t tile, unsigned long long* st,
                                                uint32_t* tw_all, JagSharedT<Cfg>& sh, JagWarpT<Cfg>& sw) {
  constexpr int W = MRN_WIN_WORDS;
  constexpr int K = Cfg::kTile / Cfg::kThreads;  // parents per thread
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint32_t* tw = tw_all + warp * MRN_TW_WORDS(W);
  const ConvPlan& P = jp.parent;
  const uint64_t t0 = tile * Cfg::kTile;

  // The tile's aggregate first, from the lengths alone, published at once:
  // the tiles after this one sum it in their look-back, which otherwise
  // waits for this tile's whole parent conversion.  (The records' lines
  // stay in cache for the conversion below.)
  // (The fall-back pass of a split conversion reads each base from the
  // finished offsets and publishes nothing.)
  const uint32_t mode = jp.mode;
  const bool publish = mode != JAG_CHILDREN && (long long)tile != jp.skip_publish_tile;
  if (mode != JAG_CHILDREN) {
    unsigned long long own = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const uint64_t r = t0 + k * Cfg::kThreads + tid;
      if (r < P.n) {
        const char* q = P.src.base + r * P.stride + jp.len_off;
        if (P.vec >= 4) {
          own += __ldg(reinterpret_cast<const unsigned int*>(q));
        } else {  // a base aligned to less than 4 bytes: byte by byte
          uint32_t v = 0;
#pragma unroll
          for (int b = 0; b < 4; ++b) v |= (uint32_t)__ldg(reinterpret_cast<const unsigned char*>(q + b)) << (8 * b);
          own += v;
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) own += __shfl_xor_sync(0xffffffffu, own, o);
    if (lane == 0) sw.lsum[warp] = own;
    __syncthreads();
    if (tid == 0) {
      unsigned long long a = 0;
#pragma unroll
      for (int w = 0; w < Cfg::kWarps; ++w) a += sw.lsum[w];
      if (publish)
        st_release_u64(&st[tile], (tile == 0 ? MRN_TS_PREFIX : MRN_TS_AGG) | (a & MRN_TS_VALUE));
    }
  }

  // Parents q = k * Cfg::kThreads + tid of the tile (consecutive records
  // per warp); then their lengths go to excl[] for the scan and their
  // begins (all ones for a parent whose children lie outside the pool) to
  // beg[].
  uint32_t len[K];
  uint64_t beg[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const uint64_t r = t0 + k * Cfg::kThreads + tid;
    const bool ok = r < P.n;
    len[k] = 0;
    beg[k] = 0;
    // slots after n of a destination's last AoSoA block are written as zero
    aos_to_fm_lane<VP, W>(P, r, ok, r < P.n_fm_pad, P.src.base + r * P.stride, tw, lane, &len[k], &beg[k]);
    if (!ok) len[k] = 0;
    if (ok && (beg[k] > jp.pool_n || (uint64_t)len[k] > jp.pool_n - beg[k])) {
      flag_error(MRN_EINVAL);
      beg[k] = ~0ull;
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) {
    sh.excl[k * Cfg::kThreads + tid] = len[k];
    sh.beg[k * Cfg::kThreads + tid] = beg[k];
  }
  __syncthreads();

  // CTA-wide exclusive scan in parent order: thread t owns parents K t ..
  // K t + K - 1 (64-bit sums).
  unsigned long long own = 0;
#pragma unroll
  for (int k = 0; k < K; ++k) own += sh.excl[K * tid + k];
  unsigned long long x = own;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sw.warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    unsigned long long t = lane < Cfg::kWarps ? sw.warp[lane] : 0ull;
#pragma unroll
    for (int o = 1; o < Cfg::kWarps; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < Cfg::kWarps) sw.warp[lane] = t;
  }
  __syncthreads();
  const unsigned long long agg = sw.warp[Cfg::kWarps - 1];
  // Exclusive offsets of the thread's parents written back in place; the
  // run test on the way: beg - excl equal for every parent with children
  // (a parent outside the pool fails it: min 0, max all ones).
  unsigned long long kmin = ~0ull, kmax = 0ull;
  {
    unsigned long long e = x - own + (warp > 0 ? sw.warp[warp - 1] : 0ull);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const unsigned long long l = sh.excl[K * tid + k], b = sh.beg[K * tid + k];
      if (b == ~0ull) {
        kmin = 0ull;
        kmax = ~0ull;
      } else if (l > 0) {
        kmin = min(kmin, b - e);
        kmax = max(kmax, b - e);
      }
      sh.excl[K * tid + k] = e;
      e += l;
    }
  }
  if (tid == Cfg::kThreads - 1) sh.excl[Cfg::kTile] = agg;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    kmin = min(kmin, __shfl_xor_sync(0xffffffffu, kmin, o));
    kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
  }
  if (lane == 0) {
    sw.kmin[warp] = kmin;
    sw.kmax[warp] = kmax;
  }

  // Decoupled look-back for the number of children of all earlier tiles
  // (the tile's aggregate was published as soon as its lengths were in).
  if (warp == 0) {
    unsigned long long prefix = 0;
    if (mode == JAG_CHILDREN) {  // the finished offset of the tile's first parent
      if (t0 < P.n) prefix = read_offset(jp.offsets, jp.off_size, t0) - jp.offset_base;
    } else if (tile > 0) {
      prefix = jagged_lookback(jp.timeout_ns, tile, st, lane);
      if (publish && lane == 0) st_release_u64(&st[tile], MRN_TS_PREFIX | ((prefix + agg) & MRN_TS_VALUE));
    }
    if (lane == 0) sw.base = prefix;
  }
  __syncthreads();
  const unsigned long long base = sw.base;
  // Children in one run of the pool: start pulling their source range into
  // L2 while the offsets are written.
  kmin = ~0ull;
  kmax = 0ull;
#pragma unroll
  for (int w = 0; w < Cfg::kWarps; ++w) {
    kmin = min(kmin, sw.kmin[w]);
    kmax = max(kmax, sw.kmax[w]);
  }
  const bool run = kmin == kmax;
  if (run && warp == 0 && agg > 0) {
    const uint32_t cs = jp.child.stride;
    const uintptr_t a = reinterpret_cast<uintptr_t>(jp.child.src.base + kmin * cs);
    const uintptr_t b = reinterpret_cast<uintptr_t>(jp.child.src.base + (kmin + agg) * cs);
    const uintptr_t lo = a & ~(uintptr_t)15, hi = (b + 15) & ~(uintptr_t)15;
    for (uintptr_t q = lo + (uintptr_t)lane * 32768; q < hi; q += 32 * 32768)
      bulk_prefetch_l2(reinterpret_cast<const void*>(q), (uint32_t)min((uintptr_t)32768, hi - q));
  }

  // Tile 0 of a single conversion zeroes the destination's gap bytes.
  if (tile == 0 && jp.ngaps && mode != JAG_CHILDREN)
    for (uint32_t k = 0; k < jp.ngaps; ++k)
      for (uint32_t b = tid; b < jp.gap_len[k]; b += Cfg::kThreads) jp.gap_base[jp.gap_off[k] + b] = 0;

  // Offsets: offset_base + children before this parent (a collection of
  // no objects, given one tile, has the single offset offset_base).  Every
  // parent's exclusive offset and the next one are in excl[] (excl[TILE] =
  // the tile's sum), written before the look-back's barrier.
  if (P.n == 0 && tid == 0) write_offset(jp.offsets, jp.off_size, 0, jp.offset_base);
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const uint64_t r = t0 + K * tid + k;
    const unsigned long long excl = sh.excl[K * tid + k], len = sh.excl[K * tid + k + 1] - excl;
    if (r < P.n) {
      const unsigned long long o = jp.offset_base + base + excl;
      write_offset(jp.offsets, jp.off_size, r, o);
      if (r == P.n - 1) {
        const unsigned long long end = o + len;
        write_offset(jp.offsets, jp.off_size, P.n, end);
        if (jp.total_out) *jp.total_out = base + excl + len;
        if (jp.off_size == 4 && (end > 0xffffffffull || end < o)) flag_error(MRN_EOVERFLOW);
      } else if (jp.off_size == 4 && o + len > 0xffffffffull) {
        flag_error(MRN_EOVERFLOW);
      }
    }
  }

  // Children, as one run of the pool when they form one.
  if (run && jp.child.stride <= 8)
    jagged_run_small<kJagSlots, Cfg>(jp, agg, base, kmin, lane, warp);
  else if (run)
    jagged_children<true, Cfg>(jp, sh, agg, base, kmin, lane, warp);
  else
    jagged_children<false, Cfg>(jp, sh, agg, base, 0ull, lane, warp);
}

template <int VP, int VC>
__global__ void __launch_bounds__(MRN_JAG_THREADS, MRN_JAG_CTAS) k_jagged_a2s(const __grid_constant__ JagPlan jp) {
  // The tile windows serve the parent conversion only; the per-parent
  // arrays are written after every warp has finished it.
  constexpr size_t kTw = MRN_JAG_WARPS * MRN_TW_WORDS_PER_WARP * sizeof(uint32_t);
  __shared__ __align__(16) unsigned char jag_raw[kTw > sizeof(JagShared) ? kTw : sizeof(JagShared)];
  uint32_t* tw_all = reinterpret_cast<uint32_t*>(jag_raw);
  JagShared& sh = *reinterpret_cast<JagShared*>(jag_raw);
  __shared__ JagWarp sw;
  __shared__ unsigned int s_tile;
  if (threadIdx.x == 0) s_tile = atomicAdd(jp.tile_counter, 1u);
  __syncthreads();
  jagged_a2s_tile<VP, VC>(jp, s_tile, jp.tile_state, tw_all, sh, sw);
}

// The same conversion in tiles of JagSmall (256 parents, one per thread),
// for single conversions of few tiles (generic access widths).
__global__ void __launch_bounds__(MRN_JAG_SMALL_THREADS, 6) k_jagged_a2s_small(const __grid_constant__ JagPlan jp) {
  constexpr size_t kTw = JagSmall::kWarps * MRN_TW_WORDS_PER_WARP * sizeof(uint32_t);
  __shared__ __align__(16) unsigned char jag_raw[kTw > sizeof(JagSharedT<JagSmall>) ? kTw : sizeof(JagSharedT<JagSmall>)];
  uint32_t* tw_all = reinterpret_cast<uint32_t*>(jag_raw);
  JagSharedT<JagSmall>& sh = *reinterpret_cast<JagSharedT<JagSmall>*>(jag_raw);
  __shared__ JagWarpT<JagSmall> sw;
  __shared__ unsigned int s_tile;
  if (threadIdx.x == 0) s_tile = atomicAdd(jp.tile_counter, 1u);
  __syncthreads();
  jagged_a2s_tile<0, 0, JagSmall>(jp, s_tile, jp.tile_state, tw_all, sh, sw);
}

// Fall-back pass of a split jagged AoS -> field-major conversion (plan mode
// JAG_CHILDREN): nothing to do unless the scan pass found the pool not
// canonical; then the CTAs take the tiles in turn and gather their
// children (no look-back: every base is in the tile words).
__global__ void __launch_bounds__(MRN_JAG_THREADS, MRN_JAG_CTAS) k_jagged_a2s_rest(const __grid_constant__ JagPlan jp) {
  if (ld_relaxed_u32(jp.noncanon) == 0) return;
  constexpr size_t kTw = MRN_JAG_WARPS * MRN_TW_WORDS_PER_WARP * sizeof(uint32_t);
  __shared__ __align__(16) unsigned char jag_raw[kTw > sizeof(JagShared) ? kTw : sizeof(JagShared)];
  uint32_t* tw_all = reinterpret_cast<uint32_t*>(jag_raw);
  JagShared& sh = *reinterpret_cast<JagShared*>(jag_raw);
  __shared__ JagWarp sw;
  for (uint64_t t = blockIdx.x; t < jp.ntiles; t += gridDim.x) {
    jagged_a2s_tile<0, 0>(jp, t, nullptr, tw_all, sh, sw);
    __syncthreads();  // the next tile's parent windows overlay this tile's arrays
  }
}

// Fall-back pass of a split single conversion in the local form (plan mode
// JAG_FUSED here, the parents' checks done): block 0 first zeroes the
// destination's gap bytes, which the staged jobs leave, and (a canonical
// pool) writes the children's count, the pool's size, to total_out;
// nothing else unless the checks found the pool not canonical, and then
// the whole conversion again, fused, tiles taken by ticket in increasing
// order (look-back over tile_state; its tiles write total_out).
__global__ void __launch_bounds__(MRN_JAG_THREADS, MRN_JAG_CTAS) k_jagged_a2s_whole_if(const __grid_constant__ JagPlan jp) {
  if (blockIdx.x == 0)
    for (uint32_t k = 0; k < jp.ngaps; ++k)
      for (uint32_t b = threadIdx.x; b < jp.gap_len[k]; b += blockDim.x) jp.gap_base[jp.gap_off[k] + b] = 0;
  if (ld_relaxed_u32(jp.noncanon) == 0) {
    if (blockIdx.x == 0 && threadIdx.x == 0 && jp.total_out) *jp.total_out = jp.pool_n;
    return;
  }
  constexpr size_t kTw = MRN_JAG_WARPS * MRN_TW_WORDS_PER_WARP * sizeof(uint32_t);
  __shared__ __align__(16) unsigned char jag_raw[kTw > sizeof(JagShared) ? kTw : sizeof(JagShared)];
  uint32_t* tw_all = reinterpret_cast<uint32_t*>(jag_raw);
  JagShared& sh = *reinterpret_cast<JagShared*>(jag_raw);
  __shared__ JagWarp sw;
  __shared__ unsigned int s_tile;
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(jp.tile_counter, 1u);
    __syncthreads();
    const uint64_t t = s_tile;
    if (t >= jp.ntiles) break;
    jagged_a2s_tile<0, 0>(jp, t, jp.tile_state, tw_all, sh, sw);
    __syncthreads();  // the next ticket (and tile) overlay this tile's state
  }
}

// The jagged AoS -> field-major jobs of a batch: one CTA per tile as in
// k_jagged_a2s, 3 CTAs (48 warps) per SM, tiles taken in increasing order
// over all the jobs,
// each tile's job read from a host-built map.  A tile's look-back only
// visits its own job's earlier tiles, which hold earlier tickets.  The
// job's plan is copied into shared memory first: the tile reads its fields
// all along, and from global memory (not the constant bank, where a single
// conversion's plan sits) those reads cost the batch a quarter of its speed.
__global__ void __launch_bounds__(MRN_JAG_THREADS, MRN_JAG_CTAS) k_batch_jag(const BatchJob* __restrict__ jobs,
                                                                 const unsigned int* __restrict__ tile_job,
                                                                 unsigned long long total, unsigned int* counter,
                                                                 unsigned long long* states) {
  // The tile windows serve the parent conversion only; the per-parent
  // arrays are written after every warp has finished it.
  constexpr size_t kTw = MRN_JAG_WARPS * MRN_TW_WORDS_PER_WARP * sizeof(uint32_t);
  __shared__ __align__(16) unsigned char jag_raw[kTw > sizeof(JagShared) ? kTw : sizeof(JagShared)];
  uint32_t* tw_all = reinterpret_cast<uint32_t*>(jag_raw);
  JagShared& sh = *reinterpret_cast<JagShared*>(jag_raw);
  __shared__ JagWarp sw;
  __shared__ unsigned int s_tile;
  __shared__ __align__(16) unsigned long long jps[(sizeof(JagPlan) + 7) / 8];
  if (threadIdx.x == 0) s_tile = atomicAdd(counter, 1u);
  __syncthreads();
  const uint64_t t = s_tile;
  if (t >= total) return;
  const BatchJob& J = jobs[__ldg(tile_job + t)];
  const unsigned long long* g = reinterpret_cast<const unsigned long long*>(&J.jp);
  for (uint32_t i = threadIdx.x; i < sizeof(JagPlan) / 8; i += blockDim.x) jps[i] = __ldg(g + i);
  const uint64_t tb = J.tile_begin;
  __syncthreads();
  jagged_a2s_tile<0, 0>(*reinterpret_cast<const JagPlan*>(jps), t - tb, states + tb, tw_all, sh, sw);
}

// Fall-back pass of a batch's split jagged jobs (JAG_LOCAL): nothing to do
// unless a parents job's local check found its pool not canonical (*any);
// then every CTA walks the jobs, 32 flags at a time, and converts each
// flagged job whole again (plan mode JAG_FUSED in the shared copy: the
// parents job wrote the begins as offsets, which the fused tiles write
// again, with the children gathered), tiles taken by ticket in increasing
// order for the look-back.
__global__ void __launch_bounds__(MRN_JAG_THREADS, MRN_JAG_CTAS) k_batch_jag_rest(const BatchJob* __restrict__ jobs,
                                                                      unsigned int njobs,
                                                                      const unsigned int* flags,
                                                                      const unsigned int* any) {
  if (ld_relaxed_u32(any) == 0) return;
  constexpr size_t kTw = MRN_JAG_WARPS * MRN_TW_WORDS_PER_WARP * sizeof(uint32_t);
  __shared__ __align__(16) unsigned char jag_raw[kTw > sizeof(JagShared) ? kTw : sizeof(JagShared)];
  uint32_t* tw_all = reinterpret_cast<uint32_t*>(jag_raw);
  JagShared& sh = *reinterpret_cast<JagShared*>(jag_raw);
  __shared__ JagWarp sw;
  __shared__ unsigned int s_mask, s_tile;
  __shared__ __align__(16) unsigned long long jps[(sizeof(JagPlan) + 7) / 8];
  JagPlan& jp = *reinterpret_cast<JagPlan*>(jps);
  for (unsigned int j0 = 0; j0 < njobs; j0 += 32) {
    if (threadIdx.x < 32) {
      const unsigned int j = j0 + threadIdx.x;
      const unsigned int m = __ballot_sync(0xffffffffu, j < njobs && ld_relaxed_u32(flags + j) != 0);
      if (threadIdx.x == 0) s_mask = m;
    }
    __syncthreads();
    unsigned int mask = s_mask;
    __syncthreads();  // s_mask is written again in the next round
    while (mask) {
      const unsigned int j = j0 + (unsigned int)__ffs(mask) - 1u;
      mask &= mask - 1u;
      const BatchJob& J = jobs[j];
      const uint64_t nt = J.ntiles;
      const unsigned long long* g = reinterpret_cast<const unsigned long long*>(&J.jp);
      for (uint32_t i = threadIdx.x; i < sizeof(JagPlan) / 8; i += blockDim.x) jps[i] = __ldg(g + i);
      __syncthreads();
      if (threadIdx.x == 0) jp.mode = JAG_FUSED;
      __syncthreads();
      for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(jp.tile_counter, 1u);
        __syncthreads();
        const uint64_t t = s_tile;
        if (t >= nt) break;
        jagged_a2s_tile<0, 0>(jp, t, jp.tile_state, tw_all, sh, sw);
        __syncthreads();  // the next ticket (and tile) overlay this tile's state
      }
      __syncthreads();  // s_tile and the plan are written again for the next job
    }
  }
}

// ---------------------------------------------------- split jagged scan

// A u32 / u64 field of an AoS record whose base is aligned to `vec` bytes.
__device__ __forceinline__ uint32_t ld_u32_rec(const char* p, uint32_t vec) {
  if (vec >= 4) return __ldg(reinterpret_cast<const unsigned int*>(p));
  uint32_t v = 0;
#pragma unroll
  for (int b = 0; b < 4; ++b) v |= (uint32_t)__ldg(reinterpret_cast<const unsigned char*>(p + b)) << (8 * b);
  return v;
}
__device__ __forceinline__ uint64_t ld_u64_rec(const char* p, uint32_t vec) {
  if (vec >= 8) return __ldg(reinterpret_cast<const unsigned long long*>(p));
  return (uint64_t)ld_u32_rec(p, vec) | ((uint64_t)ld_u32_rec(p + 4, vec) << 32);
}

__device__ __forceinline__ unsigned long long warp_incl_scan_u64(unsigned long long x, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

constexpr uint32_t kScanThreads = 256;
constexpr uint32_t kScanGroups = MRN_SCAN_CHUNK / 32;                    // groups of 32 parents per chunk
constexpr uint32_t kScanWarpGroups = kScanGroups / (kScanThreads / 32);  // groups per warp
static_assert(kScanWarpGroups == 32, "a warp's groups are one per lane");

struct ScanShared {
  unsigned long long wsum[kScanThreads / 32];
  unsigned long long base;
};

// Chunk c (of MRN_SCAN_CHUNK parents) of a split jagged AoS -> field-major
// conversion: warp w sums the lengths of groups 32 w .. 32 w + 31 of the
// chunk (lane l of a pass holds parent 32 g + l; lane i ends up holding group
// i's sum and the begin - exclusive offset its parents with children
// share, if they do), the chunk's aggregate is published and the children before the
// chunk come from a decoupled look-back over st[]; then every group's base
// (children before it) goes to group_base.  The pool is canonical where each
// group with children has begin - exclusive offset equal to its base for all
// those parents; the group of the last parent writes offsets[n] and checks
// that the children are exactly the pool's records.
__device__ __forceinline__ void jag_scan_chunk(const JagPlan& jp, uint64_t c, unsigned long long* st, ScanShared& sh) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint64_t n = jp.parent.n, pool_n = jp.pool_n;
  const char* base = jp.parent.src.base;
  const uint32_t stride = jp.parent.stride, vec = jp.parent.vec, len_off = jp.len_off, begin_off = jp.begin_off;
  const uint64_t g0 = c * kScanGroups + (uint64_t)warp * kScanWarpGroups;
  // lane i: group g0 + i's sum, the common begin - exclusive offset of its
  // parents with children (gd), and whether they all share it (guni)
  unsigned long long gsum = 0, gd = 0;
  bool guni = true;
  // groups per pass (loads in flight per lane: 2 U); measured on 105 M
  // parents: U = 4 at 6 CTAs per SM 0.477 ms, U = 8 at 4 (its registers) 0.512,
  // U = 2 at 8 0.507, U = 4 at 8 0.525
  constexpr int U = 4;
#pragma unroll 1
  for (uint32_t i0 = 0; i0 < kScanWarpGroups; i0 += U) {
    uint32_t len[U];
    uint64_t beg[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint64_t r = (g0 + i0 + u) * 32 + lane;
      len[u] = 0;
      beg[u] = 0;
      if (r < n) {
        const char* q = base + r * stride;
        len[u] = ld_u32_rec(q + len_off, vec);
        beg[u] = ld_u64_rec(q + begin_off, vec);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint64_t r = (g0 + i0 + u) * 32 + lane;
      const bool bad = r < n && (beg[u] > pool_n || (uint64_t)len[u] > pool_n - beg[u]);
      if (bad) flag_error(MRN_EINVAL);
      // the exclusive prefix inside the group: 32-bit unless some length
      // could carry past 32 bits (32 lengths below 2^26 cannot)
      unsigned long long excl, tot;
      if (__any_sync(0xffffffffu, len[u] >= (1u << 26))) {
        const unsigned long long x = warp_incl_scan_u64(len[u], lane);
        excl = x - len[u];
        tot = __shfl_sync(0xffffffffu, x, 31);
      } else {
        uint32_t x = len[u];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
          if (lane >= o) x += y;
        }
        excl = x - len[u];
        tot = __reduce_add_sync(0xffffffffu, len[u]);
      }
      // canonical here: every parent valid, and begin - exclusive offset
      // the same for all parents with children
      const unsigned long long d = beg[u] - excl;
      const unsigned int has = __ballot_sync(0xffffffffu, len[u] > 0);
      const unsigned long long d0 = __shfl_sync(0xffffffffu, d, has ? __ffs(has) - 1 : 0);
      const bool uni = __all_sync(0xffffffffu, !bad && (len[u] == 0 || d == d0));
      if ((uint32_t)lane == i0 + u) {
        gsum = tot;
        gd = d0;
        guni = uni;
      }
    }
  }
  const unsigned long long x = warp_incl_scan_u64(gsum, lane);
  if (lane == 31) sh.wsum[warp] = x;
  __syncthreads();
  unsigned long long agg = 0, wbase = 0;
#pragma unroll
  for (int w = 0; w < (int)(kScanThreads / 32); ++w) {
    const unsigned long long v = sh.wsum[w];
    if (w < warp) wbase += v;
    agg += v;
  }
  const bool publish = (long long)c != jp.skip_publish_tile;
  if (tid == 0 && publish) st_release_u64(&st[c], (c == 0 ? MRN_TS_PREFIX : MRN_TS_AGG) | (agg & MRN_TS_VALUE));
  if (warp == 0) {
    unsigned long long prefix = 0;
    if (c > 0) {
      prefix = jagged_lookback(jp.timeout_ns, c, st, lane);
      if (publish && lane == 0) st_release_u64(&st[c], MRN_TS_PREFIX | ((prefix + agg) & MRN_TS_VALUE));
    }
    if (lane == 0) sh.base = prefix;
  }
  // chunk 0 of a single conversion zeroes the destination's gap bytes
  if (c == 0 && jp.ngaps)
    for (uint32_t k = 0; k < jp.ngaps; ++k)
      for (uint32_t b = tid; b < jp.gap_len[k]; b += kScanThreads) jp.gap_base[jp.gap_off[k] + b] = 0;
  __syncthreads();
  const uint64_t g = g0 + lane;
  const bool have = g * 32 < n;
  const unsigned long long gb = sh.base + wbase + (x - gsum);
  bool bad = have && (!guni || (gsum > 0 && gd != gb));
  if (have) jp.group_base[g] = gb;
  if (have && (n - 1) / 32 == g) {
    const unsigned long long total = gb + gsum, end = jp.offset_base + total;
    write_offset(jp.offsets, jp.off_size, n, end);
    if (jp.total_out) *jp.total_out = total;
    if (jp.off_size == 4 && (end > 0xffffffffull || end < total)) flag_error(MRN_EOVERFLOW);
    if (total != pool_n) bad = true;
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) {
    atomicExch(jp.noncanon, 1u);
    if (jp.any_noncanon) atomicExch(jp.any_noncanon, 1u);
  }
}

// Chunk c of a column scan (ColScan): the same sums, pool check and
// look-back as jag_scan_chunk, the lengths and begins read from their
// columns.  Each parent's offset inside its group is kept in shared memory
// (`ex`: [warp][group][lane]), so that once the chunk's base is known each
// warp writes its parents' offsets without a second scan; a group whose
// lengths could carry past 32 bits is scanned again from its lengths.
struct ColScanShared {
  uint32_t ex[kScanThreads / 32][kScanWarpGroups][32];
  unsigned long long gb[kScanThreads / 32][32];
};
__device__ __forceinline__ void col_scan_chunk(const ColScan& cs, uint64_t n, uint64_t c, ScanShared& sh,
                                               ColScanShared& cx) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint64_t pool_n = cs.pool_n;
  const uint64_t g0 = c * kScanGroups + (uint64_t)warp * kScanWarpGroups;
  unsigned long long gsum = 0, gd = 0;
  bool guni = true;
  uint32_t big = 0;  // groups scanned in 64 bits (bit i: group g0 + i)
  constexpr int U = 4;
#pragma unroll 1
  for (uint32_t i0 = 0; i0 < kScanWarpGroups; i0 += U) {
    uint32_t len[U];
    uint64_t beg[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint64_t r = (g0 + i0 + u) * 32 + lane;
      len[u] = r < n ? __ldg(cs.len + r) : 0u;
      beg[u] = r < n ? __ldg(cs.beg + r) : 0ull;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint64_t r = (g0 + i0 + u) * 32 + lane;
      const bool bad = r < n && (beg[u] > pool_n || (uint64_t)len[u] > pool_n - beg[u]);
      if (bad) flag_error(MRN_EINVAL);
      unsigned long long excl, tot;
      if (__any_sync(0xffffffffu, len[u] >= (1u << 26))) {
        const unsigned long long x = warp_incl_scan_u64(len[u], lane);
        excl = x - len[u];
        tot = __shfl_sync(0xffffffffu, x, 31);
        big |= 1u << (i0 + u);
      } else {
        uint32_t x = len[u];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
          if (lane >= o) x += y;
        }
        excl = x - len[u];
        tot = __reduce_add_sync(0xffffffffu, len[u]);
      }
      cx.ex[warp][i0 + u][lane] = (uint32_t)excl;
      const unsigned long long d = beg[u] - excl;
      const unsigned int has = __ballot_sync(0xffffffffu, len[u] > 0);
      const unsigned long long d0 = __shfl_sync(0xffffffffu, d, has ? __ffs(has) - 1 : 0);
      const bool uni = __all_sync(0xffffffffu, !bad && (len[u] == 0 || d == d0));
      if ((uint32_t)lane == i0 + u) {
        gsum = tot;
        gd = d0;
        guni = uni;
      }
    }
  }
  const unsigned long long x = warp_incl_scan_u64(gsum, lane);
  if (lane == 31) sh.wsum[warp] = x;
  __syncthreads();
  unsigned long long agg = 0, wbase = 0;
#pragma unroll
  for (int w = 0; w < (int)(kScanThreads / 32); ++w) {
    const unsigned long long v = sh.wsum[w];
    if (w < warp) wbase += v;
    agg += v;
  }
  const bool publish = (long long)c != cs.skip_publish_tile;
  if (tid == 0 && publish) st_release_u64(&cs.state[c], (c == 0 ? MRN_TS_PREFIX : MRN_TS_AGG) | (agg & MRN_TS_VALUE));
  if (warp == 0) {
    unsigned long long prefix = 0;
    if (c > 0) {
      prefix = jagged_lookback(cs.timeout_ns, c, cs.state, lane);
      if (publish && lane == 0) st_release_u64(&cs.state[c], MRN_TS_PREFIX | ((prefix + agg) & MRN_TS_VALUE));
    }
    if (lane == 0) sh.base = prefix;
  }
  __syncthreads();
  const uint64_t g = g0 + lane;
  const bool have = g * 32 < n;
  const unsigned long long gb = sh.base + wbase + (x - gsum);  // lane i: group g0 + i's base
  bool bad = have && (!guni || (gsum > 0 && gd != gb));
  if (have && (n - 1) / 32 == g) {
    const unsigned long long total = gb + gsum;
    write_offset(cs.offsets, cs.off_size, n, total);
    if (cs.off_size == 4 && total > 0xffffffffull) flag_error(MRN_EOVERFLOW);
    if (total != pool_n) bad = true;
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicExch(cs.noncanon, 1u);
  // the offsets, group by group (the warp's own shared rows: no barrier)
  cx.gb[warp][lane] = gb;
  __syncwarp();
#pragma unroll 4
  for (uint32_t i = 0; i < kScanWarpGroups; ++i) {
    const uint64_t r = (g0 + i) * 32 + lane;
    if ((g0 + i) * 32 >= n) break;
    unsigned long long e = cx.ex[warp][i][lane];
    if ((big >> i) & 1u) {  // 64-bit group: scanned again
      const uint32_t len = r < n ? __ldg(cs.len + r) : 0u;
      e = warp_incl_scan_u64(len, lane) - len;
    }
    if (r < n) write_offset(cs.offsets, cs.off_size, r, cx.gb[warp][i] + e);
  }
}

// The grid covers cs.n entries; the count (read from device memory, where
// the level above wrote it) may be smaller, and the chunks past it return.
__global__ void __launch_bounds__(kScanThreads, 6) k_col_scan(const __grid_constant__ ColScan cs) {
  if (cs.only_if && ld_relaxed_u32(cs.only_if) == 0) return;
  __shared__ ScanShared sh;
  __shared__ ColScanShared cx;
  __shared__ unsigned int s_chunk;
  if (threadIdx.x == 0) s_chunk = atomicAdd(cs.counter, 1u);
  __syncthreads();
  const uint64_t c = s_chunk;
  const uint64_t n = cs.count ? min((uint64_t)ld_acquire_u64(cs.count), cs.n) : cs.n;
  if (n == 0) {  // no entries: the single offset, and a pool with records is not theirs
    if (c == 0 && threadIdx.x == 0) {
      write_offset(cs.offsets, cs.off_size, 0, 0);
      if (cs.pool_n != 0) atomicExch(cs.noncanon, 1u);
    }
    return;
  }
  if (c * MRN_SCAN_CHUNK >= n) return;
  col_scan_chunk(cs, n, c, sh, cx);
}

// The local form of a column-scanned level: a pool is canonical for the
// entries exactly when beg[0] = 0, beg[h] + len[h] = beg[h + 1] and the last
// entry's end is pool_n, and its offsets are then the begins.  Every entry
// writes its begin as its offset (the last also offsets[count] = pool_n),
// and a failed check sets *local_bad, on which the scan then runs and
// writes the offsets and the pool word as usual.  The grid covers cs.n
// entries, the count being read from device memory.
__global__ void __launch_bounds__(256) k_col_local(const __grid_constant__ ColScan cs) {
  const uint64_t n = cs.count ? min((uint64_t)ld_acquire_u64(cs.count), cs.n) : cs.n;
  const uint64_t step = (uint64_t)gridDim.x * blockDim.x;
  bool bad = false;
  uint64_t h = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  // four entries per thread and pass, their loads issued together
  constexpr int U = 4;
  for (; h + (U - 1) * step < n; h += U * step) {
    uint32_t len[U];
    unsigned long long beg[U], next[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint64_t e = h + u * step;
      len[u] = __ldg(cs.len + e);
      beg[u] = __ldg(cs.beg + e);
      next[u] = e + 1 < n ? __ldg(cs.beg + e + 1) : cs.pool_n;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint64_t e = h + u * step;
      bad |= beg[u] + len[u] != next[u] || (e == 0 && beg[u] != 0);
      write_offset(cs.offsets, cs.off_size, e, beg[u]);
      if (e + 1 == n) write_offset(cs.offsets, cs.off_size, n, cs.pool_n);
    }
  }
  for (; h < n; h += step) {
    const uint32_t len = __ldg(cs.len + h);
    const unsigned long long beg = __ldg(cs.beg + h);
    const unsigned long long next = h + 1 < n ? __ldg(cs.beg + h + 1) : cs.pool_n;
    bad |= beg + len != next || (h == 0 && beg != 0);
    write_offset(cs.offsets, cs.off_size, h, beg);
    if (h + 1 == n) write_offset(cs.offsets, cs.off_size, n, cs.pool_n);
  }
  if (n == 0 && blockIdx.x == 0 && threadIdx.x == 0) bad = true;  // the scan's own empty case
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicExch(cs.local_bad, 1u);
}

// The gathering form of a column-scanned level, for a pool that is not
// canonical (or whose conversion cannot be staged: `force`): every entry's
// children are copied one by one from the pool (`P`: the pool's records ->
// the level's columns) to the rows its offset gives.  Returns at once for
// a canonical pool.  Entries whose children lie outside the pool were
// recorded by the scan and are passed over; rows at or past `capacity`
// record MRN_ESIZE.
__global__ void __launch_bounds__(256) k_col_gather(const __grid_constant__ ColScan cs,
                                                    const __grid_constant__ ConvPlan P, unsigned long long capacity,
                                                    unsigned int force) {
  if (!force && ld_relaxed_u32(cs.noncanon) == 0) return;
  const uint64_t n = cs.count ? min((uint64_t)ld_acquire_u64(cs.count), cs.n) : cs.n;
  for (uint64_t h = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; h < n; h += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t len = __ldg(cs.len + h);
    const uint64_t beg = __ldg(cs.beg + h);
    if (beg > cs.pool_n || (uint64_t)len > cs.pool_n - beg) continue;
    const uint64_t row0 = read_offset(cs.offsets, cs.off_size, h);
    for (uint32_t k = 0; k < len; ++k) {
      const uint64_t row = row0 + k;
      if (row >= capacity) {
        flag_error(MRN_ESIZE);
        break;
      }
      const char* rec = P.src.base + (beg + k) * P.stride;
      for (uint32_t c = 0; c < P.naos; ++c) {
        const ColPlan cp = P.aos_cols[c];
        if (cp.fm < 0) continue;
        st_elem(P.dst.col[cp.fm] + row * cp.size, cp.size, ld_elem(rec + cp.aos_off, cp.size));
      }
    }
  }
}

// The split scan of one conversion: chunks handed out in increasing order,
// so that every chunk a look-back waits for is already running.
__global__ void __launch_bounds__(kScanThreads, 6) k_jag_scan_one(const __grid_constant__ JagPlan jp) {
  __shared__ ScanShared sh;
  __shared__ unsigned int s_chunk;
  if (threadIdx.x == 0) s_chunk = atomicAdd(jp.tile_counter, 1u);
  __syncthreads();
  jag_scan_chunk(jp, s_chunk, jp.chunk_state, sh);
}

// Offsets of the parents of a split jagged job, group by group (32
// parents, starting at a multiple of 32): offset_base + the group's base +
// the exclusive prefix of the lengths inside the group.  From staged tile
// `local` of R records (`stage`: the tile's AoS records; consumer warp w
// takes groups w, w + 8, w + 16 of it, their bases loaded together first),
// or from global memory.
constexpr int kJagTileGroups = 3;  // groups per consumer warp of a staged tile (T <= 768)
__device__ __forceinline__ void jag_offsets_staged(const JagPlan& jp, uint64_t local, uint32_t R, const char* stage,
                                                   const TileHdr& h, int lane, int warp) {
  const uint64_t r0 = local * h.T;
  unsigned long long gb[kJagTileGroups];
#pragma unroll
  for (int k = 0; k < kJagTileGroups; ++k) {
    const uint32_t q = (uint32_t)(warp + 8 * k) * 32;
    gb[k] = q < R ? __ldg(jp.group_base + (r0 + q) / 32) : 0ull;
  }
#pragma unroll
  for (int k = 0; k < kJagTileGroups; ++k) {
    const uint32_t q = (uint32_t)(warp + 8 * k) * 32;
    if (q >= R) break;
    const uint32_t len = *reinterpret_cast<const unsigned int*>(stage + (size_t)(q + lane) * h.stride + jp.len_off);
    const unsigned long long x = warp_incl_scan_u64(len, lane);
    write_offset(jp.offsets, jp.off_size, r0 + q + lane, jp.offset_base + gb[k] + x - len);
  }
}

__device__ __forceinline__ void jag_offsets_direct(const JagPlan& jp, uint64_t r0, uint64_t r1, int lane, int warp,
                                                   int nwarps) {
  const ConvPlan& P = jp.parent;
  if (r1 > P.n) r1 = P.n;
  for (uint64_t q = r0 + (uint64_t)warp * 32; q < r1; q += (uint64_t)nwarps * 32) {
    const uint64_t r = q + lane;
    const uint32_t len = r < r1 ? ld_u32_rec(P.src.base + r * P.stride + jp.len_off, P.vec) : 0u;
    const unsigned long long x = warp_incl_scan_u64(len, lane);
    const unsigned long long gbase = __ldg(jp.group_base + q / 32);
    if (r < r1) write_offset(jp.offsets, jp.off_size, r, jp.offset_base + gbase + x - len);
  }
}

// Parents of a JAG_LOCAL job (see JagPlan): offsets = offset_base + the
// begins, offsets[n] = offset_base + pool_n, and the local checks of the
// pool (begin[0] = 0, begin[r] + length[r] = begin[r + 1], the last parent's
// end = pool_n); a warp whose check failed sets the job's pool word (the
// pool launch skips the pool, the fall-back pass redoes the job).
__device__ __forceinline__ void jag_local_flag(const JagPlan& jp, bool bad, int lane) {
  if (__any_sync(0xffffffffu, bad) && lane == 0) {
    atomicExch(jp.noncanon, 1u);
    atomicExch(jp.any_noncanon, 1u);
  }
}

// From staged tile `local` of R records (`stage`: its AoS records; consumer
// warp w takes groups w, w + 8, w + 16): a lane's successor is the next
// lane's record, the group's last lane's the next group's first record (in
// the tile, else in global memory, else the pool's end).
__device__ __forceinline__ void jag_local_staged(const JagPlan& jp, uint64_t local, uint32_t R, const char* stage,
                                                 const TileHdr& h, int lane, int warp) {
  const ConvPlan& P = jp.parent;
  const uint64_t r0 = local * h.T, n = P.n;
  bool bad = false;
#pragma unroll 1
  for (int k = 0; k < kJagTileGroups; ++k) {
    const uint32_t q = (uint32_t)(warp + 8 * k) * 32;
    if (q >= R) break;
    const char* rec = stage + (size_t)(q + lane) * h.stride;
    const uint32_t len = *reinterpret_cast<const unsigned int*>(rec + jp.len_off);
    const unsigned long long beg = *reinterpret_cast<const unsigned long long*>(rec + jp.begin_off);
    unsigned long long next = __shfl_down_sync(0xffffffffu, beg, 1);
    const uint64_t r = r0 + q + lane;
    if (lane == 31) {
      if (q + 32 < R)
        next = *reinterpret_cast<const unsigned long long*>(stage + (size_t)(q + 32) * h.stride + jp.begin_off);
      else if (r + 1 < n)
        next = ld_u64_rec(P.src.base + (r + 1) * P.stride + jp.begin_off, P.vec);
      else
        next = jp.pool_n;
    }
    bad |= beg + len != next || (r == 0 && beg != 0);
    write_offset(jp.offsets, jp.off_size, r, jp.offset_base + beg);
    if (r + 1 == n) write_offset(jp.offsets, jp.off_size, n, jp.offset_base + jp.pool_n);
  }
  jag_local_flag(jp, bad, lane);
}

// The same for records [r0, r1) of a direct tile (from global memory).
__device__ __forceinline__ void jag_local_direct(const JagPlan& jp, uint64_t r0, uint64_t r1, int lane, int warp,
                                                 int nwarps) {
  const ConvPlan& P = jp.parent;
  const uint64_t n = P.n;
  if (r1 > n) r1 = n;
  bool bad = false;
  for (uint64_t r = r0 + (uint64_t)warp * 32 + lane; r < r1; r += (uint64_t)nwarps * 32) {
    const char* rec = P.src.base + r * P.stride;
    const uint32_t len = ld_u32_rec(rec + jp.len_off, P.vec);
    const unsigned long long beg = ld_u64_rec(rec + jp.begin_off, P.vec);
    const unsigned long long next = r + 1 < n ? ld_u64_rec(rec + P.stride + jp.begin_off, P.vec) : jp.pool_n;
    bad |= beg + len != next || (r == 0 && beg != 0);
    write_offset(jp.offsets, jp.off_size, r, jp.offset_base + beg);
    if (r + 1 == n) write_offset(jp.offsets, jp.off_size, n, jp.offset_base + jp.pool_n);
  }
  jag_local_flag(jp, bad, lane);
}

// One warp group of a jagged SoA -> AoS conversion: groups [0,
// parent_groups) build 32 parent records each (length and begin from the
// offsets), the following groups convert MRN_JAG_CHILD_GROUP of the m_src
// children each into the pool.
template <int VP, int VC, int W = MRN_WIN_WORDS, bool Ilp = false>
__device__ __forceinline__ void jagged_s2a_group(const JagPlan& jp, uint64_t w, uint64_t parent_groups,
                                                 uint32_t* tw, int lane) {
  if (w < parent_groups) {
    const ConvPlan& P = jp.parent;
    const uint64_t r = w * 32 + lane;
    const bool ok = r < P.n;
    uint64_t a = 0, b = 0;
    if (ok) {
      a = read_offset(jp.offsets, jp.off_size, r);
      b = read_offset(jp.offsets, jp.off_size, r + 1);
    }
    // Ilp: the offsets and the parent columns are all loaded before any is
    // used (the offsets are checked after the record is written).
    if constexpr (Ilp)
      fm_to_aos_lane_ilp<VP, W>(P, r, ok, P.dst.base + r * P.stride, tw, lane, (uint32_t)(b - a), a);
    else
      fm_to_aos_lane<VP, W>(P, r, ok, P.dst.base + r * P.stride, tw, lane, (uint32_t)(b - a), a);
    if (ok && (b < a || b - a > 0xffffffffull)) flag_error(MRN_EINVAL);
  } else {
    jagged_s2a_children<VC, W>(jp, (w - parent_groups) * MRN_JAG_CHILD_GROUP, tw, lane);
  }
}

template <int VP, int VC>
__global__ void __launch_bounds__(256) k_jagged_s2a(const __grid_constant__ JagPlan jp,
                                                    unsigned long long parent_groups) {
  extern __shared__ uint32_t smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t* tw = smem + warp * MRN_TW_WORDS_PER_WARP;
  const uint64_t wpb = blockDim.x >> 5;
  const uint64_t all = parent_groups + (jp.m_src + MRN_JAG_CHILD_GROUP - 1) / MRN_JAG_CHILD_GROUP;
  const uint64_t total_warps = (uint64_t)gridDim.x * wpb;
  for (uint64_t w = (uint64_t)blockIdx.x * wpb + warp; w < all; w += total_warps)
    jagged_s2a_group<VP, VC, MRN_WIN_WORDS, true>(jp, w, parent_groups, tw, lane);
}

// Sum of the jagged lengths of AoS parents.
__global__ void k_jagged_count(const char* base, uint64_t n, uint32_t stride, uint32_t len_off,
                               unsigned long long* total) {
  unsigned long long s = 0;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x)
    s += __ldg(reinterpret_cast<const unsigned int*>(base + i * stride + len_off));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0 && s) atomicAdd(total, s);
}

// The {length, begin} of every parent of a field-major jagged side, from
// its offsets (length = offsets[i+1] - offsets[i], begin = offsets[i]), as
// two columns: uint32 lengths and uint64 begins.  Decreasing offsets or a
// length beyond uint32 record MRN_EINVAL.
__global__ void k_len_begin(const char* offs, uint32_t osz, uint64_t n, unsigned int* len,
                            unsigned long long* beg) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t a = read_offset(offs, osz, i), b = read_offset(offs, osz, i + 1);
    if (b < a || b - a > 0xffffffffull) flag_error(MRN_EINVAL);
    len[i] = (unsigned int)(b - a);
    beg[i] = a;
  }
}

__global__ void k_write_offset0(char* offs, uint32_t osz, unsigned long long v) {
  write_offset(offs, osz, 0, v);
}

// ----------------------------------------------------------------- batched

// ----------------------------------------------------------------- batched
//
// Every job of a batch in one persistent, warp-specialized launch of 320
// threads per CTA.
//  - Warp 8 (loader) takes chunks of up to `chunk` consecutive global tiles
//    (fewer as the tiles run out) from an atomic tile counter (chunks are
//    handed out in increasing order), publishes
//    the child counts of the chunk's jagged tiles at once (so a jagged
//    tile's look-back waits only for chunks taken earlier), decides each
//    tile and issues the TMA loads of staged tiles up to kBNS stages ahead
//    (lane c loads SoA column c).
//  - Warps 0-7 (consumers) take the decided tiles in order.  A staged tile
//    is transformed shared -> shared, each warp on its own records; every
//    other tile (jagged, zero-fill, partial or unstaged conversions) runs
//    directly on global memory with a private scratch.
//  - Warp 9 (storer) writes each finished staged tile back with bulk stores
//    (lane c stores SoA column c) and frees its destination buffer once they
//    have read it.
// The warps meet only on mbarriers:
//   ready[i] / rel[i]   ring slot i written / read by all consumer warps
//   full[s] / empty[s]  source stage s loaded / read by all consumer warps
//   done[d] / dfree[d]  destination buffer d written / read by its stores
// Each stage carries its job's column descriptors, written by the loader
// before the stage's loads.  Every wait is bounded; on expiry the warp that
// saw it records MRN_ETIMEOUT and stops, and the others follow.
constexpr uint32_t kBStage = MRN_BATCH_STAGE_BYTES;
constexpr uint32_t kBNS = 3;      // source stages
constexpr uint32_t kBND = 2;      // destination buffers
constexpr uint32_t kRing = 8;     // decided tiles in flight
constexpr uint32_t kSQ = 8;       // staged tiles between loader and storer
constexpr uint64_t kChunk = 16;   // most consecutive tiles per chunk
constexpr uint32_t kBThreads = 320;
constexpr unsigned long long kSkipTile = ~0ull;

struct TileSlot {
  unsigned long long t;  // global tile; >= total_tiles: no more tiles
  unsigned long long local;  // kSkipTile: a tile of a job whose condition failed
  unsigned int job;
  unsigned int staged;  // records of a staged tile; 0: the tile runs directly
  unsigned int jag;     // 1: a tile of the parents of a split jagged job (offsets too)
  unsigned int pad;
};

// A stage's table in shared memory: the layout of StageRec, read as uint4.
struct StageDesc {
  TileHdr h;
  unsigned int pad[2];
  uint4 d[MRN_MAX_COLS];
};
static_assert(sizeof(StageDesc) == sizeof(StageRec), "a stage table is a StageRec");
static_assert(sizeof(StageDesc) % 16 == 0, "stage tables are whole bulk copies");

struct StoreItem {
  unsigned long long local;
  unsigned int job;
  unsigned int records;  // records of the tile (T, or fewer for a job's partial staged tile)
};

// Consumer scratch: 8 warps' lane words in 32-byte windows.
constexpr uint32_t kBWin = 8;
constexpr size_t kBTw = 8 * MRN_TW_WORDS(kBWin) * sizeof(uint32_t);
constexpr size_t kBScratch = (kBTw + 15) / 16 * 16;
constexpr size_t kBOffDst = (size_t)kBNS * kBStage;
constexpr size_t kBOffScratch = kBOffDst + (size_t)kBND * kBStage;
constexpr size_t kBOffDesc = kBOffScratch + kBScratch;
constexpr size_t kBOffBar = kBOffDesc + kBNS * sizeof(StageDesc);
constexpr size_t kBNumBars = 2 * kBNS + 2 * kBND + 2 * kRing;
constexpr size_t kBOffRing = kBOffBar + kBNumBars * 8;
constexpr size_t kBOffSQ = kBOffRing + kRing * sizeof(TileSlot);
constexpr size_t kBOffFlag = kBOffSQ + kSQ * sizeof(StoreItem);
constexpr size_t kBOffSJob = kBOffFlag + 16;
constexpr size_t kBatchSmem = kBOffSJob + 16;

struct BatchSmem {
  char* base;
  __device__ __forceinline__ char* src(uint32_t s) const { return base + (size_t)s * kBStage; }
  __device__ __forceinline__ char* dst(uint32_t d) const { return base + kBOffDst + (size_t)d * kBStage; }
  __device__ __forceinline__ uint32_t* scratch() const { return reinterpret_cast<uint32_t*>(base + kBOffScratch); }
  __device__ __forceinline__ StageDesc* desc(uint32_t s) const {
    return reinterpret_cast<StageDesc*>(base + kBOffDesc) + s;
  }
  __device__ __forceinline__ unsigned long long* bar(uint32_t i) const {
    return reinterpret_cast<unsigned long long*>(base + kBOffBar) + i;
  }
  __device__ __forceinline__ unsigned long long* full(uint32_t s) const { return bar(s); }
  __device__ __forceinline__ unsigned long long* empty(uint32_t s) const { return bar(kBNS + s); }
  __device__ __forceinline__ unsigned long long* done(uint32_t d) const { return bar(2 * kBNS + d); }
  __device__ __forceinline__ unsigned long long* dfree(uint32_t d) const { return bar(2 * kBNS + kBND + d); }
  __device__ __forceinline__ unsigned long long* ready(uint32_t i) const { return bar(2 * kBNS + 2 * kBND + i); }
  __device__ __forceinline__ unsigned long long* rel(uint32_t i) const {
    return bar(2 * kBNS + 2 * kBND + kRing + i);
  }
  __device__ __forceinline__ TileSlot* ring(uint32_t i) const {
    return reinterpret_cast<TileSlot*>(base + kBOffRing) + i;
  }
  __device__ __forceinline__ StoreItem* sq(uint32_t i) const {
    return reinterpret_cast<StoreItem*>(base + kBOffSQ) + i;
  }
  // [0] abort, [1] loader finished, [2] staged tiles issued in total,
  // [3] tiles decided so far (the storer's sign that the loader is alive)
  __device__ __forceinline__ volatile int* flags() const { return reinterpret_cast<volatile int*>(base + kBOffFlag); }
  // the job whose table each stage holds (the loader's own record)
  __device__ __forceinline__ unsigned int* sjob() const { return reinterpret_cast<unsigned int*>(base + kBOffSJob); }
};

__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Bytes of the first R records (a multiple of the staging granule) of a
// tile side whose full tile is `full` bytes.
__device__ __forceinline__ uint32_t side_tile_bytes(const ConvPlan& p, const SidePlan& sp, uint32_t full, uint32_t R) {
  if (R == p.tg.T) return full;
  if (sp.kind == K_AOS) return R * p.stride;
  if (sp.kind == K_AOSOA) return R / sp.block * (uint32_t)sp.block_bytes;
  return full / p.tg.T * R;  // SoA: T * (sum of storage columns' element bytes), packed
}

// Warp-wide bulk stores of the first R records of destination tile lt;
// every lane commits its own bulk group.
template <bool kInter>
__device__ __forceinline__ void tma_store_tile_warp(const ConvPlan& p, uint64_t lt, uint32_t R, const char* tile,
                                                    int lane) {
  const TileGeom& g = p.tg;
  const uint64_t t0 = lt * g.T;
  const SidePlan& sp = p.dst;
  const uint32_t bytes = side_tile_bytes(p, sp, g.dst_bytes, R);
  if (sp.kind == K_AOS) {
    if (lane == 0) bulk_s2g(sp.base + t0 * p.stride, tile, bytes);
  } else if (sp.kind == K_AOSOA) {
    if (lane == 0) bulk_s2g(sp.base + (t0 / sp.block) * sp.block_bytes, tile, bytes);
  } else if (kInter) {  // a range per storage column (an interleaved array's rows once)
    for (uint32_t c = lane; c < p.ncols; c += 32)
      if (!(g.col[c] & MRN_COL_SUB)) bulk_s2g(sp.col[c] + t0 * p.fm_es[c], tile + g.dst_off[c], R * p.fm_es[c]);
  } else {
    for (uint32_t c = lane; c < p.ncols; c += 32)
      bulk_s2g(sp.col[c] + t0 * p.fm_size[c], tile + g.dst_off[c], R * p.fm_size[c]);
  }
  bulk_commit();
}

// Loader warp, one conversion per launch: the plan's column descriptors and
// header into stage s's table (lane c writes column c), padding absorbed in
// widened field stores where the plan has them.
template <bool Inter>
__device__ __forceinline__ void fill_stage_desc(const ConvPlan& p, const BatchSmem& m, uint32_t s, int lane,
                                                bool wide) {
  StageDesc* sd = m.desc(s);
  for (uint32_t c = lane; c < p.ncols; c += 32) sd->d[c] = tile_desc<Inter>(p, c, wide);
  if (lane == 0) sd->h = tile_hdr<Inter>(p, wide);
}

static_assert(sizeof(BatchJob) % 16 == 0, "a job descriptor is one whole L2 prefetch");

// The job of tile t: the last job j >= cur with first_tile[j] <= t, given
// first_tile[cur] <= t (jobs without tiles are passed over).  Called by a
// whole warp: the next job is one load; a jump over many jobs is a 32-way
// search, each round one coalesced load of 32 tile starts, so a CTA's first
// chunk finds its job in one or two round trips instead of a chain.
__device__ __forceinline__ unsigned int advance_job(const unsigned long long* __restrict__ first_tile,
                                                    unsigned int njobs, unsigned int cur, uint64_t t,
                                                    int lane) {
  if (cur + 1 >= njobs || __ldg(first_tile + cur + 1) > t) return cur;
  unsigned int lo = cur + 1, hi = njobs;  // first_tile[lo] <= t < first_tile[hi]
  while (hi - lo > 1) {
    const unsigned int step = (hi - lo + 31) / 32;
    const unsigned int j = lo + (unsigned int)lane * step;
    const bool le = j < hi && __ldg(first_tile + j) <= t;
    const unsigned int mask = __ballot_sync(0xffffffffu, le);  // lane 0 (j = lo) is set
    const unsigned int k = 31u - (unsigned int)__clz(mask);
    lo += k * step;
    hi = min(hi, lo + step);
  }
  return lo;
}

// What the loader warp reads of its current job for every tile, kept in
// registers from one job switch to the next (a batch's job table is in
// global memory, and the plan fields of one tile are a chain of loads on
// the way to its bulk copies): the tile numbering and the source side, with
// lane c holding columns c and c + 32.
struct LoadCache {
  unsigned int job;
  bool staged_job;
  bool skip;  // the job converts a jagged pool that the scan found not canonical
  bool jag_parents;
  uint32_t T, rs, kind, ncols, stride, src_bytes, block;
  uint64_t tile_begin, nfull, block_bytes;
  const char* base;
  const char* col[2];
  uint32_t size[2], off[2];
};

__device__ __forceinline__ void load_cache(const BatchJob& J, unsigned int job, int lane, LoadCache* c,
                                           const unsigned int* conds) {
  const ConvPlan& P = J.jp.parent;
  c->job = job;
  c->skip = J.cond && conds && ld_relaxed_u32(conds + J.cond - 1) != 0;
  c->tile_begin = J.tile_begin;
  c->staged_job = (J.kind == JOB_CONVERT || J.kind == JOB_JAG_PARENTS) && P.tg.tma;
  c->jag_parents = J.kind == JOB_JAG_PARENTS;
  c->T = P.tg.T;
  const StagedTiles st = staged_tiles(P.n, 0, P.tg.T, P.tg.G);
  c->nfull = st.nfull;
  c->rs = (uint32_t)st.rs;
  c->kind = P.src.kind;
  c->ncols = P.ncols;
  c->stride = P.stride;
  c->src_bytes = P.tg.src_bytes;
  c->block = (uint32_t)P.src.block;
  c->block_bytes = P.src.block_bytes;
  c->base = P.src.base;
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const uint32_t col = (uint32_t)lane + 32u * k;
    // a range per storage column: an interleaved array's rows are loaded
    // with its first column
    const bool have = col < P.ncols && P.src.kind == K_SOA && !(P.tg.col[col] & MRN_COL_SUB);
    c->col[k] = have ? P.src.col[col] : nullptr;
    c->size[k] = have ? P.fm_es[col] : 0u;
    c->off[k] = have ? P.tg.src_off[col] : 0u;
  }
}

// Warp-wide bulk loads of the first R records of source tile lt, from the
// cached fields: lane 0 sets the transaction count, then lane c copies SoA
// columns c and c + 32 (lane 0 copies an AoS / AoSoA tile, which is one
// range).  With `rec`, lane 0 also copies that stage table into `table` on
// the same barrier.
__device__ __forceinline__ void tma_load_tile_cached(const LoadCache& c, uint64_t lt, uint32_t R, char* stage,
                                                     unsigned long long* bar, int lane, const StageRec* rec,
                                                     StageDesc* table) {
  const uint64_t t0 = lt * c.T;
  uint32_t bytes;
  if (R == c.T) bytes = c.src_bytes;
  else if (c.kind == K_AOS) bytes = R * c.stride;
  else if (c.kind == K_AOSOA) bytes = R / c.block * (uint32_t)c.block_bytes;
  else bytes = c.src_bytes / c.T * R;
  if (lane == 0) {
    mbar_expect_tx(bar, bytes + (rec ? (uint32_t)sizeof(StageRec) : 0u));
    if (rec) bulk_g2s(table, rec, (uint32_t)sizeof(StageRec), bar);
  }
  __syncwarp();
  if (c.kind == K_AOS) {
    if (lane == 0) bulk_g2s(stage, c.base + t0 * c.stride, bytes, bar);
  } else if (c.kind == K_AOSOA) {
    if (lane == 0) bulk_g2s(stage, c.base + (t0 / c.block) * c.block_bytes, bytes, bar);
  } else {
#pragma unroll
    for (int k = 0; k < 2; ++k)
      if (c.col[k]) bulk_g2s(stage + c.off[k], c.col[k] + t0 * c.size[k], R * c.size[k], bar);
  }
}

// The loader's decision for a tile of the cached job: skipped (a pool that
// is not canonical), or staged with its records, or direct.
__device__ __forceinline__ void decide_tile(const LoadCache& lc, TileSlot* cand) {
  if (lc.skip)
    cand->local = kSkipTile;
  else if (lc.staged_job)
    cand->staged = cand->local < lc.nfull ? lc.T : (cand->local == lc.nfull ? lc.rs : 0u);
}

// Loader warp: decides tiles in order (lane 0 decides, the warp follows)
// and issues the loads of staged ones; returns after publishing the
// end-of-work slot, or on abort once its loads in flight have landed.
template <bool kStatic, bool kWide, bool kInter>
__device__ __forceinline__ void batch_loader(const BatchJob* __restrict__ jobs,
                                             const unsigned long long* __restrict__ first_tile,
                                             unsigned int njobs, unsigned long long total_tiles,
                                             unsigned int* counter,
                                             uint32_t chunk, unsigned int first_start, unsigned int first_size,
                                             const BatchSmem& m, int lane, const unsigned int* conds) {
  uint64_t k_issue = 0;  // tiles decided
  uint32_t c_issue = 0;  // staged tiles loaded
  unsigned int cursor = 0;
  uint64_t next_t = 0, chunk_end = 0;
  uint32_t n_chunks = 0;  // static assignment: chunks taken so far
  uint64_t seen = 0;      // dynamic assignment: end of the last chunk taken
  uint64_t snap = 0;      // the counter, read while deciding a chunk's last tile
  LoadCache lc;           // the fields of job lc.job the loader reads per tile
  lc.job = 0xffffffffu;
  bool have = false;
  TileSlot cand;
  cand.t = 0;
  unsigned long long idle_since = global_ns();
  for (;;) {
    if (m.flags()[0]) break;
    if (!have) {
      if (next_t == chunk_end) {
        if (kStatic && !counter) {
          next_t = ((uint64_t)n_chunks * gridDim.x + blockIdx.x) * chunk;
          ++n_chunks;
          chunk_end = next_t + chunk;
        } else {
          // guided chunks: up to `chunk` tiles, fewer as the tiles run out
          // (the remaining tiles' share per CTA), so the CTAs finish
          // together; the counter counts tiles, handed out in increasing
          // order.  The remaining tiles are judged by the counter as it
          // stood when the last chunk's last tile was decided: this CTA's
          // own last chunk says little about the others'.
          unsigned int start = 0, size = 0;
          if (lane == 0 && first_size) {  // taken at entry (lane 0's values)
            start = first_start;
            size = first_size;
            first_size = 0;
          } else if (lane == 0) {
            seen = max(seen, snap);
            const unsigned long long rem = total_tiles > seen ? total_tiles - seen : 0ull;
            const unsigned long long share = rem / (1ull * gridDim.x);
            size = (unsigned int)(share < 1ull ? 1ull : (share > chunk ? (unsigned long long)chunk : share));
            start = atomicAdd(counter, size);
          }
          next_t = __shfl_sync(0xffffffffu, start, 0);
          chunk_end = next_t + __shfl_sync(0xffffffffu, size, 0);
          seen = chunk_end;
        }
      }
      // read early, so that the load's latency hides behind this tile's
      // stage wait
      if (counter && lane == 0 && next_t + 1 == chunk_end) snap = ld_relaxed_u32(counter);
      cand.t = next_t++;
      cand.staged = 0;
      cand.job = 0;
      cand.local = 0;
      cand.jag = 0;
      if (cand.t < total_tiles) {
        if constexpr (!kStatic) cursor = advance_job(first_tile, njobs, cursor, cand.t, lane);
        if (cursor != lc.job) load_cache(jobs[cursor], cursor, lane, &lc, conds);
        cand.job = cursor;
        cand.local = cand.t - lc.tile_begin;
        cand.jag = lc.jag_parents ? 1u : 0u;
        decide_tile(lc, &cand);
      }
      have = true;
    }
    const uint32_t slot = k_issue % kRing;
    const uint32_t s = c_issue % kBNS;
    int go = 0;
    if (lane == 0) {
      go = k_issue < kRing || mbar_try_wait(m.rel(slot), (uint32_t)(((k_issue / kRing) - 1) & 1));
      if (go && cand.staged && c_issue >= kBNS) go = mbar_try_wait(m.empty(s), ((c_issue / kBNS) - 1) & 1);
    }
    go = __shfl_sync(0xffffffffu, go, 0);
    if (go) {
      if (cand.staged) {
        const ConvPlan& P = jobs[cand.job].jp.parent;
        if (lane == 0) {
          StoreItem it;
          it.local = cand.local;
          it.job = cand.job;
          it.records = cand.staged;
          *m.sq(c_issue % kSQ) = it;
        }
        // the stage's table changes with the job: one conversion's is
        // written in place (first use of each stage), a batch job's comes
        // from its record with the tile's data
        const StageRec* rec = nullptr;
        if (m.sjob()[s] != cand.job) {
          if constexpr (kStatic)
            fill_stage_desc<kInter>(P, m, s, lane, kWide);
          else
            rec = &jobs[cand.job].stage;
          __syncwarp();
          if (lane == 0) m.sjob()[s] = cand.job;
        }
        __syncwarp();
        tma_load_tile_cached(lc, cand.local, cand.staged, m.src(s), m.full(s), lane, rec, m.desc(s));
        ++c_issue;
      }
      if (lane == 0) {
        *m.ring(slot) = cand;
        if (cand.t >= total_tiles) {
          m.flags()[2] = (int)c_issue;
          __threadfence_block();
          m.flags()[1] = 1;
        }
        mbar_arrive(m.ready(slot));
        m.flags()[3] = (int)(k_issue + 1);
      }
      ++k_issue;
      have = false;
      if (cand.t >= total_tiles) return;
      idle_since = global_ns();
    } else {
      int late = global_ns() - idle_since > 2000000000ull;
      late = __shfl_sync(0xffffffffu, late, 0);
      if (late) {
        if (lane == 0) {
          flag_error(MRN_ETIMEOUT);
          m.flags()[0] = 1;
        }
        break;
      }
      __nanosleep(20);
    }
  }
  // aborted: the most recent loads land before the CTA may exit (bounded)
  if (lane == 0)
    for (uint32_t q = (c_issue > kBNS ? c_issue - kBNS : 0); q < c_issue; ++q)
      mbar_wait_bounded(m.full(q % kBNS), (q / kBNS) & 1);
}

// Storer warp: stores staged tiles in order as the consumers finish them
// (lane c stores SoA column c); each destination buffer is freed once its
// stores have read it.
template <bool kInter>
__device__ __forceinline__ void batch_storer(const BatchJob* __restrict__ jobs, const BatchSmem& m, int lane) {
  uint32_t c = 0;
  int seen = 0;
  unsigned long long idle_since = global_ns();
  for (;;) {
    if (m.flags()[0]) break;
    const uint32_t d = c % kBND;
    int ready = 0;
    if (lane == 0) ready = mbar_try_wait(m.done(d), (c / kBND) & 1);
    ready = __shfl_sync(0xffffffffu, ready, 0);
    if (ready) {
      __syncwarp();  // orders lane 0's acquire before the other lanes' stores
      const StoreItem it = *m.sq(c % kSQ);
      tma_store_tile_warp<kInter>(jobs[it.job].jp.parent, it.local, it.records, m.dst(d), lane);
      bulk_wait_read<0>();
      __syncwarp();
      if (lane == 0) mbar_arrive(m.dfree(d));
      ++c;
      idle_since = global_ns();
      continue;
    }
    int stop = 0, late = 0;
    if (lane == 0) {
      if (m.flags()[1]) {
        __threadfence_block();
        stop = (int)c >= m.flags()[2];  // every staged tile is stored
      }
      const int decided = m.flags()[3];
      if (decided != seen) {
        seen = decided;
        idle_since = global_ns();
      }
      late = global_ns() - idle_since > 4000000000ull;
      if (late && !stop) {
        flag_error(MRN_ETIMEOUT);
        m.flags()[0] = 1;
      }
    }
    stop = __shfl_sync(0xffffffffu, stop | late, 0);
    if (stop) break;
    __nanosleep(20);
  }
  bulk_wait_all();
}

// kJag: the parents jobs of split jagged conversions the instance meets,
// whose offsets epilogue it compiles in: 1 those of JAG_SPLIT (single
// conversions: offsets from the scan's group bases), 2 those of JAG_LOCAL
// (batches: offsets from the begins, and the pool's check), 0 none.  Where
// an epilogue cannot occur, leaving it out keeps the transform's register
// allocation (single points AoS -> SoA at 2^26 records 0.718 ms with the
// first, 0.672 without; the batch 0.6% slower with both than with its one).
template <bool kStatic, bool kWide, int kJag, bool kInter>
__device__ __forceinline__ void batch_main(const BatchJob* __restrict__ jobs,
                                           const unsigned long long* __restrict__ first_tile, unsigned int njobs,
                                           unsigned long long total_tiles, unsigned int* counter,
                                           uint32_t chunk, char* batch_smem, const unsigned int* conds) {
  BatchSmem m{batch_smem};
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if constexpr (!kStatic) {
    // the first tiles' job descriptors and the job index are read in a
    // chain of dependent loads: bring them into L2 while the CTA starts
    // (CTA b fetches job b; CTA 0 the tile index of the jobs)
    if (warp == 9 && lane == 0) {
      if (blockIdx.x < njobs) bulk_prefetch_l2(jobs + blockIdx.x, (uint32_t)sizeof(BatchJob));
      if (blockIdx.x == 0)
        for (uint32_t q = 0; q < njobs; q += 2048)
          bulk_prefetch_l2(first_tile + q, (min(njobs - q, 2048u) * 8 + 15) & ~15u);
    }
  }
  // warp 0 initializes the barriers, one per lane
  if (warp == 0) {
    constexpr uint32_t kBars = (uint32_t)kBNumBars;
    static_assert(kBars <= 32, "one barrier per lane");
    if ((uint32_t)lane < kBars) {
      const uint32_t i = lane;
      uint32_t count;
      if (i < kBNS) count = 1;                                  // full
      else if (i < 2 * kBNS) count = 8;                         // empty
      else if (i < 2 * kBNS + kBND) count = 8;                  // done
      else if (i < 2 * kBNS + 2 * kBND) count = 1;              // dfree
      else if (i < 2 * kBNS + 2 * kBND + kRing) count = 1;      // ready
      else count = 8;                                           // rel
      mbar_init(m.bar(i), count);
      fence_mbar_init();
    }
    if ((uint32_t)lane < kBNS) m.sjob()[lane] = 0xffffffffu;
    if (lane < 4) m.flags()[lane] = 0;
  }
  // the loader takes its first chunk now, so that the atomic's round trip
  // overlaps the barrier set-up
  unsigned int first_start = 0, first_size = 0;
  if (warp == 8 && lane == 0 && counter) {
    const unsigned long long share = total_tiles / gridDim.x;
    first_size = (unsigned int)(share < 1ull ? 1ull : (share > chunk ? (unsigned long long)chunk : share));
    first_start = atomicAdd(counter, first_size);
  }
  __syncthreads();
  if (warp == 8) {
    batch_loader<kStatic, kWide, kInter>(jobs, first_tile, njobs, total_tiles, counter, chunk, first_start, first_size, m,
                                 lane, conds);
    return;
  }
  if (warp == 9) {
    batch_storer<kInter>(jobs, m, lane);
    return;
  }
  // consumers
  uint32_t* scratch = m.scratch();
  uint32_t* tw = scratch + warp * MRN_TW_WORDS(kBWin);
  bool ok = true;
  uint32_t c = 0;  // staged tiles consumed
  for (uint64_t k = 0;; ++k) {
    const uint32_t slot = k % kRing;
    if (!mbar_wait_bounded(m.ready(slot), (uint32_t)((k / kRing) & 1))) ok = false;
    const TileSlot ts = *m.ring(slot);
    __syncwarp();
    if (lane == 0) mbar_arrive(m.rel(slot));
    if (!ok || m.flags()[0]) break;
    if (ts.staged) {
      const uint32_t s = c % kBNS, d = c % kBND;
      if (!mbar_wait_bounded(m.full(s), (c / kBNS) & 1) ||
          (c >= kBND && !mbar_wait_bounded(m.dfree(d), ((c / kBND) - 1) & 1))) {
        ok = false;
        break;
      }
      const StageDesc* sd = m.desc(s);
      tma_transform<kWide, kStatic, kInter>(sd->h, smem_u32(sd->d), m.src(s), m.dst(d), ts.staged, lane, warp);
      // parents of a split jagged job: the offsets, from the staged lengths
      // (or, with the local check, begins) before the source stage is released
      if (kJag == 1 && ts.jag) jag_offsets_staged(jobs[ts.job].jp, ts.local, ts.staged, m.src(s), sd->h, lane, warp);
      if (kJag == 2 && ts.jag) jag_local_staged(jobs[ts.job].jp, ts.local, ts.staged, m.src(s), sd->h, lane, warp);
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(m.empty(s));
        mbar_arrive(m.done(d));
      }
      ++c;
    } else {
      if (ts.t >= total_tiles) break;
      if (ts.local == kSkipTile) continue;
      const BatchJob& J = jobs[ts.job];
      const unsigned long long local = ts.local;
      if (J.kind == JOB_CONVERT || J.kind == JOB_JAG_PARENTS) {
        const ConvPlan& P = J.jp.parent;
        uint64_t r0, r1;
        if (P.tg.tma) {  // the records after a staged job's staged tiles
          r0 = staged_tiles(P.n, 0, P.tg.T, P.tg.G).d0;
          r1 = ~0ull;
        } else {
          r0 = local * J.tile_records;
          r1 = r0 + J.tile_records;
        }
        conv_range<0, kBWin>(P, r0, r1, tw, lane, warp, 8);
        if (kJag == 1 && J.kind == JOB_JAG_PARENTS) jag_offsets_direct(J.jp, r0, r1, lane, warp, 8);
        if (kJag == 2 && J.kind == JOB_JAG_PARENTS) jag_local_direct(J.jp, r0, r1, lane, warp, 8);
      } else if (J.kind == JOB_JAG_S2A) {
        jagged_s2a_group<0, 0, kBWin>(J.jp, local * 8 + warp, J.parent_groups, tw, lane);
      } else {
        const uint64_t q = local * 256 + tid;
        if (q < J.gp.nblocks * J.gp.ngaps) zero_gap_item(J.gp, q);
      }
    }
  }
  if (!ok) {
    if (lane == 0) flag_error(MRN_ETIMEOUT);
    m.flags()[0] = 1;
  }
}

// Batched conversions: tiles handed out dynamically in increasing order.
// A job with a condition (cond > 0) is skipped when conds[cond - 1] != 0.
__global__ void __launch_bounds__(kBThreads, 3) k_batch(const BatchJob* __restrict__ jobs,
                                                        const unsigned long long* __restrict__ first_tile,
                                                        unsigned int njobs, unsigned long long total_tiles,
                                                        unsigned int* counter, uint32_t chunk,
                                                        const unsigned int* conds) {
  extern __shared__ __align__(128) char batch_smem[];
  batch_main<false, false, 2, false>(jobs, first_tile, njobs, total_tiles, counter, chunk, batch_smem, conds);
}

// One staged conversion through the same warp-specialized pipeline: the
// job travels as a kernel parameter (it has no jagged tiles).  Without a
// counter, chunk c of tiles belongs to CTA c % gridDim.x; with one (a
// zeroed word), chunks are guided as in a batch, so that CTAs that run
// faster take more of them.  kWide: the instance for conversions whose
// plan stores fields wider over an AoS destination's padding.
// With `cond`, the launch does nothing when *cond != 0 (the child pool of a
// split jagged conversion that the scan found not canonical).  kJag: the
// instance for the parents job of a split jagged conversion (1: the scan
// form's, JAG_SPLIT; 2: the local check's, JAG_LOCAL).  kInter: the
// instance for plans with an interleaved array.
template <bool kWide, int kJag, bool kInter>
__global__ void __launch_bounds__(kBThreads, 3) k_convert_ws(const __grid_constant__ BatchJob job,
                                                             uint32_t chunk, unsigned int* counter,
                                                             const unsigned int* cond) {
  if (cond && ld_relaxed_u32(cond) != 0) return;
  extern __shared__ __align__(128) char batch_smem[];
  batch_main<true, kWide, kJag, kInter>(&job, nullptr, 1u, job.ntiles, counter, chunk, batch_smem, nullptr);
}

// ================================================================== host

namespace mrn {

namespace {

std::mutex g_mu;
int g_sm_count = 0;

constexpr size_t kConvSmem = 8 * MRN_TW_WORDS_PER_WARP * sizeof(uint32_t);

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return MRN_OK;
  if (e == cudaErrorMemoryAllocation) return MRN_ENOMEM;
  return MRN_ECUDA;
}

void* conv_kernel(uint32_t vec) {
  switch (vec) {
    case 16: return reinterpret_cast<void*>(&k_convert<16>);
    case 8: return reinterpret_cast<void*>(&k_convert<8>);
    case 4: return reinterpret_cast<void*>(&k_convert<4>);
    case 2: return reinterpret_cast<void*>(&k_convert<2>);
    default: return reinterpret_cast<void*>(&k_convert<1>);
  }
}

// Resident CTAs per SM of a kernel (cached per kernel and shape).
int occupancy(const void* fn, int threads, size_t smem) {
  static std::mutex mu;
  static std::vector<std::tuple<const void*, int, size_t, int>> cache;
  std::lock_guard<std::mutex> lk(mu);
  for (auto& e : cache)
    if (std::get<0>(e) == fn && std::get<1>(e) == threads && std::get<2>(e) == smem) return std::get<3>(e);
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, threads, smem) != cudaSuccess || n < 1) n = 1;
  cache.emplace_back(fn, threads, smem, n);
  return n;
}

}  // namespace

// Scratch of the library's calls: stream-ordered allocations from a memory
// pool the library owns, one per device.  The device's default pool
// returns its free memory at every synchronisation, and a call whose
// scratch must be mapped again then spends longer on the host than its
// kernels take at small sizes (and, for the half-gigabyte scratch of a
// 2,097,152-parent nested conversion, about 0.4 ms of a 0.8 ms call).  So
// the pool keeps reserved between calls the most its calls have held at
// once: its release threshold starts at kScratchKeepBytes and follows
// that high-water mark up to 1/64 of the device's memory (at most
// kScratchKeepMax); mrn_scratch_release returns it.  Under stream capture
// the allocation is an ordinary cudaMallocAsync.
namespace {
constexpr uint64_t kScratchKeepBytes = 256ull << 20;
constexpr uint64_t kScratchKeepMax = 4ull << 30;
std::mutex g_pool_mu;
cudaMemPool_t g_pools[64] = {};
uint64_t g_pool_keep[64] = {};  // current release threshold
uint64_t g_pool_cap[64] = {};   // its bound on this device

cudaMemPool_t scratch_pool(int dev) {
  if (dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (!g_pools[dev]) {
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    uint64_t keep = kScratchKeepBytes;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    cudaDeviceProp prop;
    const uint64_t total = cudaGetDeviceProperties(&prop, dev) == cudaSuccess ? (uint64_t)prop.totalGlobalMem : 0ull;
    cudaGetLastError();
    g_pool_cap[dev] = std::max<uint64_t>(kScratchKeepBytes, std::min<uint64_t>(kScratchKeepMax, total / 64));
    g_pool_keep[dev] = keep;
    g_pools[dev] = pool;
  }
  return g_pools[dev];
}

// Raises device dev's release threshold to the memory its pool has in use
// now (in 2 MiB steps, within the bound).
void keep_in_use(cudaMemPool_t pool, int dev) {
  uint64_t used = 0;
  if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (used <= g_pool_keep[dev] || g_pool_keep[dev] >= g_pool_cap[dev]) return;
  const uint64_t step = 2ull << 20;
  uint64_t keep = std::min<uint64_t>(g_pool_cap[dev], (used + step - 1) / step * step);
  if (cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep) == cudaSuccess) g_pool_keep[dev] = keep;
  cudaGetLastError();
}
}  // namespace

int scratch_alloc(void** p, size_t bytes, void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  *p = nullptr;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  int dev = -1;
  cudaMemPool_t pool = nullptr;
  if (cudaStreamIsCapturing(s, &cap) == cudaSuccess && cap == cudaStreamCaptureStatusNone &&
      cudaStreamGetDevice(s, &dev) == cudaSuccess)
    pool = scratch_pool(dev);
  cudaGetLastError();
  const cudaError_t e = pool ? cudaMallocFromPoolAsync(p, bytes, pool, s) : cudaMallocAsync(p, bytes, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return MRN_ENOMEM;
  }
  if (pool && bytes > kScratchKeepBytes / 4) keep_in_use(pool, dev);
  return MRN_OK;
}

int scratch_release(int dev) {
  if (dev < 0 || dev >= 64) return MRN_EINVAL;
  std::lock_guard<std::mutex> lk(g_pool_mu);
  cudaMemPool_t pool = g_pools[dev];
  if (!pool) return MRN_OK;
  uint64_t keep = kScratchKeepBytes;
  if (cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess ||
      cudaMemPoolTrimTo(pool, 0) != cudaSuccess) {
    cudaGetLastError();
    return MRN_ECUDA;
  }
  g_pool_keep[dev] = keep;
  return MRN_OK;
}

void scratch_free(void* p, void* stream) {
  if (p) cudaFreeAsync(p, static_cast<cudaStream_t>(stream));
}

int device_sm_count() {
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_sm_count == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&g_sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      g_sm_count = 1;
  }
  return g_sm_count;
}

int status_from_bits(uint32_t bits) {
  static const int order[] = {MRN_ETIMEOUT, MRN_EOVERFLOW, MRN_EINVAL, MRN_ESIZE, MRN_EALIGN, MRN_ECUDA};
  for (int c : order)
    if (bits & (1u << c)) return c;
  return MRN_OK;
}

int read_and_clear_status(void* stream, uint32_t* bits) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return MRN_ECUDA;
  unsigned int v = 0, zero = 0;
  e = cudaMemcpyFromSymbolAsync(&v, g_mrn_status_bits, sizeof(v), 0, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess)
    e = cudaMemcpyToSymbolAsync(g_mrn_status_bits, &zero, sizeof(zero), 0, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return MRN_ECUDA;
  *bits = v;
  return MRN_OK;
}

// Opts a kernel into the batch pipeline's dynamic shared memory, once per
// kernel and device.
void allow_batch_smem(const void* fn) {
  static std::mutex mu;
  static std::vector<std::pair<const void*, int>> done;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  for (const auto& f : done)
    if (f.first == fn && f.second == dev) return;
  cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBatchSmem);
  done.emplace_back(fn, dev);
}

// Tiles per CTA from which a single staged conversion takes guided chunks.
constexpr uint64_t kDynamicTilesPerCta = 32;

// Tiles per chunk by default: up to 8 (fewer job switches per CTA), but
// small enough that every CTA of the grid gets about four chunks.
uint32_t chunk_for(uint64_t tiles, uint64_t ctas) {
  return (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(8, tiles / (4 * std::max<uint64_t>(1, ctas))));
}

// One staged job (JOB_CONVERT or JOB_JAG_PARENTS, plan in job.jp.parent)
// through the warp-specialized pipeline of the batch kernel.
int launch_staged_job(BatchJob& job, void* stream, const LaunchShape& sh, const unsigned int* cond) {
  const ConvPlan& p = job.jp.parent;
  const uint64_t nrec = p.dir == DIR_FM_AOS ? p.n : p.n_fm_pad;
  {
    job.tile_records = p.tg.T;
    job.ntiles = staged_tile_count(p.n, nrec, p.tg.T, p.tg.G);
    // the instance with the widened-field transform only for plans that
    // have widened fields: the branch costs the others a few percent
    const void* fn =
        job.kind == JOB_JAG_PARENTS
            ? (job.jp.mode == JAG_LOCAL ? reinterpret_cast<const void*>(&k_convert_ws<false, 2, false>)
                                        : reinterpret_cast<const void*>(&k_convert_ws<false, 1, false>))
        : p.tg.inter ? (p.dst.kind == K_AOS && p.tg.nwide ? reinterpret_cast<const void*>(&k_convert_ws<true, 0, true>)
                                                          : reinterpret_cast<const void*>(&k_convert_ws<false, 0, true>))
        : p.dst.kind == K_AOS && p.tg.nwide ? reinterpret_cast<const void*>(&k_convert_ws<true, 0, false>)
                                            : reinterpret_cast<const void*>(&k_convert_ws<false, 0, false>);
    allow_batch_smem(fn);
    const int occ = occupancy(fn, kBThreads, kBatchSmem);
    const int per_sm = sh.ctas_per_sm ? std::min((int)sh.ctas_per_sm, occ) : occ;
    const uint64_t cap = (uint64_t)device_sm_count() * (uint64_t)per_sm;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    uint32_t chunk = chunk_for(job.ntiles, cap);
    unsigned int* counter = nullptr;
    // Large conversions take guided chunks from a counter: CTAs do not all
    // run at the same speed, and a static split leaves the fast ones idle
    // at the end.  The counter costs an allocation and a memset, which
    // conversions of fewer than kDynamicTilesPerCta tiles per CTA do not
    // earn back.
    if (job.ntiles >= kDynamicTilesPerCta * cap) {
      if (scratch_alloc(reinterpret_cast<void**>(&counter), 256, st) != MRN_OK) {
        counter = nullptr;
      } else if (cudaMemsetAsync(counter, 0, sizeof(unsigned int), st) != cudaSuccess) {
        scratch_free(counter, st);
        return MRN_ECUDA;
      } else {
        chunk = (uint32_t)kChunk;
      }
    }
    const uint64_t chunks = (job.ntiles + chunk - 1) / chunk;
    const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(chunks, cap));
    void* args[] = {&job, &chunk, &counter, &cond};
    const int rc = cuda_status(cudaLaunchKernel(fn, dim3(grid), dim3(kBThreads), args, kBatchSmem, st));
    if (counter) scratch_free(counter, st);
    return rc;
  }
}

int launch_convert(const ConvPlan& p, void* stream, const LaunchShape* shape, const unsigned int* cond) {
  const uint64_t nrec = p.dir == DIR_FM_AOS ? p.n : p.n_fm_pad;
  if (nrec == 0) return MRN_OK;
  LaunchShape sh = shape ? *shape : LaunchShape{};
  if (p.tg.tma && !sh.generic) {
    BatchJob job;
    std::memset(&job, 0, sizeof(job));
    job.kind = JOB_CONVERT;
    job.jp.parent = p;
    return launch_staged_job(job, stream, sh, cond);
  }
  if (cond) return MRN_EINVAL;  // only staged launches take a condition
  if (sh.threads != 64 && sh.threads != 128 && sh.threads != 256) sh.threads = 256;
  if (sh.tile_records == 0 || sh.tile_records % 32) sh.tile_records = sh.threads * 2;
  void* fn = conv_kernel(p.dir == DIR_FM_FM ? 1 : p.vec);
  const size_t smem = (sh.threads / 32) * MRN_TW_WORDS_PER_WARP * sizeof(uint32_t);
  const int occ = occupancy(fn, (int)sh.threads, smem);
  const int per_sm = sh.ctas_per_sm ? std::min((int)sh.ctas_per_sm, occ) : occ;
  const uint64_t need = (nrec + sh.tile_records - 1) / sh.tile_records;
  const uint64_t cap = (uint64_t)device_sm_count() * (uint64_t)per_sm;
  const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min(need, cap));
  uint32_t tr = sh.tile_records;
  void* args[] = {const_cast<ConvPlan*>(&p), &tr};
  cudaError_t e = cudaLaunchKernel(fn, dim3(grid), dim3(sh.threads), args, smem,
                                   static_cast<cudaStream_t>(stream));
  return cuda_status(e);
}

int launch_zero_gaps(const GapPlan& g, void* stream) {
  const uint64_t total = g.nblocks * g.ngaps;
  if (total == 0) return MRN_OK;
  const unsigned grid = (unsigned)std::min<uint64_t>((total + 255) / 256, 4096);
  k_zero_gaps<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(g);
  return cuda_status(cudaGetLastError());
}

void fill_stage_rec(const ConvPlan& p, StageRec* out) {
  std::memset(out, 0, sizeof(*out));
  out->h = tile_hdr<false>(p);  // batches stage no plan with an interleaved array
  for (uint32_t c = 0; c < p.ncols; ++c) {
    const uint4 d = tile_desc<false>(p, c);
    out->d[c][0] = d.x;
    out->d[c][1] = d.y;
    out->d[c][2] = d.z;
    out->d[c][3] = d.w;
  }
}

uint64_t jagged_scratch_bytes(uint64_t n, uint32_t tile) {
  const uint64_t ntiles = (n + tile - 1) / tile;
  return 256 + ntiles * sizeof(unsigned long long);
}

namespace {
template <int VP, int VC>
void* jag_a2s_ptr() { return reinterpret_cast<void*>(&k_jagged_a2s<VP, VC>); }
template <int VP>
void* jag_a2s_for(uint32_t vc) {
  switch (vc) {
    case 16: return jag_a2s_ptr<VP, 16>();
    case 8: return jag_a2s_ptr<VP, 8>();
    case 4: return jag_a2s_ptr<VP, 4>();
    case 2: return jag_a2s_ptr<VP, 2>();
    default: return jag_a2s_ptr<VP, 1>();
  }
}
void* jag_a2s(uint32_t vp, uint32_t vc) {
  switch (vp) {
    case 16: return jag_a2s_for<16>(vc);
    case 8: return jag_a2s_for<8>(vc);
    case 4: return jag_a2s_for<4>(vc);
    case 2: return jag_a2s_for<2>(vc);
    default: return jag_a2s_for<1>(vc);
  }
}
template <int VP, int VC>
void* jag_s2a_ptr() { return reinterpret_cast<void*>(&k_jagged_s2a<VP, VC>); }
template <int VP>
void* jag_s2a_for(uint32_t vc) {
  switch (vc) {
    case 16: return jag_s2a_ptr<VP, 16>();
    case 8: return jag_s2a_ptr<VP, 8>();
    case 4: return jag_s2a_ptr<VP, 4>();
    case 2: return jag_s2a_ptr<VP, 2>();
    default: return jag_s2a_ptr<VP, 1>();
  }
}
void* jag_s2a(uint32_t vp, uint32_t vc) {
  switch (vp) {
    case 16: return jag_s2a_for<16>(vc);
    case 8: return jag_s2a_for<8>(vc);
    case 4: return jag_s2a_for<4>(vc);
    case 2: return jag_s2a_for<2>(vc);
    default: return jag_s2a_for<1>(vc);
  }
}
}  // namespace

int launch_jagged_a2s(JagPlan& jp, void* scratch, void* stream, bool small) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const uint64_t n = jp.parent.n;
  if (n == 0) {
    k_write_offset0<<<1, 1, 0, s>>>(jp.offsets, jp.off_size, jp.offset_base);
    return cuda_status(cudaGetLastError());
  }
  const uint64_t nt = jagged_tile_records(jp);  // AoSoA: whole blocks
  const uint32_t tile = small ? MRN_JAG_SMALL_TILE : MRN_JAG_TILE;
  jp.ntiles = (nt + tile - 1) / tile;
  if (jp.ntiles > 0x7fffffffull) return MRN_EUNSUPPORTED;
  char* sc = static_cast<char*>(scratch);
  jp.tile_counter = reinterpret_cast<unsigned int*>(sc);
  jp.tile_state = reinterpret_cast<unsigned long long*>(sc + 256);
  cudaError_t e = cudaMemsetAsync(sc, 0, jagged_scratch_bytes(nt, tile), s);
  if (e != cudaSuccess) return cuda_status(e);
  void* fn = small ? reinterpret_cast<void*>(&k_jagged_a2s_small) : jag_a2s(jp.parent.vec, jp.child.vec);
  void* args[] = {&jp};
  e = cudaLaunchKernel(fn, dim3((unsigned)jp.ntiles), dim3(small ? MRN_JAG_SMALL_THREADS : MRN_JAG_THREADS), args, 0,
                       s);
  return cuda_status(e);
}

uint64_t jagged_split_scratch_bytes(uint64_t n, size_t* group_at) {
  const uint64_t nchunks = (n + MRN_SCAN_CHUNK - 1) / MRN_SCAN_CHUNK;
  const uint64_t at = align_up(256 + nchunks * sizeof(unsigned long long), 256);
  if (group_at) *group_at = (size_t)at;
  return at + (n + 31) / 32 * sizeof(unsigned long long);
}

int launch_jagged_a2s_split(JagPlan& jp, const ConvPlan& pool, void* scratch, void* stream, bool local) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const uint64_t n = jp.parent.n;
  if (n == 0 || !pool.tg.tma || !jp.parent.tg.tma) return MRN_EINVAL;
  jp.nchunks = (n + MRN_SCAN_CHUNK - 1) / MRN_SCAN_CHUNK;
  jp.ntiles = (jagged_tile_records(jp) + MRN_JAG_TILE - 1) / MRN_JAG_TILE;  // tiles of the fall-back pass
  if (jp.nchunks > 0x7fffffffull || jp.ntiles > 0x7fffffffull) return MRN_EUNSUPPORTED;
  if (local) {
    // The local form (see JagPlan, JAG_LOCAL): no scan.  Scratch: the
    // fall-back's ticket at 0, the pool word at 128 (and its copy at 192),
    // the fall-back's look-back words from 256.
    char* sc = static_cast<char*>(scratch);
    jp.mode = JAG_LOCAL;
    jp.noncanon = reinterpret_cast<unsigned int*>(sc + 128);
    jp.any_noncanon = reinterpret_cast<unsigned int*>(sc + 192);
    cudaError_t e = cudaMemsetAsync(sc, 0, 256 + jp.ntiles * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return cuda_status(e);
    // 1. the parents' data columns, their begins as offsets and the checks
    BatchJob job;
    std::memset(&job, 0, sizeof(job));
    job.kind = JOB_JAG_PARENTS;
    job.jp = jp;
    int rc = launch_staged_job(job, stream, LaunchShape{}, nullptr);
    if (rc) return rc;
    // 2. a canonical pool: its records -> the child rows, one staged conversion
    if ((rc = launch_convert(pool, stream, nullptr, jp.noncanon))) return rc;
    // 3. the gaps, and otherwise the whole conversion again, fused
    jp.mode = JAG_FUSED;
    jp.tile_counter = reinterpret_cast<unsigned int*>(sc);
    jp.tile_state = reinterpret_cast<unsigned long long*>(sc + 256);
    const int per_sm = occupancy(reinterpret_cast<const void*>(&k_jagged_a2s_whole_if), MRN_JAG_THREADS, 0);
    const uint64_t grid = std::min<uint64_t>(jp.ntiles, (uint64_t)device_sm_count() * (uint64_t)per_sm);
    k_jagged_a2s_whole_if<<<(unsigned)std::max<uint64_t>(1, grid), MRN_JAG_THREADS, 0, s>>>(jp);
    return cuda_status(cudaGetLastError());
  }
  size_t group_at = 0;
  jagged_split_scratch_bytes(n, &group_at);
  char* sc = static_cast<char*>(scratch);
  jp.mode = JAG_SPLIT;
  jp.tile_counter = reinterpret_cast<unsigned int*>(sc);
  jp.noncanon = reinterpret_cast<unsigned int*>(sc + 128);
  jp.any_noncanon = nullptr;
  jp.chunk_state = reinterpret_cast<unsigned long long*>(sc + 256);
  jp.group_base = reinterpret_cast<unsigned long long*>(sc + group_at);
  cudaError_t e = cudaMemsetAsync(sc, 0, group_at, s);
  if (e != cudaSuccess) return cuda_status(e);
  // 1. the scan: group bases, offsets[n], the pool check
  k_jag_scan_one<<<(unsigned)jp.nchunks, kScanThreads, 0, s>>>(jp);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e);
  // 2. the parents' data columns and offsets, one staged conversion
  BatchJob job;
  std::memset(&job, 0, sizeof(job));
  job.kind = JOB_JAG_PARENTS;
  job.jp = jp;
  int rc = launch_staged_job(job, stream, LaunchShape{}, nullptr);
  if (rc) return rc;
  // 3. a canonical pool: its records -> the child rows, one staged conversion
  if ((rc = launch_convert(pool, stream, nullptr, jp.noncanon))) return rc;
  // 4. otherwise the tiles gather their children
  jp.mode = JAG_CHILDREN;
  const int per_sm = occupancy(reinterpret_cast<const void*>(&k_jagged_a2s_rest), MRN_JAG_THREADS, 0);
  const uint64_t grid = std::min<uint64_t>(jp.ntiles, (uint64_t)device_sm_count() * (uint64_t)per_sm);
  k_jagged_a2s_rest<<<(unsigned)grid, MRN_JAG_THREADS, 0, s>>>(jp);
  return cuda_status(cudaGetLastError());
}

int launch_col_scan(ColScan& cs, void* scratch, void* stream, bool local) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const uint64_t nchunks = std::max<uint64_t>(1, (cs.n + MRN_SCAN_CHUNK - 1) / MRN_SCAN_CHUNK);
  if (nchunks > 0x7fffffffull) return MRN_EUNSUPPORTED;
  char* sc = static_cast<char*>(scratch);
  cs.counter = reinterpret_cast<unsigned int*>(sc);
  cs.noncanon = reinterpret_cast<unsigned int*>(sc + 128);
  cs.local_bad = reinterpret_cast<unsigned int*>(sc + 192);
  cs.only_if = nullptr;
  cs.state = reinterpret_cast<unsigned long long*>(sc + 256);
  cudaError_t e = cudaMemsetAsync(sc, 0, col_scan_scratch_bytes(cs.n), s);
  if (e != cudaSuccess) return cuda_status(e);
  if (local) {
    const unsigned grid = (unsigned)std::max<uint64_t>(
        1, std::min<uint64_t>((cs.n + 255) / 256, (uint64_t)device_sm_count() * 8));
    k_col_local<<<grid, 256, 0, s>>>(cs);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e);
    cs.only_if = cs.local_bad;
  }
  k_col_scan<<<(unsigned)nchunks, kScanThreads, 0, s>>>(cs);
  return cuda_status(cudaGetLastError());
}

uint64_t col_scan_scratch_bytes(uint64_t n) {
  return 256 + std::max<uint64_t>(1, (n + MRN_SCAN_CHUNK - 1) / MRN_SCAN_CHUNK) * sizeof(unsigned long long);
}

int launch_col_gather(const ColScan& cs, const ConvPlan& P, uint64_t capacity, bool force, void* stream) {
  const unsigned grid = (unsigned)std::max<uint64_t>(
      1, std::min<uint64_t>((cs.n + 255) / 256, (uint64_t)device_sm_count() * 8));
  k_col_gather<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(cs, P, capacity, force ? 1u : 0u);
  return cuda_status(cudaGetLastError());
}

int launch_jagged_s2a(const JagPlan& jp, void* stream) {
  const uint64_t pw = (jp.parent.n + 31) / 32;
  const uint64_t cw = (jp.m_src + MRN_JAG_CHILD_GROUP - 1) / MRN_JAG_CHILD_GROUP;
  if (pw + cw == 0) return MRN_OK;
  void* fn = jag_s2a(jp.parent.vec, jp.child.vec);
  const int per_sm = occupancy(fn, 256, kConvSmem);
  const uint64_t need = (pw + cw + 7) / 8;
  const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(need, (uint64_t)device_sm_count() * per_sm));
  unsigned long long pgroups = pw;
  void* args[] = {const_cast<JagPlan*>(&jp), &pgroups};
  return cuda_status(cudaLaunchKernel(fn, dim3(grid), dim3(256), args, kConvSmem,
                                      static_cast<cudaStream_t>(stream)));
}

int launch_len_begin(const char* offsets, uint32_t off_size, uint64_t n, unsigned int* len,
                     unsigned long long* beg, void* stream) {
  if (n == 0) return MRN_OK;
  const unsigned grid = (unsigned)std::min<uint64_t>((n + 255) / 256, (uint64_t)device_sm_count() * 8);
  k_len_begin<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(offsets, off_size, n, len, beg);
  return cuda_status(cudaGetLastError());
}

int launch_jagged_count(const ConvPlan& parent, uint64_t* dev_total, void* stream) {
  uint32_t len_off = 0;
  for (uint32_t i = 0; i < parent.naos; ++i)
    if (parent.aos_cols[i].fm == FM_JLEN) len_off = parent.aos_cols[i].aos_off;
  const unsigned grid = (unsigned)std::max<uint64_t>(
      1, std::min<uint64_t>((parent.n + 255) / 256, (uint64_t)device_sm_count() * 8));
  k_jagged_count<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(
      parent.src.base, parent.n, parent.stride, len_off, reinterpret_cast<unsigned long long*>(dev_total));
  return cuda_status(cudaGetLastError());
}

int batch_occupancy() {
  const void* fn = reinterpret_cast<const void*>(&k_batch);
  allow_batch_smem(fn);
  return occupancy(fn, kBThreads, kBatchSmem);
}

int launch_batch_jag(const BatchJob* jobs, const unsigned int* tile_job, unsigned long long total,
                     unsigned int* counter, unsigned long long* states, void* stream) {
  if (total == 0) return MRN_OK;
  k_batch_jag<<<(unsigned)total, MRN_JAG_THREADS, 0, static_cast<cudaStream_t>(stream)>>>(jobs, tile_job, total,
                                                                                       counter, states);
  return cuda_status(cudaGetLastError());
}

int launch_batch_jag_rest(const BatchJob* jobs, unsigned int njobs, unsigned long long max_tiles,
                          const unsigned int* flags, const unsigned int* any, void* stream) {
  if (max_tiles == 0 || njobs == 0) return MRN_OK;
  const int per_sm = occupancy(reinterpret_cast<const void*>(&k_batch_jag_rest), MRN_JAG_THREADS, 0);
  const uint64_t grid = std::min<uint64_t>(max_tiles, (uint64_t)device_sm_count() * (uint64_t)per_sm);
  k_batch_jag_rest<<<(unsigned)grid, MRN_JAG_THREADS, 0, static_cast<cudaStream_t>(stream)>>>(jobs, njobs, flags,
                                                                                           any);
  return cuda_status(cudaGetLastError());
}

int launch_batch(const BatchJob* jobs, const unsigned long long* first_tile, unsigned int njobs,
                 unsigned long long total_tiles, unsigned int* counter,
                 unsigned int ctas_per_sm, unsigned int max_chunk, void* stream, const unsigned int* conds) {
  if (total_tiles == 0) return MRN_OK;
  const int occ = batch_occupancy();
  const int per_sm = ctas_per_sm ? std::min((int)ctas_per_sm, occ) : occ;
  const uint64_t cap = (uint64_t)device_sm_count() * (uint64_t)per_sm;
  // max_chunk caps the default choice; a tuned value above 8 is taken as is
  // (up to kChunk) while every CTA still gets a chunk
  uint32_t chunk = std::min<uint32_t>(std::max(1u, max_chunk), chunk_for(total_tiles, cap));
  if (max_chunk > 8)
    chunk = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>({(uint64_t)max_chunk, kChunk, total_tiles / cap}));
  const uint64_t chunks = (total_tiles + chunk - 1) / chunk;
  const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(cap, chunks));
  k_batch<<<grid, kBThreads, kBatchSmem, static_cast<cudaStream_t>(stream)>>>(jobs, first_tile, njobs,
                                                                                total_tiles, counter, chunk, conds);
  return cuda_status(cudaGetLastError());
}

}  // namespace mrn

// ------------------------------------------------ overlapping moves


// One range of an overlapping move: `bytes` bytes from src to dst, read and
// written `w` bytes at a time.  With elem (4 or 8) the range holds unsigned
// integers of that size and `delta` is added to each as it moves (jagged
// offsets after an insertion or deletion).
struct MoveSeg {
  const char* src;
  char* dst;
  uint64_t bytes;
  uint64_t chunk_begin;  // first chunk of this range among the launch's chunks
  uint64_t nchunks;
  long long delta;
  uint32_t w;
  uint32_t elem;
  uint32_t up;  // 1: dst above src; chunks are taken from the top down
  uint32_t pad;
};

constexpr uint32_t kMoveSegs = 136;     // a schema's 64 columns, offsets, 64 child columns
constexpr uint32_t kMoveThreads = 256;
constexpr uint32_t kMoveBytes = 64;     // bytes per thread per chunk, whatever the access width
// k_move runs 8 CTAs per SM (32 registers): measured 25-40% faster than the
// 64-register build at 4 CTAs per SM, and than double-buffered chunks

struct MovePlan {
  MoveSeg seg[kMoveSegs];
  uint32_t nseg;
  uint32_t pad;
  uint64_t total_chunks;
  unsigned int* counter;  // [0] chunk tickets, [1] set once a wait has expired
  unsigned int* flags;    // per chunk: 1 once its source has been read
  unsigned long long timeout_ns;
};

__device__ __forceinline__ void st_release_u32(unsigned int* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <int W>
struct MoveWord;
template <> struct MoveWord<1> { using T = uint8_t; };
template <> struct MoveWord<2> { using T = uint16_t; };
template <> struct MoveWord<4> { using T = uint32_t; };
template <> struct MoveWord<8> { using T = unsigned long long; };
template <> struct MoveWord<16> { using T = uint4; };

// Read phase: the chunk's source words into shared memory (the stores there
// consume the loads, so the reads are complete at the barrier that follows).
template <int W>
__device__ __forceinline__ void move_read(const MoveSeg& S, uint64_t lo, uint64_t hi, unsigned char* buf) {
  using T = typename MoveWord<W>::T;
  const T* src = reinterpret_cast<const T*>(S.src + lo);
  T* b = reinterpret_cast<T*>(buf);
  const uint64_t nw = (hi - lo) / W;
#pragma unroll 4
  for (uint32_t i = 0; i < kMoveBytes / W; ++i) {
    const uint64_t k = threadIdx.x + (uint64_t)i * kMoveThreads;
    if (k < nw) b[k] = src[k];
  }
}

template <int W>
__device__ __forceinline__ void move_write(const MoveSeg& S, uint64_t lo, uint64_t hi, const unsigned char* buf) {
  using T = typename MoveWord<W>::T;
  T* dst = reinterpret_cast<T*>(S.dst + lo);
  const T* b = reinterpret_cast<const T*>(buf);
  const uint64_t nw = (hi - lo) / W;
#pragma unroll 4
  for (uint32_t i = 0; i < kMoveBytes / W; ++i) {
    const uint64_t k = threadIdx.x + (uint64_t)i * kMoveThreads;
    if (k < nw) {
      T v = b[k];
      if constexpr (W == 4 || W == 8)
        if (S.elem) v = (T)(v + (T)S.delta);
      dst[k] = v;
    }
  }
}

// Waits until every chunk of S whose source overlaps [a, b) (the
// destination of chunk p) has been read; those chunks hold earlier tickets.
__device__ bool move_wait_sources(const MovePlan& P, const MoveSeg& S, uint64_t p, uint64_t CB, uintptr_t a,
                                  uintptr_t b) {
  const uintptr_t s0 = reinterpret_cast<uintptr_t>(S.src), s1 = s0 + S.bytes;
  if (b <= s0 || a >= s1) return true;
  const uint64_t q0 = (uint64_t)((a > s0 ? a : s0) - s0) / CB;
  const uint64_t q1 = (uint64_t)((b < s1 ? b : s1) - 1 - s0) / CB;
  const unsigned long long deadline = global_ns() + P.timeout_ns;
  for (uint64_t q = q0; q <= q1; ++q) {
    if (q == p) continue;
    const uint64_t c = S.chunk_begin + (S.up ? S.nchunks - 1 - q : q);
    for (uint32_t i = 0; ld_acquire_u32(P.flags + c) == 0; ++i) {
      // after another chunk gave up, this wait may never end: give up too
      if ((i & 63) == 63 && (global_ns() > deadline || ld_acquire_u32(P.counter + 1))) return false;
      __nanosleep(64);
    }
  }
  return true;
}

// Persistent grid: each CTA takes chunks by ticket (chunks of a range in
// the order that makes every overlap point back to an earlier ticket), reads
// one into shared memory, marks it read, waits for the chunks its
// destination overlaps to have been read, then writes it.  A chunk's read
// never waits, so the chunks a CTA waits for always finish their reads.
__global__ void __launch_bounds__(kMoveThreads, 8) k_move(const __grid_constant__ MovePlan P) {
  __shared__ __align__(16) unsigned char buf[kMoveThreads * kMoveBytes];
  __shared__ unsigned long long s_chunk;
  __shared__ int s_ok;
  for (;;) {
    if (threadIdx.x == 0) s_chunk = atomicAdd(P.counter, 1u);
    __syncthreads();
    const uint64_t c = s_chunk;
    if (c >= P.total_chunks) return;
    uint32_t si = 0;
    while (si + 1 < P.nseg && P.seg[si + 1].chunk_begin <= c) ++si;
    const MoveSeg& S = P.seg[si];
    const uint64_t k = c - S.chunk_begin;
    const uint64_t p = S.up ? S.nchunks - 1 - k : k;
    const uint64_t CB = (uint64_t)kMoveThreads * kMoveBytes;
    const uint64_t lo = p * CB, hi = min(lo + CB, S.bytes);
    switch (S.w) {
      case 16: move_read<16>(S, lo, hi, buf); break;
      case 8: move_read<8>(S, lo, hi, buf); break;
      case 4: move_read<4>(S, lo, hi, buf); break;
      case 2: move_read<2>(S, lo, hi, buf); break;
      default: move_read<1>(S, lo, hi, buf); break;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      st_release_u32(P.flags + c, 1u);
      const uintptr_t a = reinterpret_cast<uintptr_t>(S.dst) + lo, b = reinterpret_cast<uintptr_t>(S.dst) + hi;
      s_ok = move_wait_sources(P, S, p, CB, a, b);
      if (!s_ok) {
        flag_error(MRN_ETIMEOUT);
        st_release_u32(P.counter + 1, 1u);
      }
    }
    __syncthreads();
    if (!s_ok) return;
    switch (S.w) {
      case 16: move_write<16>(S, lo, hi, buf); break;
      case 8: move_write<8>(S, lo, hi, buf); break;
      case 4: move_write<4>(S, lo, hi, buf); break;
      case 2: move_write<2>(S, lo, hi, buf); break;
      default: move_write<1>(S, lo, hi, buf); break;
    }
    __syncthreads();  // the buffer and s_chunk are reused
  }
}

// Fills count unsigned integers of `elem` bytes at dst with the value at
// `from` (read on the device: the new objects' offsets after a resize).
__global__ void k_fill_from(char* dst, const char* from, uint64_t count, uint32_t elem) {
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i >= count) return;
  if (elem == 8)
    reinterpret_cast<unsigned long long*>(dst)[i] = *reinterpret_cast<const unsigned long long*>(from);
  else
    reinterpret_cast<unsigned int*>(dst)[i] = *reinterpret_cast<const unsigned int*>(from);
}


namespace mrn {

int launch_moves(const MoveRange* r, size_t nr, void* stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  MovePlan* P = new (std::nothrow) MovePlan;
  if (!P) return MRN_ENOMEM;
  std::memset(P, 0, sizeof(*P));
  uint64_t chunks = 0;
  int rc = MRN_OK;
  for (size_t i = 0; i < nr && rc == MRN_OK; ++i) {
    const MoveRange& m = r[i];
    if (m.bytes == 0 || (m.src == m.dst && !m.elem)) continue;
    const uintptr_t s0 = reinterpret_cast<uintptr_t>(m.src), d0 = reinterpret_cast<uintptr_t>(m.dst);
    const bool overlap = s0 < d0 + m.bytes && d0 < s0 + m.bytes;
    if (!overlap && !m.elem) {
      rc = cuda_status(cudaMemcpyAsync(m.dst, m.src, m.bytes, cudaMemcpyDeviceToDevice, st));
      continue;
    }
    if (P->nseg == kMoveSegs) {
      rc = MRN_EINVAL;
      break;
    }
    // widest access that divides both addresses and the length
    uint32_t w = m.elem ? m.elem : 16;
    const uintptr_t x = s0 | d0 | (uintptr_t)m.bytes;
    while (w > 1 && (x & (w - 1))) w >>= 1;
    if (m.elem && w != m.elem) {
      rc = MRN_EALIGN;
      break;
    }
    MoveSeg& S = P->seg[P->nseg++];
    S.src = m.src;
    S.dst = m.dst;
    S.bytes = m.bytes;
    S.w = w;
    S.elem = m.elem;
    S.delta = m.delta;
    S.up = d0 > s0;
    const uint64_t CB = (uint64_t)kMoveThreads * kMoveBytes;
    S.chunk_begin = chunks;
    S.nchunks = (m.bytes + CB - 1) / CB;
    chunks += S.nchunks;
  }
  if (rc == MRN_OK && P->nseg) {
    void* scratch = nullptr;
    const size_t sb = 256 + chunks * sizeof(unsigned int);
    rc = scratch_alloc(&scratch, sb, st);
    if (rc == MRN_OK) {
      rc = cuda_status(cudaMemsetAsync(scratch, 0, sb, st));
      P->counter = static_cast<unsigned int*>(scratch);
      P->flags = reinterpret_cast<unsigned int*>(static_cast<char*>(scratch) + 256);
      P->total_chunks = chunks;
      P->timeout_ns = 2000000000ull;
      const int per_sm = occupancy(reinterpret_cast<const void*>(&k_move), kMoveThreads, 0);
      const uint64_t cap = (uint64_t)device_sm_count() * (uint64_t)per_sm;
      const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(cap, chunks));
      if (rc == MRN_OK) {
        void* args[] = {P};
        rc = cuda_status(cudaLaunchKernel(reinterpret_cast<const void*>(&k_move), dim3(grid), dim3(kMoveThreads),
                                          args, 0, st));
      }
      scratch_free(scratch, st);
    }
  }
  delete P;
  return rc;
}

int launch_fill_from(char* dst, const char* from, uint64_t count, uint32_t elem, void* stream) {
  if (count == 0) return MRN_OK;
  const unsigned grid = (unsigned)((count + 255) / 256);
  k_fill_from<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(dst, from, count, elem);
  return cuda_status(cudaGetLastError());
}

}  // namespace mrn
