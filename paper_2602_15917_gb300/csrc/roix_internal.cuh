// Internal declarations of libroix: device helpers shared by the kernel files
// and the launch functions the host API calls. Not installed; the public
// interface is include/roix.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "roix.h"

namespace roix {

typedef unsigned long long u64;
typedef unsigned int u32;
typedef unsigned char u8;

constexpr u32 kHeaderBytes = 256;   // container header
constexpr u32 kLMax = 24;           // longest Huffman code
constexpr u32 kMaxRadius = 2048;    // R limit: 2R symbols fit the codebook block
constexpr u32 kMaxSym = 2 * kMaxRadius;
constexpr u32 kVersion = 1;

// Status word codes (first error wins).
__device__ __forceinline__ void set_status(u32* status, u32 code) {
  atomicCAS(status, 0u, code);
}

// ---------------------------------------------------------------- memory
__device__ __forceinline__ u32 ld_acquire(const u32* p) {
  u32 v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(u32* p, u32 v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ u64 ld_relaxed(const u64* p) {
  u64 v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed(u64* p, u64 v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ u32 ld_relaxed32(const u32* p) {
  u32 v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// ------------------------------------------------------------ look-back
// Single-pass decoupled look-back scan (Merrill & Garland 2016) over tiles
// taken in increasing order from an atomic counter: a tile publishes its
// aggregate, walks back over predecessors until one has published an
// inclusive prefix, then publishes its own inclusive prefix. NV 64-bit sums
// are carried. Every wait is bounded: after `limit` polls (0: kSpinLimit) the
// tile gives up, records ROIX_ETIMEOUT, treats the missing value as 0 and
// returns true (results invalid, the kernel still ends; the kernels after it
// in the same call see the status and do nothing).
constexpr u32 kSpinLimit = 1u << 22;
__host__ __device__ __forceinline__ u32 spin_limit_of(u32 limit) {
  return limit ? limit : kSpinLimit;
}

template <int NV>
struct LookBack {
  u32* flags;  // [tiles], zero before the launch
  u64* agg;    // [tiles * NV]
  u64* inc;    // [tiles * NV]
};

// hold: tile 0 publishes nothing (a flag that nobody sets; test hook for the
// bounded waits of the tiles after it)
template <int NV>
__device__ bool lookback(LookBack<NV> lb, u64 t, const u64 (&mine)[NV], u64 (&excl)[NV],
                         u32* status, u32 limit, bool hold = false) {
  for (int i = 0; i < NV; ++i) excl[i] = 0;
  if (t == 0) {
    if (hold) return false;
    for (int i = 0; i < NV; ++i) st_relaxed(&lb.inc[i], mine[i]);
    st_release(&lb.flags[0], 2u);
    return false;
  }
  limit = spin_limit_of(limit);
  bool timed_out = false;
  for (int i = 0; i < NV; ++i) st_relaxed(&lb.agg[t * NV + i], mine[i]);
  st_release(&lb.flags[t], 1u);
  u64 j = t - 1;
  u32 spins = 0;
  while (true) {
    u32 f = ld_acquire(&lb.flags[j]);
    if (f == 0) {
      if (++spins > limit) {
        set_status(status, ROIX_ETIMEOUT);
        timed_out = true;
        break;
      }
      __nanosleep(64);
      continue;
    }
    if (f == 2) {
      for (int i = 0; i < NV; ++i) excl[i] += ld_relaxed(&lb.inc[j * NV + i]);
      break;
    }
    for (int i = 0; i < NV; ++i) excl[i] += ld_relaxed(&lb.agg[j * NV + i]);
    if (j == 0) break;  // tile 0 always publishes an inclusive prefix; guard only
    --j;
  }
  for (int i = 0; i < NV; ++i) st_relaxed(&lb.inc[t * NV + i], excl[i] + mine[i]);
  st_release(&lb.flags[t], 2u);
  return timed_out;
}

// Warp-parallel form (Merrill & Garland's window variant): all 32 lanes of one
// warp call it; lane j inspects predecessor t-1-j, so a window of 32 flags is
// read per L2 round trip. Lanes up to the nearest inclusive prefix must have
// published; their aggregates and that prefix are summed by a warp reduction.
// Returns the exclusive prefix in every lane. Bounded like lookback().
template <int NV>
__device__ bool lookback_warp(LookBack<NV> lb, u64 t, const u64 (&mine)[NV], u64 (&excl)[NV],
                              u32* status, u32 limit, bool hold = false) {
  const int lane = threadIdx.x & 31;
  for (int i = 0; i < NV; ++i) excl[i] = 0;
  if (t == 0) {
    if (lane == 0 && !hold) {
      for (int i = 0; i < NV; ++i) st_relaxed(&lb.inc[i], mine[i]);
      st_release(&lb.flags[0], 2u);
    }
    return false;
  }
  limit = spin_limit_of(limit);
  bool timed_out = false;
  if (lane == 0) {
    for (int i = 0; i < NV; ++i) st_relaxed(&lb.agg[t * NV + i], mine[i]);
    st_release(&lb.flags[t], 1u);
  }
  long long base = (long long)t - 1;
  u32 spins = 0;
  while (true) {
    const long long j = base - lane;
    const u32 f = j >= 0 ? ld_acquire(&lb.flags[j]) : 2u;
    const u32 incl = __ballot_sync(0xffffffffu, f == 2u);
    const u32 zero = __ballot_sync(0xffffffffu, f == 0u);
    const int first = incl ? __ffs(incl) - 1 : 32;
    const u32 need = first == 32 ? 0xffffffffu : (0xffffffffu >> (31 - first));
    if (zero & need) {
      if (++spins > limit) {
        if (lane == 0) set_status(status, ROIX_ETIMEOUT);
        timed_out = true;
        break;
      }
      __nanosleep(32);
      continue;
    }
    u64 v[NV];
    for (int i = 0; i < NV; ++i) {
      v[i] = 0;
      if (lane < first) v[i] = ld_relaxed(&lb.agg[(u64)j * NV + i]);
      else if (lane == first && j >= 0) v[i] = ld_relaxed(&lb.inc[(u64)j * NV + i]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
      excl[i] += v[i];
    }
    if (first < 32) break;
    base -= 32;
  }
  if (lane == 0) {
    for (int i = 0; i < NV; ++i) st_relaxed(&lb.inc[t * NV + i], excl[i] + mine[i]);
    st_release(&lb.flags[t], 2u);
  }
  return timed_out;
}

// A kernel of the compression path that runs after a tile scan: true when a
// bounded wait of this call gave up (ROIX_ETIMEOUT), so that nothing is
// computed from the scan's invalid offsets.
__device__ __forceinline__ bool halted(const u32* status) {
  return ld_relaxed32(status) == (u32)ROIX_ETIMEOUT;
}

// ------------------------------------------------------------------- scans
template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    T o = __shfl_up_sync(0xffffffffu, v, d);
    if (lane >= d) v += o;
  }
  return v;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
  return v;
}

// Block-wide exclusive scan of one value per thread; `scratch` holds 33 T.
// Returns the exclusive prefix; *total receives the block sum.
template <typename T>
__device__ T block_excl_scan(T v, T* scratch, T* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = (blockDim.x + 31) >> 5;
  T inc = warp_incl_scan(v);
  if (lane == 31) scratch[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    T s = lane < nwarps ? scratch[lane] : T(0);
    T si = warp_incl_scan(s);
    if (lane < nwarps) scratch[lane] = si - s;
    if (lane == nwarps - 1) scratch[32] = si;
  }
  __syncthreads();
  T out = scratch[warp] + inc - v;
  *total = scratch[32];
  __syncthreads();
  return out;
}

// Exclusive scans of two count arrays a[0..n), b[0..n) into ao, bo by one
// block: thread i sums its contiguous range of ceil(n / blockDim) entries
// (eight loads in flight), one block scan combines the sums, each thread
// writes its range. Returns the totals (in every thread). `scratch` holds 33
// u64. Writers and later readers of ao / bo in the same block need a barrier.
__device__ __forceinline__ void block_scan2(const u32* __restrict__ a, const u32* __restrict__ b,
                                            u64 n, u64* __restrict__ ao, u64* __restrict__ bo,
                                            u64* scratch, u64* ta, u64* tb) {
  const u64 per = (n + blockDim.x - 1) / blockDim.x;
  const u64 lo = umin(n, (u64)threadIdx.x * per), hi = umin(n, lo + per);
  u64 sa = 0, sb = 0;
  for (u64 i0 = lo; i0 < hi; i0 += 8) {
    u32 va[8], vb[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      va[k] = i0 + k < hi ? __ldg(a + i0 + k) : 0u;
      vb[k] = i0 + k < hi ? __ldg(b + i0 + k) : 0u;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      sa += va[k];
      sb += vb[k];
    }
  }
  u64 ea = block_excl_scan<u64>(sa, scratch, ta);
  u64 eb = block_excl_scan<u64>(sb, scratch, tb);
  for (u64 i0 = lo; i0 < hi; i0 += 8) {
    u32 va[8], vb[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      va[k] = i0 + k < hi ? __ldg(a + i0 + k) : 0u;
      vb[k] = i0 + k < hi ? __ldg(b + i0 + k) : 0u;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      if (i0 + k < hi) {
        ao[i0 + k] = ea;
        bo[i0 + k] = eb;
      }
      ea += va[k];
      eb += vb[k];
    }
  }
}

// Exclusive scan of one count array a[0..n) into ao by one block (as
// block_scan2); returns the total in every thread.
__device__ __forceinline__ u64 block_scan1(const u32* __restrict__ a, u64 n,
                                           u64* __restrict__ ao, u64* scratch) {
  const u64 per = (n + blockDim.x - 1) / blockDim.x;
  const u64 lo = umin(n, (u64)threadIdx.x * per), hi = umin(n, lo + per);
  u64 sa = 0;
  for (u64 i0 = lo; i0 < hi; i0 += 8) {
    u32 va[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) va[k] = i0 + k < hi ? __ldg(a + i0 + k) : 0u;
#pragma unroll
    for (int k = 0; k < 8; ++k) sa += va[k];
  }
  u64 ta;
  u64 ea = block_excl_scan<u64>(sa, scratch, &ta);
  for (u64 i0 = lo; i0 < hi; i0 += 8) {
    u32 va[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) va[k] = i0 + k < hi ? __ldg(a + i0 + k) : 0u;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      if (i0 + k < hi) ao[i0 + k] = ea;
      ea += va[k];
    }
  }
  return ta;
}

// ------------------------------------------------------------ fast division
// Division of 32-bit numerators by an invariant divisor with a multiply-high
// and shifts (Granlund & Montgomery 1994, round-up method).
// floor((2^64 - 1) / d), the multiplier of div_by (host side, once per item).
__host__ __device__ inline u64 recip64(u64 d) { return d ? ~0ull / d : 0ull; }

// floor(a / d) for d >= 1 from m = recip64(d). With m = (2^64 - 1 - rho) / d,
// 0 <= rho < d: a m / 2^64 = a / d - a (1 + rho) / (d 2^64) > a / d - 1, so the
// high word of a m is floor(a / d) or one less, and one remainder test fixes it.
// Integer pipes only (a binary64 or 64-bit division would run on the FP64 pipe,
// which is narrow on this part).
__device__ __forceinline__ u64 div_by(u64 a, u64 d, u64 m) {
  u64 q = __umul64hi(a, m);
  if (a - q * d >= d) ++q;
  return q;
}

struct FastDiv {
  u32 d, m, s;
  u32 p2;  // d is a power of two (= 2^s)
  __host__ __device__ FastDiv(u32 div = 1) : d(div ? div : 1), m(0), s(0), p2(0) {
    u32 l = 0;
    while ((1ull << l) < d) ++l;
    s = l;
    m = l ? (u32)(((1ull << 32) * ((1ull << l) - d)) / d + 1) : 0u;
    p2 = (d & (d - 1)) == 0 ? 1u : 0u;
  }
  __device__ __forceinline__ u32 div(u32 n) const {
    if (s == 0) return n;
    const u32 t = __umulhi(m, n);
    return (t + ((n - t) >> 1)) >> (s - 1);
  }
};

__device__ __forceinline__ int quant_u16_fd(unsigned raw, int dark, int eb_int,
                                            const FastDiv& fd) {
  const int v = (int)raw - dark;  // in [-65535, 65535]
  if (eb_int == 0) return v;
  const int num = v + eb_int;
  if (fd.p2) return num >> fd.s;  // floor of num / 2^s (arithmetic shift)
  return num >= 0 ? (int)fd.div((u32)num) : -(int)fd.div((u32)(-num + 2 * eb_int - 1));
}

// ------------------------------------------------------- ordered float keys
// Monotone map of binary32 bit patterns to uint32 (for atomicMin/Max).
__device__ __forceinline__ u32 f32_key(float f) {
  u32 b = __float_as_uint(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float key_f32(u32 k) {
  u32 b = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
  return __uint_as_float(b);
}

// ----------------------------------------------------------------- layout
__host__ __device__ __forceinline__ u64 align16(u64 v) { return (v + 15) & ~u64(15); }
__host__ __device__ __forceinline__ u64 umin(u64 a, u64 b) { return a < b ? a : b; }
__host__ __device__ __forceinline__ u64 umax(u64 a, u64 b) { return a > b ? a : b; }

// Section offsets of a container (all little-endian, 16-byte aligned).
struct Layout {
  u64 off_lens, off_counts, off_bounds, off_outk, off_outv, off_chunks, off_payload, total;
};
__host__ __device__ __forceinline__ Layout make_layout(u64 S, u64 rows, u64 nb, u64 nout,
                                                       u64 nchunks, u64 nwords) {
  Layout L;
  L.off_lens = kHeaderBytes;
  L.off_counts = align16(L.off_lens + S);
  L.off_bounds = align16(L.off_counts + 2 * rows);
  L.off_outk = align16(L.off_bounds + 2 * nb);
  L.off_outv = align16(L.off_outk + 8 * nout);
  L.off_chunks = align16(L.off_outv + 4 * nout);
  L.off_payload = align16(L.off_chunks + 8 * nchunks);
  L.total = align16(L.off_payload + 4 * nwords);
  return L;
}

// Device-side state of one compressed item (zeroed per call, except the
// first word of the context's first state, which is the context status).
struct State {
  u32 status;                          // context status word (state 0 only)
  u32 ctr_front, ctr_quant, ctr_pack;  // dynamic tile counters (state 0: batch tickets)
  u32 ctr_write, ctr_front2;           // pack-write and compaction-write tickets
  u32 ctr_scan_f, ctr_scan_p;          // tile scans of the compaction and of the pack
  u64 n, nb, nout, nwords;             // sizes found on the device
  u32 vmin_key, vmax_key;              // range of retained finite values
  u32 cap_flag, pad0;
  u32 done_front, done_pack;           // tiles / chunks counted (the last one scans)
  u64 total;
  roix_eb_info eb;
};

// Static description of one volume and its coder settings (kernel argument).
struct Desc {
  u64 nx, ny, nz, rows, W, N;  // W = mask words per row
  int dtype;                   // ROIX_F32 / ROIX_U16
  int cmp, keep, conn, dilate;
  float thr_f;                 // float32: x > thr_f (cmp 0) or x < thr_f (cmp 1)
  int thr_i;                   // uint16: v > thr_i or v < thr_i, v = raw - dark
  int thr_never;               // NaN threshold: nothing passes
  int dark;
  double threshold, dark_d, fill;
  int eb_mode;
  double eb_value;
  u32 R, S, C;
  u32 front_words;             // compaction tile size (mask words), from the tuning
  u32 order;                   // Lorenzo order of the prediction: 1 or 2
  u32 spin_limit;              // polls of a bounded device wait (0: kSpinLimit)
  u32 hold_scans;              // test hook: the first tile of each tile scan never publishes
};

// ------------------------------------------------------------------ batches
// A batch is up to kMaxBatch independent items (volumes or images) sharing
// the ROI / error-bound / coder settings. Kernels take it as a
// __grid_constant__ parameter and map global work tickets to (item, tile)
// through prefix sums; every item has its own state, look-back descriptors,
// histogram, codebook and container. A single volume is a batch of one.
constexpr int kMaxBatch = 64;
// Rows of a compaction tile, at most: the warp-per-tile counting kernel keeps
// one warp's row totals (2 x 4 bytes a row) in shared memory.
constexpr u32 kMaxTileRows = 256;

struct Item {
  u64 nx, ny, nz, rows, W, N;          // geometry
  const void* in;                      // input values
  uint8_t* out;                        // container
  u64 cap;
  u64* size_dev;                       // container size (output)
  State* st;
  State* rst;                          // state holding the value range (st, or a state
                                       // shared by the z-slabs of one volume)
  u32* T;                              // thresholded mask (fused path)
  void* P;                             // pixel section
  uint16_t* sym;
  u64 rec_cap;                         // records the container can hold
  unsigned long long* hist;
  uint8_t* lens;
  u32* codes;
  const int32_t* q;                    // staged codes (encode from codes), else null
  const u32* obits;
  const roix_eb_info* info_in;         // staged error-bound constants, else null
  uint16_t* counts;                    // row geometry destinations
  u64 counts_cap;
  uint16_t* bounds;
  u64 bounds_cap;
  const uint16_t* counts_src;          // staged geometry to copy into the container
  const uint16_t* bounds_src;
  u64* sizes;                          // [n, nb]
  u32* D;                              // retained words (dilated mask), when dilating
  u32* ftn;                            // [tiles] retained voxels per compaction tile
  u32* ftb;                            // [tiles] boundaries per compaction tile
  u64* ftno;                           // [tiles] first retained voxel of each tile
  u64* ftbo;                           // [tiles] first boundary of each tile
  LookBack<2> lbsf, lbsp;              // look-backs of the tile scans (8192 entries a tile)
  u32* rno;                            // [rows] first retained voxel of the row in its tile
  u32* rbo;                            // [rows] first boundary of the row in its tile
  u32* crec;                           // [chunks] records per pack chunk (zeroed)
  u32* rbits;                          // [n / 32] record bitmap (bit k: symbol k is 0)
  u32* cw;                             // [chunks] payload words per chunk
  u64* cwoff;                          // [chunks] first payload word of each chunk
  u64* crecoff;                        // [chunks] first record of each chunk
  u32 rpt;                             // rows per front tile
  u32 vec;                             // rows are 16-byte aligned (vector loads)
  u32 flat;                            // binarisation reads the volume as a flat array
  u32 zhalo;                           // z-slab: bit 0 = T holds the plane before z = 0,
                                       // bit 1 = T holds the plane after z = nz - 1
  u64 ftiles;                          // front tiles
  u32 fscan;                           // the counting kernel scans the tile totals
                                       // (ftiles <= kInScanMax), not k_scan_pairs<0>
  u32 pscan;                           // k_pack_count scans the chunk word counts
                                       // (chunks <= kInScanMax), not k_scan_pairs<1>
  u64 m_nx, m_spr, m_rpt, m_ny;        // recip64 of nx, of the 1024-voxel segments per
                                       // row, of rpt and of ny (divisions by multiply-high)
};

struct Batch {
  Desc c;                              // shared settings (geometry fields unused)
  u32 n;                               // items
  u32* status;                         // context status word
  u32* ctr;                            // [7] tickets: front count (block kernel), symbols,
                                       // (unused), pack write, front write, front scan,
                                       // pack scan
  u64 seg0[kMaxBatch + 1];             // prefix of threshold row segments (row-form items)
  u64 fseg0[kMaxBatch + 1];            // prefix of threshold flat spans (flat-form items)
  u64 ftile0[kMaxBatch + 1];           // prefix of front tiles
  u64 row0[kMaxBatch + 1];             // prefix of rows
  Item it[kMaxBatch];
};
// Kernels take the batch by value as a __grid_constant__ parameter: it must
// stay within the 32,764 bytes of kernel parameters a launch may carry.
static_assert(sizeof(Batch) <= 32764, "Batch exceeds the kernel parameter limit");

__device__ __forceinline__ Desc desc_of(const Batch& B, const Item& I) {
  Desc d = B.c;
  d.nx = I.nx;
  d.ny = I.ny;
  d.nz = I.nz;
  d.rows = I.rows;
  d.W = I.W;
  d.N = I.N;
  return d;
}

// Largest i in [0, n) with prefix[i] <= x (prefix[0] = 0, nondecreasing).
template <typename P>
__device__ __forceinline__ u32 find_item(const P& prefix, u32 n, u64 x) {
  u32 lo = 0, hi = n;  // invariant: prefix[lo] <= x < prefix[hi] (prefix[n] = total)
  while (hi - lo > 1) {
    const u32 mid = (lo + hi) >> 1;
    if (prefix[mid] <= x) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Error-bound constants from the mode, the value and the range keys; the same
// sequence of binary64 operations as the definition (Sec. 4.2.3, Sz3 range).
__device__ __forceinline__ roix_eb_info make_eb(const Desc& d, u32 vmin_key, u32 vmax_key) {
  roix_eb_info e;
  double vmin, vmax;
  if (d.dtype == ROIX_F32) {
    vmin = vmin_key == 0xffffffffu ? __longlong_as_double(0x7ff0000000000000ll)
                                   : (double)key_f32(vmin_key);
    vmax = vmax_key == 0u ? -__longlong_as_double(0x7ff0000000000000ll)
                          : (double)key_f32(vmax_key);
  } else {
    vmin = vmin_key == 0xffffffffu ? __longlong_as_double(0x7ff0000000000000ll)
                                   : (double)(vmin_key - 1);
    vmax = vmax_key == 0u ? -__longlong_as_double(0x7ff0000000000000ll) : (double)(vmax_key - 1);
  }
  e.vmin = vmin;
  e.vmax = vmax;
  double eb;
  if (d.eb_mode == 0) eb = d.eb_value;
  else eb = (vmax >= vmin) ? __dmul_rn(d.eb_value, __dsub_rn(vmax, vmin)) : 0.0;
  e.eb_abs = eb;
  double two_d = __dmul_rn(2.0, eb);
  float two = __double2float_rn(two_d);
  float inv = eb > 0.0 ? __double2float_rn(__ddiv_rn(1.0, two_d)) : 0.0f;
  bool ok = eb > 0.0 && isfinite(eb) && isfinite(two) && two > 0.0f && isfinite(inv) &&
            inv > 0.0f;
  if (ok) {
    e.two_eb = two;
    e.inv2eb = inv;
    e.bound = __double2float_rz(__dmul_rn(eb, 1.0 - 0x1p-23));
  } else {
    e.two_eb = 0.0f;
    e.inv2eb = 0.0f;
    e.bound = -1.0f;
  }
  double ebi = floor(eb);
  if (!(ebi >= 0.0)) ebi = 0.0;
  if (ebi > 65535.0) ebi = 65535.0;
  e.eb_int = (int)ebi;
  return e;
}

// Linear quantiser of one value (Sec. 4.2.3 contract): returns the code, sets
// `out` for an outlier (code 0). Binary32 operations rounded to nearest, no
// contraction: the decoder repeats the reconstruction bit for bit.
__device__ __forceinline__ int quant_f32(float x, const roix_eb_info& e, bool& out) {
  // a non-finite x gives a non-finite y (inf * positive, NaN, or inf * 0 =
  // NaN for the degenerate bound), so the range test below also rejects it
  float y = __fmul_rn(x, e.inv2eb);
  if (!(fabsf(y) < 1073741824.0f)) {
    out = true;
    return 0;
  }
  int q = __float2int_rn(y);
  float xh = __fmul_rn(__int2float_rn(q), e.two_eb);
  float dd = __fsub_rn(x, xh);
  out = !(fabsf(dd) <= e.bound);
  return out ? 0 : q;
}
__device__ __forceinline__ int quant_u16(unsigned raw, int dark, int eb_int) {
  int v = (int)raw - dark;
  if (eb_int == 0) return v;
  int num = v + eb_int, den = 2 * eb_int;
  return num >= 0 ? num / den : -((-num + den - 1) / den);
}
// Same value with the division by 2*eb_int done by `fd` (a FastDiv of it).
__device__ __forceinline__ int quant_u16_fd(unsigned raw, int dark, int eb_int,
                                            const struct FastDiv& fd);

// Launch shapes that leave every output byte unchanged (picked by roix_tune).
struct Tuning {
  u32 front_words = 2048;      // mask words per compaction tile
  u32 thr_blocks_per_sm = 8;   // binarisation, row form (blocks of 256 threads)
  u32 flat_blocks_per_sm = 4;  // binarisation, flat form
  u32 sym_blocks_per_sm = 0;   // symbols: 0 = as many as fit
  u32 pack_blocks_per_sm = 0;  // pack: 0 = as many as fit
  u32 front_kernel = 0;        // compaction counts: 0 = block per tile, 1 = warp per tile
};

}  // namespace roix

// A context: device, workspace, status carry-over, profiling events.
struct roix_ctx {
  int device = 0;
  int sms = 0;
  char* ws = nullptr;
  size_t ws_bytes = 0;
  bool ws_borrowed = false;  // ws belongs to a server's arena (never grown or freed here)
  roix::u32 pending = 0;  // status carried over a workspace reallocation
  std::string err;
  int profile = 0;        // per-stage events in the fused path
  roix::Tuning tune{};    // launch shapes (roix_tune / roix_set_tuning)
  roix::u32 spin_limit = 0;  // polls of a bounded device wait (0: the default)
  int hold_scans = 0;        // test hook (roix_debug_hold_scans)
  cudaEvent_t ev[16] = {};
  int nev = 0;
};

namespace roix {

// Host: grows the context workspace (synchronises the device); exact = no headroom.
roix_status ensure_ws(roix_ctx* ctx, size_t bytes, bool exact = false);
// Host: the context works in a caller's region [ws, ws + bytes) from now on
// (the serving loop's arena); the region is not grown or freed by the context.
void borrow_ws(roix_ctx* ctx, char* ws, size_t bytes);
// Host: workspace bytes of one fused group of items sharing the settings `c`.
size_t batch_workspace(const Desc& c, const roix_item* items, u32 n);

// Host: argument checks and descriptor (roix_api.cu); ctx may be null.
roix_status make_desc(roix_ctx* ctx, roix_dtype dtype, roix_dims dims, const roix_roi* roi,
                      const roix_eb* eb, const roix_params* prm, Desc* d);

// Host: a one-item batch for the binarisation kernel alone (roix_api.cu).
void make_threshold_batch(Batch& B, const Desc& d, const void* in, u32* T);
// Host: the binarisation work units of every item (B.seg0), from each item's
// input pointer and geometry; sets the items' vec / flat forms.
void set_threshold_units(Batch& B);
size_t front_smem(u32 rpt, u64 W, int dilate);

// ------------------------------------------------------ launch functions
struct Launch {
  cudaStream_t stream;
  int sms;
  Tuning t{};
};

// mask kernels (k_mask.cu)
constexpr u32 kScanTile = 8192;  // entries per block of the tile scans
// Items with at most this many compaction tiles (pack chunks) have their tile
// scan done inside the counting kernel, by the warp that counts the item's
// last tile; larger ones go through k_scan_pairs.
constexpr u32 kInScanMax = 1024;

// Exclusive scans of two u32 arrays a, b (b may be null) of an item's nt
// entries into u64 ao, bo by one warp (loads in batches of 8 per lane, through
// L2: the entries were written by other blocks of the running kernel); returns
// the totals.
__device__ __forceinline__ void warp_scan2(const u32* a, const u32* b, u64 nt, u64* ao,
                                           u64* bo, u64& ta, u64& tb) {
  const int lane = threadIdx.x & 31;
  u64 ca = 0, cb = 0;
  for (u64 i0 = 0; i0 < nt; i0 += 256) {
    u32 va[8], vb[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const u64 i = i0 + (u64)k * 32 + lane;
      va[k] = i < nt ? __ldcg(a + i) : 0u;
      vb[k] = (b && i < nt) ? __ldcg(b + i) : 0u;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const u64 i = i0 + (u64)k * 32 + lane;
      const u32 ia = warp_incl_scan(va[k]), ib = warp_incl_scan(vb[k]);
      if (i < nt) {
        ao[i] = ca + ia - va[k];
        if (bo) bo[i] = cb + ib - vb[k];
      }
      ca += __shfl_sync(0xffffffffu, ia, 31);
      cb += __shfl_sync(0xffffffffu, ib, 31);
    }
  }
  ta = ca;
  tb = cb;
}

// One more tile (chunk) of an item counted: true in the warp that counted the
// last of its `total`, which may then read every tile's totals. Called by all
// lanes of a warp after lane 0 wrote the tile's totals.
__device__ __forceinline__ bool count_done(u32* done, u64 total) {
  u32 old = 0;
  if ((threadIdx.x & 31) == 0) {
    __threadfence();  // the tile's totals before the count
    old = atomicAdd(done, 1u);
  }
  old = __shfl_sync(0xffffffffu, old, 0);
  const bool last = (u64)old + 1 == total;
  if (last) __threadfence();  // the other tiles' totals after the count
  return last;
}
// Exclusive scans of the pairs (ftn, ftb) over compaction tiles (mode 0: into
// ftno, ftbo and the item's n, nb) or (cw, crec) over pack chunks (mode 1:
// into cwoff, crecoff and the item's nwords, nout); tiles_cap bounds the scan
// tiles of the batch.
void launch_scan_pairs(const Launch& L, const Batch& B, int mode, u64 tiles_cap);
void launch_threshold(const Launch& L, const Batch& B);
void launch_dilate(const Launch& L, const Desc& d, const u32* T, u32* D, u64* popcount);
void launch_front(const Launch& L, const Batch& B);

// coder kernels (k_encode.cu)
constexpr u32 kQuantTile = 4096;  // values per symbol segment (one warp's unit of work)
constexpr u32 kPackRange = 1;     // chunks per pack ticket (one warp's unit of work)
void launch_init(const Launch& L, State* st, u32 nstates, void* zero, size_t zero_bytes);
void launch_quantize_stage(const Launch& L, const Desc& d, const void* P, u64 n_cap,
                           const u64* n_dev, int32_t* q, u32* obits, roix_eb_info* info_out,
                           State* st);
// tiles_cap / ranges_cap: upper bounds of the batch's symbol tiles / pack ranges
void launch_symbols(const Launch& L, const Batch& B, u64 tiles_cap);
void launch_codebook(const Launch& L, const Batch& B);
void launch_pack(const Launch& L, const Batch& B, u64 ranges_cap);
void launch_finalize(const Launch& L, const Batch& B);

// largest component (k_ccl.cu)
struct CclWs {
  u32* row_runs;              // [rows]
  u64* row_off;               // [rows]
  uint16_t* xs;               // [max runs]
  uint16_t* xe;               // [max runs]
  u32* par;                   // [max runs]
  unsigned long long* size;   // [max runs]
  u64* total;                 // run count
  unsigned long long* best;   // largest size (zeroed)
  u32* best_root;             // ~root of that component (zeroed: none)
  LookBack<1> lb;             // scan of the run counts (flags zeroed)
  u32* ctr;                   // scan tickets (zeroed)
  u32* status;
};
// Largest connected component of the mask T (rows x W words) into `out`
// (same layout; every word written).
void launch_keep_largest(const Launch& L, const Desc& d, const u32* T, u32* out,
                         const CclWs& w);
inline u64 ccl_max_runs(const Desc& d) { return d.rows * ((d.nx + 1) / 2); }

// decoder kernels (k_decode.cu)
struct DecodeWs {
  u32* status;
  u64* plan;          // decoded header values (kPlanWords), zeroed by the header kernel
  void* table;        // canonical decode table (dec_table_bytes(), zeroed by the host)
  uint16_t* sym;      // [N]
  u64* agg;           // [max chunks * 2] chunk aggregates (reset flag, value)
  u64* carry;         // [max chunks]
  void* vals;         // [N] values in retained order
  u64* row_boff;      // [rows]
  u64* row_voff;      // [rows]
  LookBack<1> lb_rows_b, lb_rows_v;  // flags zeroed by the host
  u32* row_ctr;       // zeroed by the host
};
constexpr int kPlanWords = 32;
constexpr u64 kDecRowTile = 1024;
size_t dec_table_bytes();
void launch_decode(const Launch& L, const Desc& d, const uint8_t* in, u64 size, void* out,
                   const DecodeWs& ws, u64 max_chunks);

// ------------------------------------- 8-bit normalisation, greedy quantiser
// imax_key: one zeroed uint32 (the largest value's bits); imax_out may be null.
void launch_normalize8(const Launch& L, int dtype, const void* in, u64 N, int dark, u8* out,
                       u32* imax_key, double* imax_out);

constexpr u32 kGreedyMaxItems = 64;
struct GreedyItem {
  const u8* P;      // pixel sections of the rows, row after row
  const u32* mask;  // rows x W words
  u8* Q;            // quantised sections (may equal P)
  u64* n_out;       // total pixels (may be null)
  u64 rows, W;
  u32 inplace;      // Q == P: pixel loads bypass the non-coherent cache
};
struct GreedyBatch {
  u32 n;
  u32 e2;                            // 2 floor(E_abs), at most 510
  u64 tile0[kGreedyMaxItems + 1];    // prefix of 32-row tiles over the items
  u64 row0[kGreedyMaxItems + 1];     // prefix of rows over the items
  GreedyItem it[kGreedyMaxItems];
  u32* lens;                         // [rows of all items]
  u32* rpre;                         // [rows]: prefix of lengths within the row's tile
  u64* rowctr;                       // zeroed: next row to scan
  u32* tsum;                         // [tiles]
  u64* toff;                         // [tiles + 1]
};
void launch_greedy(const Launch& L, const GreedyBatch& B);

// ------------------------------------------------ paper-mode ROI
// Planar union-find (d.conn = 4 or 8): components of T (complemented when
// inv = ~0u) touching their slice border (keep_border) or the largest of every
// slice, into `out`; w.best / w.best_root hold one entry per slice, zeroed.
void launch_ccl_planar(const Launch& L, const Desc& d, const u32* T, u32 inv, int keep_border,
                       u32* out, const CclWs& w);
void launch_paper_hist_otsu(const Launch& L, const u8* img, u64 nx, u64 ny, u64 nz, u32* hist,
                            u32* thr);
void launch_paper_binarize(const Launch& L, const u8* img, u64 nx, u64 ny, u64 nz,
                           const u32* thr, u32* T);
void launch_paper_spans(const Launch& L, const u32* K, u64 rows, u64 W, u32* D, u64* popcount);

// ------------------------------------------------ evaluation metrics
size_t roi_quality_ws_bytes(u64 nx, u64 ny, u64 nz, int distances);
void launch_roi_quality(const Launch& L, const u32* A, const u32* B, u64 nx, u64 ny, u64 nz,
                        int distances, char* ws, roix_roi_metrics* out);
void launch_ssim(const Launch& L, int dtype, const void* X, const void* Y, u64 nx, u64 ny, u64 nz,
                 double data_range, char* ws, double* out);

}  // namespace roix
