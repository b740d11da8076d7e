// Region-of-interest kernels: binarisation (Sec. 4.1.1, 4.1.3-4.1.4), the
// cube dilation of the retained set, and the extraction of row geometry and
// pixel section (Sec. 4.2.2) by a compaction in count, scan and write passes.
//
// Mask layout: rows = ny*nz rows of W = ceil(nx/32) uint32 words; voxel x of a
// row is bit x%32 of word x/32; bits at x >= nx are 0.
#include "roix_internal.cuh"

namespace roix {

namespace {

constexpr int kThreads = 256;

// Threshold test (Sec. 4.1.1) in one form for either direction. float32: x
// passes when s x > t, s = -1 turning x < thr into -x > -thr exactly (NaN never
// passes; no threshold gives t = +inf). Integer values: the values above
// dark + thr, or below it, are one interval [lo, lo + span] of [0, 65535], so
// raw passes when raw - lo, taken unsigned, is at most span (none: lo = 65536,
// span = 0). Formed once per work unit from the settings.
struct PassTest {
  float s, t;
  u32 lo, span;
};

__device__ __forceinline__ PassTest pass_test(const Desc& d) {
  PassTest p;
  p.s = d.cmp == 0 ? 1.0f : -1.0f;
  p.t = d.thr_never ? __int_as_float(0x7f800000) : (d.cmp == 0 ? d.thr_f : -d.thr_f);
  long long lo = 0, hi = 65535;
  if (d.cmp == 0) lo = (long long)d.dark + d.thr_i + 1;
  else hi = (long long)d.dark + d.thr_i - 1;
  if (lo < 0) lo = 0;
  if (hi > 65535) hi = 65535;
  if (d.thr_never || lo > hi) {
    p.lo = 65536u;
    p.span = 0u;
  } else {
    p.lo = (u32)lo;
    p.span = (u32)(hi - lo);
  }
  return p;
}
__device__ __forceinline__ bool passes(const PassTest& p, float x) {
  return __fmul_rn(x, p.s) > p.t;
}
__device__ __forceinline__ bool passes(const PassTest& p, u32 raw) { return raw - p.lo <= p.span; }

__device__ __forceinline__ u32 last_mask(const Desc& d, u64 w) {
  u32 rem = (u32)(d.nx & 31);
  return (w == d.W - 1 && rem) ? ((1u << rem) - 1u) : 0xffffffffu;
}

// ----------------------------------------------------------- binarisation
// One warp turns a row segment of up to 1024 voxels into 32 mask words. All of
// the segment's loads are issued before any is used (32 coalesced lines per
// warp in flight per batch of 8), then one ballot per 32 voxels forms each
// word. Used for rows that are not 16-byte aligned.
template <typename TV>
__device__ __forceinline__ void thr_segment(const Desc& d, const TV* __restrict__ in,
                                            u32* __restrict__ T, u64 r, u32 x0, int lane) {
  const PassTest pt = pass_test(d);
  const u32 nx = (u32)d.nx;
  const u32 nw = min(32u, (nx - x0 + 31) >> 5);
  const TV* row = in + r * d.nx;
  u32 mine = 0;
  for (u32 i = 0; i < nw; i += 8) {
    TV v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const u32 x = x0 + (i + j) * 32 + lane;
      v[j] = x < nx ? __ldg(row + x) : TV(0);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const u32 x = x0 + (i + j) * 32 + lane;
      bool p;
      if constexpr (sizeof(TV) == 4) p = passes(pt, v[j]);
      else p = passes(pt, (u32)v[j]);
      const u32 bl = __ballot_sync(0xffffffffu, p && x < nx);
      if (lane == (int)(i + j)) mine = bl;
    }
  }
  if ((u32)lane < nw) T[r * d.W + (x0 >> 5) + lane] = mine;
}

// Non-pass flags of two uint16 values in one word: bits 15 and 31 set where
// the value lies outside [lo, hi] (lo2, hi2: the bounds in both halves). The
// value is clamped with packed 16-bit max and min, and a half differs from its
// clamp exactly when it fails; a half is nonzero when its low 15 bits plus
// 0x7fff carry into its top bit, or the top bit is set already.
__device__ __forceinline__ u32 fail2_u16(u32 v, u32 lo2, u32 hi2) {
  u32 c;
  asm("max.u16x2 %0, %1, %2;" : "=r"(c) : "r"(v), "r"(lo2));
  asm("min.u16x2 %0, %0, %1;" : "+r"(c) : "r"(hi2));
  const u32 e = c ^ v;
  return ((e & 0x7fff7fffu) + 0x7fff7fffu) | e;
}

// Four non-pass flags (bits 15, 31 of f0, then of f1) as bits 0..3: the
// bytes holding them gathered by one byte permute, then their top bits
// collected by one multiply (the products land on distinct bit positions, so
// nothing carries into bits 28..31).
__device__ __forceinline__ u32 flags4(u32 f0, u32 f1) {
  const u32 p = __byte_perm(f0, f1, 0x7531) & 0x80808080u;
  return (p * 0x00204081u) >> 28;
}

// The kPer pass bits of one 16-byte vector of values (bit k = element k).
template <typename TV>
__device__ __forceinline__ u32 vec_pass_bits(const PassTest& pt, const uint4& v) {
  u32 bits = 0;
  if constexpr (sizeof(TV) == 2) {
    if (pt.lo > 65535u) return 0u;  // nothing passes
    const u32 lo = pt.lo, hi = pt.lo + pt.span;  // hi <= 65535
    const u32 lo2 = lo | (lo << 16), hi2 = hi | (hi << 16);
    const u32 f = flags4(fail2_u16(v.x, lo2, hi2), fail2_u16(v.y, lo2, hi2)) |
                  (flags4(fail2_u16(v.z, lo2, hi2), fail2_u16(v.w, lo2, hi2)) << 4);
    return ~f & 0xffu;
  } else if constexpr (sizeof(TV) == 4) {
    bits = (passes(pt, __uint_as_float(v.x)) ? 1u : 0u) |
           (passes(pt, __uint_as_float(v.y)) ? 2u : 0u) |
           (passes(pt, __uint_as_float(v.z)) ? 4u : 0u) |
           (passes(pt, __uint_as_float(v.w)) ? 8u : 0u);
  } else {
    const u32 q[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int b = 0; b < 4; ++b)
        bits |= (passes(pt, (q[k] >> (8 * b)) & 0xffu) ? 1u : 0u) << (4 * k + b);
  }
  return bits;
}

// Vector form for 16-byte aligned rows (float32: nx % 4 == 0, uint16: nx % 8
// == 0, uint8: nx % 16 == 0). A warp reads a 1024-voxel segment with 8
// (float4), 4 or 2 (uint4) coalesced 512-byte loads, all in flight before use.
// Each lane turns its 4, 8 or 16 voxels into a nibble, byte or half-word;
// XOR-shuffles OR those of a mask word together, and lane w picks word w.
template <typename TV>
__device__ __forceinline__ void thr_segment_vec(const Desc& d, const TV* __restrict__ in,
                                                u32* __restrict__ T, u64 r, u32 x0, int lane) {
  const PassTest pt = pass_test(d);
  constexpr int kPer = 16 / sizeof(TV);  // voxels per lane and load
  constexpr int kLoads = 1024 / (32 * kPer);      // loads per segment
  constexpr int kLanesPerWord = 32 / kPer;        // lanes contributing to one word
  constexpr int kWordsPerLoad = 32 / kLanesPerWord;
  const u32 nx = (u32)d.nx;
  const u32 nw = min(32u, (nx - x0 + 31) >> 5);
  const uint4* row = reinterpret_cast<const uint4*>(in + r * d.nx);
  uint4 v[kLoads];
#pragma unroll
  for (int i = 0; i < kLoads; ++i) {
    const u32 x = x0 + (u32)i * (32 * kPer) + (u32)lane * kPer;
    v[i] = x < nx ? __ldg(row + x / kPer) : make_uint4(0u, 0u, 0u, 0u);
  }
  u32 mine = 0;
#pragma unroll
  for (int i = 0; i < kLoads; ++i) {
    const u32 x = x0 + (u32)i * (32 * kPer) + (u32)lane * kPer;
    const u32 bits = x < nx ? vec_pass_bits<TV>(pt, v[i]) : 0u;
    u32 t = bits << (kPer * (lane & (kLanesPerWord - 1)));
#pragma unroll
    for (int o = 1; o < kLanesPerWord; o <<= 1) t |= __shfl_xor_sync(0xffffffffu, t, o);
    const u32 wv = __shfl_sync(0xffffffffu, t, kLanesPerWord * (lane & (kWordsPerLoad - 1)));
    if (lane / kWordsPerLoad == i) mine = wv;
  }
  if ((u32)lane < nw) T[r * d.W + (x0 >> 5) + lane] = mine;
}

// Flat form for a 16-byte aligned volume with nx >= 256 whose rows are not
// 16-byte aligned or do not fill whole 1024-voxel segments: the volume is read
// as one flat array in steps of kFlatSpan voxels. In a step, lane j forms flat
// word j (bit b = voxel 32 j + b of the step) from its own 16-byte vectors,
// without shuffles; each mask word of a row, whose 32 voxels start anywhere in
// the flat array, is then a funnel shift of two flat words fetched by
// shuffles. Warps take contiguous ranges of steps (every item's steps in
// order) and carry the item, its pass test and the row holding the step's
// first voxel from step to step; the next step's words are loaded before the
// current step's mask words are written, and give the first flat word after
// the step (at the end of a warp's range, a ballot over its 32 voxels does).
constexpr u32 kFlatSpan = 1024;

// The flat word of voxels [x0, x0 + 32) (x0 a multiple of 32, the volume
// 16-byte aligned): 16-byte loads when all 32 lie inside, else one value at a
// time (voxels at or past N give 0).
template <typename TV>
__device__ __forceinline__ u32 flat_word(const PassTest& pt, const TV* __restrict__ in, u64 x0,
                                         u64 N) {
  constexpr int kPer = 16 / sizeof(TV);
  constexpr int kVec = 32 / kPer;
  u32 bits = 0;
  if (x0 + 32 <= N) {
    const uint4* p = reinterpret_cast<const uint4*>(in + x0);
    uint4 v[kVec];
#pragma unroll
    for (int i = 0; i < kVec; ++i) v[i] = __ldg(p + i);
#pragma unroll
    for (int i = 0; i < kVec; ++i) bits |= vec_pass_bits<TV>(pt, v[i]) << (i * kPer);
  } else {
    for (u32 k = 0; k < 32; ++k) {
      if (x0 + k < N) {
        bool q;
        if constexpr (sizeof(TV) == 4) q = passes(pt, __ldg(in + x0 + k));
        else q = passes(pt, (u32)__ldg(in + x0 + k));
        bits |= (q ? 1u : 0u) << k;
      }
    }
  }
  return bits;
}

// Mask words of the rows whose voxels x = 32 w .. start in flat step [a, a +
// 1024): F = that step's flat words (lane j: word j), f32 = the next step's
// word 0; r / rel0: the row holding voxel a and its first voxel's position
// relative to a (<= 0). Positions within the step are 32-bit. NR bounds the
// rows that start words in a step: 2 when nx >= 1024, 3 when nx >= 512, 5
// when nx >= 256.
template <int NR>
__device__ __forceinline__ void flat_emit(const Desc& d, u32* __restrict__ T, u64 a, u32 F,
                                          u32 f32, u64 r, int rel0, int lim, int lane) {
  const int nx = (int)d.nx, W = (int)d.W;
  const u32 tail = (nx & 31) ? (1u << (nx & 31)) - 1u : 0xffffffffu;  // last word's bits
  const u64 rows_left = d.rows - r;
  int cnt[NR], wlo[NR];
  int total = 0;
#pragma unroll
  for (int k = 0; k < NR; ++k) {
    const int rel = rel0 + k * nx;  // row r + k starts at a + rel
    int lo = 0, hi = 0;
    if ((u64)k < rows_left && rel < lim) {
      lo = rel >= 0 ? 0 : (-rel + 31) >> 5;
      hi = min(W, (lim - rel + 31) >> 5);  // words with start < lim
      if (hi < lo) hi = lo;
    }
    cnt[k] = hi - lo;
    wlo[k] = lo;
    total += cnt[k];
  }
  int pre[NR];  // words of the rows before row r + k (constant indices: registers)
  pre[0] = 0;
#pragma unroll
  for (int k = 1; k < NR; ++k) pre[k] = pre[k - 1] + cnt[k - 1];
  for (int o0 = 0; o0 < total; o0 += 32) {
    const int o = o0 + lane;
    int k = 0, acc = 0, wl = wlo[0];
#pragma unroll
    for (int q = 1; q < NR; ++q)
      if (o >= pre[q]) {
        k = q;
        acc = pre[q];
        wl = wlo[q];
      }
    const bool have = o < total;
    const int w = wl + (o - acc);
    const int off = have ? rel0 + k * nx + 32 * w : 0;  // in [0, 1024)
    const u32 j = (u32)off >> 5, sh = (u32)off & 31;
    const u32 lo = __shfl_sync(0xffffffffu, F, j & 31);
    u32 hi = __shfl_sync(0xffffffffu, F, (j + 1) & 31);
    if (j == 31) hi = f32;
    if (have) {
      u32 v = sh ? __funnelshift_r(lo, hi, sh) : lo;
      if (w == W - 1) v &= tail;
      T[(r + k) * d.W + w] = v;
    }
  }
}

// A warp's contiguous range [s0, s1) of the batch's flat steps.
template <typename TV>
__device__ __forceinline__ void thr_flat_range(const Batch& B, u64 s0, u64 s1, int lane) {
  u64 s = s0;
  while (s < s1) {
    // enter the item holding step s
    const u32 i = find_item(B.fseg0, B.n, s);
    const Item& I = B.it[i];
    const Desc d = desc_of(B, I);
    const PassTest pt = pass_test(d);
    const TV* __restrict__ in = (const TV*)I.in;
    u32* __restrict__ T = I.T;
    const u64 N = d.rows * d.nx;
    const u64 end = umin(s1, B.fseg0[i + 1]);  // the warp's steps of this item
    u64 a = (s - B.fseg0[i]) * kFlatSpan;
    u64 r = div_by(a, d.nx, I.m_nx);  // the row holding voxel a
    int rel0 = (int)((long long)(r * d.nx) - (long long)a);
    const int nx = (int)d.nx;
    u32 F = flat_word<TV>(pt, in, a + 32u * (u32)lane, N);
    for (; s < end; ++s) {
      const u64 an = a + kFlatSpan;
      u32 Fn = 0, f32;
      if (s + 1 < end) {  // the next step is this warp's: its words now
        Fn = flat_word<TV>(pt, in, an + 32u * (u32)lane, N);
        f32 = __shfl_sync(0xffffffffu, Fn, 0);
      } else {  // the first flat word after the step: a ballot over its 32 voxels
        const u64 x = an + lane;
        bool p = false;
        if (x < N) {
          if constexpr (sizeof(TV) == 4) p = passes(pt, __ldg(in + x));
          else p = passes(pt, (u32)__ldg(in + x));
        }
        f32 = __ballot_sync(0xffffffffu, p);
      }
      const int lim = (int)umin(kFlatSpan, N - a);
      if (nx >= 1024) flat_emit<2>(d, T, a, F, f32, r, rel0, lim, lane);
      else if (nx >= 512) flat_emit<3>(d, T, a, F, f32, r, rel0, lim, lane);
      else flat_emit<5>(d, T, a, F, f32, r, rel0, lim, lane);
      F = Fn;
      a = an;
      rel0 -= (int)kFlatSpan;
      while (rel0 <= -nx) {  // nx >= 256: at most four rows start in a step
        rel0 += nx;
        ++r;
      }
    }
  }
}

// Warps take the batch's work units (all items, in order): 1024-voxel row
// segments of the row-form items, strided over the warps, or contiguous ranges
// of the kFlatSpan-voxel steps of the flat-form items (FLAT; a launch of its
// own, so that each form keeps its registers).
template <typename TV, bool FLAT>
__global__ void __launch_bounds__(kThreads, 4) k_threshold(const __grid_constant__ Batch B) {
  const int lane = threadIdx.x & 31;
  const u64 warp = ((u64)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const u64 nwarps = ((u64)gridDim.x * blockDim.x) >> 5;
  if constexpr (FLAT) {
    const u64 total = B.fseg0[B.n];
    const u64 per = (total + nwarps - 1) / nwarps;
    const u64 s0 = warp * per;
    if (s0 < total) thr_flat_range<TV>(B, s0, umin(total, s0 + per), lane);
    return;
  }
  const u64 total = B.seg0[B.n];
  for (u64 s = warp; s < total; s += nwarps) {
    const u32 i = find_item(B.seg0, B.n, s);
    const u64 local = s - B.seg0[i];
    const Item& I = B.it[i];
    const Desc d = desc_of(B, I);
    const u64 spr = (I.nx + 1023) >> 10;
    const u64 r = spr == 1 ? local : div_by(local, spr, I.m_spr);
    const u32 x0 = (u32)(local - r * spr) << 10;
    if (I.vec) thr_segment_vec<TV>(d, (const TV*)I.in, I.T, r, x0, lane);
    else thr_segment<TV>(d, (const TV*)I.in, I.T, r, x0, lane);
  }
}

// Cube dilation of the mask on its own (the fused path dilates inside the
// compaction). A block takes a tile of rpt consecutive rows of one z slice:
// it stages their band, one row above and below, already OR-ed over the three
// slices z-1, z, z+1 (coalesced, three loads per word), then forms each word
// from the three band rows around it, the x shift taking its carries from the
// neighbouring words. Tiles never cross a slice, so the row's y and z come
// from the tile index alone.
__global__ void __launch_bounds__(kThreads) k_dilate(Desc d, const u32* __restrict__ T,
                                                     u32* __restrict__ D, u64* popcount,
                                                     u32 rpt, FastDiv fdW) {
  extern __shared__ u32 band[];  // (rpt + 2) x W
  const u64 W = d.W;
  const u64 tps = (d.ny + rpt - 1) / rpt;  // tiles per slice
  const u64 tiles = tps * d.nz;
  u64 cnt = 0;
  for (u64 t = blockIdx.x; t < tiles; t += gridDim.x) {
    const u64 z = t / tps;
    const u64 y0 = (t - z * tps) * rpt;
    const u32 nr = (u32)umin((u64)rpt, d.ny - y0);
    const u64 y_lo = y0 ? y0 - 1 : 0, y_hi = umin(y0 + nr + 1, d.ny);  // staged rows [y_lo, y_hi)
    const u32 nb = (u32)((y_hi - y_lo) * W);  // at most (rpt + 2) W <= 6144
    for (u32 k = threadIdx.x; k < nb; k += blockDim.x) {
      const u32 q = fdW.div(k);
      const u64 yy = y_lo + q, w = k - q * (u32)W;
      const u64 r = z * d.ny + yy;
      u32 v = __ldg(T + r * W + w);
      if (d.dilate) {
        if (z > 0) v |= __ldg(T + (r - d.ny) * W + w);
        if (z + 1 < d.nz) v |= __ldg(T + (r + d.ny) * W + w);
      }
      band[(yy - y0 + 1) * W + w] = v;  // band row 0 is y0 - 1
    }
    __syncthreads();
    const u32 nw = nr * (u32)W;
    for (u32 k = threadIdx.x; k < nw; k += blockDim.x) {
      const u32 ly32 = fdW.div(k);
      const u64 ly = ly32, w = k - ly32 * (u32)W;
      const u64 y = y0 + ly;
      u32 v;
      if (d.dilate) {
        u32 c = 0, lo = 0, hi = 0;
        for (int dy = -1; dy <= 1; ++dy) {
          if ((dy < 0 && y == 0) || (dy > 0 && y + 1 >= d.ny)) continue;
          const u32* b = band + (ly + 1 + dy) * W;
          c |= b[w];
          if (w > 0) lo |= b[w - 1];
          if (w + 1 < W) hi |= b[w + 1];
        }
        v = c | (c << 1) | (lo >> 31) | (c >> 1) | (hi << 31);
      } else {
        v = band[(ly + 1) * W + w];
      }
      v &= last_mask(d, w);
      D[(z * d.ny + y) * W + w] = v;
      cnt += __popc(v);
    }
    __syncthreads();
  }
  cnt = warp_sum(cnt);
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd((unsigned long long*)popcount, cnt);
}

// ------------------------------------------------------------ compaction
// Tiles of `rpt` consecutive rows: a counting kernel forms each tile's retained
// words and per-row counts, a scan turns the tile totals into offsets, and
// k_front_write writes every row's boundaries and values at its offset.
constexpr u32 kListCap = 512;  // boundaries of one row kept per warp for run copies

// Range of the retained finite values of one item: warp-reduced per-thread
// keys, one atomic per warp; the keys restart for the next item.
__device__ __forceinline__ void flush_range(State* st, u32& kmin, u32& kmax, int lane) {
  for (int o = 16; o > 0; o >>= 1) {
    kmin = min(kmin, __shfl_xor_sync(0xffffffffu, kmin, o));
    kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
  }
  if (st && lane == 0) {
    if (kmin != 0xffffffffu) atomicMin(&st->vmin_key, kmin);
    if (kmax != 0u) atomicMax(&st->vmax_key, kmax);
  }
  kmin = 0xffffffffu;
  kmax = 0u;
}

// Range key of one value (float32: order-preserving bits of a finite value;
// uint16: value + 1, so that 0 means none).
template <typename TV>
__device__ __forceinline__ void range_add(TV v, u32& kmin, u32& kmax) {
  if constexpr (sizeof(TV) == 4) {
    if (isfinite(v)) {
      const u32 kq = f32_key(__fadd_rn(v, 0.0f));
      kmin = min(kmin, kq);
      kmax = max(kmax, kq);
    }
  } else {
    kmin = min(kmin, (u32)v + 1u);
    kmax = max(kmax, (u32)v + 1u);
  }
}

// The compaction runs in three launches, none of whose blocks waits on
// another: a counting kernel forms the retained words of each tile of rows
// (dilated from T, stored to the item's D when dilating), the rows' boundary
// counts (into the container), each row's offsets within its tile and the
// tile's totals; k_scan_pairs turns the tiles' totals into offsets;
// k_front_write has warps take rows and write their boundaries and values.
// Two counting kernels give the same results: k_front_count_blk (rows staged
// by a block, better for narrow rows without dilation) and k_front_count (a
// warp per tile, better for dilated volumes); the tuning picks one.
constexpr int kStage = 16;  // mask words a thread has in flight while staging a band

struct FrontSmem {
  u32 wn[kThreads / 32], wb[kThreads / 32];  // per-warp totals, then offsets
  u64 base_n, base_nb, tile;
  u32 scratch[40];
};

// k_front_count_blk: a block per tile (tickets in order). The block stages
// the tile's band of mask rows in shared memory (three loads per word for the
// z part of the dilation), forms the retained words from the staged band,
// then its warps count whole rows and one warp scans the per-warp totals.
__global__ void __launch_bounds__(kThreads, 4) k_front_count_blk(const __grid_constant__ Batch B) {
  extern __shared__ u32 smem_dyn[];
  __shared__ FrontSmem sh;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int dilate = B.c.dilate;
  const u64 total_tiles = B.ftile0[B.n];
  while (true) {
    if (threadIdx.x == 0) sh.tile = atomicAdd(&B.ctr[0], 1u);
    __syncthreads();
    const u64 gt = sh.tile;
    if (gt >= total_tiles) break;
    const u32 item = find_item(B.ftile0, B.n, gt);
    const Item& I = B.it[item];
    const Desc d = desc_of(B, I);
    const u64 t = gt - B.ftile0[item];
    const u32 rpt = I.rpt;
    const u32* __restrict__ T = I.T;
    uint16_t* __restrict__ counts = I.counts;
    const u64 counts_cap = I.counts_cap;
    const u32 zhalo = I.zhalo;  // z-slab: T continues across the slab's z borders
    const u32 W = (u32)d.W;
    const FastDiv divW(W);
    u32* Dw = smem_dyn;                                 // [rpt * W]
    u32* rowcnt = Dw + (u64)rpt * W;                    // [rpt] boundaries per row
    u32* rown = rowcnt + rpt;                           // [rpt] retained voxels per row
    u32* bflag = rown + rpt;                            // [rpt + 2]
    u32* U = bflag + rpt + 2;                           // [rpt + 2][W] when dilating
    const bool end_extra = (d.nx & 31) == 0;  // boundary at x = nx lives past the last word
    const u64 zstride = d.ny * (u64)W;
    const u64 r0 = t * rpt;
    const u32 nrows = (u32)umin(rpt, d.rows - r0);
    const u32 nw = nrows * W;

    // ---- retained words D. Dilation by the 3x3x3 cube is separable: U = OR
    // over z of T (staged once per band row), V = OR over y of U, D = V
    // dilated in x. Band row j is row r0 - 1 + j; its flags say which
    // neighbours exist (bit 16 = the row itself exists).
    u32 any = 0u;
    if (dilate) {
      for (u32 j = threadIdx.x; j < rpt + 2; j += blockDim.x) {
        const int64_t rr = (int64_t)r0 - 1 + j;
        u32 f = 0u;
        if (rr >= 0 && rr < (int64_t)d.rows) {
          const u64 z = (u64)rr / d.ny, y = (u64)rr - z * d.ny;
          f = 16u | (y > 0 ? 1u : 0u) | (y + 1 < d.ny ? 2u : 0u) |
              ((z > 0 || (zhalo & 1u)) ? 4u : 0u) | ((z + 1 < d.nz || (zhalo & 2u)) ? 8u : 0u);
        }
        bflag[j] = f;
      }
      __syncthreads();
      // the loads of kStage words per thread are issued before any is used
      const u32 nu = (nrows + 2) * W;
      for (u32 i0 = threadIdx.x; i0 < nu; i0 += kStage * blockDim.x) {
        u32 u[kStage];
#pragma unroll
        for (int k = 0; k < kStage; ++k) {
          const u32 i = i0 + (u32)k * blockDim.x;
          u[k] = 0u;
          if (i < nu) {
            const u32 j = divW.div(i), w = i - j * W;
            const u32 f = bflag[j];
            if (f & 16u) {
              const u32* tr = T + (u64)((int64_t)r0 - 1 + j) * W + w;
              u[k] = __ldg(tr);
              if (f & 4u) u[k] |= __ldg(tr - zstride);
              if (f & 8u) u[k] |= __ldg(tr + zstride);
            }
          }
        }
#pragma unroll
        for (int k = 0; k < kStage; ++k) {
          const u32 i = i0 + (u32)k * blockDim.x;
          if (i < nu) {
            U[i] = u[k];
            any |= u[k];
          }
        }
      }
      any = __syncthreads_or(any);
      if (any) {
        for (u32 i = threadIdx.x; i < nw; i += blockDim.x) {
          const u32 lr = divW.div(i), w = i - lr * W;
          const u32 f = bflag[lr + 1];
          const u32* um = U + lr * W;  // row above (band row lr)
          const u32* uc = um + W;      // the row itself
          const u32* up = uc + W;      // row below
          auto vword = [&](u32 ww) {
            u32 v = uc[ww];
            if (f & 1u) v |= um[ww];
            if (f & 2u) v |= up[ww];
            return v;
          };
          const u32 c = vword(w);
          const u32 lo = w > 0 ? vword(w - 1) : 0u;
          const u32 hi = w + 1 < W ? vword(w + 1) : 0u;
          Dw[i] = (c | (c << 1) | (lo >> 31) | (c >> 1) | (hi << 31)) & last_mask(d, w);
        }
      }
    } else {
      for (u32 i0 = threadIdx.x; i0 < nw; i0 += kStage * blockDim.x) {
        u32 v[kStage];
#pragma unroll
        for (int k = 0; k < kStage; ++k) {
          const u32 i = i0 + (u32)k * blockDim.x;
          v[k] = i < nw ? __ldg(T + r0 * W + i) : 0u;
        }
#pragma unroll
        for (int k = 0; k < kStage; ++k) {
          const u32 i = i0 + (u32)k * blockDim.x;
          if (i < nw) {
            const u32 w = i - divW.div(i) * W;
            const u32 x = v[k] & last_mask(d, w);
            Dw[i] = x;
            any |= x;
          }
        }
      }
      any = __syncthreads_or(any);
    }
    __syncthreads();

    // ---- per-warp totals: warps own whole rows (in order), lanes walk words
    const u32 pwr = (nrows + (kThreads / 32) - 1) / (kThreads / 32);
    const u32 rbeg = min(nrows, warp * pwr), rend = min(nrows, rbeg + pwr);
    {
      u32 cn = 0, cb = 0;
      if (!any)
        for (u32 lr = rbeg + lane; lr < rend; lr += 32) {
          rowcnt[lr] = 0;
          rown[lr] = 0;
        }
      for (u32 lr = any ? rbeg : rend; lr < rend; ++lr) {
        const u32* drow = Dw + lr * W;
        u32 rn = 0, rb = 0;
        for (u32 w = lane; w < W; w += 32) {
          const u32 dv = drow[w];
          const u32 pv = w ? drow[w - 1] : 0u;
          rn += __popc(dv);
          rb += __popc(dv ^ ((dv << 1) | (pv >> 31))) +
                ((end_extra && w == W - 1) ? (dv >> 31) : 0u);
        }
        rn = warp_sum(rn);
        rb = warp_sum(rb);
        if (lane == 0) {
          rowcnt[lr] = rb;
          rown[lr] = rn;
        }
        cn += rn;
        cb += rb;
      }
      if (lane == 0) {
        sh.wn[warp] = cn;
        sh.wb[warp] = cb;
      }
    }
    __syncthreads();
    if (warp == 0) {
      const u32 a = lane < kThreads / 32 ? sh.wn[lane] : 0u;
      const u32 b = lane < kThreads / 32 ? sh.wb[lane] : 0u;
      const u32 ia = warp_incl_scan(a), ib = warp_incl_scan(b);
      const u64 tn = __shfl_sync(0xffffffffu, ia, kThreads / 32 - 1);
      const u64 tb = __shfl_sync(0xffffffffu, ib, kThreads / 32 - 1);
      if (lane < kThreads / 32) {
        sh.wn[lane] = ia - a;
        sh.wb[lane] = ib - b;
      }
      if (lane == 0) {
        I.ftn[t] = (u32)tn;
        I.ftb[t] = (u32)tb;
      }
      if (I.fscan && count_done(&I.st->done_front, I.ftiles)) {  // the item's tile scan
        u64 an, ab;
        warp_scan2(I.ftn, I.ftb, I.ftiles, I.ftno, I.ftbo, an, ab);
        if (lane == 0) {
          I.sizes[0] = an;
          I.sizes[1] = ab;
        }
      }
    }
    __syncthreads();
    // each row's offsets within the tile (a warp walks its own rows in order)
    {
      u32 on = sh.wn[warp], ob = sh.wb[warp];
      for (u32 lr = rbeg; lr < rend; ++lr) {
        if (lane == 0) {
          I.rno[r0 + lr] = on;
          I.rbo[r0 + lr] = ob;
        }
        on += rown[lr];
        ob += rowcnt[lr];
      }
    }
    // the rows' boundary counts into the container, the retained words to D
    for (u32 lr = threadIdx.x; lr < nrows; lr += blockDim.x) {
      const u64 r = r0 + lr;
      if (r < counts_cap) counts[r] = (uint16_t)rowcnt[lr];
    }
    if (dilate)  // (Dw holds nothing when the band is empty)
      for (u32 i = threadIdx.x; i < nw; i += blockDim.x) I.D[r0 * W + i] = any ? Dw[i] : 0u;
    __syncthreads();
  }
}

// Raw mask loads of one word of one row: T of the row and, when dilating, of
// the rows one slice before and after (present only where those slices are).
struct URaw {
  u32 c, zlo, zhi;
};

template <bool DIL>
__device__ __forceinline__ void u_issue(const u32* p, bool ok, bool zlo, bool zhi, u64 zstride,
                                        URaw& q) {
  q.c = q.zlo = q.zhi = 0u;
  if (ok) {
    q.c = __ldg(p);
    if constexpr (DIL) {
      if (zlo) q.zlo = __ldg(p - zstride);
      if (zhi) q.zhi = __ldg(p + zstride);
    }
  }
}

__device__ __forceinline__ u32 u_of(const URaw& q) { return q.c | q.zlo | q.zhi; }

// k_front_count: one warp per tile, no block barriers. The warp walks the
// tile's rows in 32-word columns (lane = word); the 3x3x3 dilation is
// separable: U = OR over z of T (three loads), V = OR of U over the rows y-1,
// y, y+1 (a window of three rows in registers, the next row's loads issued one
// row ahead), D = V dilated in x (neighbour words by shuffles; for rows of
// more than one column, lanes 0 and 31 also hold the words just outside the
// column). Per row one warp reduction of the packed counts gives the retained
// voxels and boundaries; the tile's rows are then scanned in parallel for
// their offsets within the tile.

template <bool DIL>
__device__ __forceinline__ void front_count_tile(const Batch& B, const Item& I, const Desc& d,
                                                 u64 t, u32* rown, u32* rowcnt, int lane) {
  const u64 W = d.W;
  const u32 rpt = I.rpt;
  const u64 r0 = t * rpt;
  const u32 nrows = (u32)umin(rpt, d.rows - r0);
  const bool end_extra = (d.nx & 31) == 0;  // boundary at x = nx lives past the last word
  const bool multi = W > 32;                // rows span more than one column
  const u64 zstride = d.ny * W;
  const u32* __restrict__ T = I.T;
  u32* __restrict__ Dm = I.D;
  const u32 zhalo = I.zhalo;  // z-slab: T continues across the slab's z borders
  // slice position of the first row
  const u64 zc064 = div_by(r0, d.ny, I.m_ny);
  const u32 ny = (u32)d.ny, nz = (u32)d.nz;  // slice sizes fit 32 bits
  const u32 zc0 = (u32)zc064, yc0 = (u32)(r0 - zc064 * d.ny);
  // rows from r0 on that exist (loads past the item's last row are skipped)
  const u64 avail = d.rows - r0;
  for (u32 w0 = 0; w0 < (u32)W; w0 += 32) {
    const u32 w = w0 + lane;
    const bool wv = w < W;
    const u32 lmask = wv ? last_mask(d, w) : 0u;
    // lanes 0 and 31 also hold the word left / right of the column
    const u32 hw = lane == 0 ? w0 - 1u : w0 + 32u;
    const bool hv = multi && ((lane == 0 && w0 > 0) || (DIL && lane == 31 && (u64)w0 + 32 < W));
    // issue position: row r0 + ii with slice coordinates (zi, yi)
    const u32* pw = T + r0 * W + w;   // this lane's word of the issue row
    const u32* ph = T + r0 * W + hw;  // the halo word of the issue row
    u64 ii = 0;
    u32 zi = zc0, yi = yc0;
    bool zl = zc0 > 0 || (zhalo & 1u), zh = zc0 + 1 < nz || (zhalo & 2u);
    auto issue = [&](URaw& q, URaw& hq) {
      const bool ok = ii < avail;
      u_issue<DIL>(pw, ok && wv, zl, zh, zstride, q);
      if (multi) u_issue<DIL>(ph, ok && hv, zl, zh, zstride, hq);
      ++ii;
      pw += W;
      ph += W;
      if (++yi == ny) {
        yi = 0;
        ++zi;
        zl = true;
        zh = zi + 1 < nz || (zhalo & 2u);
      }
    };
    u32 um = 0u, hm = 0u;  // U of the row above (used only when it is in the slice)
    if (DIL && yc0 > 0) {
      URaw a, ha;
      u_issue<DIL>(pw - W, wv, zl, zh, zstride, a);
      um = u_of(a);
      if (multi) {
        u_issue<DIL>(ph - W, hv, zl, zh, zstride, ha);
        hm = u_of(ha);
      }
    }
    // two load buffers used in turn (no register copies of loads in flight):
    // dilating, the buffer read at row r holds row r + 1 and row r + 2 is
    // issued into the other; otherwise it holds row r and row r + 1 is issued
    URaw qa, hqa{0u, 0u, 0u}, qb, hqb{0u, 0u, 0u};
    issue(qa, hqa);  // row r0
    u32 uc = 0u, hc = 0u;
    if (DIL) {
      uc = u_of(qa);
      hc = u_of(hqa);
      issue(qa, hqa);  // row r0 + 1
    }
    u32 y = yc0;
    u32* pd_out = DIL ? Dm + r0 * W + w : nullptr;
    auto step = [&](u32 lr, const URaw& cur, const URaw& hcur, URaw& nxt, URaw& hnxt) {
      issue(nxt, hnxt);
      u32 v, vh = 0u;
      if constexpr (DIL) {
        const u32 up = u_of(cur);
        const bool ym = y > 0, yp = y + 1 < ny;
        v = uc | (ym ? um : 0u) | (yp ? up : 0u);
        um = uc;
        uc = up;
        if (multi) {
          const u32 hp = u_of(hcur);
          vh = hc | (ym ? hm : 0u) | (yp ? hp : 0u);
          hm = hc;
          hc = hp;
        }
      } else {
        v = u_of(cur);
        if (multi) vh = u_of(hcur);
      }
      if (++y == ny) y = 0;
      // retained word of this lane, and the top bit of the word left of it
      u32 hlo = 0u, hhi = 0u;  // words w0 - 1 and w0 + 32 (zero for one column)
      if (multi) {
        hlo = __shfl_sync(0xffffffffu, vh, 0);
        hhi = __shfl_sync(0xffffffffu, vh, 31);
      }
      u32 dv, ptop;
      if constexpr (DIL) {
        const u32 vlo = __shfl_up_sync(0xffffffffu, v, 1);
        const u32 vhi = __shfl_down_sync(0xffffffffu, v, 1);
        const u32 lo = lane == 0 ? hlo : vlo;
        const u32 hi = lane == 31 ? hhi : vhi;
        dv = (v | (v << 1) | (lo >> 31) | (v >> 1) | (hi << 31)) & lmask;
        const u32 pd = __shfl_up_sync(0xffffffffu, dv, 1);
        // bit 31 of the dilated word w0 - 1 (never the last word of the row)
        ptop = lane == 0 ? ((hlo >> 31) | (hlo >> 30) | (w0 > 0 ? v : 0u)) & 1u : pd >> 31;
      } else {
        dv = v & lmask;
        const u32 pd = __shfl_up_sync(0xffffffffu, dv, 1);
        ptop = lane == 0 ? hlo >> 31 : pd >> 31;
      }
      // (lanes past the row's last word count nothing: the carried top bit of
      // the last word is the x = nx boundary, counted by end_extra)
      const u32 nb = wv ? __popc(dv ^ ((dv << 1) | ptop)) +
                              ((end_extra && w == W - 1) ? (dv >> 31) : 0u)
                        : 0u;
      // both at most 1025 per column
      const u32 packed = __reduce_add_sync(0xffffffffu, __popc(dv) | (nb << 16));
      if (lane == 0) {
        const u32 a0 = w0 ? rown[lr] : 0u, b0 = w0 ? rowcnt[lr] : 0u;
        rown[lr] = a0 + (packed & 0xffffu);
        rowcnt[lr] = b0 + (packed >> 16);
      }
      if (DIL) {
        if (wv) *pd_out = dv;
        pd_out += W;
      }
    };
    for (u32 lr = 0; lr < nrows; lr += 2) {
      step(lr, qa, hqa, qb, hqb);
      if (lr + 1 < nrows) step(lr + 1, qb, hqb, qa, hqa);
    }
  }
  __syncwarp();
  // the rows' offsets within the tile, their boundary counts, the tile totals
  uint16_t* __restrict__ counts = I.counts;
  const u64 counts_cap = I.counts_cap;
  u32 on = 0, ob = 0;
  for (u32 b = 0; b < nrows; b += 32) {
    const u32 lr = b + lane;
    const u32 n_ = lr < nrows ? rown[lr] : 0u, c_ = lr < nrows ? rowcnt[lr] : 0u;
    const u32 in_ = warp_incl_scan(n_), ic = warp_incl_scan(c_);
    if (lr < nrows) {
      const u64 r = r0 + lr;
      I.rno[r] = on + in_ - n_;
      I.rbo[r] = ob + ic - c_;
      if (r < counts_cap) counts[r] = (uint16_t)c_;
    }
    on += __shfl_sync(0xffffffffu, in_, 31);
    ob += __shfl_sync(0xffffffffu, ic, 31);
  }
  if (lane == 0) {
    I.ftn[t] = on;
    I.ftb[t] = ob;
  }
  if (I.fscan && count_done(&I.st->done_front, I.ftiles)) {  // the item's tile scan
    u64 an, ab;
    warp_scan2(I.ftn, I.ftb, I.ftiles, I.ftno, I.ftbo, an, ab);
    if (lane == 0) {
      I.sizes[0] = an;
      I.sizes[1] = ab;
    }
  }
  __syncwarp();
}

template <bool DIL>
__global__ void __launch_bounds__(kThreads, 4) k_front_count(const __grid_constant__ Batch B) {
  __shared__ u32 rows_all[kThreads / 32][2 * kMaxTileRows];  // per warp: row totals
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  u32* rown = rows_all[warp];
  u32* rowcnt = rown + kMaxTileRows;
  const u64 total_tiles = B.ftile0[B.n];
  const u64 nwarps = ((u64)gridDim.x * blockDim.x) >> 5;
  for (u64 gt = ((u64)blockIdx.x * blockDim.x + threadIdx.x) >> 5; gt < total_tiles;
       gt += nwarps) {
    const u32 item = find_item(B.ftile0, B.n, gt);
    const Item& I = B.it[item];
    const Desc d = desc_of(B, I);
    const u64 t = gt - B.ftile0[item];
    front_count_tile<DIL>(B, I, d, t, rown, rowcnt, lane);
  }
}

// Exclusive scans of two counts per tile or chunk, several blocks per item:
// a block takes kScanTile entries (8 consecutive ones per thread), scans them,
// and a decoupled look-back over the item's few scan tiles gives its offset.
// MODE 0: compaction tiles (ftn, ftb -> ftno, ftbo; totals n, nb); MODE 1:
// pack chunks (cw, crec -> cwoff, crecoff; totals nwords, nout).
template <int MODE>
__global__ void __launch_bounds__(1024) k_scan_pairs(const __grid_constant__ Batch B) {
  if (MODE == 1 && halted(B.status)) return;  // the compaction scan of this call gave up
  __shared__ u64 pre[kMaxBatch + 1];
  __shared__ u64 scratch[40];
  __shared__ u64 s_tile, s_ex[2];
  const int tid = threadIdx.x, lane = tid & 31;
  for (u32 i = tid; i < B.n; i += blockDim.x) {  // counts read in parallel
    const Item& I = B.it[i];
    const u64 cnt = MODE == 0 ? I.ftiles : (umin(I.sizes[0], I.N) + B.c.C - 1) / B.c.C;
    const bool done = MODE == 0 ? I.fscan != 0 : I.pscan != 0;  // scanned by the counting kernel
    pre[i + 1] = done ? 0 : (cnt + kScanTile - 1) / kScanTile;
  }
  __syncthreads();
  if (tid == 0) {
    u64 acc = 0;
    for (u32 i = 0; i < B.n; ++i) {
      const u64 c = pre[i + 1];
      pre[i] = acc;
      acc += c;
    }
    pre[B.n] = acc;
  }
  __syncthreads();
  const u64 total = pre[B.n];
  while (true) {
    if (tid == 0) s_tile = atomicAdd(&B.ctr[5 + MODE], 1u);
    __syncthreads();
    const u64 gt = s_tile;
    if (gt >= total) break;
    const u32 item = find_item(pre, B.n, gt);
    const Item& I = B.it[item];
    const u64 t = gt - pre[item];
    const u64 cnt = MODE == 0 ? I.ftiles : (umin(I.sizes[0], I.N) + B.c.C - 1) / B.c.C;
    const u64 ntiles = (cnt + kScanTile - 1) / kScanTile;
    const u32* __restrict__ a = MODE == 0 ? I.ftn : I.cw;
    const u32* __restrict__ b = MODE == 0 ? I.ftb : I.crec;
    u64* __restrict__ ao = MODE == 0 ? I.ftno : I.cwoff;
    u64* __restrict__ bo = MODE == 0 ? I.ftbo : I.crecoff;
    const u64 i0 = t * kScanTile + (u64)tid * 8;
    u32 va[8], vb[8];
    u64 sa = 0, sb = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      va[k] = i0 + k < cnt ? __ldg(a + i0 + k) : 0u;
      vb[k] = i0 + k < cnt ? __ldg(b + i0 + k) : 0u;
      sa += va[k];
      sb += vb[k];
    }
    u64 ta, tb;
    u64 ea = block_excl_scan<u64>(sa, scratch, &ta);
    u64 eb = block_excl_scan<u64>(sb, scratch, &tb);
    if (tid < 32) {
      u64 mine[2] = {ta, tb}, excl[2];
      lookback_warp<2>(MODE == 0 ? I.lbsf : I.lbsp, t, mine, excl, B.status, B.c.spin_limit,
                       B.c.hold_scans && item == 0);
      if (lane == 0) {
        s_ex[0] = excl[0];
        s_ex[1] = excl[1];
        if (t == ntiles - 1) {
          if (MODE == 0) {
            I.sizes[0] = excl[0] + ta;
            I.sizes[1] = excl[1] + tb;
          } else {
            I.st->nwords = excl[0] + ta;
            I.st->nout = excl[1] + tb;
            if (excl[1] + tb > I.rec_cap) I.st->cap_flag = 1u;
          }
        }
      }
    }
    __syncthreads();
    ea += s_ex[0];
    eb += s_ex[1];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      if (i0 + k < cnt) {
        ao[i0 + k] = ea;
        bo[i0 + k] = eb;
      }
      ea += va[k];
      eb += vb[k];
    }
    __syncthreads();
  }
}

// Warps take up to kRowsPerTicket consecutive rows of the batch (all items' rows
// in order) per ticket: lane j looks up row j's item, boundary count and offsets (the
// tile's offset plus the row's offset in its tile); then the warp walks the
// rows that retain anything: the boundaries (x positions where D turns on or
// off) are written in order, and the values of each run [x_start, x_end) are
// copied with coalesced loads and stores while the value range is gathered.
constexpr u32 kRowsPerTicket = 8;
constexpr u32 kRunCap = 128;  // runs a warp gathers before copying them

// Runs of one warp waiting to be copied: source and destination byte
// addresses, length in elements.
struct RunList {
  u64 src[kRunCap], dst[kRunCap];
  u32 len[kRunCap];
  u32 cpre[kRunCap + 1];  // prefix of the runs' 16-byte destination chunks
  u32 ppre[kRunCap + 1];  // prefix of the runs' head and tail elements
};

// Largest i < n with pre[i] <= x (pre nondecreasing), given pre[lo] <= x: a
// lane's chunks rise, so the search gallops forward from the run of its
// previous chunk and then bisects the last step.
__device__ __forceinline__ u32 run_from(const u32* pre, u32 n, u32 x, u32 lo) {
  u32 hi = lo + 1, step = 2;
  while (hi < n && pre[hi] <= x) {
    lo = hi;
    hi = lo + step;
    step <<= 1;
  }
  if (hi > n) hi = n;
  while (hi - lo > 1) {
    const u32 mid = (lo + hi) >> 1;
    if (pre[mid] <= x) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Copies the gathered runs with the whole warp at once: every lane takes
// 16-byte destination chunks across all runs (funnel-shifted out of five
// aligned source words), then the runs' unaligned head and tail elements;
// loads of many runs are in flight together. The value range is gathered.
template <typename TV>
__device__ void flush_runs(RunList& rl, u32 nr, int lane, u32& kmin, u32& kmax) {
  constexpr u32 kPer = 16 / sizeof(TV);
  __syncwarp();
  // per run: head elements (to the destination's 16-byte boundary), chunks
  u32 cacc = 0, pacc = 0;
  for (u32 i0 = 0; i0 < nr; i0 += 32) {
    const u32 i = i0 + lane;
    u32 ch = 0, pc = 0;
    if (i < nr) {
      const u32 len = rl.len[i];
      const u32 h = umin((u32)(((16u - (rl.dst[i] & 15u)) & 15u) / sizeof(TV)), len);
      ch = (len - h) / kPer;
      pc = len - ch * kPer;
    }
    const u32 ci = warp_incl_scan(ch), pi = warp_incl_scan(pc);
    if (i < nr) {
      rl.cpre[i] = cacc + ci - ch;
      rl.ppre[i] = pacc + pi - pc;
    }
    cacc += __shfl_sync(0xffffffffu, ci, 31);
    pacc += __shfl_sync(0xffffffffu, pi, 31);
  }
  if (lane == 0) {
    rl.cpre[nr] = cacc;
    rl.ppre[nr] = pacc;
  }
  __syncwarp();
  // whole 16-byte chunks, four per lane at a time (their loads issued together)
  constexpr int kU = 4;
  u32 ri = 0;  // run of the lane's latest chunk
  for (u32 u0 = lane; u0 < cacc; u0 += 32 * kU) {
    u32 w[kU][5];
    u64 dq[kU];
    u32 shq[kU];
#pragma unroll
    for (int q = 0; q < kU; ++q) {
      const u32 u = u0 + 32u * q;
      dq[q] = 0;
      shq[q] = 0;
#pragma unroll
      for (int e = 0; e < 5; ++e) w[q][e] = 0u;
      if (u < cacc) {
        const u32 i = ri = run_from(rl.cpre, nr, u, ri);
        const u32 k = u - rl.cpre[i];
        const u32 len = rl.len[i];
        const u64 db = rl.dst[i];
        const u32 h = umin((u32)(((16u - (db & 15u)) & 15u) / sizeof(TV)), len);
        const uintptr_t sa = (uintptr_t)rl.src[i] + (uintptr_t)(h + k * kPer) * sizeof(TV);
        shq[q] = (u32)(sa & 3u) * 8u;
        const u32* sw = reinterpret_cast<const u32*>(sa & ~(uintptr_t)3);
        w[q][0] = __ldg(sw);
        w[q][1] = __ldg(sw + 1);
        w[q][2] = __ldg(sw + 2);
        w[q][3] = __ldg(sw + 3);
        if (shq[q]) w[q][4] = __ldg(sw + 4);
        dq[q] = db + (u64)h * sizeof(TV) + 16ull * k;
      }
    }
#pragma unroll
    for (int q = 0; q < kU; ++q) {
      if (u0 + 32u * q < cacc) {
        const u32 sh = shq[q];
        const uint4 v = make_uint4(
            __funnelshift_r(w[q][0], w[q][1], sh), __funnelshift_r(w[q][1], w[q][2], sh),
            __funnelshift_r(w[q][2], w[q][3], sh), __funnelshift_r(w[q][3], w[q][4], sh));
        *reinterpret_cast<uint4*>(dq[q]) = v;
        if constexpr (sizeof(TV) == 4) {
          range_add<float>(__uint_as_float(v.x), kmin, kmax);
          range_add<float>(__uint_as_float(v.y), kmin, kmax);
          range_add<float>(__uint_as_float(v.z), kmin, kmax);
          range_add<float>(__uint_as_float(v.w), kmin, kmax);
        } else if constexpr (sizeof(TV) == 2) {  // eight values: packed 16-bit minima, maxima
          const u32 mn = __vminu2(__vminu2(v.x, v.y), __vminu2(v.z, v.w));
          const u32 mx = __vmaxu2(__vmaxu2(v.x, v.y), __vmaxu2(v.z, v.w));
          kmin = min(kmin, min(mn & 0xffffu, mn >> 16) + 1u);
          kmax = max(kmax, max(mx & 0xffffu, mx >> 16) + 1u);
        }  // (8-bit values carry no range)
      }
    }
  }
  // head and tail elements, four per lane at a time
  ri = 0;
  for (u32 e0 = lane; e0 < pacc; e0 += 32 * kU) {
    TV vq[kU];
    TV* dp[kU];
#pragma unroll
    for (int q = 0; q < kU; ++q) {
      const u32 e = e0 + 32u * q;
      dp[q] = nullptr;
      vq[q] = TV(0);
      if (e < pacc) {
        const u32 i = ri = run_from(rl.ppre, nr, e, ri);
        const u32 k = e - rl.ppre[i];
        const u32 len = rl.len[i];
        const u64 db = rl.dst[i];
        const u32 h = umin((u32)(((16u - (db & 15u)) & 15u) / sizeof(TV)), len);
        const u32 mid = (len - h) / kPer * kPer;
        const u32 x = k < h ? k : h + mid + (k - h);  // element index within the run
        vq[q] = __ldg(reinterpret_cast<const TV*>(rl.src[i]) + x);
        dp[q] = reinterpret_cast<TV*>(db) + x;
      }
    }
#pragma unroll
    for (int q = 0; q < kU; ++q) {
      if (dp[q]) {
        *dp[q] = vq[q];
        if constexpr (sizeof(TV) != 1) range_add<TV>(vq[q], kmin, kmax);
      }
    }
  }
  __syncwarp();
}


template <typename TV>
__global__ void __launch_bounds__(kThreads, 4) k_front_write(const __grid_constant__ Batch B) {
  if (halted(B.status)) return;  // a tile scan of this call gave up
  __shared__ uint16_t blist_all[kThreads / 32][kListCap];
  __shared__ RunList runs_all[kThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const u32 below = (1u << lane) - 1u;
  uint16_t* lst = blist_all[warp];
  RunList& rl = runs_all[warp];
  u32 nruns = 0;  // runs gathered and not yet copied
  const u64 total_rows = B.row0[B.n];
  u32 kmin = 0xffffffffu, kmax = 0u;
  u32 cur = 0xffffffffu;  // item whose range the warp accumulates
  // rows per ticket: kRowsPerTicket, fewer when the batch has too few rows to
  // give every warp about four tickets (a warp walks a ticket's rows one after
  // another; with rows of unequal lengths, as in a batch of images of several
  // sizes, the last tickets decide when the kernel ends)
  const u64 nwarps = ((u64)gridDim.x * blockDim.x) >> 5;
  const u32 per = (u32)umax(1, umin(kRowsPerTicket, total_rows / (4 * nwarps)));
  while (true) {
    u64 g0 = 0;
    if (lane == 0) g0 = atomicAdd(&B.ctr[4], per);
    g0 = __shfl_sync(0xffffffffu, g0, 0);
    if (g0 >= total_rows) break;
    // lane j < per: row g0 + j's item, boundary count, offsets
    const u64 g = lane < (int)per ? g0 + lane : total_rows;
    u32 my_item = 0, my_nbr = 0;
    u64 my_on = 0, my_ob = 0;
    if (g < total_rows) {
      my_item = find_item(B.row0, B.n, g);
      const Item& I = B.it[my_item];
      const u64 r = g - B.row0[my_item];
      const u64 t = div_by(r, I.rpt, I.m_rpt);
      my_nbr = r < I.counts_cap ? (u32)I.counts[r] : 0xffffffffu;
      my_on = I.ftno[t] + I.rno[r];
      my_ob = I.ftbo[t] + I.rbo[r];
    }
    u32 todo = __ballot_sync(0xffffffffu, g < total_rows && my_nbr != 0u);
    while (todo) {
      const int j = __ffs(todo) - 1;
      todo &= todo - 1;
      const u32 item = __shfl_sync(0xffffffffu, my_item, j);
      u32 nbr = __shfl_sync(0xffffffffu, my_nbr, j);
      u64 on = __shfl_sync(0xffffffffu, my_on, j);
      const u64 ob = __shfl_sync(0xffffffffu, my_ob, j);
      const Item& I = B.it[item];
      if (item != cur) {  // copy the previous item's runs, flush its value range
        if (nruns) flush_runs<TV>(rl, nruns, lane, kmin, kmax);
        nruns = 0;
        flush_range(cur == 0xffffffffu ? nullptr : B.it[cur].rst, kmin, kmax, lane);
        cur = item;
      }
      const u64 r = g0 + j - B.row0[item];
      const u32 W = (u32)I.W, nx = (u32)I.nx;  // nx < 2^16 (boundaries are 16-bit)
      const bool end_extra = (nx & 31) == 0;
      const u32 tail = end_extra ? 0xffffffffu : (1u << (nx & 31)) - 1u;  // last word's bits
      auto lmask = [&](u32 w) { return w == W - 1 ? tail : 0xffffffffu; };
      const u32* drow = (B.c.dilate ? I.D : I.T) + r * W;
      const TV* irow = (const TV*)I.in + (u64)r * nx;
      TV* __restrict__ P = (TV*)I.P;
      uint16_t* __restrict__ bounds = I.bounds;
      const u64 bounds_cap = I.bounds_cap;
      if (nbr == 0xffffffffu) {  // container too small for the counts: count again
        u32 rb = 0;
        for (u32 w = lane; w < W; w += 32) {
          const u32 dv = __ldg(drow + w) & lmask(w);
          const u32 pv = w ? __ldg(drow + w - 1) & lmask(w - 1) : 0u;
          rb += __popc(dv ^ ((dv << 1) | (pv >> 31))) + ((end_extra && w == W - 1) ? (dv >> 31) : 0u);
        }
        nbr = warp_sum(rb);
        if (nbr == 0) continue;
      }
      const bool fast = nbr <= kListCap;
      u32 bo = 0;
      for (u32 w0 = 0; w0 < W; w0 += 32) {
        const u32 w = w0 + lane;
        u32 ev = 0u, ex = 0u;
        if (w < W) {
          const u32 dv = __ldg(drow + w) & lmask(w);
          const u32 pv = w ? __ldg(drow + w - 1) & lmask(w - 1) : 0u;
          ev = dv ^ ((dv << 1) | (pv >> 31));
          ex = (end_extra && w == W - 1) ? (dv >> 31) : 0u;
        }
        const u32 pb = __popc(ev) + ex;
        const u32 inc = warp_incl_scan(pb);
        u32 o = bo + inc - pb;
        while (ev) {
          const u32 x = w * 32 + (__ffs(ev) - 1);
          ev &= ev - 1;
          if (ob + o < bounds_cap) bounds[ob + o] = (uint16_t)x;
          else set_status(B.status, ROIX_ECAPACITY);
          if (fast && o < kListCap) lst[o] = (uint16_t)x;
          ++o;
        }
        if (ex) {
          if (ob + o < bounds_cap) bounds[ob + o] = (uint16_t)nx;
          else set_status(B.status, ROIX_ECAPACITY);
          if (fast && o < kListCap) lst[o] = (uint16_t)nx;
        }
        bo += __shfl_sync(0xffffffffu, inc, 31);
      }
      __syncwarp();
      if (bo != nbr) {  // the row's count disagrees with its mask: copy nothing
        set_status(B.status, ROIX_ECORRUPT);
        continue;
      }
      if (fast) {
        for (u32 i = 0; i < nbr; i += 2) {
          const u32 xs = lst[i], xe = lst[i + 1];
          const TV* src = irow + xs;
          TV* dst = P + on;
          const u32 len = xe - xs;
          if (nruns == kRunCap) {  // the list is full: copy what it holds
            flush_runs<TV>(rl, nruns, lane, kmin, kmax);
            nruns = 0;
          }
          if (lane == 0) {
            rl.src[nruns] = (u64)(uintptr_t)src;
            rl.dst[nruns] = (u64)(uintptr_t)dst;
            rl.len[nruns] = len;
          }
          ++nruns;
          on += len;
        }
      } else {
        // many short runs: lanes take the bits of one word at a time
        for (u32 w0 = 0; w0 < W; w0 += 32) {
          const u32 dv_l = w0 + lane < W ? __ldg(drow + w0 + lane) & lmask(w0 + lane) : 0u;
          const u32 pn = __popc(dv_l);
          const u32 sn = warp_incl_scan(pn) - pn;
          u32 nz = __ballot_sync(0xffffffffu, dv_l != 0u);
          while (nz) {
            const int k = __ffs(nz) - 1;
            nz &= nz - 1;
            const u32 dv = __shfl_sync(0xffffffffu, dv_l, k);
            const u32 so = __shfl_sync(0xffffffffu, sn, k);
            if ((dv >> lane) & 1u) {
              const TV v = __ldg(irow + (u64)(w0 + k) * 32 + lane);
              P[on + so + __popc(dv & below)] = v;
              if constexpr (sizeof(TV) == 4) {
                if (isfinite(v)) {
                  const u32 kq = f32_key(__fadd_rn(v, 0.0f));
                  kmin = min(kmin, kq);
                  kmax = max(kmax, kq);
                }
              } else {
                kmin = min(kmin, (u32)v + 1u);
                kmax = max(kmax, (u32)v + 1u);
              }
            }
          }
          on += __shfl_sync(0xffffffffu, sn + pn, 31);
        }
      }
      __syncwarp();
    }
    if (nruns) flush_runs<TV>(rl, nruns, lane, kmin, kmax);  // the ticket's runs
    nruns = 0;
  }
  flush_range(cur == 0xffffffffu ? nullptr : B.it[cur].rst, kmin, kmax, lane);
}

int occupancy_grid(const void* fn, int threads, size_t smem, int sms) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem);
  if (per_sm < 1) per_sm = 1;
  return per_sm * sms;
}

}  // namespace

void launch_scan_pairs(const Launch& L, const Batch& B, int mode, u64 tiles_cap) {
  if (tiles_cap == 0) return;
  const u64 grid = umin(tiles_cap, (u64)L.sms * 2);
  if (mode == 0) k_scan_pairs<0><<<(unsigned)grid, 1024, 0, L.stream>>>(B);
  else k_scan_pairs<1><<<(unsigned)grid, 1024, 0, L.stream>>>(B);
}

void launch_threshold(const Launch& L, const Batch& B) {
  // blocks per SM: the tuned value, but never more than fit at once (a second
  // partial wave of equally loaded blocks would leave SMs idle at the end)
  auto run = [&](auto kernel, u64 units, u64 per_sm) {
    if (units == 0) return;
    const u64 warps_per_block = kThreads / 32;
    u64 blocks = (units + warps_per_block - 1) / warps_per_block;
    int fit = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, (const void*)kernel, kThreads, 0);
    const u64 cap = (u64)L.sms * umax(1, umin(per_sm, (u64)(fit > 0 ? fit : 1)));
    if (blocks > cap) blocks = cap;
    kernel<<<(unsigned)blocks, kThreads, 0, L.stream>>>(B);
  };
  const u64 segs = B.seg0[B.n], spans = B.fseg0[B.n];
  const u64 rb = L.t.thr_blocks_per_sm ? L.t.thr_blocks_per_sm : 8;
  const u64 fb = L.t.flat_blocks_per_sm ? L.t.flat_blocks_per_sm : 4;
  if (B.c.dtype == ROIX_F32) {
    run(k_threshold<float, false>, segs, rb);
    run(k_threshold<float, true>, spans, fb);
  } else if (B.c.dtype == ROIX_U16) {
    run(k_threshold<unsigned short, false>, segs, rb);
    run(k_threshold<unsigned short, true>, spans, fb);
  } else {
    run(k_threshold<unsigned char, false>, segs, rb);
    run(k_threshold<unsigned char, true>, spans, fb);
  }
}

void launch_dilate(const Launch& L, const Desc& d, const u32* T, u32* D, u64* popcount) {
  const u64 total = d.rows * d.W;
  if (total == 0) return;
  u64 rpt = 2048 / d.W;  // about 2048 words per tile
  if (rpt < 1) rpt = 1;
  if (rpt > d.ny) rpt = d.ny;
  const size_t smem = (size_t)(rpt + 2) * d.W * 4;
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(k_dilate, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const u64 tiles = (d.ny + rpt - 1) / rpt * d.nz;
  u64 blocks = tiles;
  if (blocks > (u64)L.sms * 8) blocks = (u64)L.sms * 8;
  k_dilate<<<(unsigned)blocks, kThreads, smem, L.stream>>>(d, T, D, popcount, (u32)rpt,
                                                            FastDiv((u32)d.W));
}


size_t front_smem(u32 rpt, u64 W, int dilate) {
  return (size_t)rpt * W * 4 + (size_t)rpt * 12 + 8 + (dilate ? (size_t)(rpt + 2) * W * 4 : 0);
}

void launch_front(const Launch& L, const Batch& B) {
  const u64 tiles = B.ftile0[B.n];
  if (tiles == 0) return;
  if (L.t.front_kernel == 0) {
    size_t smem = 0;
    for (u32 i = 0; i < B.n; ++i) {
      const size_t s = front_smem(B.it[i].rpt, B.it[i].W, B.c.dilate);
      if (s > smem) smem = s;
    }
    cudaFuncSetAttribute((const void*)k_front_count_blk,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    u64 grid = (u64)occupancy_grid((const void*)k_front_count_blk, kThreads, smem, L.sms);
    if (grid > tiles) grid = tiles;
    k_front_count_blk<<<(unsigned)grid, kThreads, smem, L.stream>>>(B);
  } else {
    auto count = [&](auto kernel) {
      u64 grid = (u64)occupancy_grid((const void*)kernel, kThreads, 0, L.sms);
      const u64 need = (tiles + kThreads / 32 - 1) / (kThreads / 32);
      if (grid > need) grid = need;
      kernel<<<(unsigned)grid, kThreads, 0, L.stream>>>(B);
    };
    if (B.c.dilate) count(k_front_count<true>);
    else count(k_front_count<false>);
  }
  u64 scan_tiles = 0;
  for (u32 i = 0; i < B.n; ++i)
    if (!B.it[i].fscan) scan_tiles += (B.it[i].ftiles + kScanTile - 1) / kScanTile;
  launch_scan_pairs(L, B, 0, scan_tiles);
  auto run = [&](auto kernel) {
    u64 g = (u64)occupancy_grid((const void*)kernel, kThreads, 0, L.sms);
    const u64 need = (B.row0[B.n] + (kThreads / 32) - 1) / (kThreads / 32);  // a row per warp
    if (g > need) g = need;
    if (g < 1) g = 1;
    kernel<<<(unsigned)g, kThreads, 0, L.stream>>>(B);
  };
  if (B.c.dtype == ROIX_F32) run(k_front_write<float>);
  else if (B.c.dtype == ROIX_U16) run(k_front_write<unsigned short>);
  else run(k_front_write<unsigned char>);
}

}  // namespace roix
