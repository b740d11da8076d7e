// Coder kernels: error-bounded quantisation (Sec. 4.2.3 contract, Sz3-style
// linear lattice of Sec. 4.3), 1D Lorenzo prediction with symbolisation and a
// histogram, the canonical Huffman codebook, the chunked bit packer and the
// container finaliser.
#include <type_traits>

#include "roix_internal.cuh"

namespace roix {

namespace {

constexpr int kThreads = 256;

// ------------------------------------------------------------------ range
template <typename TV>
__global__ void __launch_bounds__(kThreads) k_range(const TV* __restrict__ P, u64 n_cap,
                                                    const u64* n_dev, State* st) {
  const u64 n = n_dev ? min(*n_dev, n_cap) : n_cap;
  u32 kmin = 0xffffffffu, kmax = 0u;
  for (u64 k = (u64)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (u64)gridDim.x * blockDim.x) {
    const TV v = __ldg(P + k);
    if constexpr (sizeof(TV) == 4) {
      if (isfinite(v)) {
        const u32 kk = f32_key(__fadd_rn(v, 0.0f));
        kmin = min(kmin, kk);
        kmax = max(kmax, kk);
      }
    } else {
      kmin = min(kmin, (u32)v + 1u);
      kmax = max(kmax, (u32)v + 1u);
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    kmin = min(kmin, __shfl_xor_sync(0xffffffffu, kmin, o));
    kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
  }
  if ((threadIdx.x & 31) == 0) {
    if (kmin != 0xffffffffu) atomicMin(&st->vmin_key, kmin);
    if (kmax != 0u) atomicMax(&st->vmax_key, kmax);
  }
}

// ------------------------------------------------------ staged quantiser
// One warp per 32 values: codes written as int32, outliers as one ballot word.
template <typename TV>
__global__ void __launch_bounds__(kThreads) k_quantize_stage(Desc d, const TV* __restrict__ P,
                                                             u64 n_cap, const u64* n_dev,
                                                             int32_t* __restrict__ q,
                                                             u32* __restrict__ obits,
                                                             roix_eb_info* info_out,
                                                             State* st) {
  const u64 n = n_dev ? min(*n_dev, n_cap) : n_cap;
  const roix_eb_info e = make_eb(d, st->vmin_key, st->vmax_key);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *info_out = e;
    st->eb = e;
  }
  const int lane = threadIdx.x & 31;
  const u64 nwords = (n + 31) >> 5;
  for (u64 w = ((u64)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < nwords;
       w += ((u64)gridDim.x * blockDim.x) >> 5) {
    const u64 k = (w << 5) + lane;
    bool out = false;
    int c = 0;
    if (k < n) {
      if constexpr (sizeof(TV) == 4) c = quant_f32(__ldg(P + k), e, out);
      else c = quant_u16(__ldg(P + k), d.dark, e.eb_int);
      q[k] = c;
    }
    const u32 b = __ballot_sync(0xffffffffu, out);
    if (lane == 0) obits[w] = b;
  }
}

// -------------------------------------------------------------- symbols
// Code of value k and its outlier flag, either quantised on the fly from the
// pixel section (fused path) or read from the staged codes. Loads and the
// evaluation are separate so that a batch of loads can be issued first.
template <typename TV, bool FROM_Q>
struct Src {
  const TV* P;
  const int32_t* q;
  const u32* obits;
  roix_eb_info e;
  int dark;
  FastDiv fd;  // division by 2 * eb_int (uint16 path)
  struct R {
    TV x;
    int q;
    u32 o;
  };
  __device__ __forceinline__ R load1(u64 k) const {
    R r{TV(0), 0, 0u};
    if constexpr (FROM_Q) {
      r.q = __ldg(q + k);
      r.o = (__ldg(obits + (k >> 5)) >> (k & 31)) & 1u;
    } else {
      r.x = __ldg(P + k);
    }
    return r;
  }
  // k0 even and k0 + 1 < n: one vector load for the pair
  __device__ __forceinline__ void load2(u64 k0, R& a, R& b) const {
    a = R{TV(0), 0, 0u};
    b = R{TV(0), 0, 0u};
    if constexpr (FROM_Q) {
      const int2 v = __ldg(reinterpret_cast<const int2*>(q + k0));
      const u32 w = __ldg(obits + (k0 >> 5));
      a.q = v.x;
      b.q = v.y;
      a.o = (w >> (k0 & 31)) & 1u;
      b.o = (w >> ((k0 + 1) & 31)) & 1u;
    } else if constexpr (sizeof(TV) == 4) {
      const float2 v = __ldg(reinterpret_cast<const float2*>(P + k0));
      a.x = v.x;
      b.x = v.y;
    } else {
      const ushort2 v = __ldg(reinterpret_cast<const ushort2*>(P + k0));
      a.x = v.x;
      b.x = v.y;
    }
  }
  __device__ __forceinline__ int eval(const R& r, bool& out) const {
    if constexpr (FROM_Q) {
      out = r.o != 0u;
      return out ? 0 : r.q;
    } else if constexpr (sizeof(TV) == 4) {
      return quant_f32(r.x, e, out);
    } else {
      out = false;
      return quant_u16_fd(r.x, dark, e.eb_int, fd);
    }
  }
  __device__ __forceinline__ int code(u64 k, bool& out) const { return eval(load1(k), out); }
  __device__ __forceinline__ u32 raw_bits(u64 k) const {
    if constexpr (sizeof(TV) == 4) return __float_as_uint(__ldg(P + k));
    else return (u32)__ldg(P + k);
  }
};

// Symbol of the two-layer residual d = c - (2 p1 - p2), exact in 64 bits: d + R
// when -R < d < R, else 0.
__device__ __forceinline__ u32 symbol2_of(int c, int p1, int p2, bool out, u32 R) {
  if (out) return 0u;
  const long long d = (long long)c - (2ll * p1 - (long long)p2);
  return (d > -(long long)R && d < (long long)R) ? (u32)(d + R) : 0u;
}

// Symbol of a delta: d + R when -R < d < R, else 0. Codes lie in
// [-2^30, 2^30], so the true delta lies in [-2^31, 2^31]; its two's-complement
// wrap to 0x80000000 at the extremes still fails the unsigned range test.
__device__ __forceinline__ u32 symbol_of(int c, int prev, bool out, u32 R) {
  if (out) return 0u;
  const u32 dd = (u32)c - (u32)prev;
  return (dd + R - 1u < 2u * R - 1u) ? dd + R : 0u;
}

// Segments of `per` values (a power of two), every item's segments in order:
// prefix of ceil(n_i / per) over the items (n_i found by the compaction),
// formed by warp 0 of each block at start (lane l holds items 2l and 2l + 1;
// kMaxBatch = 64) with one warp scan.
__device__ __forceinline__ void tile_prefix(const Batch& B, u64* pre, u64 per,
                                            u64* counts = nullptr) {
  static_assert(kMaxBatch <= 64, "two items per lane");
  if (threadIdx.x < 32) {
    const u32 lane = threadIdx.x, sh = (u32)(__ffsll((long long)per) - 1);
    u64 c[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const u32 i = 2 * lane + k;
      c[k] = 0;
      if (i < B.n) {
        const Item& I = B.it[i];
        const u64 n = umin(I.sizes[0], I.N);
        c[k] = (n + per - 1) >> sh;
        if (counts) counts[i] = n;
      }
    }
    const u64 inc = warp_incl_scan<u64>(c[0] + c[1]);
    const u64 ex = inc - c[0] - c[1];
    if (2 * lane < B.n) pre[2 * lane] = ex;
    if (2 * lane + 1 < B.n) pre[2 * lane + 1] = ex + c[0];
    if (lane == 31) pre[B.n] = inc;
  }
  __syncthreads();
}

// Per-lane vector of one step: V consecutive values kept as the raw words of
// one 16-byte load of the pixel section (elements unpacked when used, so that
// a lane's loads in flight take four registers each), or two staged codes and
// their outlier bits.
template <typename TV, bool FROM_Q>
struct SymVec {
  static constexpr int V = FROM_Q ? 2 : 16 / (int)sizeof(TV);
  u32 w[FROM_Q ? 2 : 4];
  u32 o;
};

template <typename TV, bool FROM_Q>
__device__ __forceinline__ void sym_load(const Src<TV, FROM_Q>& src, u64 k0, u64 n,
                                         SymVec<TV, FROM_Q>& r) {
  constexpr int V = SymVec<TV, FROM_Q>::V;
  r.o = 0u;
  if constexpr (FROM_Q) {
    if (k0 + V <= n) {
      const int2 v = __ldg(reinterpret_cast<const int2*>(src.q + k0));
      r.w[0] = (u32)v.x;
      r.w[1] = (u32)v.y;
    } else {
#pragma unroll
      for (int j = 0; j < V; ++j) r.w[j] = k0 + j < n ? (u32)__ldg(src.q + k0 + j) : 0u;
    }
    r.o = k0 < n ? (__ldg(src.obits + (k0 >> 5)) >> (k0 & 31)) & 3u : 0u;  // V = 2, k0 even
  } else {
    if (k0 + V <= n) {
      const uint4 v = __ldg(reinterpret_cast<const uint4*>(src.P + k0));
      r.w[0] = v.x;
      r.w[1] = v.y;
      r.w[2] = v.z;
      r.w[3] = v.w;
    } else {
#pragma unroll
      for (int i = 0; i < 4; ++i) r.w[i] = 0u;
#pragma unroll
      for (int j = 0; j < V; ++j) {
        if (k0 + j < n) {
          if constexpr (sizeof(TV) == 4) r.w[j] = __float_as_uint(__ldg(src.P + k0 + j));
          else r.w[j >> 1] |= (u32)__ldg(src.P + k0 + j) << (16 * (j & 1));
        }
      }
    }
  }
}

// Code of element j of a loaded vector (0 and out = true for an outlier).
template <typename TV, bool FROM_Q>
__device__ __forceinline__ int sym_eval(const Src<TV, FROM_Q>& src,
                                        const SymVec<TV, FROM_Q>& r, int j, bool& out) {
  if constexpr (FROM_Q) {
    out = ((r.o >> j) & 1u) != 0u;
    return out ? 0 : (int)r.w[j];
  } else if constexpr (sizeof(TV) == 4) {
    return quant_f32(__uint_as_float(r.w[j]), src.e, out);
  } else {
    out = false;
    const TV x = (TV)((r.w[j >> 1] >> (16 * (j & 1))) & 0xffffu);
    return quant_u16_fd(x, src.dark, src.e.eb_int, src.fd);
  }
}

// Error-bound constants of every item of the batch, formed once per block
// (one thread per item) into shared memory: warps that move between items
// then read them instead of repeating the binary64 derivation.
struct ItemEb {
  roix_eb_info e;
  FastDiv fd;
};

__device__ __forceinline__ void items_eb(const Batch& B, ItemEb* out) {
  for (u32 i = threadIdx.x; i < B.n; i += blockDim.x) {
    const Item& I = B.it[i];
    const Desc d = desc_of(B, I);
    out[i].e = make_eb(d, I.rst->vmin_key, I.rst->vmax_key);
    out[i].fd = FastDiv(2u * (u32)out[i].e.eb_int);
  }
}

// One warp's histogram (shared memory) added to the item's global one.
__device__ __forceinline__ void flush_hist(u32* h, unsigned long long* g, u32 S, int lane) {
  __syncwarp();
  for (u32 i = lane; i < S; i += 32) {
    const u32 v = h[i];
    if (v) {
      atomicAdd(g + i, (unsigned long long)v);
      h[i] = 0;
    }
  }
  __syncwarp();
}

// Persistent warps, each on its own: a warp takes the next segment of
// kQuantTile values (global ticket, every item's segments in order) and walks
// it in steps of 32 V values, lane l holding V consecutive values of a step
// (one vector load each; the loads of kBatch steps are issued before any is
// used). Codes are formed on the fly from the pixel section (or read from the
// staged codes); the predecessor of a lane's first value comes from the lane
// before it, of lane 0's from the warp's previous step, of the segment's first
// from value base - 1, quantised again. Symbols leave as one vector store per
// lane and step; the histogram is the warp's own in shared memory (no block
// barrier anywhere in the loop) and goes to the item's global histogram when
// the warp moves to another item. Symbol-0 positions (records) are only
// counted here, per pack chunk (an atomic per lane and step that has one);
// they are written by k_pack_count once the codebook kernel has turned the
// counts into offsets, so that no segment waits for another.
// (first-order forms: registers for four blocks per SM for uint16 values,
// three for float32)
template <typename TV, bool FROM_Q, int ORDER>
__global__ void __launch_bounds__(kThreads, ORDER != 1 || FROM_Q ? 1 : (sizeof(TV) == 2 ? 4 : 3))
k_symbols(const __grid_constant__ Batch B) {
  if (halted(B.status)) return;  // a tile scan of this call gave up
  using Vec = SymVec<TV, FROM_Q>;
  constexpr int V = Vec::V;
  constexpr u32 kStep = 32u * V;                 // values per warp and step
  constexpr int kSteps = (int)(kQuantTile / kStep);
  constexpr int kBatch = V >= 8 ? 4 : (kSteps < 8 ? kSteps : 8);  // loads in flight per lane
  static_assert(kQuantTile % kStep == 0 && kSteps % kBatch == 0, "whole steps and batches");
  extern __shared__ u32 hsm[];  // [warps][S]
  __shared__ u64 pre[kMaxBatch + 1];
  __shared__ ItemEb ieb[kMaxBatch];
  if constexpr (!FROM_Q) items_eb(B, ieb);
  const u32 R_ = B.c.R, S = B.c.S;
  const u32 csh = (u32)(__ffs((int)B.c.C) - 1);  // log2 of the pack chunk
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  u32* h = hsm + (u32)warp * S;
  for (u32 i = lane; i < S; i += 32) h[i] = 0;
  tile_prefix(B, pre, kQuantTile);
  const u64 total = pre[B.n];
  u32 cur = 0xffffffffu;
  u32 since_flush = 0;
  Src<TV, FROM_Q> src{};
  u64 n = 0;
  while (true) {
    u64 gt = 0;
    if (lane == 0) gt = atomicAdd(&B.ctr[1], 1u);
    gt = __shfl_sync(0xffffffffu, gt, 0);
    if (gt >= total) break;
    const u32 item = find_item(pre, B.n, gt);
    const Item& I = B.it[item];
    if (item != cur || since_flush >= (1u << 19)) {  // 2^19 segments keep u32 counts exact
      if (cur != 0xffffffffu) flush_hist(h, B.it[cur].hist, S, lane);
      since_flush = 0;
      if (item != cur) {
        cur = item;
        const Desc d = desc_of(B, I);
        src.P = (const TV*)I.P;
        src.q = I.q;
        src.obits = I.obits;
        src.dark = d.dark;
        if constexpr (!FROM_Q) {
          src.e = ieb[item].e;
          src.fd = ieb[item].fd;
        }
        n = umin(I.sizes[0], I.N);
      }
    }
    ++since_flush;
    const u64 t = gt - pre[item];
    const u64 base = t * kQuantTile;
    uint16_t* __restrict__ sym = I.sym;
    int carry = 0, carry2 = 0;  // codes of values base - 1, base - 2 (0: outlier or none)
    if (lane == 0 && base > 0) {
      bool o;
      carry = src.code(base - 1, o);
      if (ORDER == 2 && base > 1) carry2 = src.code(base - 2, o);
    }
    carry = __shfl_sync(0xffffffffu, carry, 0);
    if (ORDER == 2) carry2 = __shfl_sync(0xffffffffu, carry2, 0);
    u32* __restrict__ crec = I.crec;
    u32* __restrict__ rbits = I.rbits;
    // one step: V codes per lane, deltas, symbols, histogram, record bits;
    // GUARD = the segment reaches past n (the item's last segment)
    auto step = [&](auto guard_tag, const int st, const Vec& r) {
      constexpr bool GUARD = decltype(guard_tag)::value;
      const u64 k0 = base + (u64)st * kStep + (u64)lane * V;
      int c[V];
      bool o[V];
#pragma unroll
      for (int j = 0; j < V; ++j) {
        if (!GUARD || k0 + j < n) c[j] = sym_eval<TV, FROM_Q>(src, r, j, o[j]);
        else {
          c[j] = 0;
          o[j] = false;
        }
      }
      int prev = __shfl_up_sync(0xffffffffu, c[V - 1], 1);
      int prev2 = 0;
      if constexpr (ORDER == 2) prev2 = __shfl_up_sync(0xffffffffu, c[V - 2], 1);
      if (lane == 0) {
        prev = carry;
        prev2 = carry2;
      }
      if constexpr (ORDER == 2) carry2 = __shfl_sync(0xffffffffu, c[V - 2], 31);
      carry = __shfl_sync(0xffffffffu, c[V - 1], 31);
      u32 sv[V];
      u32 rb = 0;
#pragma unroll
      for (int j = 0; j < V; ++j) {
        const bool in = !GUARD || k0 + j < n;
        if constexpr (ORDER == 2)
          sv[j] = symbol2_of(c[j], j ? c[j - 1] : prev, j > 1 ? c[j - 2] : (j ? prev : prev2),
                             o[j], R_);
        else
          sv[j] = symbol_of(c[j], j ? c[j - 1] : prev, o[j], R_);
        if (in) {
          atomicAdd(&h[sv[j]], 1u);
          rb |= (sv[j] == 0u ? 1u : 0u) << j;
        }
      }
      if (!GUARD || k0 + V <= n) {
        if constexpr (V == 8) {
          *reinterpret_cast<uint4*>(sym + k0) =
              make_uint4(sv[0] | (sv[1] << 16), sv[2] | (sv[3] << 16), sv[4] | (sv[5] << 16),
                         sv[6] | (sv[7] << 16));
        } else if constexpr (V == 4) {
          *reinterpret_cast<uint2*>(sym + k0) =
              make_uint2(sv[0] | (sv[1] << 16), sv[2] | (sv[3] << 16));
        } else {
          *reinterpret_cast<u32*>(sym + k0) = sv[0] | (sv[1] << 16);
        }
      } else {
#pragma unroll
        for (int j = 0; j < V; ++j)
          if (k0 + j < n) sym[k0 + j] = (uint16_t)sv[j];
      }
      if (rb) atomicAdd(crec + (k0 >> csh), (u32)__popc(rb));  // records of the pack chunk
      // record bitmap: bit k % 32 of word k / 32 (the 32 / V lanes of a word OR-ed)
      {
        constexpr int kLanesPerWord = 32 / V;
        u32 wv = rb << (u32)(k0 & 31);
#pragma unroll
        for (int o = 1; o < kLanesPerWord; o <<= 1) wv |= __shfl_xor_sync(0xffffffffu, wv, o);
        if ((lane & (kLanesPerWord - 1)) == 0 && (!GUARD || k0 < n)) rbits[k0 >> 5] = wv;
      }
    };
    if (base + kQuantTile <= n) {  // a whole segment: no bounds checks
      // (the batches are not unrolled: one copy of kBatch step bodies keeps
      // the loop inside the instruction cache; all kSteps copies missed it)
#pragma unroll 1
      for (int b0 = 0; b0 < kSteps; b0 += kBatch) {
        Vec r[kBatch];
#pragma unroll
        for (int i = 0; i < kBatch; ++i)
          sym_load<TV, FROM_Q>(src, base + (u64)(b0 + i) * kStep + (u64)lane * V, ~0ull, r[i]);
#pragma unroll
        for (int i = 0; i < kBatch; ++i) step(std::false_type{}, b0 + i, r[i]);
      }
    } else {
      for (int b0 = 0; b0 < kSteps; b0 += kBatch) {
        Vec r[kBatch];
#pragma unroll
        for (int i = 0; i < kBatch; ++i)
          sym_load<TV, FROM_Q>(src, base + (u64)(b0 + i) * kStep + (u64)lane * V, n, r[i]);
#pragma unroll
        for (int i = 0; i < kBatch; ++i) step(std::true_type{}, b0 + i, r[i]);
      }
    }
  }
  if (cur != 0xffffffffu) flush_hist(h, B.it[cur].hist, S, lane);
}

// ------------------------------------------------------------- codebook
// One block of 1024 threads builds the canonical length-limited Huffman code:
// bitonic sort of (count, symbol) keys, the two-queue construction on one
// thread (van Leeuwen), depths by pointer jumping, the per-length fold for
// lengths over 24 (ITU-T T.81 Annex K.3 procedure), lengths handed out
// shortest-first from the most frequent leaf, canonical codes (RFC 1951).
constexpr int kCbThreads = 1024;

__device__ void bitonic_sort(u64* key, u32 M) {
  // one thread per compare-exchange pair (M / 2 pairs per stage)
  for (u32 k = 2; k <= M; k <<= 1) {
    for (u32 j = k >> 1; j > 0; j >>= 1) {
      for (u32 p = threadIdx.x; p < M / 2; p += blockDim.x) {
        const u32 i = 2 * j * (p / j) + (p % j), l = i + j;
        const u64 a = key[i], b = key[l];
        const bool up = (i & k) == 0;
        if ((a > b) == up) {
          key[i] = b;
          key[l] = a;
        }
      }
      __syncthreads();
    }
  }
}

// Same network for M <= blockDim.x keys with thread i holding key i in a
// register: distances below 32 by warp shuffles (no barrier), larger ones
// through shared memory.
__device__ void bitonic_sort_reg(u64* key, u32 M) {
  const u32 i = threadIdx.x;
  u64 v = i < M ? key[i] : ~0ull;
  for (u32 k = 2; k <= M; k <<= 1) {
    for (u32 j = k >> 1; j > 0; j >>= 1) {
      u64 o;
      if (j >= 32) {
        __syncthreads();
        if (i < M) key[i] = v;
        __syncthreads();
        o = i < M ? key[i ^ j] : ~0ull;
      } else {
        o = __shfl_xor_sync(0xffffffffu, v, j);
      }
      const bool up = (i & k) == 0, lower = (i & j) == 0;
      const u64 lo = v < o ? v : o, hi = v < o ? o : v;
      v = (up == lower) ? lo : hi;
    }
  }
  __syncthreads();
  if (i < M) key[i] = v;
  __syncthreads();
}

__host__ __device__ __forceinline__ u32 next_pow2(u32 v) {
  u32 p = 1;
  while (p < v) p <<= 1;
  return p;
}

// leaves-per-depth entries: depths up to m - 1 < S while building, and the
// lengths 0..kLMax + 1 when they are summed
__host__ __device__ __forceinline__ u32 bl_entries(u32 S) {
  return S + 2 > kLMax + 2 ? S + 2 : kLMax + 2;
}

size_t codebook_smem(u32 S) {
  return (size_t)next_pow2(S) * 8  // key (sorted with a power-of-two bitonic network)
         + (size_t)S * 8      // internal weights
         + (size_t)2 * S * 4  // parent / ancestor
         + (size_t)2 * S * 4  // depth
         + (size_t)bl_entries(S) * 4  // leaves per depth
         + (size_t)S;         // lengths
}

#ifdef ROIX_CB_PROBE
__device__ long long g_cb_probe[16];
#define CB_MARK(i) \
  if (threadIdx.x == 0 && blockIdx.x == 0) g_cb_probe[i] = clock64();
#else
#define CB_MARK(i)
#endif

// Two-queue Huffman construction (van Leeuwen 1976) by a team of threads, in
// rounds. The sequential form pops the two lightest fronts of the leaf queue
// (leaves 0..m-1 sorted ascending) and of the internal queue (nodes m.. in
// creation order), a leaf winning ties, and appends their sum to the internal
// queue. Every node created from now on weighs at least 2 x_min (x_min = the
// lighter front), so every known leaf or internal node of weight <= T =
// 2 x_min is popped before any of them, in merged order (weight, leaves before
// internal nodes on a tie, queue order within a queue); a round therefore
// takes those K nodes at once (K rounded down to even; the odd one waits for
// the next round), places each in the merged order by its rank (a leaf: its
// index plus the internal nodes lighter than it; an internal node: its index
// plus the leaves no heavier than it; binary searches in the other run), and
// pairs merged positions 2p, 2p + 1 into new nodes m + created + p, which is
// the sequential algorithm's order of pops and of creations. When K < 2 the two
// lightest fronts are popped as one sequential step. Rounds: about
// log2(total weight / lightest leaf) plus those steps, each a few team
// barriers. par[] receives every node's parent; mid[] (2m entries) is scratch;
// rstart[] (rounds + 1 entries) receives each round's first created node and
// *nrounds their number, for the depths. Called by every thread of the team.
constexpr u64 kNoWeight = ~0ull;

// The construction runs on a team of the block's first kTeam threads, which
// synchronise on named barrier 1 (a round's steps are short: the whole block
// spends more on its barriers than it saves; 64 threads are too few).
constexpr u32 kTeam = 256;
__device__ __forceinline__ void team_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(kTeam) : "memory");
}
// Number of team threads whose p is true (a barrier of the team).
__device__ __forceinline__ u32 team_count(bool p) {
  u32 r;
  asm volatile(
      "{\n .reg .pred q;\n setp.ne.u32 q, %1, 0;\n bar.red.popc.u32 %0, 1, %2, q;\n}\n"
      : "=r"(r)
      : "r"((u32)p), "n"(kTeam)
      : "memory");
  return r;
}

// Number of i in [0, len) with pred(i), by the team (len uniform); with
// `prefix`, pred holds on a prefix of the range, and counting stops at the
// first team-sized part where it fails.
template <typename F>
__device__ __forceinline__ u32 team_count_range(u32 len, bool prefix, F pred) {
  u32 c = 0;
  for (u32 b0 = 0; b0 < len; b0 += kTeam) {
    const u32 i = b0 + threadIdx.x;
    const u32 k = team_count(i < len && pred(i));
    c += k;
    if (prefix && k < min(kTeam, len - b0)) break;
  }
  return c;
}

__device__ void huffman_merge_team(const u64* key, u64* wi, int32_t* par, int32_t* mid,
                                    u32* rstart, u32* nrounds, u32 m) {
  const u32 tid = threadIdx.x;
  auto lw = [&](u32 i) -> u64 { return key[i] >> 16; };
  u32 lf = 0, in = 0, created = 0, rounds = 0;
  while (created + 1 < m) {
    if (tid == 0) rstart[rounds] = created;  // first node of this round
    ++rounds;
    const u64 a0 = lf < m ? lw(lf) : kNoWeight;
    const u64 b0 = in < created ? wi[in] : kNoWeight;
    const u64 xmin = a0 < b0 ? a0 : b0;
    const u64 T = xmin > (kNoWeight >> 1) ? kNoWeight : 2 * xmin;
    const u32 na = team_count_range(m - lf, true, [&](u32 i) { return lw(lf + i) <= T; });
    const u32 nb = team_count_range(created - in, true, [&](u32 i) { return wi[in + i] <= T; });
    const u32 K = na + nb;
    if (K < 2) {
      // one sequential step: the two lightest fronts, a leaf winning ties (every
      // thread follows it; thread 0 writes)
      u32 l = lf, q = in;
      int32_t id[2];
      u64 w[2];
      for (int t = 0; t < 2; ++t) {
        const u64 la = l < m ? lw(l) : kNoWeight, ib = q < created ? wi[q] : kNoWeight;
        if (la <= ib) {
          id[t] = (int32_t)l;
          w[t] = la;
          ++l;
        } else {
          id[t] = (int32_t)(m + q);
          w[t] = ib;
          ++q;
        }
      }
      team_sync();  // every thread has read the fronts
      if (tid == 0) {
        wi[created] = w[0] + w[1];
        par[id[0]] = (int32_t)(m + created);
        par[id[1]] = (int32_t)(m + created);
      }
      team_sync();
      lf = l;
      in = q;
      ++created;
      continue;
    }
    const u32 P = K >> 1, out = 2 * P;
    // merged positions of the K nodes; those below `out` are paired
    const u32 ca = team_count_range(K, false, [&](u32 e) {
      if (e < na) {  // leaf lf + e: after the internal nodes strictly lighter
        const u64 w = lw(lf + e);
        u32 lo = 0, hi = nb;
        while (lo < hi) {
          const u32 c = (lo + hi) >> 1;
          if (wi[in + c] < w) lo = c + 1;
          else hi = c;
        }
        const u32 pos = e + lo;
        if (pos < out) mid[pos] = (int32_t)(lf + e);
        return pos < out;
      }
      const u32 j = e - na;  // internal node in + j: after the leaves no heavier
      const u64 w = wi[in + j];
      u32 lo = 0, hi = na;
      while (lo < hi) {
        const u32 c = (lo + hi) >> 1;
        if (lw(lf + c) <= w) lo = c + 1;
        else hi = c;
      }
      const u32 pos = j + lo;
      if (pos < out) mid[pos] = (int32_t)(m + in + j);
      return false;
    });  // (its barriers also order the mid[] writes before the pairing)
    for (u32 p = tid; p < P; p += kTeam) {
      const u32 x = (u32)mid[2 * p], y = (u32)mid[2 * p + 1];
      const u64 wx = x < m ? lw(x) : wi[x - m], wy = y < m ? lw(y) : wi[y - m];
      wi[created + p] = wx + wy;
      par[x] = (int32_t)(m + created + p);
      par[y] = (int32_t)(m + created + p);
    }
    team_sync();
    lf += ca;
    in += out - ca;
    created += P;
  }
  if (tid == 0) {
    par[2 * m - 2] = -1;
    rstart[rounds] = created;
    *nrounds = rounds;
  }
  team_sync();
}

// Depths by the rounds in reverse (a node's parent is created in a later
// round), then the leaves; by the team.
__device__ void huffman_depths_team(const int32_t* par, int32_t* dep, const u32* rstart,
                                    u32 nrounds, u32 m) {
  if (threadIdx.x == 0) dep[2 * m - 2] = 0;
  team_sync();
  for (int r = (int)nrounds - 1; r >= 0; --r) {
    for (u32 v = rstart[r] + threadIdx.x; v < rstart[r + 1]; v += kTeam) {
      if (v + 2 < m) dep[m + v] = dep[par[m + v]] + 1;  // the root (v = m - 2) keeps 0
    }
    team_sync();
  }
  for (u32 i = threadIdx.x; i < m; i += kTeam) dep[i] = dep[par[i]] + 1;
  team_sync();
}

__global__ void __launch_bounds__(kCbThreads) k_codebook(const __grid_constant__ Batch B) {
  if (halted(B.status)) return;  // a tile scan of this call gave up
  extern __shared__ __align__(16) unsigned char cb_smem[];
  CB_MARK(0)
  const Item& I = B.it[blockIdx.x];
  const unsigned long long* hist = I.hist;
  uint8_t* lens_ws = I.lens;
  u32* codes_ws = I.codes;
  uint8_t* out = I.out;
  const u64 cap = I.cap;
  const u32 S = B.c.S;
  u64* key = (u64*)cb_smem;                       // [next_pow2(S)] (count << 16 | symbol)
  u64* wint = key + next_pow2(S);                 // [S] internal node weights
  int32_t* par = (int32_t*)(wint + S);            // [2S]
  int32_t* dep = par + 2 * S;                     // [2S]
  u32* bl = (u32*)(dep + 2 * S);                  // [bl_entries(S)]
  uint8_t* len = (uint8_t*)(bl + bl_entries(S));  // [S]
  __shared__ u32 scratch[40];
  __shared__ u32 s_maxl, s_next[kLMax + 2], s_cum[kLMax + 2];
  const int tid = threadIdx.x;
  // used symbols, compacted in symbol order
  u32 m = 0;
  for (u32 c0 = 0; c0 < S; c0 += kCbThreads) {
    const u32 s = c0 + tid;
    const u64 hv = s < S ? hist[s] : 0ull;
    u32 tot;
    const u32 pos = block_excl_scan<u32>(hv ? 1u : 0u, scratch, &tot);
    if (hv) key[m + pos] = (hv << 16) | s;
    m += tot;
  }
  for (u32 s = tid; s < S; s += kCbThreads) len[s] = 0;
  for (u32 i = tid; i < bl_entries(S); i += kCbThreads) bl[i] = 0;
  u32 M = 1;
  while (M < m) M <<= 1;
  for (u32 i = m + tid; i < M; i += kCbThreads) key[i] = ~0ull;
  __syncthreads();
  CB_MARK(1)
  if (m <= 128u) {
    // rank of each (count, symbol) key among the m distinct keys: one key per
    // thread, every thread reads the keys in the same order (smem broadcast);
    // O(m^2) work, so only for small alphabets
    u64 mine = tid < (int)m ? key[tid] : 0ull;
    u32 rank = 0;
    if (tid < (int)m)  // only the warps holding keys read them
      for (u32 j = 0; j < m; ++j) rank += key[j] < mine;
    __syncthreads();
    if (tid < (int)m) key[rank] = mine;
    __syncthreads();
  } else if (M <= (u32)kCbThreads) {
    bitonic_sort_reg(key, M);  // ascending (count, symbol)
  } else {
    bitonic_sort(key, M);
  }
  CB_MARK(2)
  if (m == 1) {
    if (tid == 0) {
      len[key[0] & 0xffffu] = 1;
      bl[1] = 1;
    }
  } else if (m >= 2) {
    // two-queue construction by the team, in rounds (dep is scratch until the
    // depths, bl holds the rounds' first nodes until the lengths are counted)
    __shared__ u32 s_rounds;
    if (tid < (int)kTeam) {
      huffman_merge_team(key, wint, par, dep, bl, &s_rounds, m);
      CB_MARK(3)
      huffman_depths_team(par, dep, bl, s_rounds, m);
    }
    __syncthreads();
    CB_MARK(4)
    for (u32 i = tid; i < bl_entries(S); i += kCbThreads) bl[i] = 0;
    __syncthreads();
    if (tid == 0) s_maxl = 0;
    __syncthreads();
    for (u32 i = tid; i < m; i += kCbThreads) {
      atomicAdd(&bl[dep[i]], 1u);
      atomicMax(&s_maxl, (u32)dep[i]);
    }
    __syncthreads();
    if (tid == 0) {  // fold lengths above kLMax back (per-length counts)
      for (u32 l = s_maxl; l > kLMax; --l) {
        while (bl[l] > 0) {
          u32 j = l - 2;
          while (bl[j] == 0) --j;
          bl[l] -= 2;
          bl[l - 1] += 1;
          bl[j + 1] += 2;
          bl[j] -= 1;
        }
      }
    }
  }
  __syncthreads();
  if (tid == 0) {
    u32 c = 0;
    s_cum[0] = 0;
    for (u32 l = 1; l <= kLMax; ++l) {
      c += bl[l];
      s_cum[l] = c;
    }
    u32 code = 0;
    s_next[0] = 0;
    for (u32 l = 1; l <= kLMax; ++l) {
      code = (code + (l >= 2 ? bl[l - 1] : 0u)) << 1;
      s_next[l] = code;
    }
  }
  __syncthreads();
  if (m >= 2) {
    // the leaf at sorted position i has rank m-1-i counted from the most frequent
    for (u32 i = tid; i < m; i += kCbThreads) {
      const u32 rank = m - 1 - i;
      u32 l = 1;
      while (l < kLMax && s_cum[l] <= rank) ++l;
      len[key[i] & 0xffffu] = (uint8_t)l;
    }
  }
  __syncthreads();
  CB_MARK(5)
  // canonical codes: code = first code of its length + rank of the symbol
  // among the symbols of that length. Ranks in symbol order, chunk by chunk of
  // kCbThreads symbols: lanes of equal length found with __match_any_sync,
  // per-warp counts per length scanned across warps, carried across chunks.
  {
    __shared__ u32 wcnt[32][kLMax + 1];  // per warp and length: count, then offset
    __shared__ u32 s_carry[kLMax + 1];
    if (tid <= (int)kLMax) s_carry[tid] = 0;
    const int lane = tid & 31, warp = tid >> 5;
    for (u32 c0 = 0; c0 < S; c0 += kCbThreads) {
      for (u32 i = tid; i < 32 * (kLMax + 1); i += kCbThreads) (&wcnt[0][0])[i] = 0u;
      __syncthreads();
      const u32 s = c0 + tid;
      const u32 l = s < S ? len[s] : 0u;
      const u32 same = __match_any_sync(0xffffffffu, l);
      const u32 below = __popc(same & ((1u << lane) - 1u));
      if (lane == __ffs(same) - 1) wcnt[warp][l] = __popc(same);
      __syncthreads();
      if (tid <= (int)kLMax) {  // exclusive scan over warps, one thread per length
        u32 acc = s_carry[tid];
        for (int w = 0; w < 32; ++w) {
          const u32 present = wcnt[w][tid];
          wcnt[w][tid] = acc;
          acc += present;
        }
        s_carry[tid] = acc;
      }
      __syncthreads();
      // the pack kernel's entry: the code left-justified in 32 bits, its
      // length in the low byte (lengths are at most 24, so the two never meet)
      if (s < S) codes_ws[s] = l ? ((s_next[l] + wcnt[warp][l] + below) << (32u - l)) | l : 0u;
      __syncthreads();
    }
  }
  CB_MARK(6)
  for (u32 s = tid; s < S; s += kCbThreads) {
    lens_ws[s] = len[s];
    if (kHeaderBytes + s < cap) out[kHeaderBytes + s] = len[s];
  }
  // the records of an item with at most kInScanMax chunks: per-chunk counts
  // (from the symbol kernel) into offsets (larger items: k_scan_pairs<1>)
  if (I.pscan) {
    __shared__ u64 scratch64[40];
    const u64 n = umin(I.sizes[0], I.N);
    const u64 nch = (n + B.c.C - 1) / B.c.C;
    const u64 nout = block_scan1(I.crec, nch, I.crecoff, scratch64);
    if (tid == 0) {
      I.st->nout = nout;
      if (nout > I.rec_cap) I.st->cap_flag = 1u;
    }
  }
  CB_MARK(7)
}

// ------------------------------------------------------------------- pack
// The records of chunk t of item I (a whole warp): the chunk's symbol-0
// positions in order, from the record bitmap the symbol kernel wrote (all of
// the lane's bitmap words, j = 32 g + lane, loaded before any is used; a warp
// scan of their popcounts per group g), each written straight into the
// container's record sections (keys at byte offset okey, values at oval) as
// (k | kind << 63, payload) from record idx on; the code or the raw value is
// formed again from the pixel section (or the staged codes).
template <typename TV, bool FROM_Q>
__device__ __forceinline__ void chunk_records(const Item& I, const Src<TV, FROM_Q>& src, u64 t,
                                              u64 n, u32 C, u64 idx, u64 okey, u64 oval,
                                              int lane) {
  constexpr int kG = 16;  // 32-word groups of a chunk (C <= 16384)
  const u32* __restrict__ rbits = I.rbits;
  uint8_t* out = I.out;
  const u64 cap = I.cap, rec_cap = I.rec_cap;
  const u64 w0 = t * (C / 32);
  const u32 nw = (u32)((umin(n, (t + 1) * (u64)C) - t * (u64)C + 31) / 32);
  u32 zm[kG];
#pragma unroll
  for (int g = 0; g < kG; ++g) {
    const u32 j = (u32)g * 32 + (u32)lane;
    zm[g] = j < nw ? __ldg(rbits + w0 + j) : 0u;
  }
#pragma unroll
  for (int g = 0; g < kG; ++g) {
    if ((u32)g * 32 >= nw) break;
    u32 z = zm[g];
    const u32 cnt = __popc(z);
    const u32 inc = warp_incl_scan(cnt);
    u64 o = idx + inc - cnt;
    while (z) {
      const int q = __ffs(z) - 1;
      z &= z - 1;
      const u64 k = (w0 + (u64)g * 32 + lane) * 32 + q;
      bool outl;
      const int c = src.code(k, outl);
      if (o < rec_cap) {
        const u64 ok = okey + 8 * o, ov = oval + 4 * o;
        if (ok + 8 <= cap) *reinterpret_cast<u64*>(out + ok) = k | (outl ? (1ull << 63) : 0ull);
        if (ov + 4 <= cap) *reinterpret_cast<u32*>(out + ov) = outl ? src.raw_bits(k) : (u32)c;
      }
      ++o;
    }
    idx += __shfl_sync(0xffffffffu, inc, 31);
  }
}

// Passes none of whose blocks waits on another: k_pack_count sums the code
// lengths of every chunk; the chunks' word and record counts become offsets
// (for items with at most kInScanMax chunks in the codebook kernel and in
// k_pack_count, which then also writes their records; for larger items in
// k_scan_pairs<1>, followed by k_records), and k_pack writes every chunk's
// words at its offset (chunks from global tickets in order).

// Warps, one chunk at a time: lane l holds symbols [8 l, 8 l + 8) of each
// round of 256 (coalesced 16-byte loads); the code lengths come from the
// item's byte table (2R bytes, read through L1). For an item with at most
// kInScanMax chunks the warp also writes the chunk's records, if it holds
// any: the symbol-0 positions in order, from the
// record bitmap the symbol kernel wrote (lane l with words l, l + 32, ...; a
// warp scan of their popcounts), each as (k | kind << 63, payload) at the
// chunk's record offset (scanned by the codebook kernel); the code or the raw
// value is formed again from the pixel section (or the staged codes). For an
// item with at most kInScanMax chunks, the warp that counts the item's last
// chunk scans the chunks' word counts into their offsets.
template <typename TV, bool FROM_Q>
__global__ void __launch_bounds__(kThreads, 4) k_pack_count(const __grid_constant__ Batch B) {
  if (halted(B.status)) return;  // a tile scan of this call gave up
  __shared__ u64 pre[kMaxBatch + 1];
  __shared__ u64 nn[kMaxBatch];
  const u32 C = B.c.C;
  const int lane = threadIdx.x & 31;
  tile_prefix(B, pre, C, nn);
  const u64 total = pre[B.n];
  const u64 nwarps = ((u64)gridDim.x * blockDim.x) >> 5;
  constexpr u32 kIn = 4;  // vector loads of a lane in flight at once
  u32 cur = 0xffffffffu;  // item whose records source is set
  Src<TV, FROM_Q> src{};
  for (u64 gt = ((u64)blockIdx.x * blockDim.x + threadIdx.x) >> 5; gt < total; gt += nwarps) {
    const u32 item = find_item(pre, B.n, gt);
    const Item& I = B.it[item];
    const u64 n = nn[item];
    const uint16_t* __restrict__ sym = I.sym;
    const uint8_t* __restrict__ len = I.lens;  // 2R bytes: stays in L1
    const u64 t = gt - pre[item];
    const u64 c0 = t * C + (u64)lane * 8;
    const u32 steps = C / 256;  // 8 symbols per lane and step
    u32 bits = 0;
    if (t * C + C <= n) {  // a full chunk: no bounds tests
      for (u32 r0 = 0; r0 < steps; r0 += kIn) {
        uint4 v[kIn];
#pragma unroll
        for (u32 q = 0; q < kIn; ++q)
          if (r0 + q < steps)
            v[q] = __ldg(reinterpret_cast<const uint4*>(sym + c0 + (u64)(r0 + q) * 256));
#pragma unroll
        for (u32 q = 0; q < kIn; ++q)
          if (r0 + q < steps)
            bits += __ldg(len + (v[q].x & 0xffffu)) + __ldg(len + (v[q].x >> 16)) +
                    __ldg(len + (v[q].y & 0xffffu)) + __ldg(len + (v[q].y >> 16)) +
                    __ldg(len + (v[q].z & 0xffffu)) + __ldg(len + (v[q].z >> 16)) +
                    __ldg(len + (v[q].w & 0xffffu)) + __ldg(len + (v[q].w >> 16));
      }
    } else {
      for (u32 r = 0; r < steps; ++r) {
        const u64 k = c0 + (u64)r * 256;
#pragma unroll
        for (int q = 0; q < 8; ++q)
          if (k + q < n) bits += __ldg(len + __ldg(sym + k + q));
      }
    }
    bits = __reduce_add_sync(0xffffffffu, bits);
    if (lane == 0) I.cw[t] = (bits + 31) >> 5;
    if (I.pscan && I.crec[t] != 0u) {  // the chunk's records (a small item's)
      if (item != cur) {
        cur = item;
        const Desc d = desc_of(B, I);
        src.P = (const TV*)I.P;
        src.q = I.q;
        src.obits = I.obits;
        src.dark = d.dark;
        if constexpr (!FROM_Q) {
          src.e = make_eb(d, I.rst->vmin_key, I.rst->vmax_key);
          src.fd = FastDiv(2u * (u32)src.e.eb_int);
        }
      }
      // record sections of the container: offsets from the item's sizes
      const Layout Lo = make_layout(B.c.S, I.rows, I.sizes[1], I.st->nout, (n + C - 1) / C, 0);
      chunk_records<TV, FROM_Q>(I, src, t, n, C, I.crecoff[t], Lo.off_outk, Lo.off_outv, lane);
    }
    const u64 nch = pre[item + 1] - pre[item];
    if (I.pscan && count_done(&I.st->done_pack, nch)) {  // the item's chunk offsets
      u64 tw, tr;
      warp_scan2(I.cw, nullptr, nch, I.cwoff, nullptr, tw, tr);
      if (lane == 0) I.st->nwords = tw;
    }
  }
}

// Warps, one chunk at a time, only chunks that hold records of items with
// more than kInScanMax chunks (k_pack_count writes those of the others): the
// symbol-0 positions of the chunk in order, from the record bitmap the symbol
// kernel wrote (lane l with words l, l + 32, ...; a warp scan of their
// popcounts), each written as (k | kind << 63, payload) at the chunk's record
// offset (from k_scan_pairs<1>); the code or the raw value is formed again from
// the pixel section (or the staged codes).
template <typename TV, bool FROM_Q>
__global__ void __launch_bounds__(kThreads) k_records(const __grid_constant__ Batch B) {
  if (halted(B.status)) return;  // a tile scan of this call gave up
  __shared__ u64 pre[kMaxBatch + 1];
  const u32 C = B.c.C;
  const int lane = threadIdx.x & 31;
  tile_prefix(B, pre, C);
  const u64 total = pre[B.n];
  const u64 warp0 = ((u64)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const u64 nwarps = ((u64)gridDim.x * blockDim.x) >> 5;
  u32 cur = 0xffffffffu;
  Src<TV, FROM_Q> src{};
  u64 n = 0, okey = 0, oval = 0;
  for (u64 gt = warp0; gt < total; gt += nwarps) {
    const u32 item = find_item(pre, B.n, gt);
    const Item& I = B.it[item];
    const u64 t = gt - pre[item];
    if (I.pscan || I.crec[t] == 0u) continue;
    if (item != cur) {  // the item's error-bound constants, formed only for chunks with records
      cur = item;
      const Desc d = desc_of(B, I);
      src.P = (const TV*)I.P;
      src.q = I.q;
      src.obits = I.obits;
      src.dark = d.dark;
      if constexpr (!FROM_Q) {
        src.e = make_eb(d, I.rst->vmin_key, I.rst->vmax_key);
        src.fd = FastDiv(2u * (u32)src.e.eb_int);
      }
      n = umin(I.sizes[0], I.N);
      const Layout Lo = make_layout(B.c.S, I.rows, I.sizes[1], I.st->nout, (n + C - 1) / C, 0);
      okey = Lo.off_outk;
      oval = Lo.off_outv;
    }
    chunk_records<TV, FROM_Q>(I, src, t, n, C, I.crecoff[t], okey, oval, lane);
  }
}

// Bulk copies into shared memory (cp.async.bulk, completion on an mbarrier).
__device__ __forceinline__ u32 smem_addr(const void* p) {
  return (u32)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(u64* bar, u32 count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(u64* bar, u32 bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
// global -> shared, 16-byte aligned addresses, bytes a multiple of 16
__device__ __forceinline__ void bulk_to_smem(void* dst, const void* src, u32 bytes, u64* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
// true once the phase of the given parity has completed; false after `limit`
// unsuccessful polls
__device__ __forceinline__ bool mbar_wait(u64* bar, u32 parity, u32 limit) {
  for (u32 i = 0; i < limit; ++i) {
    u32 ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// Shared memory of k_pack: two buffers of C symbols, two code tables (each
// rounded to 16 bytes), the chunk's stream.
__host__ __device__ __forceinline__ u32 pack_tab_words(u32 S) { return (S + 3u) & ~3u; }
__host__ __device__ __forceinline__ size_t pack_smem(u32 C, u32 S) {
  return (size_t)4 * C + (size_t)8 * pack_tab_words(S) + ((size_t)C * kLMax / 64 + 2) * 8;
}

// Persistent blocks, one chunk of C symbols at a time, double-buffered: the
// chunk's symbols (and the item's code table, when it differs from the one
// already in that buffer) arrive in shared memory by bulk copies issued a
// chunk ahead, and the ticket of the chunk after that is requested while the
// current one is packed. Thread i takes its EPT = C / 256 consecutive symbols
// and keeps their table entries (code left-justified, length in the low
// byte) in registers; a block scan of the per-thread bit counts gives each
// thread its bit offset; each thread ORs its codes into the chunk's words
// (MSB first) in a shared buffer: the word being filled stays in a register,
// a code is placed by one shift (and the part that runs past the word by one
// funnel shift), and a full word leaves by one shared OR (so the words shared
// with the neighbouring threads need no other care); the words are stored
// with coalesced stores at the chunk's offset. Waits on the copies are
// bounded (ROIX_ETIMEOUT).
template <int EPT>
__global__ void __launch_bounds__(kThreads, EPT <= 16 ? 5 : 1) k_pack(const __grid_constant__ Batch B) {
  if (halted(B.status)) return;  // a tile scan of this call gave up
  extern __shared__ __align__(16) unsigned char pk_smem[];
  __shared__ u32 scratch[40];
  __shared__ __align__(8) u64 mbar[2];
  __shared__ u64 s_tick[2];
  __shared__ u32 s_titem[2];  // item whose code table a buffer holds
  __shared__ u32 s_item[2], s_t[2];  // a buffer's chunk: item, chunk of the item
  __shared__ int s_bad;
  __shared__ u64 pre[kMaxBatch + 1];
  __shared__ u64 nval[kMaxBatch], pay0s[kMaxBatch], tab0s[kMaxBatch];
  const u32 C = B.c.C, S = B.c.S, tabw = pack_tab_words(S);
  uint16_t* sbuf = reinterpret_cast<uint16_t*>(pk_smem);                          // [2][C]
  u32* tabs = reinterpret_cast<u32*>(pk_smem + 4 * (size_t)C);                      // [2][tabw]
  unsigned long long* wb =
      reinterpret_cast<unsigned long long*>(pk_smem + 4 * (size_t)C + 8 * (size_t)tabw);
  const int tid = threadIdx.x;
  const u32 limit = spin_limit_of(B.c.spin_limit);
  tile_prefix(B, pre, C, nval);
  // per item: byte offsets of the payload and of the chunk table
  for (u32 i = tid; i < B.n; i += blockDim.x) {
    const Item& I = B.it[i];
    const Layout Lo = make_layout(S, I.rows, I.sizes[1], I.st->nout, (nval[i] + C - 1) / C, 0);
    pay0s[i] = Lo.off_payload;
    tab0s[i] = Lo.off_chunks;
  }
  const u64 total = pre[B.n];
  const u32 wb_words = C * kLMax / 64 + 2;
  for (u32 i = tid; i < wb_words; i += blockDim.x) wb[i] = 0ull;
  // (thread 0) the copies of ticket gt's chunk into buffer b
  auto issue = [&](int b, u64 gt) {
    const u32 item = find_item(pre, B.n, gt);
    const Item& I = B.it[item];
    const u64 t = gt - pre[item];
    s_item[b] = item;
    s_t[b] = (u32)t;  // (n < 2^32 C)
    const u32 nsym = (u32)umin(C, nval[item] - t * C);
    const u32 sb = (2u * nsym + 15u) & ~15u;  // (the symbol buffer has 16 bytes of slack)
    const u32 tb = s_titem[b] != item ? 4u * tabw : 0u;
    s_titem[b] = item;
    mbar_expect_tx(&mbar[b], sb + tb);
    bulk_to_smem(sbuf + (size_t)b * C, I.sym + t * C, sb, &mbar[b]);
    if (tb) bulk_to_smem(tabs + (size_t)b * tabw, I.codes, tb, &mbar[b]);
  };
  if (tid == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_titem[0] = s_titem[1] = 0xffffffffu;
    for (int b = 0; b < 2; ++b) {
      const u64 gt = atomicAdd(&B.ctr[3], 1u);
      s_tick[b] = gt;
      if (gt < total) issue(b, gt);
    }
  }
  __syncthreads();
  u32 phase = 0u;  // bit b: parity of buffer b's next completion
  for (int b = 0;; b ^= 1) {
    const u64 gt = s_tick[b];
    if (gt >= total) break;
    u64 nt = 0;  // the ticket buffer b takes next, requested now
    if (tid == 0) nt = atomicAdd(&B.ctr[3], 1u);
    const u32 item = s_item[b], t = s_t[b];
    const Item& I = B.it[item];
    const u64 n = nval[item];
    const u64 k0 = (u64)t * C + (u64)tid * EPT;
    const u64 cw0 = __ldg(I.cwoff + t);
    const bool ok = mbar_wait(&mbar[b], (phase >> b) & 1u, limit);
    if (__syncthreads_or(!ok)) {  // a copy never completed: give up, and wait for the other
      if (tid == 0) {
        s_bad = 1;
        set_status(B.status, ROIX_ETIMEOUT);
        if (s_tick[b ^ 1] < total) mbar_wait(&mbar[b ^ 1], (phase >> (b ^ 1)) & 1u, limit);
      }
      __syncthreads();
      return;
    }
    phase ^= 1u << b;
    const uint16_t* sy = sbuf + (size_t)b * C + (size_t)tid * EPT;
    const u32* tab = tabs + (size_t)b * tabw;
    const bool whole = k0 + EPT <= n;
    u32 e[EPT];
    u32 bits = 0;
    if constexpr (EPT % 8 == 0) {
      if (whole) {
#pragma unroll
        for (int v = 0; v < EPT / 8; ++v) {
          const uint4 r = reinterpret_cast<const uint4*>(sy)[v];
          const u32 w4[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            e[8 * v + 2 * q] = tab[w4[q] & 0xffffu];
            e[8 * v + 2 * q + 1] = tab[w4[q] >> 16];
          }
        }
      } else {
#pragma unroll
        for (int j = 0; j < EPT; ++j) e[j] = k0 + j < n ? tab[sy[j]] : 0u;
      }
    } else {
#pragma unroll
      for (int j = 0; j < EPT; ++j) e[j] = k0 + j < n ? tab[sy[j]] : 0u;
    }
#pragma unroll
    for (int j = 0; j < EPT; ++j) bits += e[j] & 0xffu;
    u32 cbits;
    const u32 off = block_excl_scan<u32>(bits, scratch, &cbits);
    const u32 words = (cbits + 31) >> 5;
    // the thread's codes are contiguous in the chunk's stream [off, off +
    // bits): `acc` holds word w's bits from position `fill` on (MSB first)
    if (bits) {
      u32* wb32 = reinterpret_cast<u32*>(wb);
      u32 w = off >> 5, fill = off & 31u, acc = 0u;
#pragma unroll
      for (int j = 0; j < EPT; ++j) {
        const u32 l = e[j] & 0xffu;
        const u32 cj = e[j] & 0xffffff00u;  // the code's bits, from bit 31 down
        acc |= cj >> fill;
        const u32 nf = fill + l;
        if (nf >= 32u) {  // word w is full (fill >= 8 here: l <= 24)
          atomicOr(&wb32[w], acc);
          ++w;
          acc = __funnelshift_r(0u, cj, fill);  // the code's bits past word w
        }
        fill = nf & 31u;
      }
      if (fill) atomicOr(&wb32[w], acc);
    }
    __syncthreads();
    const u64 tab0 = tab0s[item], cap = I.cap;
    uint8_t* out = I.out;
    if (tid == 0 && tab0 + 8ull * t + 8 <= cap)  // the chunk table entry
      *reinterpret_cast<u64*>(out + tab0 + 8ull * t) = cw0;
    const u64 pay = pay0s[item] + 4 * cw0;  // byte offset of the chunk's first word
    const u32* wb32 = reinterpret_cast<const u32*>(wb);
    for (u32 i = tid; i < words; i += blockDim.x) {
      const u64 o = pay + 4 * (u64)i;
      if (o + 4 <= cap) *reinterpret_cast<u32*>(out + o) = wb32[i];
    }
    __syncthreads();  // buffer b and the stream are read: refill, clear
    if (tid == 0) {
      s_tick[b] = nt;
      if (nt < total) issue(b, nt);
    }
    for (u32 i = tid; i < (words + 1) / 2; i += blockDim.x) wb[i] = 0ull;
  }
}

// --------------------------------------------------------------- finalize
__device__ __forceinline__ void put_bytes(uint8_t* h, u32 off, const void* src, u32 bytes) {
  const uint8_t* s = (const uint8_t*)src;
  for (u32 i = 0; i < bytes; ++i) h[off + i] = s[i];
}

__global__ void __launch_bounds__(kThreads) k_finalize(const __grid_constant__ Batch B) {
  if (halted(B.status)) return;  // a tile scan of this call gave up
  const Item& I = B.it[blockIdx.y];
  const Desc d = desc_of(B, I);
  State* st = I.st;
  uint8_t* out = I.out;
  const u64 cap = I.cap;
  const uint16_t* counts_src = I.counts_src;
  const uint16_t* bounds_src = I.bounds_src;
  const u64 n = umin(I.sizes[0], I.N), nb = I.sizes[1], nout = st->nout, nwords = st->nwords;
  const u64 nchunks = (n + d.C - 1) / d.C;
  const Layout Lo = make_layout(d.S, d.rows, nb, nout, nchunks, nwords);
  const u64 gtid = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  const u64 gstride = (u64)gridDim.x * blockDim.x;
  if (gtid == 0) {
    uint8_t h[kHeaderBytes];
    for (u32 i = 0; i < kHeaderBytes; ++i) h[i] = 0;
    const roix_eb_info e = I.info_in ? *I.info_in : make_eb(d, I.rst->vmin_key, I.rst->vmax_key);
    h[0] = 'R'; h[1] = 'O'; h[2] = 'I'; h[3] = 'X';
    const uint16_t ver = kVersion;
    put_bytes(h, 4, &ver, 2);
    h[6] = (uint8_t)d.dtype;
    h[7] = (uint8_t)d.eb_mode;
    const u32 nx = (u32)d.nx, ny = (u32)d.ny, nz = (u32)d.nz;
    put_bytes(h, 8, &nx, 4);
    put_bytes(h, 12, &ny, 4);
    put_bytes(h, 16, &nz, 4);
    h[20] = (uint8_t)d.cmp;
    h[21] = (uint8_t)d.keep;
    h[22] = (uint8_t)d.conn;
    h[23] = (uint8_t)d.dilate;
    put_bytes(h, 24, &d.threshold, 8);
    put_bytes(h, 32, &d.dark_d, 8);
    put_bytes(h, 40, &d.fill, 8);
    put_bytes(h, 48, &d.eb_value, 8);
    put_bytes(h, 56, &e.eb_abs, 8);
    put_bytes(h, 64, &e.two_eb, 4);
    put_bytes(h, 68, &e.inv2eb, 4);
    put_bytes(h, 72, &e.bound, 4);
    put_bytes(h, 76, &e.eb_int, 4);
    put_bytes(h, 80, &d.R, 4);
    put_bytes(h, 92, &d.order, 4);
    put_bytes(h, 84, &d.C, 4);
    const u32 lmax = kLMax;
    put_bytes(h, 88, &lmax, 4);
    put_bytes(h, 96, &n, 8);
    put_bytes(h, 104, &nout, 8);
    put_bytes(h, 112, &nb, 8);
    put_bytes(h, 120, &nchunks, 8);
    put_bytes(h, 128, &nwords, 8);
    put_bytes(h, 136, &e.vmin, 8);
    put_bytes(h, 144, &e.vmax, 8);
    put_bytes(h, 152, &Lo.off_lens, 8);
    put_bytes(h, 160, &Lo.off_counts, 8);
    put_bytes(h, 168, &Lo.off_bounds, 8);
    put_bytes(h, 176, &Lo.off_outk, 8);
    put_bytes(h, 184, &Lo.off_outv, 8);
    put_bytes(h, 192, &Lo.off_chunks, 8);
    put_bytes(h, 200, &Lo.off_payload, 8);
    put_bytes(h, 208, &Lo.total, 8);
    if (cap >= kHeaderBytes)
      for (u32 i = 0; i < kHeaderBytes; i += 4)
        *reinterpret_cast<u32*>(out + i) = *reinterpret_cast<const u32*>(h + i);
    *I.size_dev = Lo.total;
    st->total = Lo.total;
    if (Lo.total > cap || st->cap_flag) set_status(B.status, ROIX_ECAPACITY);
  }
  // zero the alignment gaps between sections
  const u64 gaps[7][2] = {{Lo.off_lens + d.S, Lo.off_counts},
                          {Lo.off_counts + 2 * d.rows, Lo.off_bounds},
                          {Lo.off_bounds + 2 * nb, Lo.off_outk},
                          {Lo.off_outk + 8 * nout, Lo.off_outv},
                          {Lo.off_outv + 4 * nout, Lo.off_chunks},
                          {Lo.off_chunks + 8 * nchunks, Lo.off_payload},
                          {Lo.off_payload + 4 * nwords, Lo.total}};
  if (gtid < 7 * 16) {
    const u32 g = (u32)(gtid / 16), b = (u32)(gtid % 16);
    const u64 o = gaps[g][0] + b;
    if (o < gaps[g][1] && o < cap) out[o] = 0;
  }
  // geometry from the staged buffers
  if (counts_src)
    for (u64 i = gtid; i < d.rows; i += gstride) {
      const u64 o = Lo.off_counts + 2 * i;
      if (o + 2 <= cap) *reinterpret_cast<uint16_t*>(out + o) = counts_src[i];
    }
  if (bounds_src)
    for (u64 i = gtid; i < nb; i += gstride) {
      const u64 o = Lo.off_bounds + 2 * i;
      if (o + 2 <= cap) *reinterpret_cast<uint16_t*>(out + o) = bounds_src[i];
    }
}

// Per-call reset: the state (all but its first word, the status that
// persists until it is read) and a region of look-back flags and counters.
__global__ void k_init(State* st, u32 nstates, u64* zero, u64 words) {
  const u64 gtid = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (gtid < nstates) {
    u32* s = reinterpret_cast<u32*>(st + gtid);
    for (u32 i = gtid == 0 ? 1 : 0; i < sizeof(State) / 4; ++i) s[i] = 0;
    st[gtid].vmin_key = 0xffffffffu;
  }
  for (u64 i = gtid; i < words; i += (u64)gridDim.x * blockDim.x) zero[i] = 0;
}

int grid_for(const void* fn, int threads, size_t smem, int sms) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem);
  if (per_sm < 1) per_sm = 1;
  return per_sm * sms;
}

}  // namespace

void launch_init(const Launch& L, State* st, u32 nstates, void* zero, size_t zero_bytes) {
  const u64 words = zero ? zero_bytes / 8 : 0;
  u64 blocks = (umax(words, nstates) + kThreads - 1) / kThreads;
  if (blocks < 1) blocks = 1;
  if (blocks > (u64)L.sms * 4) blocks = umax((u64)L.sms * 4, (nstates + kThreads - 1) / kThreads);
  k_init<<<(unsigned)blocks, kThreads, 0, L.stream>>>(st, nstates, (u64*)zero, words);
}

void launch_quantize_stage(const Launch& L, const Desc& d, const void* P, u64 n_cap,
                           const u64* n_dev, int32_t* q, u32* obits, roix_eb_info* info_out,
                           State* st) {
  const unsigned blocks = (unsigned)L.sms * 4;
  if (d.dtype == ROIX_F32) {
    k_range<float><<<blocks, kThreads, 0, L.stream>>>((const float*)P, n_cap, n_dev, st);
    k_quantize_stage<float><<<blocks, kThreads, 0, L.stream>>>(d, (const float*)P, n_cap,
                                                                n_dev, q, obits, info_out, st);
  } else {
    k_range<unsigned short><<<blocks, kThreads, 0, L.stream>>>((const unsigned short*)P, n_cap,
                                                               n_dev, st);
    k_quantize_stage<unsigned short><<<blocks, kThreads, 0, L.stream>>>(
        d, (const unsigned short*)P, n_cap, n_dev, q, obits, info_out, st);
  }
}

void launch_symbols(const Launch& L, const Batch& B, u64 tiles_cap) {
  if (tiles_cap == 0) return;
  const bool from_q = B.it[0].q != nullptr;
  const size_t smem = (size_t)(kThreads / 32) * B.c.S * 4;  // one histogram per warp
  auto run = [&](auto kernel) {
    cudaFuncSetAttribute((const void*)kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    u64 grid = (u64)grid_for((const void*)kernel, kThreads, smem, L.sms);
    if (L.t.sym_blocks_per_sm) grid = umin(grid, (u64)L.t.sym_blocks_per_sm * L.sms);
    const u64 need = (tiles_cap + kThreads / 32 - 1) / (kThreads / 32);  // a segment per warp
    if (grid > need) grid = need;
    kernel<<<(unsigned)grid, kThreads, smem, L.stream>>>(B);
  };
  if (B.c.dtype == ROIX_F32) {
    if (B.c.order == 2) {
      if (from_q) run(k_symbols<float, true, 2>);
      else run(k_symbols<float, false, 2>);
    } else {
      if (from_q) run(k_symbols<float, true, 1>);
      else run(k_symbols<float, false, 1>);
    }
  } else {
    if (B.c.order == 2) {
      if (from_q) run(k_symbols<unsigned short, true, 2>);
      else run(k_symbols<unsigned short, false, 2>);
    } else {
      if (from_q) run(k_symbols<unsigned short, true, 1>);
      else run(k_symbols<unsigned short, false, 1>);
    }
  }
}

void launch_codebook(const Launch& L, const Batch& B) {
  const size_t smem = codebook_smem(B.c.S);
  cudaFuncSetAttribute((const void*)k_codebook, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)smem);
  k_codebook<<<B.n, kCbThreads, smem, L.stream>>>(B);
}

void launch_pack(const Launch& L, const Batch& B, u64 ranges_cap) {
  if (ranges_cap == 0) return;
  const u64 wpb = kThreads / 32;
  {  // chunk sizes and records
    const bool from_q = B.it[0].q != nullptr;
    auto count = [&](auto kernel) {
      u64 grid = (u64)grid_for((const void*)kernel, kThreads, 0, L.sms);
      grid = umin(grid, (ranges_cap + wpb - 1) / wpb);
      kernel<<<(unsigned)grid, kThreads, 0, L.stream>>>(B);
    };
    if (B.c.dtype == ROIX_F32) {
      if (from_q) count(k_pack_count<float, true>);
      else count(k_pack_count<float, false>);
    } else {
      if (from_q) count(k_pack_count<unsigned short, true>);
      else count(k_pack_count<unsigned short, false>);
    }
  }
  // chunk and record offsets, then records, of the items too large for the
  // in-kernel scans
  u64 scan_tiles = 0;
  for (u32 i = 0; i < B.n; ++i)
    if (!B.it[i].pscan) scan_tiles += (B.it[i].N + B.c.C - 1) / B.c.C / kScanTile + 1;
  launch_scan_pairs(L, B, 1, scan_tiles);
  if (scan_tiles) {
    const bool from_q = B.it[0].q != nullptr;
    const u64 grid = umin((ranges_cap + wpb - 1) / wpb, (u64)L.sms * 8);
    if (B.c.dtype == ROIX_F32) {
      if (from_q) k_records<float, true><<<(unsigned)grid, kThreads, 0, L.stream>>>(B);
      else k_records<float, false><<<(unsigned)grid, kThreads, 0, L.stream>>>(B);
    } else {
      if (from_q) k_records<unsigned short, true><<<(unsigned)grid, kThreads, 0, L.stream>>>(B);
      else k_records<unsigned short, false><<<(unsigned)grid, kThreads, 0, L.stream>>>(B);
    }
  }
  const size_t smem = pack_smem(B.c.C, B.c.S);  // symbol buffers, code tables, stream
  auto run = [&](auto kernel) {
    cudaFuncSetAttribute((const void*)kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    u64 grid = (u64)grid_for((const void*)kernel, kThreads, smem, L.sms);
    if (L.t.pack_blocks_per_sm) grid = umin(grid, (u64)L.t.pack_blocks_per_sm * L.sms);
    if (grid > ranges_cap) grid = ranges_cap;
    kernel<<<(unsigned)grid, kThreads, smem, L.stream>>>(B);
  };
  switch (B.c.C / kThreads) {
    case 1: run(k_pack<1>); break;
    case 2: run(k_pack<2>); break;
    case 4: run(k_pack<4>); break;
    case 8: run(k_pack<8>); break;
    case 16: run(k_pack<16>); break;
    case 32: run(k_pack<32>); break;
    case 64: run(k_pack<64>); break;
    default: break;  // rejected on the host
  }
}

void launch_finalize(const Launch& L, const Batch& B) {
  const unsigned bx = B.n > 8 ? 4u : (unsigned)L.sms;
  dim3 grid(bx, B.n);
  k_finalize<<<grid, kThreads, 0, L.stream>>>(B);
}

}  // namespace roix
