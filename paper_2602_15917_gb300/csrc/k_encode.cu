// Coder kernels: error-bounded quantisation (Sec. 4.2.3 contract, Sz3-style
// linear lattice of Sec. 4.3), 1D Lorenzo prediction with symbolisation and a
// histogram, the canonical Huffman codebook, the chunked bit packer and the
// container finaliser.
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

// Symbol of a delta: d + R when -R < d < R, else 0. Codes lie in
// [-2^30, 2^30], so the true delta lies in [-2^31, 2^31]; its two's-complement
// wrap to 0x80000000 at the extremes still fails the unsigned range test.
__device__ __forceinline__ u32 symbol_of(int c, int prev, bool out, u32 R) {
  if (out) return 0u;
  const u32 dd = (u32)c - (u32)prev;
  return (dd + R - 1u < 2u * R - 1u) ? dd + R : 0u;
}

// bits 0..15 of v spread to the even positions 0, 2, ..., 30
__device__ __forceinline__ u32 spread16(u32 v) {
  v &= 0xffffu;
  v = (v | (v << 8)) & 0x00ff00ffu;
  v = (v | (v << 4)) & 0x0f0f0f0fu;
  v = (v | (v << 2)) & 0x33333333u;
  v = (v | (v << 1)) & 0x55555555u;
  return v;
}

// Persistent blocks take tiles of kQuantTile values; each warp owns a
// contiguous span of the tile and walks it 64 values (a pair per lane) per
// step, so loads and symbol stores are coalesced vectors and the predecessor
// of a step's first value is the warp's own last value of the step before.
// Loads of four steps are issued before any is used. Symbol-0 positions
// (records) are marked in a shared bitmap, counted, placed by the look-back
// and written in order. The histogram lives in shared memory per block and is
// flushed once at the end.
// Tiles of every item, in order: prefix of ceil(n_i / kQuantTile) over the
// items (n_i found by the compaction), computed by each block at start.
__device__ __forceinline__ void tile_prefix(const Batch& B, u64* pre, u64 per, u64 group) {
  if (threadIdx.x == 0) {
    u64 acc = 0;
    for (u32 i = 0; i < B.n; ++i) {
      pre[i] = acc;
      const Item& I = B.it[i];
      const u64 n = umin(I.sizes[0], I.N);
      acc += ((n + per - 1) / per + group - 1) / group;
    }
    pre[B.n] = acc;
  }
  __syncthreads();
}

template <typename TV, bool FROM_Q>
__global__ void __launch_bounds__(kThreads) k_symbols(const __grid_constant__ Batch B) {
  using R = typename Src<TV, FROM_Q>::R;
  constexpr u32 kSpan = kQuantTile / (kThreads / 32);  // values per warp and tile
  constexpr int kSteps = kSpan / 64;
  constexpr int kBatch = 4;
  __shared__ u32 h[kMaxSym];
  __shared__ u32 bitmap[kQuantTile / 32];
  __shared__ u32 scratch[40];
  __shared__ u64 s_tile, s_base;
  __shared__ u64 pre[kMaxBatch + 1];
  static_assert(kQuantTile / 32 == kThreads, "one bitmap word per thread");
  static_assert(kSteps % kBatch == 0, "whole batches");
  const u32 R_ = B.c.R, S = B.c.S;
  for (u32 i = threadIdx.x; i < S; i += blockDim.x) h[i] = 0;
  tile_prefix(B, pre, kQuantTile, 1);
  const u64 total = pre[B.n];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  u32 cur = 0xffffffffu;
  Src<TV, FROM_Q> src{};
  u64 n = 0;
  while (true) {
    if (threadIdx.x == 0) s_tile = atomicAdd(&B.ctr[1], 1u);
    __syncthreads();
    const u64 gt = s_tile;
    if (gt >= total) break;
    const u32 item = find_item(pre, B.n, gt);
    const Item& I = B.it[item];
    if (item != cur) {  // histogram of the previous item out, the next one's settings in
      if (cur != 0xffffffffu) {
        unsigned long long* hg = B.it[cur].hist;
        for (u32 i = threadIdx.x; i < S; i += blockDim.x)
          if (h[i]) {
            atomicAdd(hg + i, (unsigned long long)h[i]);
            h[i] = 0;
          }
      }
      cur = item;
      const Desc d = desc_of(B, I);
      src.P = (const TV*)I.P;
      src.q = I.q;
      src.obits = I.obits;
      src.dark = d.dark;
      if constexpr (!FROM_Q) {
        src.e = make_eb(d, I.st->vmin_key, I.st->vmax_key);
        src.fd = FastDiv(2u * (u32)src.e.eb_int);
      }
      n = umin(I.sizes[0], I.N);
      __syncthreads();
    }
    const u64 t = gt - pre[item];
    const u64 ntiles = (n + kQuantTile - 1) / kQuantTile;
    uint16_t* __restrict__ sym = I.sym;
    const u64 base = t * kQuantTile;
    const u64 span = base + (u64)warp * kSpan;
    bitmap[threadIdx.x] = 0u;
    // code of the value just before the warp's span
    int carry = 0;
    if (lane == 0 && span > 0 && span < n) {
      bool op;
      carry = src.code(span - 1, op);
    }
    carry = __shfl_sync(0xffffffffu, carry, 0);
    __syncthreads();
    for (int b0 = 0; b0 < kSteps; b0 += kBatch) {
      R ra[kBatch], rb[kBatch];
#pragma unroll
      for (int j = 0; j < kBatch; ++j) {
        const u64 k0 = span + 64 * (u64)(b0 + j) + 2 * lane;
        if (k0 + 1 < n) {
          src.load2(k0, ra[j], rb[j]);
        } else {
          ra[j] = k0 < n ? src.load1(k0) : R{TV(0), 0, 0u};
          rb[j] = R{TV(0), 0, 0u};
        }
      }
#pragma unroll
      for (int j = 0; j < kBatch; ++j) {
        const int it = b0 + j;
        const u64 k0 = span + 64 * (u64)it + 2 * lane, k1 = k0 + 1;
        bool o0 = false, o1 = false;
        const int c0 = k0 < n ? src.eval(ra[j], o0) : 0;
        const int c1 = k1 < n ? src.eval(rb[j], o1) : 0;
        int prev = __shfl_up_sync(0xffffffffu, c1, 1);
        if (lane == 0) prev = carry;
        carry = __shfl_sync(0xffffffffu, c1, 31);
        const u32 s0 = k0 < n ? symbol_of(c0, prev, o0, R_) : 1u;
        const u32 s1 = k1 < n ? symbol_of(c1, c0, o1, R_) : 1u;
        if (k1 < n) {
          *reinterpret_cast<u32*>(sym + k0) = s0 | (s1 << 16);
        } else if (k0 < n) {
          sym[k0] = (uint16_t)s0;
        }
        const bool r0 = k0 < n && s0 == 0, r1 = k1 < n && s1 == 0;
        const u32 bb0 = __ballot_sync(0xffffffffu, r0), bb1 = __ballot_sync(0xffffffffu, r1);
        if ((bb0 | bb1) && lane < 2) {  // records are rare: the bitmap starts zeroed
          const u32 wi = warp * (kSpan / 32) + 2 * it + lane;
          const u32 sh = lane ? 16u : 0u;
          bitmap[wi] = spread16(bb0 >> sh) | (spread16(bb1 >> sh) << 1);
        }
        // histogram: deltas of noisy data rarely repeat within a warp, so plain
        // shared-memory atomics beat warp aggregation here
        if (k0 < n) atomicAdd(&h[s0], 1u);
        if (k1 < n) atomicAdd(&h[s1], 1u);
      }
    }
    __syncthreads();
    // records of this tile, in order
    const u32 word = bitmap[threadIdx.x];
    u32 tot;
    const u32 off = block_excl_scan<u32>(__popc(word), scratch, &tot);
    if (warp == 0) {
      u64 mine[1] = {tot}, excl[1];
      lookback_warp<1>(I.lbq, t, mine, excl, B.status);
      if (lane == 0) {
        s_base = excl[0];
        if (t == ntiles - 1) I.st->nout = excl[0] + tot;
      }
    }
    __syncthreads();
    if (word) {
      u64 idx = s_base + off;
      u32 wv = word;
      while (wv) {
        const int j = __ffs(wv) - 1;
        wv &= wv - 1;
        const u64 k = base + (u64)threadIdx.x * 32 + j;
        bool out;
        const int c = src.code(k, out);
        if (idx < I.rec_cap) {
          I.rk[idx] = k | (out ? (1ull << 63) : 0ull);
          I.rv[idx] = out ? src.raw_bits(k) : (u32)c;
        } else {
          atomicExch(&I.st->cap_flag, 1u);
        }
        ++idx;
      }
    }
    __syncthreads();
  }
  __syncthreads();
  if (cur != 0xffffffffu) {
    unsigned long long* hg = B.it[cur].hist;
    for (u32 i = threadIdx.x; i < S; i += blockDim.x)
      if (h[i]) atomicAdd(hg + i, (unsigned long long)h[i]);
  }
}

// ------------------------------------------------------------- codebook
// One block of 1024 threads builds the canonical length-limited Huffman code:
// bitonic sort of (count, symbol) keys, the two-queue construction on one
// thread (van Leeuwen), depths by pointer jumping, the per-length fold for
// lengths over 24 (ITU-T T.81 Annex K.3 procedure), lengths handed out
// shortest-first from the most frequent leaf, canonical codes (RFC 1951).
constexpr int kCbThreads = 1024;

__device__ void bitonic_sort(u64* key, u32 M) {
  for (u32 k = 2; k <= M; k <<= 1) {
    for (u32 j = k >> 1; j > 0; j >>= 1) {
      for (u32 i = threadIdx.x; i < M; i += blockDim.x) {
        const u32 l = i ^ j;
        if (l > i) {
          const u64 a = key[i], b = key[l];
          const bool up = (i & k) == 0;
          if ((a > b) == up) {
            key[i] = b;
            key[l] = a;
          }
        }
      }
      __syncthreads();
    }
  }
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

__global__ void __launch_bounds__(kCbThreads) k_codebook(const __grid_constant__ Batch B) {
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
  if (m <= (u32)kCbThreads) {
    // rank of each (count, symbol) key among the m distinct keys: one key per
    // thread, every thread reads the keys in the same order (smem broadcast)
    u64 mine = tid < (int)m ? key[tid] : 0ull;
    u32 rank = 0;
    if (tid < (int)m)  // only the warps holding keys read them
      for (u32 j = 0; j < m; ++j) rank += key[j] < mine;
    __syncthreads();
    if (tid < (int)m) key[rank] = mine;
    __syncthreads();
  } else {
    bitonic_sort(key, M);  // ascending (count, symbol)
  }
  CB_MARK(2)
  if (m == 1) {
    if (tid == 0) {
      len[key[0] & 0xffffu] = 1;
      bl[1] = 1;
    }
  } else if (m >= 2) {
    // two-queue construction: leaves 0..m-1 in sorted order, internal m..2m-2.
    // Both queue fronts live in registers; an empty queue reads as the
    // sentinel ~0 (weights are below 2^48), so "leaf if wl <= wi" keeps the
    // leaf-first tie rule. The next front is loaded right after a pop.
    if (tid == 0) {
      constexpr u64 kNone = ~0ull;
      u32 lf = 0, in = 0, created = 0;
      u64 wl = key[0] >> 16, wi = kNone;
      u64 wl_next = m > 1 ? (key[1] >> 16) : kNone;  // the leaf after the front, prefetched
      for (u32 t = 0; t + 1 < m; ++t) {
        int32_t pa, pb;
        u64 wa, wb;
        if (wl <= wi) {
          pa = (int32_t)lf;
          wa = wl;
          ++lf;
          wl = wl_next;
          wl_next = lf + 1 < m ? (key[lf + 1] >> 16) : kNone;
        } else {
          pa = (int32_t)(m + in);
          wa = wi;
          ++in;
          wi = in < created ? wint[in] : kNone;
        }
        if (wl <= wi) {
          pb = (int32_t)lf;
          wb = wl;
          ++lf;
          wl = wl_next;
          wl_next = lf + 1 < m ? (key[lf + 1] >> 16) : kNone;
        } else {
          pb = (int32_t)(m + in);
          wb = wi;
          ++in;
          wi = in < created ? wint[in] : kNone;
        }
        const u64 w2 = wa + wb;
        wint[created] = w2;
        par[pa] = (int32_t)(m + created);
        par[pb] = (int32_t)(m + created);
        ++created;
        if (in == created - 1) wi = w2;  // the queue was empty: the new node is its front
      }
      par[2 * m - 2] = -1;
    }
    __syncthreads();
    CB_MARK(3)
    // depth = distance to the root, by pointer jumping
    const u32 nodes = 2 * m - 1;
    for (u32 i = tid; i < nodes; i += kCbThreads) dep[i] = par[i] >= 0 ? 1 : 0;
    __syncthreads();
    for (u32 round = 0; (1u << round) < nodes; ++round) {
      int32_t na[(2 * kMaxSym + kCbThreads - 1) / kCbThreads];
      int32_t nd[(2 * kMaxSym + kCbThreads - 1) / kCbThreads];
      int cnt = 0;
      for (u32 i = tid; i < nodes; i += kCbThreads, ++cnt) {
        const int32_t a = par[i];
        nd[cnt] = a >= 0 ? dep[i] + dep[a] : dep[i];
        na[cnt] = a >= 0 ? par[a] : -1;
      }
      __syncthreads();
      cnt = 0;
      for (u32 i = tid; i < nodes; i += kCbThreads, ++cnt) {
        dep[i] = nd[cnt];
        par[i] = na[cnt];
      }
      __syncthreads();
    }
    CB_MARK(4)
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
      if (s < S) codes_ws[s] = l ? s_next[l] + wcnt[warp][l] + below : 0u;
      __syncthreads();
    }
  }
  CB_MARK(6)
  for (u32 s = tid; s < S; s += kCbThreads) {
    lens_ws[s] = len[s];
    if (kHeaderBytes + s < cap) out[kHeaderBytes + s] = len[s];
  }
  CB_MARK(7)
}

// ------------------------------------------------------------------- pack
// Persistent blocks take ranges of kPackRange chunks of C symbols, in order.
// Pass 1 sums the code lengths of every chunk of the range (block scans; the
// per-thread bit offsets are kept in shared memory); one look-back per range
// gives the range's word offset. Pass 2 re-reads each chunk (from L2), shifts
// every thread's codes through a 64-bit register, stores the words that lie
// wholly inside its bit range and OR-s only its first and last (shared)
// words into the shared buffer, which is copied out with coalesced stores.

template <int EPT>
__device__ __forceinline__ void load_syms(const uint16_t* __restrict__ sym, u64 k0, u64 n,
                                          uint16_t (&sv)[EPT]) {
  if constexpr (EPT % 8 == 0) {
    if (k0 + EPT <= n) {
#pragma unroll
      for (int j = 0; j < EPT; j += 8) {
        const uint4 v = __ldg(reinterpret_cast<const uint4*>(sym + k0 + j));
        const u32 w4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          sv[j + 2 * q] = (uint16_t)(w4[q] & 0xffffu);
          sv[j + 2 * q + 1] = (uint16_t)(w4[q] >> 16);
        }
      }
      return;
    }
  }
#pragma unroll
  for (int j = 0; j < EPT; ++j) sv[j] = k0 + j < n ? __ldg(sym + k0 + j) : (uint16_t)0;
}

template <int EPT>  // symbols per thread = C / 256
__global__ void __launch_bounds__(kThreads, 4) k_pack(const __grid_constant__ Batch B) {
  extern __shared__ u32 wbuf[];  // C * 24 / 32 + 2 words
  constexpr u32 kPackWordsMax = EPT * kThreads * kLMax / 32 + 2;
  __shared__ uint8_t slen[kMaxSym];
  __shared__ u32 scode[kMaxSym];
  __shared__ u32 boffs[kPackRange][kThreads];
  __shared__ u32 cwords[kPackRange];
  __shared__ u32 scratch[40];
  __shared__ u64 s_tile, s_base;
  __shared__ u64 pre[kMaxBatch + 1];
  const u32 C = B.c.C, S = B.c.S;
  tile_prefix(B, pre, C, kPackRange);
  const u64 total = pre[B.n];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  u32 cur = 0xffffffffu;
  u64 n = 0, nchunks = 0, nranges = 0;
  Layout Lo{};
  const uint16_t* __restrict__ sym = nullptr;
  uint8_t* out = nullptr;
  u64 cap = 0;
  while (true) {
    if (threadIdx.x == 0) s_tile = atomicAdd(&B.ctr[2], 1u);
    __syncthreads();
    const u64 gr = s_tile;
    if (gr >= total) break;
    const u32 item = find_item(pre, B.n, gr);
    const Item& I = B.it[item];
    if (item != cur) {  // the item's code table into shared memory
      cur = item;
      for (u32 i = threadIdx.x; i < S; i += blockDim.x) {
        slen[i] = I.lens[i];
        scode[i] = I.codes[i];
      }
      n = umin(I.sizes[0], I.N);
      nchunks = (n + C - 1) / C;
      nranges = (nchunks + kPackRange - 1) / kPackRange;
      Lo = make_layout(S, I.rows, I.sizes[1], I.st->nout, nchunks, 0);
      sym = I.sym;
      out = I.out;
      cap = I.cap;
      __syncthreads();
    }
    const u64 r = gr - pre[item];
    const u64 c_lo = r * kPackRange;
    const u32 nc = (u32)umin(kPackRange, nchunks - c_lo);
    // pass 1: bits per thread and chunk
    for (u32 c = 0; c < nc; ++c) {
      const u64 k0 = (c_lo + c) * C + (u64)threadIdx.x * EPT;
      uint16_t sv[EPT];
      load_syms<EPT>(sym, k0, n, sv);
      u32 bits = 0;
#pragma unroll
      for (int j = 0; j < EPT; ++j) bits += (k0 + j < n) ? slen[sv[j]] : 0u;
      u32 total;
      boffs[c][threadIdx.x] = block_excl_scan<u32>(bits, scratch, &total);
      if (threadIdx.x == 0) cwords[c] = (total + 31) >> 5;
    }
    __syncthreads();
    if (warp == 0) {
      u32 rw = lane < nc ? cwords[lane] : 0u;
      rw = warp_sum(rw);
      u64 mine[1] = {rw}, excl[1];
      lookback_warp<1>(I.lbp, r, mine, excl, B.status);
      if (lane == 0) {
        s_base = excl[0];
        if (r == nranges - 1) I.st->nwords = excl[0] + rw;
      }
    }
    __syncthreads();
    // pass 2: pack and copy out each chunk
    u64 cbase = s_base;
    for (u32 c = 0; c < nc; ++c) {
      const u64 t = c_lo + c;
      const u32 words = cwords[c];
      if (threadIdx.x == 0) {
        const u64 o = Lo.off_chunks + 8 * t;
        if (o + 8 <= cap) *reinterpret_cast<u64*>(out + o) = cbase;
      }
      for (u32 i = threadIdx.x; i <= words && i < kPackWordsMax; i += blockDim.x) wbuf[i] = 0;
      __syncthreads();
      const u64 k0 = t * C + (u64)threadIdx.x * EPT;
      uint16_t sv[EPT];
      load_syms<EPT>(sym, k0, n, sv);
      const u32 boff = boffs[c][threadIdx.x];
      u64 acc = 0;
      u32 nacc = boff & 31;  // leading bits belong to earlier threads (zeros here)
      u32 wi = boff >> 5;
      bool shared_first = (boff & 31) != 0;
      u32 mybits = 0;
#pragma unroll
      for (int j = 0; j < EPT; ++j) {
        if (k0 + j < n) {
          const u32 l = slen[sv[j]];
          mybits += l;
          acc = (acc << l) | scode[sv[j]];
          nacc += l;
          if (nacc >= 32) {
            const u32 wv = (u32)(acc >> (nacc - 32));
            if (shared_first) atomicOr(&wbuf[wi], wv);
            else wbuf[wi] = wv;
            shared_first = false;
            ++wi;
            nacc -= 32;
            acc &= (1ull << nacc) - 1ull;
          }
        }
      }
      if (mybits && nacc > (shared_first ? (boff & 31) : 0u))
        atomicOr(&wbuf[wi], (u32)(acc << (32 - nacc)));
      __syncthreads();
      for (u32 i = threadIdx.x; i < words; i += blockDim.x) {
        const u64 o = Lo.off_payload + 4 * (cbase + i);
        if (o + 4 <= cap) *reinterpret_cast<u32*>(out + o) = wbuf[i];
      }
      cbase += words;
      __syncthreads();
    }
  }
}

// --------------------------------------------------------------- finalize
__device__ __forceinline__ void put_bytes(uint8_t* h, u32 off, const void* src, u32 bytes) {
  const uint8_t* s = (const uint8_t*)src;
  for (u32 i = 0; i < bytes; ++i) h[off + i] = s[i];
}

__global__ void __launch_bounds__(kThreads) k_finalize(const __grid_constant__ Batch B) {
  const Item& I = B.it[blockIdx.y];
  const Desc d = desc_of(B, I);
  State* st = I.st;
  uint8_t* out = I.out;
  const u64 cap = I.cap;
  const u64 rec_cap = I.rec_cap;
  const u64* __restrict__ rk = I.rk;
  const u32* __restrict__ rv = I.rv;
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
    const roix_eb_info e = I.info_in ? *I.info_in : make_eb(d, st->vmin_key, st->vmax_key);
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
  // outlier records
  for (u64 i = gtid; i < umin(nout, rec_cap); i += gstride) {
    const u64 ok = Lo.off_outk + 8 * i, ov = Lo.off_outv + 4 * i;
    if (ok + 8 <= cap) *reinterpret_cast<u64*>(out + ok) = rk[i];
    if (ov + 4 <= cap) *reinterpret_cast<u32*>(out + ov) = rv[i];
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
  auto run = [&](auto kernel) {
    u64 grid = (u64)grid_for((const void*)kernel, kThreads, 0, L.sms);
    if (grid > tiles_cap) grid = tiles_cap;
    kernel<<<(unsigned)grid, kThreads, 0, L.stream>>>(B);
  };
  if (B.c.dtype == ROIX_F32) {
    if (from_q) run(k_symbols<float, true>);
    else run(k_symbols<float, false>);
  } else {
    if (from_q) run(k_symbols<unsigned short, true>);
    else run(k_symbols<unsigned short, false>);
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
  const size_t smem = ((size_t)B.c.C * kLMax / 32 + 2) * 4;
  auto run = [&](auto kernel) {
    cudaFuncSetAttribute((const void*)kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    u64 grid = (u64)grid_for((const void*)kernel, kThreads, smem, L.sms);
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
