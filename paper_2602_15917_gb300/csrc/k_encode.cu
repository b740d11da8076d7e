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
// pixel section (fused path) or read from the staged codes.
template <typename TV, bool FROM_Q>
struct Src {
  const TV* P;
  const int32_t* q;
  const u32* obits;
  roix_eb_info e;
  int dark;
  __device__ __forceinline__ int code(u64 k, bool& out) const {
    if constexpr (FROM_Q) {
      out = (__ldg(obits + (k >> 5)) >> (k & 31)) & 1u;
      return out ? 0 : __ldg(q + k);
    } else if constexpr (sizeof(TV) == 4) {
      return quant_f32(__ldg(P + k), e, out);
    } else {
      out = false;
      return quant_u16(__ldg(P + k), dark, e.eb_int);
    }
  }
  __device__ __forceinline__ u32 raw_bits(u64 k) const {
    if constexpr (sizeof(TV) == 4) return __float_as_uint(__ldg(P + k));
    else return (u32)__ldg(P + k);
  }
};

__device__ __forceinline__ u32 symbol_of(int c, int prev, bool out, u32 R) {
  if (out) return 0u;
  const long long dd = (long long)c - (long long)prev;
  return (dd > -(long long)R && dd < (long long)R) ? (u32)(dd + R) : 0u;
}

__device__ __forceinline__ u32 interleave16(u32 a, u32 b) {  // bit i of a -> 2i, of b -> 2i+1
  u32 r = 0;
#pragma unroll
  for (int i = 0; i < 16; ++i) r |= (((a >> i) & 1u) << (2 * i)) | (((b >> i) & 1u) << (2 * i + 1));
  return r;
}

// Persistent blocks take tiles of kQuantTile values. A thread handles pairs
// (k, k+1) so that symbol stores are 32-bit and coalesced; the predecessor code
// of the pair comes from the neighbouring lane (lane 0 recomputes it). Symbol-0
// positions (records) are marked in a shared bitmap, counted, placed by the
// look-back and written in order. The histogram is kept in shared memory per
// block, warp-aggregated with __match_any_sync, and flushed once at the end.
template <typename TV, bool FROM_Q>
__global__ void __launch_bounds__(kThreads) k_symbols(Desc d, Src<TV, FROM_Q> src, u64 n_cap,
                                                      const u64* n_dev, State* st,
                                                      uint16_t* __restrict__ sym,
                                                      u64* __restrict__ rk, u32* __restrict__ rv,
                                                      u64 rec_cap, unsigned long long* hist,
                                                      LookBack<1> lb, int compute_eb) {
  __shared__ u32 h[kMaxSym];
  __shared__ u32 bitmap[kQuantTile / 32];
  __shared__ u32 scratch[40];
  __shared__ u64 s_tile, s_base;
  static_assert(kQuantTile / 32 == kThreads, "one bitmap word per thread");
  const u64 n = n_dev ? min(*n_dev, n_cap) : n_cap;
  if (compute_eb) {
    src.e = make_eb(d, st->vmin_key, st->vmax_key);
    if (blockIdx.x == 0 && threadIdx.x == 0) st->eb = src.e;
  }
  const u32 R = d.R;
  for (u32 i = threadIdx.x; i < d.S; i += blockDim.x) h[i] = 0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const u64 ntiles = (n + kQuantTile - 1) / kQuantTile;
  __syncthreads();
  while (true) {
    if (threadIdx.x == 0) s_tile = atomicAdd(&st->ctr_quant, 1u);
    __syncthreads();
    const u64 t = s_tile;
    if (t >= ntiles) break;
    const u64 base = t * kQuantTile;
    for (u32 it = 0; it < kQuantTile / (2 * kThreads); ++it) {
      const u32 pl = it * kThreads + threadIdx.x;  // pair within tile
      const u64 k0 = base + 2 * (u64)pl, k1 = k0 + 1;
      bool o0 = false, o1 = false;
      int c0 = 0, c1 = 0;
      if (k0 < n) c0 = src.code(k0, o0);
      if (k1 < n) c1 = src.code(k1, o1);
      int prev = __shfl_up_sync(0xffffffffu, c1, 1);
      if (lane == 0) {
        prev = 0;
        if (k0 > 0 && k0 < n) {
          bool op;
          prev = src.code(k0 - 1, op);
        }
      }
      const u32 s0 = k0 < n ? symbol_of(c0, prev, o0, R) : 1u;
      const u32 s1 = k1 < n ? symbol_of(c1, c0, o1, R) : 1u;
      if (k1 < n) {
        *reinterpret_cast<u32*>(sym + k0) = s0 | (s1 << 16);
      } else if (k0 < n) {
        sym[k0] = (uint16_t)s0;
      }
      const bool r0 = k0 < n && s0 == 0, r1 = k1 < n && s1 == 0;
      const u32 b0 = __ballot_sync(0xffffffffu, r0), b1 = __ballot_sync(0xffffffffu, r1);
      if (lane == 0) {
        const u32 wi = (it * kThreads + warp * 32) / 16;
        bitmap[wi] = interleave16(b0 & 0xffffu, b1 & 0xffffu);
        bitmap[wi + 1] = interleave16(b0 >> 16, b1 >> 16);
      }
      // histogram, one shared atomic per distinct symbol of the warp
      {
        const bool v0 = k0 < n;
        const u32 m0 = __match_any_sync(0xffffffffu, v0 ? s0 : 0xffffffffu);
        if (v0 && (__ffs(m0) - 1) == lane) atomicAdd(&h[s0], (u32)__popc(m0));
        const bool v1 = k1 < n;
        const u32 m1 = __match_any_sync(0xffffffffu, v1 ? s1 : 0xffffffffu);
        if (v1 && (__ffs(m1) - 1) == lane) atomicAdd(&h[s1], (u32)__popc(m1));
      }
    }
    __syncthreads();
    // records of this tile, in order
    const u32 word = bitmap[threadIdx.x];
    u32 total;
    const u32 off = block_excl_scan<u32>(__popc(word), scratch, &total);
    if (threadIdx.x == 0) {
      u64 mine[1] = {total}, excl[1];
      lookback<1>(lb, t, mine, excl, &st->status);
      s_base = excl[0];
      if (t == ntiles - 1) st->nout = excl[0] + total;
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
        if (idx < rec_cap) {
          rk[idx] = k | (out ? (1ull << 63) : 0ull);
          rv[idx] = out ? src.raw_bits(k) : (u32)c;
        } else {
          atomicExch(&st->cap_flag, 1u);
        }
        ++idx;
      }
    }
    __syncthreads();
  }
  __syncthreads();
  for (u32 i = threadIdx.x; i < d.S; i += blockDim.x)
    if (h[i]) atomicAdd(hist + i, (unsigned long long)h[i]);
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

size_t codebook_smem(u32 S) {
  return (size_t)next_pow2(S) * 8  // key (sorted with a power-of-two bitonic network)
         + (size_t)S * 8      // internal weights
         + (size_t)2 * S * 4  // parent / ancestor
         + (size_t)2 * S * 4  // depth
         + (size_t)(S + 2) * 4  // leaves per depth
         + (size_t)S;         // lengths
}

__global__ void __launch_bounds__(kCbThreads) k_codebook(Desc d, const unsigned long long* hist,
                                                         uint8_t* lens_ws, u32* codes_ws,
                                                         uint8_t* out, u64 cap, State* st) {
  extern __shared__ __align__(16) unsigned char cb_smem[];
  const u32 S = d.S;
  u64* key = (u64*)cb_smem;                       // [next_pow2(S)] (count << 16 | symbol)
  u64* wint = key + next_pow2(S);                 // [S] internal node weights
  int32_t* par = (int32_t*)(wint + S);            // [2S]
  int32_t* dep = par + 2 * S;                     // [2S]
  u32* bl = (u32*)(dep + 2 * S);                  // [S + 2]
  uint8_t* len = (uint8_t*)(bl + S + 2);          // [S]
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
  for (u32 i = tid; i < S + 2; i += kCbThreads) bl[i] = 0;
  u32 M = 1;
  while (M < m) M <<= 1;
  for (u32 i = m + tid; i < M; i += kCbThreads) key[i] = ~0ull;
  __syncthreads();
  bitonic_sort(key, M);  // ascending (count, symbol)
  if (m == 1) {
    if (tid == 0) {
      len[key[0] & 0xffffu] = 1;
      bl[1] = 1;
    }
  } else if (m >= 2) {
    // two-queue construction: leaves 0..m-1 in sorted order, internal m..2m-2
    if (tid == 0) {
      u32 lf = 0, in = 0, created = 0;
      u64 wl = key[0] >> 16;
      for (u32 t = 0; t + 1 < m; ++t) {
        u64 w2 = 0;
        int32_t pick[2];
        for (int a = 0; a < 2; ++a) {
          const bool leaf_ok = lf < m, int_ok = in < created;
          const u64 wiv = int_ok ? wint[in] : 0ull;
          if (leaf_ok && (!int_ok || wl <= wiv)) {
            pick[a] = (int32_t)lf;
            w2 += wl;
            ++lf;
            wl = lf < m ? (key[lf] >> 16) : 0ull;
          } else {
            pick[a] = (int32_t)(m + in);
            w2 += wiv;
            ++in;
          }
        }
        wint[created] = w2;
        par[pick[0]] = (int32_t)(m + created);
        par[pick[1]] = (int32_t)(m + created);
        ++created;
      }
      par[2 * m - 2] = -1;
    }
    __syncthreads();
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
  // canonical order: sort used symbols by (length, symbol)
  for (u32 i = tid; i < m; i += kCbThreads) {
    const u32 s = (u32)(key[i] & 0xffffu);
    key[i] = ((u64)len[s] << 16) | s;
  }
  __syncthreads();
  bitonic_sort(key, M);
  for (u32 s = tid; s < S; s += kCbThreads) codes_ws[s] = 0;
  __syncthreads();
  for (u32 i = tid; i < m; i += kCbThreads) {
    const u32 l = (u32)(key[i] >> 16), s = (u32)(key[i] & 0xffffu);
    codes_ws[s] = s_next[l] + (i - s_cum[l - 1]);
  }
  for (u32 s = tid; s < S; s += kCbThreads) {
    lens_ws[s] = len[s];
    if (kHeaderBytes + s < cap) out[kHeaderBytes + s] = len[s];
  }
}

// ------------------------------------------------------------------- pack
// Persistent blocks take chunks of C symbols. Per chunk: code lengths summed
// per thread (consecutive symbols), block scan, look-back for the chunk's word
// offset, codes OR-ed into a shared word buffer MSB first, buffer copied out.
template <int EPT>  // symbols per thread = C / 256
__global__ void __launch_bounds__(kThreads) k_pack(Desc d, const uint16_t* __restrict__ sym,
                                                   const u64* n_dev, const u64* nb_dev,
                                                   const uint8_t* lens_ws, const u32* codes_ws,
                                                   State* st, uint8_t* out, u64 cap,
                                                   LookBack<1> lb) {
  extern __shared__ u32 wbuf[];  // C * 24 / 32 + 2 words
  __shared__ uint8_t slen[kMaxSym];
  __shared__ u32 scode[kMaxSym];
  __shared__ u32 scratch[40];
  __shared__ u64 s_tile, s_base;
  const u64 n = *n_dev;
  const u32 C = d.C;
  const u64 nchunks = (n + C - 1) / C;
  const Layout Lo = make_layout(d.S, d.rows, *nb_dev, st->nout, nchunks, 0);
  for (u32 i = threadIdx.x; i < d.S; i += blockDim.x) {
    slen[i] = lens_ws[i];
    scode[i] = codes_ws[i];
  }
  __syncthreads();
  while (true) {
    if (threadIdx.x == 0) s_tile = atomicAdd(&st->ctr_pack, 1u);
    __syncthreads();
    const u64 t = s_tile;
    if (t >= nchunks) break;
    const u64 k0 = t * C + (u64)threadIdx.x * EPT;
    uint16_t sv[EPT];
    u32 bits = 0;
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
      } else {
#pragma unroll
        for (int j = 0; j < EPT; ++j) sv[j] = k0 + j < n ? __ldg(sym + k0 + j) : (uint16_t)0;
      }
    } else {
#pragma unroll
      for (int j = 0; j < EPT; ++j) sv[j] = k0 + j < n ? __ldg(sym + k0 + j) : (uint16_t)0;
    }
#pragma unroll
    for (int j = 0; j < EPT; ++j) bits += (k0 + j < n) ? slen[sv[j]] : 0u;
    u32 total;
    const u32 boff = block_excl_scan<u32>(bits, scratch, &total);
    const u32 words = (total + 31) >> 5;
    if (threadIdx.x == 0) {
      u64 mine[1] = {words}, excl[1];
      lookback<1>(lb, t, mine, excl, &st->status);
      s_base = excl[0];
      if (t == nchunks - 1) st->nwords = excl[0] + words;
      const u64 o = Lo.off_chunks + 8 * t;
      if (o + 8 <= cap) *reinterpret_cast<u64*>(out + o) = excl[0];
    }
    for (u32 i = threadIdx.x; i < words + 1; i += blockDim.x) wbuf[i] = 0;
    __syncthreads();
    u32 p = boff;
#pragma unroll
    for (int j = 0; j < EPT; ++j) {
      if (k0 + j < n) {
        const u32 l = slen[sv[j]], c = scode[sv[j]];
        const u32 wi = p >> 5, bo = p & 31;  // code occupies bits bo..bo+l-1 from the MSB
        if (bo + l <= 32) {
          atomicOr(&wbuf[wi], c << (32 - bo - l));
        } else {
          const u32 spill = bo + l - 32;
          atomicOr(&wbuf[wi], c >> spill);
          atomicOr(&wbuf[wi + 1], c << (32 - spill));
        }
        p += l;
      }
    }
    __syncthreads();
    const u64 base = s_base;
    for (u32 i = threadIdx.x; i < words; i += blockDim.x) {
      const u64 o = Lo.off_payload + 4 * (base + i);
      if (o + 4 <= cap) *reinterpret_cast<u32*>(out + o) = wbuf[i];
    }
    __syncthreads();
  }
}

// --------------------------------------------------------------- finalize
__device__ __forceinline__ void put_bytes(uint8_t* h, u32 off, const void* src, u32 bytes) {
  const uint8_t* s = (const uint8_t*)src;
  for (u32 i = 0; i < bytes; ++i) h[off + i] = s[i];
}

__global__ void __launch_bounds__(kThreads) k_finalize(Desc d, State* st, const u64* n_dev,
                                                       const u64* nb_dev,
                                                       const roix_eb_info* info,
                                                       const u64* __restrict__ rk,
                                                       const u32* __restrict__ rv, u64 rec_cap,
                                                       const uint16_t* counts_src,
                                                       const uint16_t* bounds_src, uint8_t* out,
                                                       u64 cap, u64* size_dev) {
  const u64 n = *n_dev, nb = *nb_dev, nout = st->nout, nwords = st->nwords;
  const u64 nchunks = (n + d.C - 1) / d.C;
  const Layout Lo = make_layout(d.S, d.rows, nb, nout, nchunks, nwords);
  const u64 gtid = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  const u64 gstride = (u64)gridDim.x * blockDim.x;
  if (gtid == 0) {
    uint8_t h[kHeaderBytes];
    for (u32 i = 0; i < kHeaderBytes; ++i) h[i] = 0;
    const roix_eb_info e = *info;
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
    *size_dev = Lo.total;
    st->total = Lo.total;
    if (Lo.total > cap || st->cap_flag) set_status(&st->status, ROIX_ECAPACITY);
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
__global__ void k_init(State* st, u64* zero, u64 words) {
  const u64 gtid = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (gtid == 0) {
    u32* s = reinterpret_cast<u32*>(st);
    for (u32 i = 1; i < sizeof(State) / 4; ++i) s[i] = 0;
    st->vmin_key = 0xffffffffu;
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

void launch_init(const Launch& L, State* st, void* zero, size_t zero_bytes) {
  const u64 words = zero ? zero_bytes / 8 : 0;
  u64 blocks = (words + kThreads - 1) / kThreads;
  if (blocks < 1) blocks = 1;
  if (blocks > (u64)L.sms * 4) blocks = (u64)L.sms * 4;
  k_init<<<(unsigned)blocks, kThreads, 0, L.stream>>>(st, (u64*)zero, words);
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

void launch_symbols(const Launch& L, const Desc& d, const void* P, const int32_t* q,
                    const u32* obits, u64 n_cap, const u64* n_dev, const roix_eb_info* info_in,
                    State* st, uint16_t* sym, u64* rk, u32* rv, u64 rec_cap,
                    unsigned long long* hist, LookBack<1> lb) {
  const u64 tiles_cap = (n_cap + kQuantTile - 1) / kQuantTile;
  if (tiles_cap == 0) return;
  const bool from_q = q != nullptr;
  const int compute_eb = info_in == nullptr;
  auto run = [&](auto kernel, auto src) {
    u64 grid = (u64)grid_for((const void*)kernel, kThreads, 0, L.sms);
    if (grid > tiles_cap) grid = tiles_cap;
    kernel<<<(unsigned)grid, kThreads, 0, L.stream>>>(d, src, n_cap, n_dev, st, sym, rk, rv,
                                                       rec_cap, hist, lb, compute_eb);
  };
  if (d.dtype == ROIX_F32) {
    if (from_q) {
      Src<float, true> s{(const float*)P, q, obits, {}, d.dark};
      run(k_symbols<float, true>, s);
    } else {
      Src<float, false> s{(const float*)P, nullptr, nullptr, {}, d.dark};
      run(k_symbols<float, false>, s);
    }
  } else {
    if (from_q) {
      Src<unsigned short, true> s{(const unsigned short*)P, q, obits, {}, d.dark};
      run(k_symbols<unsigned short, true>, s);
    } else {
      Src<unsigned short, false> s{(const unsigned short*)P, nullptr, nullptr, {}, d.dark};
      run(k_symbols<unsigned short, false>, s);
    }
  }
}

void launch_codebook(const Launch& L, const Desc& d, const unsigned long long* hist,
                     uint8_t* lens_ws, u32* codes_ws, uint8_t* out, u64 cap, State* st) {
  const size_t smem = codebook_smem(d.S);
  cudaFuncSetAttribute((const void*)k_codebook, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)smem);
  k_codebook<<<1, kCbThreads, smem, L.stream>>>(d, hist, lens_ws, codes_ws, out, cap, st);
}

void launch_pack(const Launch& L, const Desc& d, const uint16_t* sym, const u64* n_dev,
                 const u64* nb_dev, const uint8_t* lens_ws, const u32* codes_ws, State* st,
                 uint8_t* out, u64 cap, LookBack<1> lb, u64 chunks_cap) {
  if (chunks_cap == 0) return;
  const size_t smem = ((size_t)d.C * kLMax / 32 + 2) * 4;
  auto run = [&](auto kernel) {
    cudaFuncSetAttribute((const void*)kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    u64 grid = (u64)grid_for((const void*)kernel, kThreads, smem, L.sms);
    if (grid > chunks_cap) grid = chunks_cap;
    kernel<<<(unsigned)grid, kThreads, smem, L.stream>>>(d, sym, n_dev, nb_dev, lens_ws,
                                                         codes_ws, st, out, cap, lb);
  };
  switch (d.C / kThreads) {
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

void launch_finalize(const Launch& L, const Desc& d, State* st, const u64* n_dev,
                     const u64* nb_dev, const roix_eb_info* info, const u64* rk, const u32* rv,
                     u64 rec_cap, const uint16_t* counts_src, const uint16_t* bounds_src,
                     uint8_t* out, u64 cap, u64* size_dev) {
  const unsigned blocks = (unsigned)L.sms * 2;
  k_finalize<<<blocks, kThreads, 0, L.stream>>>(d, st, n_dev, nb_dev, info, rk, rv, rec_cap,
                                                counts_src, bounds_src, out, cap, size_dev);
}

}  // namespace roix
