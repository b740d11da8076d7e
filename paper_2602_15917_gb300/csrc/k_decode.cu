// Decoder (Sec. 4.3, decompression): header check, row geometry scan, chunked
// canonical Huffman decode, segmented prefix sum of the deltas (records reset
// it), dequantisation, and the row-by-row scatter with the background fill.
// Every read of the container is checked against its size; an inconsistency
// sets ROIX_ECORRUPT and later kernels do nothing.
#include "roix_internal.cuh"

namespace roix {

namespace {

constexpr int kThreads = 256;
constexpr u32 kLutBits = 12;

// plan word indices
enum {
  P_OK = 0, P_N, P_NOUT, P_NB, P_NCH, P_NW, P_OFF_LENS, P_OFF_COUNTS, P_OFF_BOUNDS, P_OFF_OUTK,
  P_OFF_OUTV, P_OFF_CHUNKS, P_OFF_PAYLOAD, P_R, P_C, P_S, P_TWO_EB, P_EB_INT, P_DARK, P_FILL,
  P_ZEROS, P_VOX, P_ORDER
};

// Naturally aligned read: header fields sit at multiples of their size and
// every section starts on a 16-byte boundary of a 16-byte aligned container.
template <typename T>
__device__ __forceinline__ T rd(const uint8_t* p, u64 off) {
  return *reinterpret_cast<const T*>(p + off);
}

__device__ __forceinline__ void prefetch_l1(const void* p) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

__device__ __forceinline__ void corrupt(u32* status, u64* plan) {
  set_status(status, ROIX_ECORRUPT);
  plan[P_OK] = 0;
}

// ---------------------------------------------------------------- header
__global__ void k_dec_header(Desc d, const uint8_t* in, u64 size, u32* status, u64* plan,
                             u64 max_chunks) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = 0; i < kPlanWords; ++i) plan[i] = 0;
  if (size < kHeaderBytes || in[0] != 'R' || in[1] != 'O' || in[2] != 'I' || in[3] != 'X') {
    corrupt(status, plan);
    return;
  }
  const uint16_t ver = rd<uint16_t>(in, 4);
  const u32 nx = rd<u32>(in, 8), ny = rd<u32>(in, 12), nz = rd<u32>(in, 16);
  const u32 R = rd<u32>(in, 80), C = rd<u32>(in, 84), lmax = rd<u32>(in, 88);
  const u32 order = rd<u32>(in, 92);  // Lorenzo order (0 reads as 1)
  const u64 n = rd<u64>(in, 96), nout = rd<u64>(in, 104), nb = rd<u64>(in, 112);
  const u64 nch = rd<u64>(in, 120), nw = rd<u64>(in, 128);
  const double dark = rd<double>(in, 32), fill = rd<double>(in, 40);
  bool ok = ver == kVersion && in[6] == (uint8_t)d.dtype && nx == d.nx && ny == d.ny &&
            nz == d.nz && lmax == kLMax && R >= 2 && R <= kMaxRadius && C >= 256 &&
            C <= 16384 && (C & (C - 1)) == 0 && n <= d.N && nout <= n &&
            nb <= d.rows * (d.nx + 1) && nch == (n + C - 1) / C && nch <= max_chunks &&
            order <= 2;
  if (ok && d.dtype == ROIX_U16)
    ok = fill >= 0.0 && fill <= 65535.0 && fill == floor(fill) && dark >= 0.0 &&
         dark <= 65535.0 && dark == floor(dark);
  if (ok && nw > (size >> 2)) ok = false;
  Layout Lo;
  if (ok) {
    Lo = make_layout(2ull * R, d.rows, nb, nout, nch, nw);
    ok = rd<u64>(in, 152) == Lo.off_lens && rd<u64>(in, 160) == Lo.off_counts &&
         rd<u64>(in, 168) == Lo.off_bounds && rd<u64>(in, 176) == Lo.off_outk &&
         rd<u64>(in, 184) == Lo.off_outv && rd<u64>(in, 192) == Lo.off_chunks &&
         rd<u64>(in, 200) == Lo.off_payload && rd<u64>(in, 208) == Lo.total &&
         Lo.total <= size;
  }
  if (!ok) {
    corrupt(status, plan);
    return;
  }
  plan[P_N] = n;
  plan[P_NOUT] = nout;
  plan[P_NB] = nb;
  plan[P_NCH] = nch;
  plan[P_NW] = nw;
  plan[P_OFF_LENS] = Lo.off_lens;
  plan[P_OFF_COUNTS] = Lo.off_counts;
  plan[P_OFF_BOUNDS] = Lo.off_bounds;
  plan[P_OFF_OUTK] = Lo.off_outk;
  plan[P_OFF_OUTV] = Lo.off_outv;
  plan[P_OFF_CHUNKS] = Lo.off_chunks;
  plan[P_OFF_PAYLOAD] = Lo.off_payload;
  plan[P_R] = R;
  plan[P_C] = C;
  plan[P_S] = 2ull * R;
  plan[P_TWO_EB] = rd<u32>(in, 64);
  plan[P_EB_INT] = (u64)(int64_t)rd<int32_t>(in, 76);
  plan[P_DARK] = (u64)(int64_t)dark;
  plan[P_FILL] = __double_as_longlong(fill);
  plan[P_ORDER] = order == 2 ? 2 : 1;
  plan[P_OK] = 1;
}

// ------------------------------------------------------------ decode table
// Canonical decoding data from the code lengths: per length the first code,
// the count and the index of its first symbol in (length, symbol) order, and
// a 2^12-entry lookup table for codes of up to 12 bits (entry = symbol << 8 |
// length, 0 = longer code). Lengths whose Kraft sum exceeds 1 are corrupt.
struct DecTable {
  u32 first[kLMax + 2], count[kLMax + 2], index0[kLMax + 2];
  u32 limit[kLMax + 2];  // end of the length-l codes, left-justified to kLMax bits
  uint16_t by_code[kMaxSym];
  u32 lut[1u << kLutBits];
};

__global__ void __launch_bounds__(1024) k_dec_table(const uint8_t* in, u32* status, u64* plan,
                                                    DecTable* tab) {
  __shared__ u32 cnt[kLMax + 2], first[kLMax + 2], idx0[kLMax + 2];
  __shared__ uint8_t len[kMaxSym];
  if (!plan[P_OK]) return;
  const u32 S = (u32)plan[P_S];
  const u64 off = plan[P_OFF_LENS];
  if (threadIdx.x < kLMax + 2) cnt[threadIdx.x] = 0;
  __syncthreads();
  for (u32 s = threadIdx.x; s < S; s += blockDim.x) {
    const uint8_t l = in[off + s];
    len[s] = l;
    if (l > kLMax) corrupt(status, plan);
    else if (l) atomicAdd(&cnt[l], 1u);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // Kraft sum in units of 2^-24
    u64 kraft = 0;
    for (u32 l = 1; l <= kLMax; ++l) kraft += (u64)cnt[l] << (kLMax - l);
    if (kraft > (1ull << kLMax)) corrupt(status, plan);
    u32 c = 0, ix = 0;
    for (u32 l = 1; l <= kLMax; ++l) {
      c = (c + (l >= 2 ? cnt[l - 1] : 0u)) << 1;
      first[l] = c;
      idx0[l] = ix;
      ix += cnt[l];
    }
    for (u32 l = 0; l <= kLMax; ++l) {
      tab->first[l] = first[l];
      tab->count[l] = cnt[l];
      tab->index0[l] = idx0[l];
      // canonical codes: every length-l code, left-justified, lies below every
      // longer one, so these ends do not decrease with l
      tab->limit[l] = l ? (first[l] + cnt[l]) << (kLMax - l) : 0u;
    }
  }
  __syncthreads();
  if (!plan[P_OK]) return;
  // symbol order within a length = increasing symbol: rank by counting
  for (u32 s = threadIdx.x; s < S; s += blockDim.x) {
    const u32 l = len[s];
    if (!l) continue;
    u32 r = 0;
    for (u32 s2 = 0; s2 < s; ++s2) r += (len[s2] == l);
    tab->by_code[idx0[l] + r] = (uint16_t)s;
    if (l <= kLutBits) {
      const u32 code = first[l] + r;
      const u32 lo = code << (kLutBits - l), span = 1u << (kLutBits - l);
      for (u32 i = 0; i < span; ++i) tab->lut[lo + i] = (s << 8) | l;
    }
  }
}

// ----------------------------------------------------------- row geometry
// Per tile of rows: boundary offsets (scan of the counts), then, once the
// tile's boundary base is known, the retained voxels per row (sum of run
// lengths) and their scan. Bounds are checked: even counts, increasing
// positions within [0, nx].
constexpr u32 kRowTile = (u32)kDecRowTile;

__global__ void __launch_bounds__(kThreads) k_dec_rows(Desc d, const uint8_t* in, u32* status,
                                                       u64* plan, u64* row_boff, u64* row_voff,
                                                       LookBack<1> lbb, LookBack<1> lbv,
                                                       u32* ctr, u64 ntiles) {
  __shared__ u32 scratch[40];
  __shared__ u64 s_tile, s_bb, s_vb;
  __shared__ u32 s_bad;
  if (!plan[P_OK]) return;
  const u64 off_counts = plan[P_OFF_COUNTS], off_bounds = plan[P_OFF_BOUNDS];
  const u64 nb = plan[P_NB];
  constexpr u32 RPT = kRowTile / kThreads;
  while (true) {
    if (threadIdx.x == 0) {
      s_tile = atomicAdd(ctr, 1u);
      s_bad = 0;
    }
    __syncthreads();
    const u64 t = s_tile;
    if (t >= ntiles) break;
    const u64 r0 = t * kRowTile + (u64)threadIdx.x * RPT;
    u32 c[RPT];
    u32 csum = 0;
    for (u32 j = 0; j < RPT; ++j) {
      const u64 r = r0 + j;
      c[j] = r < d.rows ? rd<uint16_t>(in, off_counts + 2 * r) : 0u;
      if (c[j] & 1u) s_bad |= 1;
      csum += c[j];
    }
    u32 ctot;
    const u32 cex = block_excl_scan<u32>(csum, scratch, &ctot);
    if (threadIdx.x == 0) {
      u64 mine[1] = {ctot}, ex[1];
      if (lookback<1>(lbb, t, mine, ex, status, d.spin_limit, d.hold_scans != 0)) s_bad |= 2;
      s_bb = ex[0];
      if (t == ntiles - 1 && ex[0] + ctot != nb) s_bad |= 1;
    }
    __syncthreads();
    u64 b = s_bb + cex;
    u64 vox[RPT];
    u64 vsum = 0;
    for (u32 j = 0; j < RPT; ++j) {
      const u64 r = r0 + j;
      vox[j] = 0;
      if (r < d.rows) {
        row_boff[r] = b;
        u32 prevx = 0;
        for (u32 i = 0; i < c[j]; i += 2) {
          if (b + i + 1 >= nb) {
            s_bad |= 1;
            break;
          }
          const u32 xs = rd<uint16_t>(in, off_bounds + 2 * (b + i));
          const u32 xe = rd<uint16_t>(in, off_bounds + 2 * (b + i + 1));
          if (xs < prevx || xe <= xs || xe > d.nx || (i > 0 && xs == prevx)) {
            s_bad |= 1;
            break;
          }
          vox[j] += xe - xs;
          prevx = xe;
        }
        b += c[j];
      }
      vsum += vox[j];
    }
    u64 vtot;
    __shared__ u64 scratch64[40];
    const u64 vex = block_excl_scan<u64>(vsum, scratch64, &vtot);
    if (threadIdx.x == 0) {
      u64 mine[1] = {vtot}, ex[1];
      if (lookback<1>(lbv, t, mine, ex, status, d.spin_limit, d.hold_scans != 0)) s_bad |= 2;
      s_vb = ex[0];
      if (t == ntiles - 1 && ex[0] + vtot != plan[P_N]) s_bad |= 1;
    }
    __syncthreads();
    u64 v = s_vb + vex;
    for (u32 j = 0; j < RPT; ++j) {
      const u64 r = r0 + j;
      if (r < d.rows) row_voff[r] = v;
      v += vox[j];
    }
    if (s_bad && threadIdx.x == 0) {
      // a wait that gave up (status ROIX_ETIMEOUT) or an inconsistent container:
      // the later kernels do nothing
      if (s_bad & 2) plan[P_OK] = 0;
      else corrupt(status, plan);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- records
// First record at or after position k (lower bound of the keys).
__device__ __forceinline__ u64 first_record(const uint8_t* in, const u64* plan, u64 k) {
  const u64 nout = plan[P_NOUT], ok_ = plan[P_OFF_OUTK];
  u64 lo = 0, hi = nout;
  while (lo < hi) {
    const u64 mid = (lo + hi) >> 1;
    if ((rd<u64>(in, ok_ + 8 * mid) & ~(1ull << 63)) < k) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// The records of one chunk in order: the first one at or after the chunk's
// first symbol 0 is found once by binary search, each later symbol 0 of the
// chunk takes the next record (records are sorted by position).
struct RecordCursor {
  const uint8_t* in;
  const u64* plan;
  u64 idx = ~0ull;
  __device__ bool next(u64 k, u64& key, u32& val) {
    if (idx == ~0ull) idx = first_record(in, plan, k);
    if (idx >= plan[P_NOUT]) return false;
    key = rd<u64>(in, plan[P_OFF_OUTK] + 8 * idx);
    if ((key & ~(1ull << 63)) != k) return false;
    val = rd<u32>(in, plan[P_OFF_OUTV] + 4 * idx);
    ++idx;
    return true;
  }
};

// ------------------------------------------------------- codeword reading
// A reader of a chunk's bit stream from any bit position: an MSB-first 64-bit
// buffer refilled from the payload words [wp, w1) through L1.
struct BitReader {
  const u32* words;
  u64 wp, w1, buf;
  int have;
  __device__ __forceinline__ void refill() {
    while (have <= 32 && wp < w1) {
      buf |= (u64)__ldg(words + wp++) << (32 - have);
      have += 32;
    }
  }
  // positioned at bit `bit` of the stream that starts at word w0
  __device__ __forceinline__ void init(const u32* w, u64 w0, u64 word1, u64 bit) {
    words = w;
    w1 = word1;
    wp = w0 + (bit >> 5);
    buf = 0;
    have = 0;
    refill();
    const int skip = (int)(bit & 31);
    if (have >= skip) {
      buf <<= skip;
      have -= skip;
    } else {
      have = 0;
    }
  }
};

// Canonical decoding tables in shared memory.
struct DecShared {
  const u32* lut;
  const u32* first;
  const u32* index0;
  const u32* limit;
  const uint16_t* by_code;
};

// One codeword at the reader's position: its symbol and length, or false when
// the bits are no code of the table or too few remain. Codes of up to
// kLutBits bits come from the lookup table; for a longer one its length is
// the first l whose left-justified end exceeds the next kLMax bits (binary
// search over the lengths).
__device__ __forceinline__ bool dec_code(BitReader& br, const DecShared& t, u32& s, u32& l) {
  br.refill();
  const u32 e = t.lut[(u32)(br.buf >> (64 - kLutBits))];
  if (e && (int)(e & 0xffu) <= br.have) {
    l = e & 0xffu;
    s = e >> 8;
  } else {
    const u32 v = (u32)(br.buf >> (64 - kLMax));
    u32 lo = 1, hi = kLMax;
    while (lo < hi) {
      const u32 mid = (lo + hi) >> 1;
      if (v < t.limit[mid]) hi = mid;
      else lo = mid + 1;
    }
    if (v >= t.limit[lo] || (int)lo > br.have) return false;
    l = lo;
    s = t.by_code[t.index0[l] + (v >> (kLMax - l)) - t.first[l]];
  }
  br.buf <<= l;
  br.have -= (int)l;
  return true;
}

// ----------------------------------------------------- symbols, order 1
// A warp per chunk, with no change to the stream: lane l decodes the codewords
// that start in the l-th of 32 equal slices of the chunk's bits, from a start
// that is a guess except for lane 0 (the slice's first bit). A Huffman code
// resynchronises: a decode begun inside a codeword soon meets the true
// boundaries. In rounds, each lane restarts from the position where the
// previous lane's decode left its slice, until no start changes; lane 0 starts
// at a true boundary, so then every start is one (by induction) and the
// lanes' codeword counts are exact. A warp scan of the counts places each
// lane's symbols; a last pass writes them (the first L of the chunk), takes the
// records of its symbols 0 in order (from the chunk's first record plus the
// zeros before it) and forms the lane's part of the chunk aggregate, and the
// parts are combined in lane order.
__global__ void __launch_bounds__(kThreads) k_dec_symbols_w(const uint8_t* in, u32* status,
                                                            u64* plan, const DecTable* tab,
                                                            uint16_t* sym, u64* agg) {
  __shared__ u32 lut[1u << kLutBits];
  __shared__ u32 first[kLMax + 2], count[kLMax + 2], index0[kLMax + 2], limit[kLMax + 2];
  __shared__ uint16_t by_code[kMaxSym];
  if (!plan[P_OK] || plan[P_ORDER] != 1) return;
  const u64 n = plan[P_N], nch = plan[P_NCH], nw = plan[P_NW];
  const u32 C = (u32)plan[P_C], R = (u32)plan[P_R], S = (u32)plan[P_S];
  const u64 off_ch = plan[P_OFF_CHUNKS], off_pl = plan[P_OFF_PAYLOAD];
  const u64 nout = plan[P_NOUT], ok_ = plan[P_OFF_OUTK], ov = plan[P_OFF_OUTV];
  for (u32 i = threadIdx.x; i < (1u << kLutBits); i += blockDim.x) lut[i] = tab->lut[i];
  for (u32 i = threadIdx.x; i < S; i += blockDim.x) by_code[i] = tab->by_code[i];
  if (threadIdx.x < kLMax + 2) {
    first[threadIdx.x] = tab->first[threadIdx.x];
    count[threadIdx.x] = tab->count[threadIdx.x];
    index0[threadIdx.x] = tab->index0[threadIdx.x];
    limit[threadIdx.x] = tab->limit[threadIdx.x];
  }
  __syncthreads();
  const DecShared t{lut, first, index0, limit, by_code};
  const int lane = threadIdx.x & 31;
  const u64 nwarps = ((u64)gridDim.x * blockDim.x) >> 5;
  const u32* words = reinterpret_cast<const u32*>(in + off_pl);
  u64 zeros = 0;
  for (u64 j = ((u64)blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < nch; j += nwarps) {
    const u64 w0 = rd<u64>(in, off_ch + 8 * j);
    const u64 w1 = j + 1 < nch ? rd<u64>(in, off_ch + 8 * (j + 1)) : nw;
    if (w0 > w1 || w1 > nw) {
      if (lane == 0) corrupt(status, plan);
      break;
    }
    const u64 k0 = j * C;
    const u32 L = (u32)umin((u64)C, n - k0);
    const u64 bmax = 32 * (w1 - w0);
    const u64 g = (bmax + 31) / 32;
    const u64 seg_lo = umin((u64)lane * g, bmax), seg_hi = umin(seg_lo + g, bmax);
    // codewords starting in [st, seg_hi): their number, their symbols 0, the end
    auto scan = [&](u64 st, u32& cnt, u32& zc, u64& end) {
      cnt = 0;
      zc = 0;
      u64 pos = st;
      if (pos < seg_hi) {
        BitReader br;
        br.init(words, w0, w1, pos);
        while (pos < seg_hi) {
          u32 sv, l;
          if (!dec_code(br, t, sv, l)) {  // a guessed start inside no codeword: slide a bit
            ++pos;
            br.init(words, w0, w1, pos);
            continue;
          }
          ++cnt;
          zc += sv == 0 ? 1u : 0u;
          pos += l;
        }
      }
      end = pos;
    };
    u64 start = lane == 0 ? 0 : seg_lo;
    u32 cnt, zc;
    u64 end;
    scan(start, cnt, zc, end);
    for (int round = 0; round < 32; ++round) {
      u64 ns = __shfl_up_sync(0xffffffffu, end, 1);
      if (lane == 0) ns = 0;
      const bool changed = ns != start;
      if (!__ballot_sync(0xffffffffu, changed)) break;
      if (changed) {
        start = ns;
        scan(start, cnt, zc, end);
      }
    }
    const u32 ci = warp_incl_scan(cnt), zi = warp_incl_scan(zc);
    const u32 base = ci - cnt, zbase = zi - zc;
    const u32 total = __shfl_sync(0xffffffffu, ci, 31);
    const bool any_zero = __ballot_sync(0xffffffffu, zc != 0u) != 0u;
    u64 rec0 = 0;
    if (any_zero) {  // the chunk's first record (lane 0 searches, the warp shares it)
      if (lane == 0) rec0 = first_record(in, plan, k0);
      rec0 = __shfl_sync(0xffffffffu, rec0, 0);
    }
    bool bad = total < L;
    bool reset = false;
    long long acc = 0;
    if (!bad && base < L) {
      const u32 todo = min(cnt, L - base);
      BitReader br;
      br.init(words, w0, w1, start);
      u64 ridx = rec0 + zbase;
      for (u32 i = 0; i < todo; ++i) {
        u32 sv, l;
        if (!dec_code(br, t, sv, l)) {
          bad = true;
          break;
        }
        const u64 k = k0 + base + i;
        sym[k] = (uint16_t)sv;
        if (sv) {
          acc += (long long)sv - (long long)R;
        } else {
          ++zeros;
          const u64 key = ridx < nout ? rd<u64>(in, ok_ + 8 * ridx) : ~0ull;
          if ((key & ~(1ull << 63)) != k) {
            bad = true;
            break;
          }
          const u32 val = rd<u32>(in, ov + 4 * ridx);
          ++ridx;
          reset = true;
          acc = (key >> 63) ? 0 : (long long)(int32_t)val;
        }
      }
    }
    if (__ballot_sync(0xffffffffu, bad)) {
      if (lane == 0) corrupt(status, plan);
      break;
    }
    // the lanes' parts in order: (r1, v1) then (r2, v2) -> (r1 | r2, r2 ? v2 : v1 + v2)
    u32 r = reset ? 1u : 0u;
    u64 v = (u64)acc;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const u32 r2 = __shfl_down_sync(0xffffffffu, r, d);
      const u64 v2 = __shfl_down_sync(0xffffffffu, v, d);
      if (lane + d < 32) {
        v = r2 ? v2 : v + v2;
        r |= r2;
      }
    }
    if (lane == 0) {
      agg[2 * j] = r;
      agg[2 * j + 1] = v;
    }
  }
  zeros = warp_sum(zeros);
  if (lane == 0 && zeros) atomicAdd((unsigned long long*)&plan[P_ZEROS], zeros);
}

// ------------------------------------------------------ symbols, order 2
// One thread per chunk: canonical decode through the lookup table (codes of up
// to 12 bits) or the per-length first-code search, the payload read one line
// ahead into L1. The chunk's aggregate for the segmented sum: (whether it
// holds a record, the code sum since the last record or since the chunk
// start); a record's own value comes from the chunk's record cursor.
__global__ void __launch_bounds__(kThreads) k_dec_symbols(const uint8_t* in, u32* status,
                                                          u64* plan, const DecTable* tab,
                                                          uint16_t* sym, u64* agg) {
  __shared__ u32 lut[1u << kLutBits];
  __shared__ u32 first[kLMax + 2], count[kLMax + 2], index0[kLMax + 2], limit[kLMax + 2];
  __shared__ uint16_t by_code[kMaxSym];
  if (!plan[P_OK] || plan[P_ORDER] == 1) return;  // order 1: k_dec_symbols_w
  const u64 n = plan[P_N], nch = plan[P_NCH], nw = plan[P_NW];
  const u32 C = (u32)plan[P_C], R = (u32)plan[P_R], S = (u32)plan[P_S];
  const u64 off_ch = plan[P_OFF_CHUNKS], off_pl = plan[P_OFF_PAYLOAD];
  for (u32 i = threadIdx.x; i < (1u << kLutBits); i += blockDim.x) lut[i] = tab->lut[i];
  for (u32 i = threadIdx.x; i < S; i += blockDim.x) by_code[i] = tab->by_code[i];
  if (threadIdx.x < kLMax + 2) {
    first[threadIdx.x] = tab->first[threadIdx.x];
    count[threadIdx.x] = tab->count[threadIdx.x];
    index0[threadIdx.x] = tab->index0[threadIdx.x];
    limit[threadIdx.x] = tab->limit[threadIdx.x];
  }
  __syncthreads();
  u64 zeros = 0;
  for (u64 j = (u64)blockIdx.x * blockDim.x + threadIdx.x; j < nch;
       j += (u64)gridDim.x * blockDim.x) {
    const u64 w0 = rd<u64>(in, off_ch + 8 * j);
    const u64 w1 = j + 1 < nch ? rd<u64>(in, off_ch + 8 * (j + 1)) : nw;
    if (w0 > w1 || w1 > nw) {
      corrupt(status, plan);
      break;
    }
    const u32* words = reinterpret_cast<const u32*>(in + off_pl);
    u64 wp = w0;           // next word to load
    u64 buf = 0;           // bit buffer, MSB first
    int have = 0;          // valid bits in buf
    const u64 k0 = j * C, k1 = min(n, k0 + C);
    bool reset = false, bad = false;
    long long acc = 0;
    // order 2: the chunk's affine map of the state (c[k-1], c[k-2]), composed
    // element by element in wrapping 64-bit arithmetic (exact modulo 2^64, and
    // every true code fits in 32 bits)
    const bool two = plan[P_ORDER] == 2;
    u64 m11 = 1, m12 = 0, m21 = 0, m22 = 1, o1 = 0, o2 = 0;
    RecordCursor rc{in, plan};
    // the payload is read one 128-byte line ahead into L1, so that the bit
    // buffer's refills do not wait on L2 or HBM
    for (u64 p = w0; p < umin(w1, w0 + 64); p += 32) prefetch_l1(words + p);
    for (u64 k = k0; k < k1; ++k) {
      while (have <= 32 && wp < w1) {
        if ((wp & 31) == 0 && wp + 64 < w1) prefetch_l1(words + wp + 64);
        buf |= (u64)words[wp++] << (32 - have);
        have += 32;
      }
      u32 s = 0, l = 0;
      const u32 e = lut[(u32)(buf >> (64 - kLutBits))];
      if (e && (int)(e & 0xffu) <= have) {
        l = e & 0xffu;
        s = e >> 8;
      } else {
        // a longer code: its length is the first l whose left-justified end
        // exceeds the next kLMax bits (binary search over the lengths)
        const u32 v = (u32)(buf >> (64 - kLMax));
        u32 lo = 1, hi = kLMax;
        while (lo < hi) {
          const u32 mid = (lo + hi) >> 1;
          if (v < limit[mid]) hi = mid;
          else lo = mid + 1;
        }
        if (v >= limit[lo] || (int)lo > have) {  // no code of the table, or past the stream
          bad = true;
          break;
        }
        l = lo;
        s = by_code[index0[l] + (v >> (kLMax - l)) - first[l]];
      }
      buf <<= l;
      have -= (int)l;
      sym[k] = (uint16_t)s;
      u64 key = 0;
      u32 val = 0;
      if (!s) {  // the next record of the chunk
        ++zeros;
        if (!rc.next(k, key, val)) {
          bad = true;
          break;
        }
      }
      if (two) {
        // element map: c' = a c1 + b c2 + v, (c1, c2) -> (c', c1); non-record:
        // (a, b, v) = (2, -1, s - R); record: (0, 0, payload)
        u64 ea = 2, eb = ~0ull, ev = (u64)((long long)s - (long long)R);
        if (!s) {
          ea = 0;
          eb = 0;
          ev = (key >> 63) ? 0ull : (u64)(long long)(int32_t)val;
        }
        const u64 n11 = ea * m11 + eb * m21, n12 = ea * m12 + eb * m22, no1 = ea * o1 + eb * o2 + ev;
        m21 = m11;
        m22 = m12;
        o2 = o1;
        m11 = n11;
        m12 = n12;
        o1 = no1;
      }
      if (s) {
        acc += (long long)s - (long long)R;
      } else {
        reset = true;
        acc = (key >> 63) ? 0 : (long long)(int32_t)val;
      }
    }
    if (bad) {
      corrupt(status, plan);
      break;
    }
    if (two) {
      u64* g = agg + 6 * j;
      g[0] = m11;
      g[1] = m12;
      g[2] = m21;
      g[3] = m22;
      g[4] = o1;
      g[5] = o2;
    } else {
      agg[2 * j] = reset ? 1ull : 0ull;
      agg[2 * j + 1] = (u64)acc;
    }
  }
  zeros = warp_sum(zeros);
  if ((threadIdx.x & 31) == 0 && zeros) atomicAdd((unsigned long long*)&plan[P_ZEROS], zeros);
}

// Segmented exclusive scan of the chunk aggregates (one block, in order).
__global__ void __launch_bounds__(1024) k_dec_carry(u32* status, u64* plan, const u64* agg,
                                                    u64* carry) {
  __shared__ u64 sv[1024];
  __shared__ u32 sr[1024];
  __shared__ u64 s_carry;
  if (!plan[P_OK] || plan[P_ORDER] != 1) return;
  const u64 nch = plan[P_NCH];
  if (threadIdx.x == 0) {
    s_carry = 0;
    if (plan[P_ZEROS] != plan[P_NOUT]) corrupt(status, plan);
  }
  __syncthreads();
  for (u64 c0 = 0; c0 < nch; c0 += 1024) {
    const u64 j = c0 + threadIdx.x;
    u32 r = j < nch ? (u32)agg[2 * j] : 0u;
    u64 v = j < nch ? agg[2 * j + 1] : 0ull;
    sr[threadIdx.x] = r;
    sv[threadIdx.x] = v;
    __syncthreads();
    // Hillis-Steele inclusive segmented scan: (r1,v1) then (r2,v2) ->
    // (r1|r2, r2 ? v2 : v1 + v2)
    for (u32 dd = 1; dd < 1024; dd <<= 1) {
      u32 pr = 0;
      u64 pv = 0;
      const bool has = threadIdx.x >= dd;
      if (has) {
        pr = sr[threadIdx.x - dd];
        pv = sv[threadIdx.x - dd];
      }
      __syncthreads();
      if (has) {
        if (!r) v += pv;
        r |= pr;
        sr[threadIdx.x] = r;
        sv[threadIdx.x] = v;
      }
      __syncthreads();
    }
    // exclusive value for chunk j, with the carry from earlier blocks
    u64 ex_v;
    u32 ex_r;
    if (threadIdx.x == 0) {
      ex_r = 0;
      ex_v = 0;
    } else {
      ex_r = sr[threadIdx.x - 1];
      ex_v = sv[threadIdx.x - 1];
    }
    const u64 cin = s_carry;
    if (j < nch) carry[j] = ex_r ? ex_v : cin + ex_v;
    __syncthreads();
    if (threadIdx.x == 1023) s_carry = sr[1023] ? sv[1023] : cin + sv[1023];
    __syncthreads();
  }
}

// ------------------------------------------------------------------ values
// One block per chunk: per-element code increments (or record resets),
// block-wide segmented scan seeded with the chunk's carry, dequantisation.
template <typename TV>
__global__ void __launch_bounds__(kThreads) k_dec_values(const uint8_t* in, u32* status,
                                                         u64* plan, const uint16_t* sym,
                                                         const u64* agg, const u64* carry,
                                                         TV* vals) {
  __shared__ u64 sv[kThreads];
  __shared__ u32 sr[kThreads];
  __shared__ u64 s_run, s_rec;
  __shared__ u32 s_wz[kThreads / 32];
  if (!plan[P_OK] || plan[P_ORDER] != 1) return;
  const u64 n = plan[P_N], nch = plan[P_NCH];
  const u32 C = (u32)plan[P_C], R = (u32)plan[P_R];
  const float two_eb = __uint_as_float((u32)plan[P_TWO_EB]);
  const long long eb_int = (long long)plan[P_EB_INT], dark = (long long)plan[P_DARK];
  const u64 ok_ = plan[P_OFF_OUTK], ov = plan[P_OFF_OUTV], nout = plan[P_NOUT];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (u64 j = blockIdx.x; j < nch; j += gridDim.x) {
    const u64 k0 = j * C, k1 = min(n, k0 + C);
    if (threadIdx.x == 0) {
      s_run = carry[j];
      // the chunk's first record, found once (the chunk holds one if it reset)
      s_rec = agg[2 * j] ? first_record(in, plan, k0) : 0ull;
    }
    __syncthreads();
    for (u64 b0 = k0; b0 < k1; b0 += kThreads) {
      const u64 k = b0 + threadIdx.x;
      u32 r = 0;
      u64 v = 0;
      u32 rawbits = 0;
      bool raw = false;
      const u32 s = k < k1 ? sym[k] : 1u;
      // a symbol 0 takes the record after the zeros before it in the chunk
      const u32 bz = __ballot_sync(0xffffffffu, s == 0u);
      if (lane == 0) s_wz[warp] = (u32)__popc(bz);
      __syncthreads();
      u64 zb = 0, zt = 0;
      for (int q = 0; q < kThreads / 32; ++q) {
        if (q < warp) zb += s_wz[q];
        zt += s_wz[q];
      }
      if (s) {
        v = (u64)((long long)s - (long long)R);
      } else {
        const u64 idx = s_rec + zb + (u64)__popc(bz & ((1u << lane) - 1u));
        const u64 key = idx < nout ? rd<u64>(in, ok_ + 8 * idx) : ~0ull;
        if ((key & ~(1ull << 63)) != k) {
          corrupt(status, plan);
        } else {
          const u32 val = rd<u32>(in, ov + 4 * idx);
          r = 1;
          raw = (key >> 63) != 0;
          rawbits = val;
          v = raw ? 0ull : (u64)(long long)(int32_t)val;
        }
      }
      sr[threadIdx.x] = r;
      sv[threadIdx.x] = v;
      __syncthreads();
      if (threadIdx.x == 0) s_rec += zt;  // read by every thread before the barrier above
      for (u32 dd = 1; dd < kThreads; dd <<= 1) {
        u32 pr = 0;
        u64 pv = 0;
        const bool has = threadIdx.x >= dd;
        if (has) {
          pr = sr[threadIdx.x - dd];
          pv = sv[threadIdx.x - dd];
        }
        __syncthreads();
        if (has) {
          if (!r) v += pv;
          r |= pr;
          sr[threadIdx.x] = r;
          sv[threadIdx.x] = v;
        }
        __syncthreads();
      }
      const u64 run = s_run;
      const long long c = (long long)(r ? v : run + v);
      if (k < k1) {
        if constexpr (sizeof(TV) == 4) {
          vals[k] = raw ? __uint_as_float(rawbits)
                        : __fmul_rn(__int2float_rn((int)c), two_eb);
        } else {
          long long x = (eb_int == 0 ? c : 2 * eb_int * c) + dark;
          x = x < 0 ? 0 : (x > 65535 ? 65535 : x);
          vals[k] = (TV)x;
        }
      }
      __syncthreads();
      if (threadIdx.x == kThreads - 1) s_run = (u64)c;
      __syncthreads();
    }
  }
}

// ------------------------------------------------- two-layer Lorenzo
// Composition of the chunks' affine maps in order (one block, Hillis-Steele
// per 1024 chunks, carried across): chunk j starts from the state that the
// maps of chunks 0..j-1 give the zero state, i.e. the offset of their
// composition.
struct Map2 {
  u64 m11, m12, m21, m22, o1, o2;
};
__device__ __forceinline__ Map2 after(const Map2& g, const Map2& f) {  // g after f
  Map2 r;
  r.m11 = g.m11 * f.m11 + g.m12 * f.m21;
  r.m12 = g.m11 * f.m12 + g.m12 * f.m22;
  r.m21 = g.m21 * f.m11 + g.m22 * f.m21;
  r.m22 = g.m21 * f.m12 + g.m22 * f.m22;
  r.o1 = g.m11 * f.o1 + g.m12 * f.o2 + g.o1;
  r.o2 = g.m21 * f.o1 + g.m22 * f.o2 + g.o2;
  return r;
}

__global__ void __launch_bounds__(1024) k_dec_carry2(u32* status, u64* plan, const u64* agg,
                                                     u64* carry) {
  __shared__ Map2 sm[1024];
  __shared__ Map2 s_run;
  if (!plan[P_OK] || plan[P_ORDER] != 2) return;
  const u64 nch = plan[P_NCH];
  if (threadIdx.x == 0) {
    s_run = Map2{1, 0, 0, 1, 0, 0};
    if (plan[P_ZEROS] != plan[P_NOUT]) corrupt(status, plan);
  }
  __syncthreads();
  for (u64 c0 = 0; c0 < nch; c0 += 1024) {
    const u64 j = c0 + threadIdx.x;
    Map2 f{1, 0, 0, 1, 0, 0};
    if (j < nch) {
      const u64* g = agg + 6 * j;
      f = Map2{g[0], g[1], g[2], g[3], g[4], g[5]};
    }
    sm[threadIdx.x] = f;
    __syncthreads();
    for (u32 dd = 1; dd < 1024; dd <<= 1) {  // inclusive: map of chunks c0..j
      Map2 p{1, 0, 0, 1, 0, 0};
      const bool has = threadIdx.x >= dd;
      if (has) p = sm[threadIdx.x - dd];
      __syncthreads();
      if (has) {
        f = after(f, p);
        sm[threadIdx.x] = f;
      }
      __syncthreads();
    }
    const Map2 run = s_run;
    const Map2 ex = threadIdx.x ? after(sm[threadIdx.x - 1], run) : run;
    if (j < nch) {
      carry[2 * j] = ex.o1;
      carry[2 * j + 1] = ex.o2;
    }
    __syncthreads();
    if (threadIdx.x == 1023) s_run = after(sm[1023], run);
    __syncthreads();
  }
}

// One thread per chunk: codes from the chunk's starting state, c = 2 c1 - c2 +
// d (records set c), dequantised.
template <typename TV>
__global__ void __launch_bounds__(kThreads) k_dec_values2(const uint8_t* in, u32* status,
                                                          u64* plan, const uint16_t* sym,
                                                          const u64* carry, TV* vals) {
  if (!plan[P_OK] || plan[P_ORDER] != 2) return;
  const u64 n = plan[P_N], nch = plan[P_NCH];
  const u32 C = (u32)plan[P_C], R = (u32)plan[P_R];
  const float two_eb = __uint_as_float((u32)plan[P_TWO_EB]);
  const long long eb_int = (long long)plan[P_EB_INT], dark = (long long)plan[P_DARK];
  for (u64 j = (u64)blockIdx.x * blockDim.x + threadIdx.x; j < nch;
       j += (u64)gridDim.x * blockDim.x) {
    u64 c1 = carry[2 * j], c2 = carry[2 * j + 1];
    const u64 k0 = j * C, k1 = min(n, k0 + C);
    RecordCursor rc{in, plan};
    for (u64 k = k0; k < k1; ++k) {
      const u32 s = sym[k];
      u64 c;
      bool raw = false;
      u32 rawbits = 0;
      if (s) {
        c = 2 * c1 - c2 + (u64)((long long)s - (long long)R);
      } else {
        u64 key;
        u32 val;
        if (!rc.next(k, key, val)) {
          corrupt(status, plan);
          return;
        }
        raw = (key >> 63) != 0;
        rawbits = val;
        c = raw ? 0ull : (u64)(long long)(int32_t)val;
      }
      const long long cv = (long long)c;
      if constexpr (sizeof(TV) == 4) {
        vals[k] = raw ? __uint_as_float(rawbits) : __fmul_rn(__int2float_rn((int)cv), two_eb);
      } else {
        long long x = (eb_int == 0 ? cv : 2 * eb_int * cv) + dark;
        x = x < 0 ? 0 : (x > 65535 ? 65535 : x);
        vals[k] = (TV)x;
      }
      c2 = c1;
      c1 = c;
    }
  }
}

// ----------------------------------------------------------------- scatter
// One warp per row: gaps get the fill value, runs their values in order.
template <typename TV>
__global__ void __launch_bounds__(kThreads) k_dec_scatter(Desc d, const uint8_t* in,
                                                          const u64* plan, const u64* row_boff,
                                                          const u64* row_voff, const TV* vals,
                                                          TV* out) {
  if (!plan[P_OK]) return;
  const int lane = threadIdx.x & 31;
  const u64 off_counts = plan[P_OFF_COUNTS], off_bounds = plan[P_OFF_BOUNDS];
  TV fill;
  if constexpr (sizeof(TV) == 4) fill = __double2float_rn(__longlong_as_double(plan[P_FILL]));
  else fill = (TV)(u32)__longlong_as_double(plan[P_FILL]);
  for (u64 r = ((u64)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < d.rows;
       r += ((u64)gridDim.x * blockDim.x) >> 5) {
    const u32 cnt = rd<uint16_t>(in, off_counts + 2 * r);
    const u64 b = row_boff[r];
    u64 v = row_voff[r];
    TV* row = out + r * d.nx;
    u32 x = 0;
    for (u32 i = 0; i <= cnt; i += 2) {
      const u32 xs = i < cnt ? rd<uint16_t>(in, off_bounds + 2 * (b + i)) : (u32)d.nx;
      const u32 xe = i < cnt ? rd<uint16_t>(in, off_bounds + 2 * (b + i + 1)) : (u32)d.nx;
      for (u32 xx = x + lane; xx < xs; xx += 32) row[xx] = fill;
      for (u32 xx = xs + lane; xx < xe; xx += 32) row[xx] = vals[v + (xx - xs)];
      v += xe - xs;
      x = xe;
    }
  }
}

}  // namespace

void launch_decode(const Launch& L, const Desc& d, const uint8_t* in, u64 size, void* out,
                   const DecodeWs& ws, u64 max_chunks) {
  // ws.plan[...] and the look-back flags are zeroed by the host
  k_dec_header<<<1, 32, 0, L.stream>>>(d, in, size, ws.status, ws.plan, max_chunks);
  DecTable* tab = reinterpret_cast<DecTable*>(ws.table);
  k_dec_table<<<1, 1024, 0, L.stream>>>(in, ws.status, ws.plan, tab);
  const u64 row_tiles = (d.rows + kRowTile - 1) / kRowTile;
  if (row_tiles) {
    unsigned g = (unsigned)umin(row_tiles, (u64)L.sms * 4);
    k_dec_rows<<<g, kThreads, 0, L.stream>>>(d, in, ws.status, ws.plan, ws.row_boff, ws.row_voff,
                                             ws.lb_rows_b, ws.lb_rows_v, ws.row_ctr, row_tiles);
  }
  if (max_chunks) {
    unsigned g = (unsigned)umin((max_chunks + kThreads - 1) / kThreads, (u64)L.sms * 4);
    k_dec_symbols<<<g, kThreads, 0, L.stream>>>(in, ws.status, ws.plan, tab, ws.sym, ws.agg);
    {  // order 1: a warp per chunk
      const u64 wpb = kThreads / 32;
      const unsigned gw = (unsigned)umin((max_chunks + wpb - 1) / wpb, (u64)L.sms * 8);
      k_dec_symbols_w<<<gw, kThreads, 0, L.stream>>>(in, ws.status, ws.plan, tab, ws.sym,
                                                      ws.agg);
    }
    k_dec_carry<<<1, 1024, 0, L.stream>>>(ws.status, ws.plan, ws.agg, ws.carry);
    k_dec_carry2<<<1, 1024, 0, L.stream>>>(ws.status, ws.plan, ws.agg, ws.carry);
    unsigned gv = (unsigned)umin(max_chunks, (u64)L.sms * 8);
    unsigned g2 = (unsigned)umin((max_chunks + kThreads - 1) / kThreads, (u64)L.sms * 8);
    if (d.dtype == ROIX_F32) {
      k_dec_values<float><<<gv, kThreads, 0, L.stream>>>(in, ws.status, ws.plan, ws.sym, ws.agg,
                                                          ws.carry, (float*)ws.vals);
      k_dec_values2<float><<<g2, kThreads, 0, L.stream>>>(in, ws.status, ws.plan, ws.sym,
                                                           ws.carry, (float*)ws.vals);
    } else {
      k_dec_values<unsigned short><<<gv, kThreads, 0, L.stream>>>(
          in, ws.status, ws.plan, ws.sym, ws.agg, ws.carry, (unsigned short*)ws.vals);
      k_dec_values2<unsigned short><<<g2, kThreads, 0, L.stream>>>(
          in, ws.status, ws.plan, ws.sym, ws.carry, (unsigned short*)ws.vals);
    }
  }
  if (d.rows) {
    unsigned g = (unsigned)umin((d.rows + 7) / 8, (u64)L.sms * 8);
    if (d.dtype == ROIX_F32)
      k_dec_scatter<float><<<g, kThreads, 0, L.stream>>>(d, in, ws.plan, ws.row_boff,
                                                         ws.row_voff, (const float*)ws.vals,
                                                         (float*)out);
    else
      k_dec_scatter<unsigned short><<<g, kThreads, 0, L.stream>>>(
          d, in, ws.plan, ws.row_boff, ws.row_voff, (const unsigned short*)ws.vals,
          (unsigned short*)out);
  }
}

size_t dec_table_bytes() { return sizeof(DecTable); }

}  // namespace roix
