// The 8-bit preprocessor path: intensity normalisation (Sec. 4.1.2) and the
// greedy absolute-error-bounded quantiser over every row's pixel sequence
// (Sec. 4.2.3).
#include "roix_internal.cuh"

namespace roix {

namespace {

constexpr int kNormThreads = 256;

// background-subtracted value, clamped at 0 (float32: non-finite counts as 0);
// non-negative binary32 patterns order like their unsigned integers
__device__ __forceinline__ u32 nv_f32(float x) {
  return (isfinite(x) && x > 0.0f) ? __float_as_uint(x) : 0u;
}
__device__ __forceinline__ u32 nv_u16(u32 raw, int dark) {
  const int v = (int)raw - dark;
  return v > 0 ? (u32)v : 0u;
}

template <typename TV>
__device__ __forceinline__ u32 nv(TV x, int dark) {
  if constexpr (sizeof(TV) == 4) return nv_f32(x);
  else return nv_u16(x, dark);
}

// the largest of the 8 (uint16) or 4 (float32) values in a 16-byte vector
template <typename TV>
__device__ __forceinline__ u32 nv_max16(uint4 v, int dark) {
  const u32 w[4] = {v.x, v.y, v.z, v.w};
  u32 m = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if constexpr (sizeof(TV) == 4) {
      m = max(m, nv_f32(__uint_as_float(w[k])));
    } else {
      m = max(m, nv_u16(w[k] & 0xffffu, dark));
      m = max(m, nv_u16(w[k] >> 16, dark));
    }
  }
  return m;
}

// Pass 1: I_max. Grid-stride over 16-byte vectors, four in flight per thread,
// one atomicMax per warp.
template <typename TV>
__global__ void __launch_bounds__(kNormThreads)
    k_norm_max(const TV* __restrict__ in, u64 N, int dark, int vec, u32* __restrict__ imax) {
  constexpr int kPer = 16 / sizeof(TV);
  const u64 tid = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  const u64 nth = (u64)gridDim.x * blockDim.x;
  u32 m = 0;
  u64 head = 0;
  if (vec) {
    const uint4* v4 = reinterpret_cast<const uint4*>(in);
    const u64 nv4 = N / kPer;
    u64 i = tid;
    for (; i + 3 * nth < nv4; i += 4 * nth) {
      uint4 a[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) a[k] = __ldg(v4 + i + k * nth);
#pragma unroll
      for (int k = 0; k < 4; ++k) m = max(m, nv_max16<TV>(a[k], dark));
    }
    for (; i < nv4; i += nth) m = max(m, nv_max16<TV>(__ldg(v4 + i), dark));
    head = nv4 * kPer;
  }
  for (u64 i = head + tid; i < N; i += nth) m = max(m, nv<TV>(__ldg(in + i), dark));
  m = __reduce_max_sync(0xffffffffu, m);
  if ((threadIdx.x & 31) == 0 && m) atomicMax(imax, m);
}

// one voxel of pass 2 (see roix_normalize8 for the arithmetic)
struct Scale {
  float fmax;  // float32: I_max
  u32 imax;    // uint16: I_max
  FastDiv fd;  // uint16: division by I_max
  int dark;
  template <typename TV>
  __device__ __forceinline__ u32 at(u32 raw_or_bits) const {
    if constexpr (sizeof(TV) == 4) {
      const u32 b = nv_f32(__uint_as_float(raw_or_bits));
      if (b == 0u || fmax == 0.0f) return 0u;
      const float y = __fmul_rn(__fdiv_rn(__uint_as_float(b), fmax), 255.0f);
      return (u32)fminf(rintf(y), 255.0f);
    } else {
      if (imax == 0u) return 0u;
      const u32 num = 255u * nv_u16(raw_or_bits, dark);
      u32 q = fd.div(num);
      const u32 r2 = 2u * (num - q * imax);
      q += (r2 > imax || (r2 == imax && (q & 1u))) ? 1u : 0u;
      return q;
    }
  }
};

// Pass 2: 16 voxels per thread and step (four float4 or two uint4 loads, one
// uint4 store) when input and output are 16-byte aligned; scalar otherwise.
template <typename TV>
__global__ void __launch_bounds__(kNormThreads)
    k_norm_scale(const TV* __restrict__ in, u64 N, int dark, int vec,
                 const u32* __restrict__ imax_key, u8* __restrict__ out, double* imax_out) {
  Scale sc;
  const u32 key = *imax_key;
  sc.dark = dark;
  sc.fmax = sizeof(TV) == 4 ? __uint_as_float(key) : 0.0f;
  sc.imax = sizeof(TV) == 4 ? 0u : key;
  sc.fd = FastDiv(sizeof(TV) == 4 ? 1u : (key ? key : 1u));
  if (imax_out && blockIdx.x == 0 && threadIdx.x == 0)
    *imax_out = sizeof(TV) == 4 ? (double)__uint_as_float(key) : (double)key;
  const u64 tid = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  const u64 nth = (u64)gridDim.x * blockDim.x;
  u64 head = 0;
  if (vec) {
    constexpr int kVec = 16 / (16 / sizeof(TV));  // 16-byte loads per 16 voxels
    const uint4* v4 = reinterpret_cast<const uint4*>(in);
    uint4* o4 = reinterpret_cast<uint4*>(out);
    const u64 n16 = N / 16;
    for (u64 i = tid; i < n16; i += nth) {
      uint4 a[kVec];
#pragma unroll
      for (int k = 0; k < kVec; ++k) a[k] = __ldg(v4 + i * kVec + k);
      u32 w[4] = {0u, 0u, 0u, 0u};
#pragma unroll
      for (int k = 0; k < kVec; ++k) {
        const u32 x[4] = {a[k].x, a[k].y, a[k].z, a[k].w};
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          if constexpr (sizeof(TV) == 4) {
            const int e = k * 4 + h;  // voxel 0..15
            w[e >> 2] |= sc.at<TV>(x[h]) << (8 * (e & 3));
          } else {
            const int e = k * 8 + h * 2;
            w[e >> 2] |= sc.at<TV>(x[h] & 0xffffu) << (8 * (e & 3));
            w[e >> 2] |= sc.at<TV>(x[h] >> 16) << (8 * ((e + 1) & 3));
          }
        }
      }
      o4[i] = make_uint4(w[0], w[1], w[2], w[3]);
    }
    head = n16 * 16;
  }
  for (u64 i = head + tid; i < N; i += nth) {
    if constexpr (sizeof(TV) == 4) out[i] = (u8)sc.at<TV>(__float_as_uint(__ldg(in + i)));
    else out[i] = (u8)sc.at<TV>((u32)__ldg(in + i));
  }
}

// ------------------------------------------------------------ greedy
constexpr int kGThreads = 256;          // 8 warps; a warp owns 32 rows at a time
constexpr int kGWarps = kGThreads / 32;
constexpr u32 kWin = 64;                // bytes of each row staged per step
constexpr u32 kPitch = 68;              // padded row pitch: 17 words, no bank conflicts

// One pixel of the greedy scan (Sec. 4.2.3 Step 3) for the lane's row: d joins
// the open group while the group's range stays within 2 floor(E_abs) (the
// acceptable sets still share an integer); otherwise the group closes with the
// value floor((u + l) / 2) = (min + max) / 2 and d opens the next one. hrel is
// the open group's first pixel relative to the step's first; a closed group's
// value is stored over that staged byte, or in the row's spare byte 64 when
// the group began in an earlier step.
struct Scan {
  int mn, mx;  // range of the open group
  int hrel;    // its first pixel, relative to the step start
  __device__ __forceinline__ bool step(int d, int j, int e2, u8* trow) {
    const int nmn = min(mn, d), nmx = max(mx, d);
    const bool close = nmx - nmn > e2;
    const int q = (mn + mx) >> 1;
    if (close) trow[hrel < 0 ? 64 : hrel] = (u8)q;
    hrel = close ? j : hrel;
    mn = close ? d : nmn;
    mx = close ? d : nmx;
    return close;
  }
};

// Row lengths of one 32-row tile: the popcounts of its mask rows, eight rows'
// loads in flight (rows of at most 64 words) or one row at a time. Lane i
// returns row i's length.
__device__ __forceinline__ u32 tile_lengths(const GreedyItem& I, u64 r0, int lane) {
  u32 mylen = 0;
  if (I.W <= 32) {
#pragma unroll 1
    for (int i0 = 0; i0 < 32; i0 += 8) {
      u32 c[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const u64 r = r0 + i0 + k;
        c[k] = (r < I.rows && (u64)lane < I.W) ? __popc(__ldg(I.mask + r * I.W + lane)) : 0u;
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const u32 sum = __reduce_add_sync(0xffffffffu, c[k]);
        if (lane == i0 + k) mylen = sum;
      }
    }
  } else if (I.W <= 64) {
#pragma unroll 1
    for (int i0 = 0; i0 < 32; i0 += 8) {
      u32 c[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const u64 r = r0 + i0 + k;
        const u32* mr = I.mask + r * I.W;
        const bool in = r < I.rows;
        const u32 a = in ? __ldg(mr + lane) : 0u;
        const u32 b = in && (u64)lane + 32 < I.W ? __ldg(mr + lane + 32) : 0u;
        c[k] = __popc(a) + __popc(b);
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const u32 sum = __reduce_add_sync(0xffffffffu, c[k]);
        if (lane == i0 + k) mylen = sum;
      }
    }
  } else {
#pragma unroll 1
    for (int i = 0; i < 32; ++i) {
      const u64 r = r0 + i;
      u32 c = 0;
      if (r < I.rows) {
        const u32* mr = I.mask + r * I.W;
#pragma unroll 4
        for (u64 w = lane; w < I.W; w += 32) c += __popc(__ldg(mr + w));
      }
      c = __reduce_add_sync(0xffffffffu, c);
      if (lane == i) mylen = c;
    }
  }
  return mylen;
}

// Pass 1: every 32-row tile of every item: the row lengths and the tile's sum.
__global__ void __launch_bounds__(kGThreads) k_greedy_count(const __grid_constant__ GreedyBatch B) {
  const int lane = threadIdx.x & 31;
  const u64 warp = ((u64)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const u64 nwarps = ((u64)gridDim.x * blockDim.x) >> 5;
  const u64 T = B.tile0[B.n];
  for (u64 g = warp; g < T; g += nwarps) {
    const u32 i = find_item(B.tile0, B.n, g);
    const GreedyItem& I = B.it[i];
    const u64 r0 = (g - B.tile0[i]) * 32;
    const u32 len = tile_lengths(I, r0, lane);
    const u32 incl = warp_incl_scan(len);
    if (r0 + lane < I.rows) {
      B.lens[B.row0[i] + r0 + lane] = len;
      B.rpre[B.row0[i] + r0 + lane] = incl - len;
    }
    if (lane == 31) B.tsum[g] = incl;
  }
}

// Pass 2 (one block of 1024 threads): exclusive prefix of the tile sums over
// the whole batch, 4096 tiles per round, and each item's pixel count.
__global__ void __launch_bounds__(1024) k_greedy_scan(const __grid_constant__ GreedyBatch B) {
  __shared__ u64 scratch[33];
  const u64 T = B.tile0[B.n];
  u64 carry = 0;
  for (u64 c0 = 0; c0 < T; c0 += 4096) {
    const u64 k = c0 + 4u * threadIdx.x;
    u64 v[4];
#pragma unroll
    for (int h = 0; h < 4; ++h) v[h] = k + h < T ? (u64)B.tsum[k + h] : 0ull;
    const u64 mine = v[0] + v[1] + v[2] + v[3];
    u64 total;
    u64 ex = block_excl_scan(mine, scratch, &total) + carry;
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      if (k + h < T) B.toff[k + h] = ex;
      ex += v[h];
    }
    carry += total;
  }
  if (threadIdx.x == 0) B.toff[T] = carry;
  __syncthreads();
  if (threadIdx.x < B.n && B.it[threadIdx.x].n_out) {
    const u32 i = threadIdx.x;
    *B.it[i].n_out = B.toff[B.tile0[i + 1]] - B.toff[B.tile0[i]];
  }
}

// Pass 3: every lane scans whole rows, taking the next non-empty row of the
// batch from a global counter when its row ends, so that the lanes of a warp
// stay busy whatever the row lengths. Per step of 64 pixels of each lane's
// row:
//  1. the warp stages the 32 rows' next 64 bytes in shared memory, two rows
//     per instruction, each lane funnel-shifting 4 bytes out of two aligned
//     words;
//  2. each lane scans its bytes, marking group starts and storing each closed
//     group's value over its first byte, then fills every byte with the value
//     of its group (forward, in place);
//  3. the warp writes the 32 rows' bytes back, two rows per instruction;
//  4. a group carried in from earlier steps that closed in this one is
//     rewritten over [head, step start) by the whole warp (those bytes were
//     written with a placeholder while the group was open).
__global__ void __launch_bounds__(kGThreads) k_greedy(const __grid_constant__ GreedyBatch B) {
  __shared__ __align__(16) u8 tiles[kGWarps][32 * kPitch];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int half = lane >> 4, l16 = lane & 15;
  const u32 lt_mask = (1u << lane) - 1u;
  u8* tb = tiles[wid];
  u8* trow = tb + lane * kPitch;
  const int e2 = (int)B.e2;
  const u64 R = B.row0[B.n];
  // this lane's row: pixel and output pointers at the row start, length, position
  const u8* src = nullptr;
  u8* dst = nullptr;
  u32 len = 0, pos = 0;
  bool has = false, done = false;
  Scan sc{0x7fffffff, -0x7fffffff, 0};
  while (true) {
    // ---- lanes without a row take the next rows of the batch
    u32 need = __ballot_sync(0xffffffffu, !has && !done);
    while (need) {
      u64 base = 0;
      if (lane == 0) base = atomicAdd(B.rowctr, (unsigned long long)__popc(need));
      base = __shfl_sync(0xffffffffu, base, 0);
      if (!has && !done) {
        const u64 r = base + __popc(need & lt_mask);
        if (r >= R) {
          done = true;
        } else {
          const u32 l = B.lens[r];
          if (l) {
            const u32 item = find_item(B.row0, B.n, r);
            const GreedyItem& I = B.it[item];
            const u64 local = r - B.row0[item];
            const u64 tile = B.tile0[item] + (local >> 5);
            const u64 off = B.toff[tile] - B.toff[B.tile0[item]] + B.rpre[r];
            src = I.P + off;
            dst = I.Q + off;
            len = l;
            pos = 0;
            has = true;
            sc = Scan{0x7fffffff, -0x7fffffff, 0};
          }
        }
      }
      need = __ballot_sync(0xffffffffu, !has && !done);
    }
    if (!__any_sync(0xffffffffu, has)) break;
    const bool inplace = src == dst;
    // ---- 1. stage
#pragma unroll 4
    for (int i2 = 0; i2 < 32; i2 += 2) {
      const int i = i2 + half;
      const u64 si = (u64)__shfl_sync(0xffffffffu, (unsigned long long)(uintptr_t)(src + pos), i);
      const u32 ai = __shfl_sync(0xffffffffu, has ? len - pos : 0u, i);
      const int ipl = __shfl_sync(0xffffffffu, (int)inplace, i);
      const u32 j = 4u * l16;
      u32 v = 0;
      if (j < ai) {
        const u64 b = si + j, end = si + ai;
        const u64 al = b & ~3ull;
        const u32 sh = (u32)(b & 3ull) * 8u;
        const u32* p = reinterpret_cast<const u32*>(al);
        const u32 lo = ipl ? __ldcg(p) : __ldg(p);
        u32 hi = 0;
        if (sh && al + 4 < end) hi = ipl ? __ldcg(p + 1) : __ldg(p + 1);
        v = __funnelshift_r(lo, hi, sh);
      }
      *reinterpret_cast<u32*>(tb + i * kPitch + j) = v;
    }
    __syncwarp();
    // ---- 2. scan and fill this lane's bytes
    const u32 cnt = has ? umin(kWin, len - pos) : 0u;
    const int hrel0 = sc.hrel;
    u64 starts = (has && pos == 0) ? 1ull : 0ull;
    const u32* trw = reinterpret_cast<const u32*>(trow);
    const u32 full = cnt & ~3u;
    for (u32 j4 = 0; j4 < full; j4 += 4) {
      const u32 w = trw[j4 >> 2];
      u32 sb = 0;
#pragma unroll
      for (int b = 0; b < 4; ++b)
        sb |= (u32)sc.step((int)((w >> (8 * b)) & 0xffu), (int)j4 + b, e2, trow) << b;
      starts |= (u64)sb << j4;
    }
    if (full < cnt) {
      const u32 w = trw[full >> 2];
      u32 sb = 0;
      for (u32 b = 0; full + b < cnt; ++b)
        sb |= (u32)sc.step((int)((w >> (8 * b)) & 0xffu), (int)(full + b), e2, trow) << b;
      starts |= (u64)sb << full;
    }
    const bool ends = has && pos + cnt == len;
    if (ends) trow[sc.hrel < 0 ? 64 : sc.hrel] = (u8)((sc.mn + sc.mx) >> 1);
    // the group carried into this step closed here: at a later start, or at the row end
    const bool carried = has && hrel0 < 0 && (ends || (starts != 0ull));
    {
      u32 v = carried ? (u32)trow[64] : 0u;  // 0: placeholder while it stays open
      u32* tw = reinterpret_cast<u32*>(trow);
      for (u32 j4 = 0; j4 < cnt; j4 += 4) {
        const u32 w = tw[j4 >> 2];
        const u32 sb = (u32)(starts >> j4) & 0xfu;
        u32 o = 0;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          if ((sb >> b) & 1u) v = (w >> (8 * b)) & 0xffu;
          o |= v << (8 * b);
        }
        tw[j4 >> 2] = o;
      }
    }
    __syncwarp();
    // ---- 3. write back
#pragma unroll 4
    for (int i2 = 0; i2 < 32; i2 += 2) {
      const int i = i2 + half;
      u8* di = reinterpret_cast<u8*>(
          (uintptr_t)__shfl_sync(0xffffffffu, (unsigned long long)(uintptr_t)(dst + pos), i));
      const u32 ci = __shfl_sync(0xffffffffu, cnt, i);
      const u32 j = 4u * l16;
      if (j < ci) {
        const u32 o = *reinterpret_cast<const u32*>(tb + i * kPitch + j);
        u8* d = di + j;
        const u32 nb = umin(4u, ci - j);
        if (nb == 4u && ((uintptr_t)d & 3u) == 0u) {
          *reinterpret_cast<u32*>(d) = o;
        } else {
          for (u32 b = 0; b < nb; ++b) d[b] = (u8)(o >> (8 * b));
        }
      }
    }
    // ---- 4. groups carried in from earlier steps that closed in this one
    u32 pm = __ballot_sync(0xffffffffu, carried);
    const u32 myval = trow[64];
    while (pm) {
      const int i = __ffs(pm) - 1;
      pm &= pm - 1;
      u8* di = reinterpret_cast<u8*>(
          (uintptr_t)__shfl_sync(0xffffffffu, (unsigned long long)(uintptr_t)dst, i));
      const u32 p0 = __shfl_sync(0xffffffffu, pos, i);
      const int h0 = __shfl_sync(0xffffffffu, hrel0, i);
      const u8 pv = (u8)__shfl_sync(0xffffffffu, myval, i);
      for (u32 k = p0 + (u32)h0 + lane; k < p0; k += 32) di[k] = pv;
    }
    __syncwarp();
    // ---- advance
    if (has) {
      if (ends) {
        has = false;
      } else {
        pos += kWin;
        sc.hrel -= (int)kWin;
      }
    }
  }
}

}  // namespace

void launch_normalize8(const Launch& L, int dtype, const void* in, u64 N, int dark, u8* out,
                       u32* imax_key, double* imax_out) {
  const bool vec_in = ((uintptr_t)in & 15) == 0;
  const bool vec_out = ((uintptr_t)out & 15) == 0;
  const u64 per = 16;
  u64 blocks = (N / per + kNormThreads - 1) / kNormThreads;
  const u64 cap = (u64)L.sms * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  if (dtype == ROIX_F32) {
    k_norm_max<float><<<(unsigned)blocks, kNormThreads, 0, L.stream>>>(
        (const float*)in, N, 0, vec_in, imax_key);
    k_norm_scale<float><<<(unsigned)blocks, kNormThreads, 0, L.stream>>>(
        (const float*)in, N, 0, vec_in && vec_out, imax_key, out, imax_out);
  } else {
    k_norm_max<unsigned short><<<(unsigned)blocks, kNormThreads, 0, L.stream>>>(
        (const unsigned short*)in, N, dark, vec_in, imax_key);
    k_norm_scale<unsigned short><<<(unsigned)blocks, kNormThreads, 0, L.stream>>>(
        (const unsigned short*)in, N, dark, vec_in && vec_out, imax_key, out, imax_out);
  }
}

void launch_greedy(const Launch& L, const GreedyBatch& B) {
  const u64 T = B.tile0[B.n];
  if (T == 0) {
    k_greedy_scan<<<1, 1024, 0, L.stream>>>(B);  // pixel counts of 0
    return;
  }
  const u64 wpb = kGThreads / 32;
  u64 blocks = (T + wpb - 1) / wpb;
  u64 cap = (u64)L.sms * 8;
  k_greedy_count<<<(unsigned)(blocks < cap ? blocks : cap), kGThreads, 0, L.stream>>>(B);
  k_greedy_scan<<<1, 1024, 0, L.stream>>>(B);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_greedy, kGThreads, 0);
  cap = (u64)(per_sm > 0 ? per_sm : 1) * L.sms;
  k_greedy<<<(unsigned)(blocks < cap ? blocks : cap), kGThreads, 0, L.stream>>>(B);
}

}  // namespace roix
