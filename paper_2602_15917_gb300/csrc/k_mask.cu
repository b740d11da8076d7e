// Region-of-interest kernels: binarisation (Sec. 4.1.1, 4.1.3-4.1.4), the
// cube dilation of the retained set, and the extraction of row geometry and
// pixel section (Sec. 4.2.2) by a single-pass decoupled look-back compaction.
//
// Mask layout: rows = ny*nz rows of W = ceil(nx/32) uint32 words; voxel x of a
// row is bit x%32 of word x/32; bits at x >= nx are 0.
#include "roix_internal.cuh"

namespace roix {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ bool pass_f32(float x, const Desc& d) {
  if (d.thr_never) return false;
  return d.cmp == 0 ? (x > d.thr_f) : (x < d.thr_f);
}
__device__ __forceinline__ bool pass_u16(unsigned raw, const Desc& d) {
  if (d.thr_never) return false;
  int v = (int)raw - d.dark;
  return d.cmp == 0 ? (v > d.thr_i) : (v < d.thr_i);
}

__device__ __forceinline__ u32 last_mask(const Desc& d, u64 w) {
  u32 rem = (u32)(d.nx & 31);
  return (w == d.W - 1 && rem) ? ((1u << rem) - 1u) : 0xffffffffu;
}

// ----------------------------------------------------------- binarisation
// One warp turns a row segment of up to 1024 voxels into 32 mask words: each
// lane reads one voxel per step (one coalesced 128-byte line per warp for
// float32), and a ballot forms the word. Eight independent loads are issued
// before the ballots so that every warp keeps several lines in flight.
template <typename TV>
__global__ void __launch_bounds__(kThreads) k_threshold(Desc d, const TV* __restrict__ in,
                                                        u32* __restrict__ T) {
  const int lane = threadIdx.x & 31;
  const u64 warp = ((u64)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const u64 nwarps = ((u64)gridDim.x * blockDim.x) >> 5;
  const u64 spr = (d.nx + 1023) >> 10;  // segments per row
  const u64 nseg = d.rows * spr;
  for (u64 s = warp; s < nseg; s += nwarps) {
    const u64 r = s / spr, sg = s - r * spr;
    const u64 x0 = sg << 10;
    const u32 nw = (u32)umin(32, (d.nx - x0 + 31) >> 5);
    const TV* row = in + r * d.nx;
    u32 mine = 0;
    for (u32 i = 0; i < nw; i += 8) {
      TV v[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const u64 x = x0 + (u64)(i + j) * 32 + lane;
        v[j] = (i + j < nw && x < d.nx) ? __ldg(row + x) : TV(0);
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const u64 x = x0 + (u64)(i + j) * 32 + lane;
        bool p;
        if constexpr (sizeof(TV) == 4) p = pass_f32(v[j], d);
        else p = pass_u16(v[j], d);
        p = p && (i + j < nw) && (x < d.nx);
        const u32 b = __ballot_sync(0xffffffffu, p);
        if (lane == (int)(i + j)) mine = b;
      }
    }
    if ((u32)lane < nw) T[r * d.W + (x0 >> 5) + lane] = mine;
  }
}

// Dilated word: OR over the 3x3 neighbour rows (clipped) of the word shifted
// by -1, 0, +1 in x, carries taken from the neighbouring words.
__device__ __forceinline__ u32 dilate_word_global(const u32* __restrict__ T, const Desc& d,
                                                  u64 r, u64 w) {
  const u64 y = r % d.ny, z = r / d.ny;
  u32 acc = 0;
  for (int dz = -1; dz <= 1; ++dz) {
    if ((dz < 0 && z == 0) || (dz > 0 && z + 1 >= d.nz)) continue;
    for (int dy = -1; dy <= 1; ++dy) {
      if ((dy < 0 && y == 0) || (dy > 0 && y + 1 >= d.ny)) continue;
      const u32* row = T + (r + (int64_t)dz * (int64_t)d.ny + dy) * d.W;
      const u32 c = __ldg(row + w);
      const u32 lo = w > 0 ? __ldg(row + w - 1) : 0u;
      const u32 hi = w + 1 < d.W ? __ldg(row + w + 1) : 0u;
      acc |= c | (c << 1) | (lo >> 31) | (c >> 1) | (hi << 31);
    }
  }
  return acc & last_mask(d, w);
}

__global__ void __launch_bounds__(kThreads) k_dilate(Desc d, const u32* __restrict__ T,
                                                     u32* __restrict__ D, u64* popcount) {
  const u64 total = d.rows * d.W;
  u64 cnt = 0;
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (u64)gridDim.x * blockDim.x) {
    const u64 r = i / d.W, w = i - r * d.W;
    const u32 v = d.dilate ? dilate_word_global(T, d, r, w) : (T[i] & last_mask(d, w));
    D[i] = v;
    cnt += __popc(v);
  }
  cnt = warp_sum(cnt);
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd((unsigned long long*)popcount, cnt);
}

// ------------------------------------------------------------ compaction
// Persistent blocks take tiles of `rpt` consecutive rows in increasing order.
// Per tile: stage the mask rows it needs (three bands of rpt+2 rows for the
// dilation) in shared memory, form the retained words D and the transition
// words E (boundaries), count both per warp, obtain the tile's output offsets
// from the decoupled look-back, then write the pixel values, the boundaries
// and the per-row boundary counts. Lanes map to the 32 bits of a word, so
// both the value loads and the compacted stores are coalesced.
struct FrontSmem {
  u32 wn[kThreads / 32], wb[kThreads / 32];  // per-warp totals, then offsets
  u64 base_n, base_nb, tile;
  u32 scratch[40];
};

__device__ __forceinline__ u32 e_word(const u32* Dw, u64 i, u64 w) {
  const u32 dv = Dw[i];
  const u32 prev = w > 0 ? Dw[i - 1] : 0u;
  return dv ^ ((dv << 1) | (prev >> 31));
}

template <typename TV>
__global__ void __launch_bounds__(kThreads) k_front(Desc d, const TV* __restrict__ in,
                                                    const u32* __restrict__ T, int dilate,
                                                    TV* __restrict__ P,
                                                    uint16_t* __restrict__ counts, u64 counts_cap,
                                                    uint16_t* __restrict__ bounds, u64 bounds_cap,
                                                    State* st, u64* sizes_out, LookBack<2> lb,
                                                    u32 rpt, u64 ntiles) {
  extern __shared__ u32 smem_dyn[];
  __shared__ FrontSmem sh;
  const u32 W = (u32)d.W;
  u32* Dw = smem_dyn;                    // [rpt * W]
  u32* band = smem_dyn + (u64)rpt * W;   // [3][rpt + 2][W] when dilating
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool end_extra = (d.nx & 31) == 0;  // boundary at x = nx lives past the last word
  u32 kmin = 0xffffffffu, kmax = 0u;

  while (true) {
    if (threadIdx.x == 0) sh.tile = atomicAdd(&st->ctr_front, 1u);
    __syncthreads();
    const u64 t = sh.tile;
    if (t >= ntiles) break;
    const u64 r0 = t * rpt;
    const u32 nrows = (u32)umin(rpt, d.rows - r0);
    const u32 nw = nrows * W;

    // ---- D words
    if (dilate) {
      const u32 bw = (rpt + 2) * W;
      for (u32 i = threadIdx.x; i < 3 * bw; i += blockDim.x) {
        const u32 b = i / bw, j = i - b * bw;
        const int64_t rr = (int64_t)r0 + ((int64_t)b - 1) * (int64_t)d.ny - 1 + j / W;
        band[i] = (rr >= 0 && rr < (int64_t)d.rows) ? __ldg(T + (u64)rr * W + (j % W)) : 0u;
      }
      __syncthreads();
      for (u32 i = threadIdx.x; i < nw; i += blockDim.x) {
        const u32 lr = i / W, w = i - lr * W;
        const u64 r = r0 + lr;
        const u64 y = r % d.ny, z = r / d.ny;
        u32 acc = 0;
#pragma unroll
        for (int dz = -1; dz <= 1; ++dz) {
          if ((dz < 0 && z == 0) || (dz > 0 && z + 1 >= d.nz)) continue;
#pragma unroll
          for (int dy = -1; dy <= 1; ++dy) {
            if ((dy < 0 && y == 0) || (dy > 0 && y + 1 >= d.ny)) continue;
            const u32* row = band + (dz + 1) * (rpt + 2) * W + (lr + 1 + dy) * W;
            const u32 c = row[w];
            const u32 lo = w > 0 ? row[w - 1] : 0u;
            const u32 hi = w + 1 < W ? row[w + 1] : 0u;
            acc |= c | (c << 1) | (lo >> 31) | (c >> 1) | (hi << 31);
          }
        }
        Dw[i] = acc & last_mask(d, w);
      }
    } else {
      for (u32 i = threadIdx.x; i < nw; i += blockDim.x) {
        const u32 w = i % W;
        Dw[i] = __ldg(T + r0 * W + i) & last_mask(d, w);
      }
    }
    __syncthreads();

    // ---- per-warp totals of retained voxels and boundaries
    const u32 per_warp = (nw + (kThreads / 32) - 1) / (kThreads / 32);
    const u32 wbeg = min(nw, warp * per_warp), wend = min(nw, wbeg + per_warp);
    {
      u32 cn = 0, cb = 0;
      for (u32 i = wbeg + lane; i < wend; i += 32) {
        const u32 w = i % W;
        cn += __popc(Dw[i]);
        cb += __popc(e_word(Dw, i, w));
        if (end_extra && w == W - 1) cb += Dw[i] >> 31;
      }
      cn = warp_sum(cn);
      cb = warp_sum(cb);
      if (lane == 0) {
        sh.wn[warp] = cn;
        sh.wb[warp] = cb;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      u64 tn = 0, tb = 0;
      for (int k = 0; k < kThreads / 32; ++k) {
        const u32 a = sh.wn[k], b = sh.wb[k];
        sh.wn[k] = (u32)tn;
        sh.wb[k] = (u32)tb;
        tn += a;
        tb += b;
      }
      u64 mine[2] = {tn, tb}, excl[2];
      lookback<2>(lb, t, mine, excl, &st->status);
      sh.base_n = excl[0];
      sh.base_nb = excl[1];
      if (t == ntiles - 1) {
        sizes_out[0] = excl[0] + tn;
        sizes_out[1] = excl[1] + tb;
      }
    }
    __syncthreads();

    // ---- writes: values and boundaries, word by word, lane = bit
    {
      u64 on = sh.base_n + sh.wn[warp];
      u64 ob = sh.base_nb + sh.wb[warp];
      const u32 below = (1u << lane) - 1u;
      for (u32 c0 = wbeg; c0 < wend; c0 += 32) {
        const u32 i_l = c0 + lane;
        const bool valid = i_l < wend;
        const u32 w_l = i_l % W;
        const u32 dv_l = valid ? Dw[i_l] : 0u;
        const u32 ev_l = valid ? e_word(Dw, i_l, w_l) : 0u;
        const u32 ex_l = (valid && end_extra && w_l == W - 1) ? (dv_l >> 31) : 0u;
        const u32 pn = __popc(dv_l), pb = __popc(ev_l) + ex_l;
        const u32 sn = warp_incl_scan(pn) - pn, sb = warp_incl_scan(pb) - pb;
        const u32 cnt = min(32u, wend - c0);
        for (u32 k0 = 0; k0 < cnt; k0 += 4) {
          TV v[4];
          bool has[4];
          u64 pos[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const u32 k = k0 + j;
            const u32 dv = __shfl_sync(0xffffffffu, dv_l, k & 31);
            const u32 so = __shfl_sync(0xffffffffu, sn, k & 31);
            const u32 i = c0 + k;
            has[j] = k < cnt && ((dv >> lane) & 1u);
            const u32 lr = i / W, w = i - lr * W;
            pos[j] = on + so + __popc(dv & below);
            v[j] = has[j] ? __ldg(in + (r0 + lr) * d.nx + (u64)w * 32 + lane) : TV(0);
          }
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            if (has[j]) {
              P[pos[j]] = v[j];
              if constexpr (sizeof(TV) == 4) {
                if (isfinite(v[j])) {
                  const u32 kk = f32_key(__fadd_rn(v[j], 0.0f));
                  kmin = min(kmin, kk);
                  kmax = max(kmax, kk);
                }
              } else {
                kmin = min(kmin, (u32)v[j] + 1u);
                kmax = max(kmax, (u32)v[j] + 1u);
              }
            }
          }
        }
        // boundaries
        for (u32 k = 0; k < cnt; ++k) {
          const u32 ev = __shfl_sync(0xffffffffu, ev_l, k);
          const u32 ex = __shfl_sync(0xffffffffu, ex_l, k);
          const u32 so = __shfl_sync(0xffffffffu, sb, k);
          if (!(ev | ex)) continue;
          const u32 i = c0 + k;
          const u32 w = i % W;
          if ((ev >> lane) & 1u) {
            const u64 p = ob + so + __popc(ev & below);
            if (p < bounds_cap) bounds[p] = (uint16_t)(w * 32 + lane);
            else atomicExch(&st->cap_flag, 1u);
          }
          if (ex && lane == 0) {
            const u64 p = ob + so + __popc(ev);
            if (p < bounds_cap) bounds[p] = (uint16_t)d.nx;
            else atomicExch(&st->cap_flag, 1u);
          }
        }
        on += __shfl_sync(0xffffffffu, sn + pn, 31);
        ob += __shfl_sync(0xffffffffu, sb + pb, 31);
      }
    }
    // ---- per-row boundary counts
    for (u32 lr = threadIdx.x; lr < nrows; lr += blockDim.x) {
      u32 c = 0;
      for (u32 w = 0; w < W; ++w) {
        const u32 i = lr * W + w;
        c += __popc(e_word(Dw, i, w));
        if (end_extra && w == W - 1) c += Dw[i] >> 31;
      }
      const u64 r = r0 + lr;
      if (r < counts_cap) counts[r] = (uint16_t)c;
    }
    __syncthreads();
  }
  // range of the retained finite values
  for (int o = 16; o > 0; o >>= 1) {
    kmin = min(kmin, __shfl_xor_sync(0xffffffffu, kmin, o));
    kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
  }
  if (lane == 0) {
    if (kmin != 0xffffffffu) atomicMin(&st->vmin_key, kmin);
    if (kmax != 0u) atomicMax(&st->vmax_key, kmax);
  }
}

int occupancy_grid(const void* fn, int threads, size_t smem, int sms) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem);
  if (per_sm < 1) per_sm = 1;
  return per_sm * sms;
}

}  // namespace

void launch_threshold(const Launch& L, const Desc& d, const void* in, u32* T) {
  const u64 segs = d.rows * ((d.nx + 1023) >> 10);
  if (segs == 0) return;
  const u64 warps_per_block = kThreads / 32;
  u64 blocks = (segs + warps_per_block - 1) / warps_per_block;
  const u64 cap = (u64)L.sms * 8;  // 8 blocks of 256 threads per SM in flight
  if (blocks > cap) blocks = cap;
  if (d.dtype == ROIX_F32)
    k_threshold<float><<<(unsigned)blocks, kThreads, 0, L.stream>>>(d, (const float*)in, T);
  else
    k_threshold<unsigned short><<<(unsigned)blocks, kThreads, 0, L.stream>>>(
        d, (const unsigned short*)in, T);
}

void launch_dilate(const Launch& L, const Desc& d, const u32* T, u32* D, u64* popcount) {
  const u64 total = d.rows * d.W;
  if (total == 0) return;
  u64 blocks = (total + kThreads - 1) / kThreads;
  if (blocks > (u64)L.sms * 8) blocks = (u64)L.sms * 8;
  k_dilate<<<(unsigned)blocks, kThreads, 0, L.stream>>>(d, T, D, popcount);
}

void launch_front(const Launch& L, const Desc& d, const void* in, const u32* T, int dilate,
                  void* P, uint16_t* counts, u64 counts_cap, uint16_t* bounds, u64 bounds_cap,
                  State* st, LookBack<2> lb, u32 rows_per_tile, u64 tiles, u64* sizes_out) {
  if (tiles == 0) return;
  const size_t smem = (size_t)rows_per_tile * d.W * 4 +
                      (dilate ? (size_t)3 * (rows_per_tile + 2) * d.W * 4 : 0);
  const void* fn = d.dtype == ROIX_F32 ? (const void*)k_front<float>
                                       : (const void*)k_front<unsigned short>;
  cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  u64 grid = (u64)occupancy_grid(fn, kThreads, smem, L.sms);
  if (grid > tiles) grid = tiles;
  if (d.dtype == ROIX_F32)
    k_front<float><<<(unsigned)grid, kThreads, smem, L.stream>>>(
        d, (const float*)in, T, dilate, (float*)P, counts, counts_cap, bounds, bounds_cap, st,
        sizes_out, lb, rows_per_tile, tiles);
  else
    k_front<unsigned short><<<(unsigned)grid, kThreads, smem, L.stream>>>(
        d, (const unsigned short*)in, T, dilate, (unsigned short*)P, counts, counts_cap, bounds,
        bounds_cap, st, sizes_out, lb, rows_per_tile, tiles);
}

}  // namespace roix
