// Largest connected component of a bit mask (Sec. 4.2.1: the largest object
// is kept). Union-find over row runs instead of voxels: the runs of every row
// are listed (counts, scan, fill), each run is joined to the overlapping runs
// of the neighbouring rows that come before it in raster order (26- or
// 6-connectivity), roots are the smallest run index of their component (the
// run holding the component's smallest voxel index), component sizes are
// summed per root, and the mask is rewritten with the runs of the component
// that has the most voxels (ties: the smallest root).
#include "roix_internal.cuh"

namespace roix {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ u32 last_word_mask(const Desc& d, u64 w) {
  const u32 rem = (u32)(d.nx & 31);
  return (w == d.W - 1 && rem) ? ((1u << rem) - 1u) : 0xffffffffu;
}

// run starts of word w: set bits whose left neighbour is clear
__device__ __forceinline__ u32 starts_of(u32 v, u32 prev) { return v & ~((v << 1) | (prev >> 31)); }
// run ends (exclusive) of word w, as positions x+1: set bits whose right neighbour is clear
__device__ __forceinline__ u32 lasts_of(u32 v, u32 next) { return v & ~((v >> 1) | (next << 31)); }

// ---- 1. runs per row (warp per row)
// word w of row `row`, complemented when inv (the background), bits >= nx clear
__device__ __forceinline__ u32 word_at(const Desc& d, const u32* row, u64 w, u32 inv) {
  return (__ldg(row + w) ^ inv) & last_word_mask(d, w);
}

__global__ void __launch_bounds__(kThreads) k_run_count(Desc d, const u32* __restrict__ T,
                                                        u32* __restrict__ row_runs,
                                                        u32* __restrict__ out, u32 inv) {
  const int lane = threadIdx.x & 31;
  for (u64 r = ((u64)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < d.rows;
       r += ((u64)gridDim.x * blockDim.x) >> 5) {
    const u32* row = T + r * d.W;
    u32 c = 0;
    for (u64 w = lane; w < d.W; w += 32) out[r * d.W + w] = 0u;  // the kept mask starts empty
    for (u64 w = lane; w < d.W; w += 32) {
      const u32 v = word_at(d, row, w, inv);
      const u32 p = w ? word_at(d, row, w - 1, inv) : 0u;
      c += __popc(starts_of(v, p));
    }
    c = warp_sum(c);
    if (lane == 0) row_runs[r] = c;
  }
}

// ---- 2. exclusive scan of the run counts (tiles of 2048 rows, look-back)
constexpr u32 kScanPer = 8;
__global__ void __launch_bounds__(kThreads) k_run_scan(u64 rows, const u32* __restrict__ cnt,
                                                       u64* __restrict__ off, LookBack<1> lb,
                                                       u32* ctr, u32* status, u64* total,
                                                       u32 limit) {
  __shared__ u64 scratch[40];
  __shared__ u64 s_tile, s_base;
  const u64 ntiles = (rows + kThreads * kScanPer - 1) / (kThreads * kScanPer);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  while (true) {
    if (threadIdx.x == 0) s_tile = atomicAdd(ctr, 1u);
    __syncthreads();
    const u64 t = s_tile;
    if (t >= ntiles) break;
    const u64 r0 = (t * kThreads + threadIdx.x) * kScanPer;
    u64 v[kScanPer], sum = 0;
    for (u32 j = 0; j < kScanPer; ++j) {
      v[j] = r0 + j < rows ? cnt[r0 + j] : 0ull;
      sum += v[j];
    }
    u64 tot;
    const u64 ex = block_excl_scan<u64>(sum, scratch, &tot);
    if (warp == 0) {
      u64 mine[1] = {tot}, excl[1];
      lookback_warp<1>(lb, t, mine, excl, status, limit);
      if (lane == 0) {
        s_base = excl[0];
        if (t == ntiles - 1) *total = excl[0] + tot;
      }
    }
    __syncthreads();
    u64 o = s_base + ex;
    for (u32 j = 0; j < kScanPer; ++j) {
      if (r0 + j < rows) off[r0 + j] = o;
      o += v[j];
    }
    __syncthreads();
  }
}

// ---- 3. run lists: x_start / x_end per run, parent = itself (warp per row)
__global__ void __launch_bounds__(kThreads) k_run_fill(Desc d, const u32* __restrict__ T,
                                                       const u64* __restrict__ off,
                                                       uint16_t* __restrict__ xs,
                                                       uint16_t* __restrict__ xe,
                                                       u32* __restrict__ par,
                                                       unsigned long long* __restrict__ size,
                                                       u32 inv) {
  const int lane = threadIdx.x & 31;
  for (u64 r = ((u64)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < d.rows;
       r += ((u64)gridDim.x * blockDim.x) >> 5) {
    const u32* row = T + r * d.W;
    u64 o = off[r];
    for (u64 w0 = 0; w0 < d.W; w0 += 32) {
      const u64 w = w0 + lane;
      u32 st = 0u, ls = 0u;
      if (w < d.W) {
        const u32 v = word_at(d, row, w, inv);
        const u32 p = w ? word_at(d, row, w - 1, inv) : 0u;
        const u32 nx = w + 1 < d.W ? word_at(d, row, w + 1, inv) : 0u;
        st = starts_of(v, p);
        ls = lasts_of(v, nx);
      }
      // starts and ends pair up in order: the k-th start of the row with the k-th end
      const u32 ns = __popc(st), ne = __popc(ls);
      const u32 is = warp_incl_scan(ns) - ns, ie = warp_incl_scan(ne) - ne;
      u32 k = 0;
      while (st) {
        const u32 b = __ffs(st) - 1;
        st &= st - 1;
        xs[o + is + k] = (uint16_t)(w * 32 + b);
        par[o + is + k] = (u32)(o + is + k);
        size[o + is + k] = 0ull;
        ++k;
      }
      k = 0;
      while (ls) {
        const u32 b = __ffs(ls) - 1;
        ls &= ls - 1;
        xe[o + ie + k] = (uint16_t)(w * 32 + b + 1);
        ++k;
      }
      o += __shfl_sync(0xffffffffu, is + ns, 31);
    }
  }
}

// ---- 4. union of overlapping runs in earlier neighbour rows
__device__ __forceinline__ u32 find_root(u32* par, u32 x) {
  u32 p = __ldcg(par + x);
  while (p != x) {
    const u32 g = __ldcg(par + p);
    if (g != p) par[x] = g;  // path halving (a stale value is still an ancestor)
    x = p;
    p = g;
  }
  return x;
}

__device__ __forceinline__ void unite(u32* par, u32 a, u32 b) {
  while (true) {
    a = find_root(par, a);
    b = find_root(par, b);
    if (a == b) return;
    if (a > b) {
      const u32 t = a;
      a = b;
      b = t;
    }
    // link the larger root under the smaller one
    const u32 old = atomicCAS(par + b, b, a);
    if (old == b) return;
    b = old;
  }
}

__global__ void __launch_bounds__(kThreads) k_run_union(Desc d, const u64* __restrict__ off,
                                                        const u64* total,
                                                        const uint16_t* __restrict__ xs,
                                                        const uint16_t* __restrict__ xe,
                                                        u32* par) {
  const int lane = threadIdx.x & 31;
  const u64 nruns = *total;
  // diagonal neighbours in x for 26- (3D) and 8-connectivity (2D, in-plane);
  // 4 and 8 join rows of the same slice only
  const int ext = (d.conn == 26 || d.conn == 8) ? 1 : 0;
  const bool planar = d.conn == 4 || d.conn == 8;
  for (u64 r = ((u64)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < d.rows;
       r += ((u64)gridDim.x * blockDim.x) >> 5) {
    const u64 b0 = off[r], b1 = r + 1 < d.rows ? off[r + 1] : nruns;
    if (b0 == b1) continue;
    const u64 z = r / d.ny, y = r - z * d.ny;
    // earlier neighbour rows: (y-1, z) and, for z-1, the rows y-1..y+1
    // (26-connectivity) or y only (6-connectivity)
    int64_t nb[4];
    int nn = 0;
    if (y > 0) nb[nn++] = (int64_t)r - 1;
    if (z > 0 && !planar) {
      const int64_t rz = (int64_t)r - (int64_t)d.ny;
      if (d.conn == 26 && y > 0) nb[nn++] = rz - 1;
      nb[nn++] = rz;
      if (d.conn == 26 && y + 1 < d.ny) nb[nn++] = rz + 1;
    }
    for (int q = 0; q < nn; ++q) {
      const u64 nr = (u64)nb[q];
      const u64 c0 = off[nr], c1 = nr + 1 < d.rows ? off[nr + 1] : nruns;
      if (c0 == c1) continue;
      for (u64 i = b0 + lane; i < b1; i += 32) {
        const int s = (int)xs[i] - ext, e = (int)xe[i] + ext;  // [s, e) touches
        // first run of the neighbour row ending after s
        u64 lo = c0, hi = c1;
        while (lo < hi) {
          const u64 mid = (lo + hi) >> 1;
          if ((int)xe[mid] <= s) lo = mid + 1;
          else hi = mid;
        }
        for (u64 j = lo; j < c1 && (int)xs[j] < e; ++j) unite(par, (u32)i, (u32)j);
      }
    }
  }
}

// ---- 5. flatten, sizes per root. The forest no longer changes, so the walk
// to the root only reads; the single write par[i] = root is thread i's own
// (a path-halving store here could overwrite it with a non-root ancestor).
__device__ __forceinline__ u32 find_root_ro(const u32* par, u32 x) {
  u32 p = __ldcg(par + x);
  while (p != x) {
    x = p;
    p = __ldcg(par + x);
  }
  return x;
}

__global__ void __launch_bounds__(kThreads) k_run_sizes(const u64* total, u32* par,
                                                        const uint16_t* __restrict__ xs,
                                                        const uint16_t* __restrict__ xe,
                                                        unsigned long long* size) {
  const u64 n = *total;
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (u64)gridDim.x * blockDim.x) {
    const u32 root = find_root_ro(par, (u32)i);
    par[i] = root;
    atomicAdd(size + root, (unsigned long long)(xe[i] - xs[i]));
  }
}

// ---- 6. the largest component (ties: smallest root)
__global__ void __launch_bounds__(kThreads) k_run_best_size(const u64* total, const u32* par,
                                                            const unsigned long long* size,
                                                            unsigned long long* best) {
  const u64 n = *total;
  unsigned long long m = 0;
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (u64)gridDim.x * blockDim.x)
    if (par[i] == (u32)i && size[i] > m) m = size[i];
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m) atomicMax(best, m);
}

__global__ void __launch_bounds__(kThreads) k_run_best_root(const u64* total, const u32* par,
                                                            const unsigned long long* size,
                                                            const unsigned long long* best,
                                                            u32* best_root) {
  const u64 n = *total;
  const unsigned long long m = *best;
  u32 r = 0xffffffffu;
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (u64)gridDim.x * blockDim.x)
    if (par[i] == (u32)i && size[i] == m && (u32)i < r) r = (u32)i;
  for (int o = 16; o > 0; o >>= 1) r = min(r, __shfl_xor_sync(0xffffffffu, r, o));
  // stored complemented so that a zeroed word means "no component" and
  // atomicMax picks the smallest root
  if ((threadIdx.x & 31) == 0 && r != 0xffffffffu) atomicMax(best_root, 0xffffffffu - r);
}

// ---- 7. rewrite the mask with the kept runs (T' zeroed first)
__global__ void __launch_bounds__(kThreads) k_run_keep(Desc d, const u64* __restrict__ off,
                                                       const u64* total, const u32* par,
                                                       const uint16_t* __restrict__ xs,
                                                       const uint16_t* __restrict__ xe,
                                                       const u32* best_root, u32* out) {
  const u64 n = *total;
  const u32 keep = 0xffffffffu - *best_root;  // ~0 (no run) when nothing was found
  // one thread per run; the row of a run by binary search over the offsets
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (u64)gridDim.x * blockDim.x) {
    if (par[i] != keep) continue;
    u64 lo = 0, hi = d.rows;  // last row with off[row] <= i
    while (hi - lo > 1) {
      const u64 mid = (lo + hi) >> 1;
      if (off[mid] <= i) lo = mid;
      else hi = mid;
    }
    u32* row = out + lo * d.W;
    const u32 s = xs[i], e = xe[i];
    for (u32 w = s >> 5; w <= (e - 1) >> 5; ++w) {
      const u32 a = w == (s >> 5) ? (s & 31) : 0u;
      const u32 b = w == ((e - 1) >> 5) ? ((e - 1) & 31) : 31u;
      const u32 m = (b == 31 ? 0xffffffffu : ((1u << (b + 1)) - 1u)) & ~((1u << a) - 1u);
      atomicOr(row + w, m);
    }
  }
}

// ---- paper mode (planar connectivity, per slice)
// row of run i: the last row whose first run index is <= i
__device__ __forceinline__ u64 row_of_run(const u64* off, u64 rows, u64 i) {
  u64 lo = 0, hi = rows;
  while (hi - lo > 1) {
    const u64 mid = (lo + hi) >> 1;
    if (off[mid] <= i) lo = mid;
    else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ void or_run(u32* row, u32 s, u32 e) {
  for (u32 w = s >> 5; w <= (e - 1) >> 5; ++w) {
    const u32 a = w == (s >> 5) ? (s & 31) : 0u;
    const u32 b = w == ((e - 1) >> 5) ? ((e - 1) & 31) : 31u;
    const u32 m = (b == 31 ? 0xffffffffu : ((1u << (b + 1)) - 1u)) & ~((1u << a) - 1u);
    atomicOr(row + w, m);
  }
}

// components touching the border of their slice (first / last row of the
// slice, first / last column): their roots are flagged (after flattening)
__global__ void __launch_bounds__(kThreads) k_run_border(Desc d, const u64* __restrict__ off,
                                                         const u64* total, const u32* par,
                                                         const uint16_t* __restrict__ xs,
                                                         const uint16_t* __restrict__ xe,
                                                         u32* flag) {
  const u64 n = *total;
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (u64)gridDim.x * blockDim.x) {
    const u64 r = row_of_run(off, d.rows, i);
    const u64 y = r % d.ny;
    if (y == 0 || y + 1 == d.ny || xs[i] == 0 || (u64)xe[i] == d.nx) flag[par[i]] = 1u;
  }
}

// the runs whose root is flagged, OR-ed into `out` (zeroed by the count pass)
__global__ void __launch_bounds__(kThreads) k_run_keep_flagged(Desc d, const u64* __restrict__ off,
                                                               const u64* total, const u32* par,
                                                               const uint16_t* __restrict__ xs,
                                                               const uint16_t* __restrict__ xe,
                                                               const u32* flag, u32* out) {
  const u64 n = *total;
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (u64)gridDim.x * blockDim.x) {
    if (!flag[par[i]]) continue;
    or_run(out + row_of_run(off, d.rows, i) * d.W, xs[i], xe[i]);
  }
}

// largest component of every slice (ties: the smallest root)
__global__ void __launch_bounds__(kThreads) k_run_best_z(Desc d, const u64* __restrict__ off,
                                                         const u64* total, const u32* par,
                                                         const unsigned long long* size,
                                                         unsigned long long* best) {
  const u64 n = *total;
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (u64)gridDim.x * blockDim.x)
    if (par[i] == (u32)i) atomicMax(best + row_of_run(off, d.rows, i) / d.ny, size[i]);
}

__global__ void __launch_bounds__(kThreads) k_run_best_root_z(Desc d, const u64* __restrict__ off,
                                                              const u64* total, const u32* par,
                                                              const unsigned long long* size,
                                                              const unsigned long long* best,
                                                              u32* best_root) {
  const u64 n = *total;
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (u64)gridDim.x * blockDim.x) {
    if (par[i] != (u32)i) continue;
    const u64 z = row_of_run(off, d.rows, i) / d.ny;
    if (size[i] == best[z]) atomicMax(best_root + z, 0xffffffffu - (u32)i);  // smallest root
  }
}

__global__ void __launch_bounds__(kThreads) k_run_keep_z(Desc d, const u64* __restrict__ off,
                                                         const u64* total, const u32* par,
                                                         const uint16_t* __restrict__ xs,
                                                         const uint16_t* __restrict__ xe,
                                                         const u32* best_root, u32* out) {
  const u64 n = *total;
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (u64)gridDim.x * blockDim.x) {
    const u64 r = row_of_run(off, d.rows, i);
    if (par[i] != 0xffffffffu - best_root[r / d.ny]) continue;
    or_run(out + r * d.W, xs[i], xe[i]);
  }
}

}  // namespace

// Paper mode, planar connectivity per slice (d.conn = 4 or 8):
//  keep_border = 1: the components of (T complemented when inv) that touch
//  their slice's border, into `out`; keep_border = 0: the largest component of
//  every slice. w.size doubles as the flag array (after the sizes are used)
//  and w.best / w.best_root hold nz entries (zeroed by the caller).
void launch_ccl_planar(const Launch& L, const Desc& d, const u32* T, u32 inv, int keep_border,
                       u32* out, const CclWs& w) {
  const unsigned gw = (unsigned)umin((d.rows + 7) / 8, (u64)L.sms * 8);
  const unsigned gr = (unsigned)L.sms * 4;
  if (d.rows == 0) return;
  k_run_count<<<gw, kThreads, 0, L.stream>>>(d, T, w.row_runs, out, inv);
  const u64 tiles = (d.rows + kThreads * kScanPer - 1) / (kThreads * kScanPer);
  k_run_scan<<<(unsigned)umin(tiles, (u64)L.sms * 4), kThreads, 0, L.stream>>>(
      d.rows, w.row_runs, w.row_off, w.lb, w.ctr, w.status, w.total, d.spin_limit);
  k_run_fill<<<gw, kThreads, 0, L.stream>>>(d, T, w.row_off, w.xs, w.xe, w.par, w.size, inv);
  k_run_union<<<gw, kThreads, 0, L.stream>>>(d, w.row_off, w.total, w.xs, w.xe, w.par);
  k_run_sizes<<<gr, kThreads, 0, L.stream>>>(w.total, w.par, w.xs, w.xe, w.size);
  if (keep_border) {
    u32* flag = reinterpret_cast<u32*>(w.size);  // sizes are not needed here
    cudaMemsetAsync(flag, 0, 4 * (size_t)ccl_max_runs(d), L.stream);
    k_run_border<<<gr, kThreads, 0, L.stream>>>(d, w.row_off, w.total, w.par, w.xs, w.xe, flag);
    k_run_keep_flagged<<<gr, kThreads, 0, L.stream>>>(d, w.row_off, w.total, w.par, w.xs, w.xe,
                                                      flag, out);
  } else {
    k_run_best_z<<<gr, kThreads, 0, L.stream>>>(d, w.row_off, w.total, w.par, w.size, w.best);
    k_run_best_root_z<<<gr, kThreads, 0, L.stream>>>(d, w.row_off, w.total, w.par, w.size,
                                                     w.best, w.best_root);
    k_run_keep_z<<<gr, kThreads, 0, L.stream>>>(d, w.row_off, w.total, w.par, w.xs, w.xe,
                                                w.best_root, out);
  }
}

void launch_keep_largest(const Launch& L, const Desc& d, const u32* T, u32* out,
                         const CclWs& w) {
  const unsigned gw = (unsigned)umin((d.rows + 7) / 8, (u64)L.sms * 8);
  const unsigned gr = (unsigned)L.sms * 4;
  if (d.rows == 0) return;
  k_run_count<<<gw, kThreads, 0, L.stream>>>(d, T, w.row_runs, out, 0u);
  const u64 tiles = (d.rows + kThreads * kScanPer - 1) / (kThreads * kScanPer);
  k_run_scan<<<(unsigned)umin(tiles, (u64)L.sms * 4), kThreads, 0, L.stream>>>(
      d.rows, w.row_runs, w.row_off, w.lb, w.ctr, w.status, w.total, d.spin_limit);
  k_run_fill<<<gw, kThreads, 0, L.stream>>>(d, T, w.row_off, w.xs, w.xe, w.par, w.size, 0u);
  k_run_union<<<gw, kThreads, 0, L.stream>>>(d, w.row_off, w.total, w.xs, w.xe, w.par);
  k_run_sizes<<<gr, kThreads, 0, L.stream>>>(w.total, w.par, w.xs, w.xe, w.size);
  k_run_best_size<<<gr, kThreads, 0, L.stream>>>(w.total, w.par, w.size, w.best);
  k_run_best_root<<<gr, kThreads, 0, L.stream>>>(w.total, w.par, w.size, w.best, w.best_root);
  k_run_keep<<<gr, kThreads, 0, L.stream>>>(d, w.row_off, w.total, w.par, w.xs, w.xe,
                                             w.best_root, out);
}

}  // namespace roix
