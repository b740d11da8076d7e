// Evaluation metrics of the paper on the GPU: the ROI quality metrics of
// Sec. 5.2 (confusion counts and the ratios built from them, the average
// Hausdorff distance through an exact Euclidean distance transform) and the
// SSIM of Sec. 5.6 (Wang et al. 2004: Gaussian window 11 x 11, sigma 1.5,
// K1 = 0.01, K2 = 0.03, per 2D slice, over the positions where the window
// fits).
#include "roix_internal.cuh"

namespace roix {

namespace {

constexpr int kMThreads = 256;
constexpr u32 kInf = 0xffffffffu;  // no feature voxel on the line

__device__ __forceinline__ u32 tail_mask(u64 nx, u64 w, u64 W) {
  const u32 rem = (u32)(nx & 31);
  return (w == W - 1 && rem) ? ((1u << rem) - 1u) : 0xffffffffu;
}

// ------------------------------------------------------ confusion counts
// A warp per row, lanes over its words; TP, FP, FN summed per thread, one
// atomic per warp and count.
__global__ void __launch_bounds__(kMThreads)
    k_confusion(const u32* __restrict__ A, const u32* __restrict__ B, u64 rows, u64 W, u64 nx,
                unsigned long long* __restrict__ cnt) {
  const int lane = threadIdx.x & 31;
  const u64 warp = ((u64)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const u64 nwarps = ((u64)gridDim.x * blockDim.x) >> 5;
  u64 tp = 0, fp = 0, fn = 0;
  for (u64 r = warp; r < rows; r += nwarps) {
    const u32* a = A + r * W;
    const u32* b = B + r * W;
    for (u64 w = lane; w < W; w += 32) {
      const u32 m = tail_mask(nx, w, W);
      const u32 x = __ldg(a + w) & m, y = __ldg(b + w) & m;
      tp += __popc(x & y);
      fp += __popc(x & ~y);
      fn += __popc(~x & y);
    }
  }
  tp = warp_sum(tp);
  fp = warp_sum(fp);
  fn = warp_sum(fn);
  if (lane == 0) {
    if (tp) atomicAdd(cnt + 0, (unsigned long long)tp);
    if (fp) atomicAdd(cnt + 1, (unsigned long long)fp);
    if (fn) atomicAdd(cnt + 2, (unsigned long long)fn);
  }
}

__device__ __forceinline__ double ddiv(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }

// The Sec. 5.2 ratios from the counts, one operation at a time (no
// contraction), in the order the equations print them.
__global__ void k_metrics_final(const unsigned long long* __restrict__ cnt, u64 N,
                                const double* __restrict__ sums, int distances,
                                roix_roi_metrics* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const u64 tp = cnt[0], fp = cnt[1], fn = cnt[2], tn = N - tp - fp - fn;
  const double TP = (double)tp, FP = (double)fp, FN = (double)fn, TN = (double)tn;
  roix_roi_metrics m;
  m.tp = tp;
  m.fp = fp;
  m.fn = fn;
  m.tn = tn;
  const double total = dadd(dadd(dadd(TP, TN), FN), FP);
  const double fc = ddiv(dadd(dmul(dadd(TN, FN), dadd(TN, FP)), dmul(dadd(FP, TP), dadd(FN, TP))),
                         total);
  m.dsc = ddiv(dmul(2.0, TP), dadd(dadd(TP, FP), dadd(TP, FN)));
  m.iou = ddiv(TP, dadd(dadd(TP, FP), FN));
  m.sensitivity = ddiv(TP, dadd(TP, FN));
  m.specificity = ddiv(TN, dadd(TN, FP));
  m.accuracy = ddiv(dadd(TP, TN), dadd(dadd(dadd(TP, TN), FP), FN));
  m.kappa = ddiv(dsub(dadd(TP, TN), fc), dsub(dadd(dadd(dadd(TP, TN), FN), FP), fc));
  m.auc = dsub(1.0, dmul(0.5, dadd(ddiv(FP, dadd(FP, TN)), ddiv(FN, dadd(FN, TP)))));
  const double nan = __longlong_as_double(0x7ff8000000000000ll);
  const u64 na = tp + fp, nb = tp + fn;
  if (distances && na && nb) {
    m.sum_ab = sums[0];
    m.sum_ba = sums[1];
    const double dab = ddiv(sums[0], (double)na), dba = ddiv(sums[1], (double)nb);
    m.ahd = dab > dba ? dab : dba;
  } else {
    m.sum_ab = nan;
    m.sum_ba = nan;
    m.ahd = nan;
  }
  *out = m;
}

// ------------------------------------------------ exact distance transform
// Meijster, Roerdink and Hesselink (2000): a 1D pass along x on the bits of
// the feature set F gives g = distance to the nearest feature of the row; two
// lower-envelope passes along y and z give the squared Euclidean distance.

// Pass x: a warp per row, a lane per 32 consecutive voxels. The nearest
// feature at or before each voxel and at or after it come from the lane's own
// bits and, across lanes, from warp max / min scans of the lanes' last and
// first features (carried over the row's 1024-voxel segments).
__global__ void __launch_bounds__(kMThreads)
    k_edt_x(const u32* __restrict__ F, u64 rows, u64 W, u64 nx, u32* __restrict__ g) {
  const int lane = threadIdx.x & 31;
  const u64 warp = ((u64)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const u64 nwarps = ((u64)gridDim.x * blockDim.x) >> 5;
  const long long none_lo = -(1ll << 40), none_hi = 1ll << 40;
  for (u64 r = warp; r < rows; r += nwarps) {
    const u32* f = F + r * W;
    u32* out = g + r * nx;
    // forward: last feature at or before x
    long long carry = none_lo;
    const u64 segs = (W + 31) / 32;
    for (u64 s = 0; s < segs; ++s) {
      const u64 w = s * 32 + lane;
      const u32 bits = w < W ? (__ldg(f + w) & tail_mask(nx, w, W)) : 0u;
      const long long mylast = bits ? (long long)(w * 32 + 31 - __clz(bits)) : none_lo;
      long long inc = mylast;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const long long v = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc = inc > v ? inc : v;
      }
      long long before = __shfl_up_sync(0xffffffffu, inc, 1);
      if (lane == 0) before = none_lo;
      before = before > carry ? before : carry;  // last feature before this lane's word
      // write the forward distance (as the candidate) for this lane's voxels
      if (w < W) {
        long long last = before;
        for (int b = 0; b < 32; ++b) {
          const u64 x = w * 32 + b;
          if (x >= nx) break;
          if ((bits >> b) & 1u) last = (long long)x;
          const long long d = last == none_lo ? -1 : (long long)x - last;
          out[x] = d < 0 ? kInf : (u32)d;
        }
      }
      const long long segmax = __shfl_sync(0xffffffffu, inc, 31);
      carry = segmax > carry ? segmax : carry;
    }
    __syncwarp();
    // backward: next feature at or after x; keep the smaller distance
    carry = none_hi;
    for (long long s = (long long)segs - 1; s >= 0; --s) {
      const u64 w = (u64)s * 32 + lane;
      const u32 bits = w < W ? (__ldg(f + w) & tail_mask(nx, w, W)) : 0u;
      const long long myfirst = bits ? (long long)(w * 32 + (__ffs(bits) - 1)) : none_hi;
      long long inc = myfirst;  // suffix minimum over lanes >= this one
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const long long v = __shfl_down_sync(0xffffffffu, inc, o);
        if (lane + o < 32) inc = inc < v ? inc : v;
      }
      long long after = __shfl_down_sync(0xffffffffu, inc, 1);
      if (lane == 31) after = none_hi;
      after = after < carry ? after : carry;
      if (w < W) {
        long long next = after;
        for (int b = 31; b >= 0; --b) {
          const u64 x = w * 32 + b;
          if (x >= nx) continue;
          if ((bits >> b) & 1u) next = (long long)x;
          if (next != none_hi) {
            const u32 d = (u32)(next - (long long)x);
            if (d < out[x]) out[x] = d;
          }
        }
      }
      const long long segmin = __shfl_sync(0xffffffffu, inc, 0);
      carry = segmin < carry ? segmin : carry;
    }
  }
}

__device__ __forceinline__ long long floor_div_ll(long long a, long long b) {
  long long q = a / b;
  if ((a % b != 0) && ((a < 0) != (b < 0))) --q;
  return q;
}

// One lower-envelope pass over lines of m values with stride `st` (voxels):
// out(u) = min over sites i of f(i) + (u - i)^2, where f is g^2 from pass x
// (pass y) or the squared distance after pass y (pass z); sites with f = kInf
// are absent. A thread per line, consecutive threads on consecutive x
// (coalesced); a thread keeps its envelope (site s[k], start t[k]) in its own
// slot of the stack workspace, entry k at stk[k * nthr + slot].
template <bool SQUARE_IN>
__device__ __forceinline__ long long fval(const u32* in, u64 base, u64 st, long long i) {
  const u32 v = in[base + (u64)i * st];
  if (v == kInf) return -1;
  return SQUARE_IN ? (long long)v * (long long)v : (long long)v;
}

// With `acc`, the square roots of the results on voxels of mask M are summed
// instead of written (the last pass).
template <bool SQUARE_IN>
__global__ void __launch_bounds__(kMThreads)
    k_edt_env(const u32* __restrict__ in, u32* __restrict__ out, u64 nx, u64 ny, u64 nz, int axis,
              const u32* __restrict__ M, u64 W, double* acc, int2* __restrict__ stk) {
  // lines: axis 1 (y): (z, x) pairs, stride nx; axis 2 (z): (y, x) pairs, stride nx*ny
  const u64 lines = axis == 1 ? nz * nx : ny * nx;
  const u64 m = axis == 1 ? ny : nz;
  const u64 st = axis == 1 ? nx : nx * ny;
  const u64 nthr = (u64)gridDim.x * blockDim.x;
  const u64 slot = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  int2* my = stk + slot;  // entry k at my[k * nthr]: (site, start)
  double sum = 0.0;
  for (u64 l = slot; l < lines; l += nthr) {
    const u64 a = l / nx, x = l - a * nx;  // axis 1: a = z; axis 2: a = y
    const u64 base = axis == 1 ? a * nx * ny + x : a * nx + x;
    // forward: the envelope of the parabolas of the sites with f finite
    long long q = -1;
    int2 top = make_int2(0, 0);  // my[q], kept in registers
    long long ftop = 0;          // f(site of top)
    for (long long u = 0; u < (long long)m; ++u) {
      const long long fu = fval<SQUARE_IN>(in, base, st, u);
      if (fu < 0) continue;
      while (q >= 0) {
        const long long ds = (long long)top.y - top.x, du = (long long)top.y - u;
        if (ftop + ds * ds <= fu + du * du) break;
        if (--q >= 0) {
          top = my[(u64)q * nthr];
          ftop = fval<SQUARE_IN>(in, base, st, top.x);
        }
      }
      if (q < 0) {
        q = 0;
        top = make_int2((int)u, 0);
        ftop = fu;
        my[0] = top;
      } else {
        const long long i = top.x;
        const long long w = 1 + floor_div_ll(u * u - i * i + fu - ftop, 2 * (u - i));
        if (w < (long long)m) {
          ++q;
          top = make_int2((int)u, (int)w);
          ftop = fu;
          my[(u64)q * nthr] = top;
        }
      }
    }
    // backward: read the envelope
    for (long long u = (long long)m - 1; u >= 0; --u) {
      u32 d = kInf;
      if (q >= 0) {
        const long long i = top.x;
        d = (u32)(ftop + (u - i) * (u - i));
        if (u == top.y && --q >= 0) {
          top = my[(u64)q * nthr];
          ftop = fval<SQUARE_IN>(in, base, st, top.x);
        }
      }
      if (acc) {
        const u64 row = axis == 1 ? a * ny + (u64)u : (u64)u * ny + a;
        if ((__ldg(M + row * W + (x >> 5)) >> (x & 31)) & 1u) sum += sqrt((double)d);
      } else {
        out[base + (u64)u * st] = d;
      }
    }
  }
  if (acc) {
    sum = warp_sum(sum);
    if ((threadIdx.x & 31) == 0 && sum != 0.0) atomicAdd(acc, sum);
  }
}

// A single row (ny = nz = 1): the distances are g itself, summed over M.
__global__ void __launch_bounds__(kMThreads)
    k_edt_rowsum(const u32* __restrict__ g, u64 N, const u32* __restrict__ M, double* acc) {
  double sum = 0.0;
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (u64)gridDim.x * blockDim.x)
    if ((__ldg(M + (i >> 5)) >> (i & 31)) & 1u) sum += (double)g[i];
  sum = warp_sum(sum);
  if ((threadIdx.x & 31) == 0 && sum != 0.0) atomicAdd(acc, sum);
}

// -------------------------------------------------------------- SSIM
constexpr int kSx = 32, kSy = 16, kR = 5;
constexpr int kTx = kSx + 2 * kR, kTy = kSy + 2 * kR;

template <typename TV>
__device__ __forceinline__ double as_double(TV v) {
  return (double)v;
}

// A block computes a 32 x 16 tile of SSIM values of one slice: the inputs of
// the tile and its 5-voxel halo are staged in binary64, the five moments are
// filtered along x (11 taps) for every staged row, then along y, and the
// per-position SSIM values are summed (binary64 atomics, order not fixed).
struct Taps {
  double w[2 * kR + 1];
};

template <typename TV>
__global__ void __launch_bounds__(kMThreads)
    k_ssim(const TV* __restrict__ X, const TV* __restrict__ Y, u64 nx, u64 ny, u64 nz,
           double c1, double c2, const Taps taps, double* acc) {
  extern __shared__ double sm[];
  double* sx = sm;                  // kTy x kTx
  double* sy = sx + kTy * kTx;      // kTy x kTx
  double* hf = sy + kTy * kTx;      // 5 x kTy x kSx
  __shared__ double w[2 * kR + 1];
  if (threadIdx.x < 2 * kR + 1) w[threadIdx.x] = taps.w[threadIdx.x];
  const u64 vx = nx - 2 * kR, vy = ny - 2 * kR;  // valid positions per slice
  const u64 tx = (vx + kSx - 1) / kSx, ty = (vy + kSy - 1) / kSy;
  const u64 tiles = tx * ty * nz;
  double sum = 0.0;
  for (u64 t = blockIdx.x; t < tiles; t += gridDim.x) {
    const u64 z = t / (tx * ty), rem = t - z * tx * ty, by = rem / tx, bx = rem - by * tx;
    const u64 x0 = bx * kSx, y0 = by * kSy;  // first staged voxel (valid output x0 + kR)
    __syncthreads();
    for (int k = threadIdx.x; k < kTy * kTx; k += blockDim.x) {
      const int ry = k / kTx, rx = k - ry * kTx;
      const u64 gx = x0 + rx, gy = y0 + ry;
      double a = 0.0, b = 0.0;
      if (gx < nx && gy < ny) {
        const u64 idx = (z * ny + gy) * nx + gx;
        a = as_double(X[idx]);
        b = as_double(Y[idx]);
      }
      sx[k] = a;
      sy[k] = b;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < kTy * kSx; k += blockDim.x) {
      const int ry = k / kSx, cx = k - ry * kSx;
      double m1 = 0, m2 = 0, m11 = 0, m22 = 0, m12 = 0;
#pragma unroll
      for (int j = 0; j < 2 * kR + 1; ++j) {
        const double a = sx[ry * kTx + cx + j], b = sy[ry * kTx + cx + j], wj = w[j];
        m1 += wj * a;
        m2 += wj * b;
        m11 += wj * (a * a);
        m22 += wj * (b * b);
        m12 += wj * (a * b);
      }
      hf[0 * kTy * kSx + k] = m1;
      hf[1 * kTy * kSx + k] = m2;
      hf[2 * kTy * kSx + k] = m11;
      hf[3 * kTy * kSx + k] = m22;
      hf[4 * kTy * kSx + k] = m12;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < kSy * kSx; k += blockDim.x) {
      const int oy = k / kSx, ox = k - oy * kSx;
      if (x0 + ox >= vx || y0 + oy >= vy) continue;
      double m[5] = {0, 0, 0, 0, 0};
#pragma unroll
      for (int j = 0; j < 2 * kR + 1; ++j) {
        const double wj = w[j];
#pragma unroll
        for (int q = 0; q < 5; ++q) m[q] += wj * hf[q * kTy * kSx + (oy + j) * kSx + ox];
      }
      const double mx = m[0], my = m[1];
      const double sxx = m[2] - mx * mx, syy = m[3] - my * my, sxy = m[4] - mx * my;
      sum += ((2 * mx * my + c1) * (2 * sxy + c2)) / ((mx * mx + my * my + c1) * (sxx + syy + c2));
    }
  }
  sum = warp_sum(sum);
  if ((threadIdx.x & 31) == 0 && sum != 0.0) atomicAdd(acc, sum);
}

__global__ void k_ssim_final(const double* acc, double count, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0)
    *out = count > 0 ? acc[0] / count : __longlong_as_double(0x7ff8000000000000ll);
}

u64 grid_for(u64 units, u64 per_block, int sms) {
  u64 b = (units + per_block - 1) / per_block;
  const u64 cap = (u64)sms * 8;
  if (b > cap) b = cap;
  return b ? b : 1;
}

}  // namespace

// threads of the envelope passes (their stack slots), and the workspace of
// launch_roi_quality: counts and sums, g and h (4 bytes per voxel each), stacks
constexpr u64 kEnvThreads = 152ull * 2 * kMThreads;
size_t roi_quality_ws_bytes(u64 nx, u64 ny, u64 nz, int distances) {
  if (!distances) return 64;
  const u64 N = nx * ny * nz, m = ny > nz ? ny : nz;
  return 64 + 2 * (4 * N + 16) + 8 * (m + 1) * kEnvThreads;
}

void launch_roi_quality(const Launch& L, const u32* A, const u32* B, u64 nx, u64 ny, u64 nz,
                        int distances, char* ws, roix_roi_metrics* out) {
  const u64 rows = ny * nz, W = (nx + 31) / 32, N = nx * ny * nz;
  unsigned long long* cnt = (unsigned long long*)ws;  // 3 counts, then 2 sums
  double* sums = (double*)(ws + 32);
  cudaMemsetAsync(ws, 0, 64, L.stream);
  if (rows && W)
    k_confusion<<<(unsigned)grid_for(rows, kMThreads / 32, L.sms), kMThreads, 0, L.stream>>>(
        A, B, rows, W, nx, cnt);
  if (distances && N) {
    u32* g = (u32*)(ws + 64);
    u32* h = (u32*)(ws + 64 + 4 * N + 16);
    int2* stk = (int2*)(ws + 64 + 2 * (4 * N + 16));
    const unsigned env_blocks = (unsigned)(kEnvThreads / kMThreads);
    for (int side = 0; side < 2; ++side) {
      const u32* F = side == 0 ? B : A;  // distances to B, summed over A; then the reverse
      const u32* Msk = side == 0 ? A : B;
      double* acc = sums + side;
      k_edt_x<<<(unsigned)grid_for(rows, kMThreads / 32, L.sms), kMThreads, 0, L.stream>>>(
          F, rows, W, nx, g);
      if (ny == 1 && nz == 1) {
        k_edt_rowsum<<<(unsigned)grid_for(N, kMThreads, L.sms), kMThreads, 0, L.stream>>>(
            g, N, Msk, acc);
      } else if (nz == 1) {
        k_edt_env<true><<<env_blocks, kMThreads, 0, L.stream>>>(g, nullptr, nx, ny, nz, 1, Msk,
                                                                 W, acc, stk);
      } else {
        k_edt_env<true><<<env_blocks, kMThreads, 0, L.stream>>>(g, h, nx, ny, nz, 1, nullptr, W,
                                                                 nullptr, stk);
        k_edt_env<false><<<env_blocks, kMThreads, 0, L.stream>>>(h, nullptr, nx, ny, nz, 2, Msk,
                                                                  W, acc, stk);
      }
    }
  }
  k_metrics_final<<<1, 32, 0, L.stream>>>(cnt, N, sums, distances, out);
}


void launch_ssim(const Launch& L, int dtype, const void* X, const void* Y, u64 nx, u64 ny, u64 nz,
                 double data_range, char* ws, double* out) {
  double* acc = (double*)ws;
  // Gaussian taps, sigma 1.5, radius 5, normalised on the host in binary64
  Taps taps;
  double s = 0;
  for (int j = -kR; j <= kR; ++j)
    s += (taps.w[j + kR] = exp(-(double)(j * j) / (2.0 * 1.5 * 1.5)));
  for (double& v : taps.w) v /= s;
  cudaMemsetAsync(acc, 0, 16, L.stream);
  double count = 0;
  if (nx >= 2 * kR + 1 && ny >= 2 * kR + 1 && nz) {
    count = (double)((nx - 2 * kR) * (ny - 2 * kR) * nz);
    const double c1 = (0.01 * data_range) * (0.01 * data_range);
    const double c2 = (0.03 * data_range) * (0.03 * data_range);
    const u64 tiles = (nx - 2 * kR + kSx - 1) / kSx * ((ny - 2 * kR + kSy - 1) / kSy) * nz;
    const size_t smem = (size_t)(2 * kTy * kTx + 5 * kTy * kSx) * 8;
    u64 grid = tiles;
    if (grid > (u64)L.sms * 4) grid = (u64)L.sms * 4;
    if (dtype == ROIX_F32) {
      cudaFuncSetAttribute(k_ssim<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      k_ssim<float><<<(unsigned)grid, kMThreads, smem, L.stream>>>(
          (const float*)X, (const float*)Y, nx, ny, nz, c1, c2, taps, acc);
    } else if (dtype == ROIX_U16) {
      cudaFuncSetAttribute(k_ssim<unsigned short>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem);
      k_ssim<unsigned short><<<(unsigned)grid, kMThreads, smem, L.stream>>>(
          (const unsigned short*)X, (const unsigned short*)Y, nx, ny, nz, c1, c2, taps, acc);
    } else {
      cudaFuncSetAttribute(k_ssim<unsigned char>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem);
      k_ssim<unsigned char><<<(unsigned)grid, kMThreads, smem, L.stream>>>(
          (const unsigned char*)X, (const unsigned char*)Y, nx, ny, nz, c1, c2, taps, acc);
    }
  }
  k_ssim_final<<<1, 32, 0, L.stream>>>(acc, count, out);
}

}  // namespace roix
