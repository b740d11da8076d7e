// Paper-mode region of interest of an 8-bit image, every 2D slice on its own:
// multi-Otsu thresholds (Sec. 4.1.3), binarisation above the lowest one
// (Sec. 4.1.4), holes filled and the largest object kept (Sec. 4.2.1,
// external contours), one span [x_start, x_end) per row (Sec. 4.2.2). The
// connected components come from the run-based union-find of k_ccl.cu in its
// planar form.
#include "roix_internal.cuh"

namespace roix {

namespace {

constexpr int kPThreads = 256;
constexpr u64 kHistChunk = 1ull << 16;  // pixels of one slice per histogram block

// 256-bin histogram of every slice: a block takes one chunk of one slice,
// counts in shared memory, then adds its bins to the slice's.
__global__ void __launch_bounds__(kPThreads)
    k_hist(const u8* __restrict__ img, u64 plane, u64 nz, u64 chunks, u32* __restrict__ hist) {
  __shared__ u32 h[256];
  for (u64 b = blockIdx.x; b < nz * chunks; b += gridDim.x) {
    const u64 z = b / chunks, c = b - z * chunks;
    for (int k = threadIdx.x; k < 256; k += blockDim.x) h[k] = 0u;
    __syncthreads();
    const u8* p = img + z * plane;
    const u64 lo = c * kHistChunk, hi = umin(lo + kHistChunk, plane);
    for (u64 i = lo + threadIdx.x; i < hi; i += blockDim.x) atomicAdd(&h[__ldg(p + i)], 1u);
    __syncthreads();
    for (int k = threadIdx.x; k < 256; k += blockDim.x)
      if (h[k]) atomicAdd(hist + z * 256 + k, h[k]);
    __syncthreads();
  }
}

// Multi-Otsu with three classes, a block per slice: every pair t1 < t2 of
// [0, 254] is scored by sum over the classes [0, t1], (t1, t2], (t2, 255] of
// (sum of values)^2 / count (binary64, one IEEE operation at a time; empty
// classes add 0); the best score wins, ties to the smallest (t1, t2).
__global__ void __launch_bounds__(kPThreads) k_multiotsu(const u32* __restrict__ hist, u64 nz,
                                                         u32* __restrict__ thr) {
  __shared__ unsigned long long P[256], S[256];
  __shared__ double bf[kPThreads];
  __shared__ u32 bt[kPThreads];
  for (u64 z = blockIdx.x; z < nz; z += gridDim.x) {
    if (threadIdx.x == 0) {
      unsigned long long p = 0, s = 0;
      for (int v = 0; v < 256; ++v) {
        const unsigned long long c = hist[z * 256 + v];
        p += c;
        s += c * (unsigned long long)v;
        P[v] = p;
        S[v] = s;
      }
    }
    __syncthreads();
    double best = -1.0;
    u32 arg = 0xffffffffu;  // t1 * 256 + t2
    const int t2off = threadIdx.x + 1;
    for (int t1 = 0; t1 < 254; ++t1) {
      const int t2 = t1 + t2off;
      if (t2 > 254) continue;
      const unsigned long long c[3] = {P[t1], P[t2] - P[t1], P[255] - P[t2]};
      const unsigned long long sm[3] = {S[t1], S[t2] - S[t1], S[255] - S[t2]};
      double f = 0.0;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        double term = 0.0;
        if (c[k]) {
          const double sv = (double)sm[k];
          term = __ddiv_rn(__dmul_rn(sv, sv), (double)c[k]);
        }
        f = __dadd_rn(f, term);
      }
      const u32 a = (u32)t1 * 256u + (u32)t2;
      if (f > best || (f == best && a < arg)) {
        best = f;
        arg = a;
      }
    }
    bf[threadIdx.x] = best;
    bt[threadIdx.x] = arg;
    __syncthreads();
    for (int o = kPThreads / 2; o > 0; o >>= 1) {
      if ((int)threadIdx.x < o) {
        const double f2 = bf[threadIdx.x + o];
        const u32 a2 = bt[threadIdx.x + o];
        if (f2 > bf[threadIdx.x] || (f2 == bf[threadIdx.x] && a2 < bt[threadIdx.x])) {
          bf[threadIdx.x] = f2;
          bt[threadIdx.x] = a2;
        }
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      thr[2 * z] = bt[0] >> 8;
      thr[2 * z + 1] = bt[0] & 255u;
    }
    __syncthreads();
  }
}

// M = [I_n > t1 of the slice]: a warp per row, 32 coalesced bytes per ballot.
__global__ void __launch_bounds__(kPThreads)
    k_binarize(const u8* __restrict__ img, u64 nx, u64 ny, u64 rows, u64 W,
               const u32* __restrict__ thr, u32* __restrict__ T) {
  const int lane = threadIdx.x & 31;
  for (u64 r = ((u64)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < rows;
       r += ((u64)gridDim.x * blockDim.x) >> 5) {
    const u32 t1 = thr[2 * (r / ny)];
    const u8* row = img + r * nx;
    for (u64 w = 0; w < W; ++w) {
      const u64 x = w * 32 + lane;
      const bool on = x < nx && (u32)__ldg(row + x) > t1;
      const u32 b = __ballot_sync(0xffffffffu, on);
      if (lane == 0) T[r * W + w] = b;
    }
  }
}

// One span per row: bits from the row's first to its last set bit; a warp
// per row; the retained count is summed into *popcount.
__global__ void __launch_bounds__(kPThreads)
    k_spans(const u32* __restrict__ K, u64 rows, u64 W, u32* __restrict__ D, u64* popcount) {
  const int lane = threadIdx.x & 31;
  u64 cnt = 0;
  for (u64 r = ((u64)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < rows;
       r += ((u64)gridDim.x * blockDim.x) >> 5) {
    const u32* k = K + r * W;
    long long first = 1ll << 40, last = -1;
    for (u64 w = lane; w < W; w += 32) {
      const u32 v = __ldg(k + w);
      if (v) {
        const long long f = (long long)(w * 32 + __ffs(v) - 1);
        const long long l = (long long)(w * 32 + 31 - __clz(v));
        first = f < first ? f : first;
        last = l > last ? l : last;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const long long f2 = __shfl_xor_sync(0xffffffffu, first, o);
      const long long l2 = __shfl_xor_sync(0xffffffffu, last, o);
      first = f2 < first ? f2 : first;
      last = l2 > last ? l2 : last;
    }
    for (u64 w = lane; w < W; w += 32) {
      u32 m = 0u;
      if (last >= 0) {
        const long long a = (long long)w * 32, b = a + 31;
        const long long lo = first > a ? first : a, hi = last < b ? last : b;
        if (lo <= hi) {
          const u32 s = (u32)(lo - a), e = (u32)(hi - a);
          m = (e == 31 ? 0xffffffffu : ((1u << (e + 1)) - 1u)) & ~((1u << s) - 1u);
        }
      }
      D[r * W + w] = m;
    }
    if (lane == 0 && last >= 0) cnt += (u64)(last - first + 1);
  }
  if (lane == 0 && cnt) atomicAdd((unsigned long long*)popcount, (unsigned long long)cnt);
}

unsigned grid_rows(u64 rows, int sms) {
  u64 b = (rows + kPThreads / 32 - 1) / (kPThreads / 32);
  const u64 cap = (u64)sms * 8;
  return (unsigned)(b < 1 ? 1 : (b > cap ? cap : b));
}

}  // namespace

void launch_paper_hist_otsu(const Launch& L, const u8* img, u64 nx, u64 ny, u64 nz, u32* hist,
                            u32* thr) {
  const u64 plane = nx * ny;
  const u64 chunks = (plane + kHistChunk - 1) / kHistChunk;
  cudaMemsetAsync(hist, 0, 4 * 256 * nz, L.stream);
  u64 blocks = nz * chunks;
  if (blocks > (u64)L.sms * 8) blocks = (u64)L.sms * 8;
  if (plane) k_hist<<<(unsigned)(blocks ? blocks : 1), kPThreads, 0, L.stream>>>(
      img, plane, nz, chunks, hist);
  u64 b2 = nz < (u64)L.sms * 4 ? nz : (u64)L.sms * 4;
  k_multiotsu<<<(unsigned)(b2 ? b2 : 1), kPThreads, 0, L.stream>>>(hist, nz, thr);
}

void launch_paper_binarize(const Launch& L, const u8* img, u64 nx, u64 ny, u64 nz,
                           const u32* thr, u32* T) {
  const u64 rows = ny * nz, W = (nx + 31) / 32;
  if (rows) k_binarize<<<grid_rows(rows, L.sms), kPThreads, 0, L.stream>>>(img, nx, ny, rows, W,
                                                                            thr, T);
}

void launch_paper_spans(const Launch& L, const u32* K, u64 rows, u64 W, u32* D, u64* popcount) {
  if (rows) k_spans<<<grid_rows(rows, L.sms), kPThreads, 0, L.stream>>>(K, rows, W, D, popcount);
}

}  // namespace roix
