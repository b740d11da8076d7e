// ROIX-Comp oracle: a plain, slow, single-threaded CPU statement of what the
// hot path computes. TEST INFRASTRUCTURE ONLY: it is loaded by the tests, by
// the smoke check and by the CPU-baseline leg of the benchmark, never by the
// product path. It shares no code, header or table with the CUDA library.
//
// Every function follows one step of the method in the paper's order:
//   threshold / binarisation ........ Sec. 4.1.3-4.1.4 (Eq. for M(x,y))
//   background subtraction ........... Sec. 4.1.1 (M = I - B), constant dark level
//   largest object ................... Sec. 4.2.1 (largest external contour),
//                                       read as the largest connected component
//   dilation ......................... 1-voxel safety margin of the workload
//   row geometry + pixel section ..... Sec. 4.2.2 (G(i) = [i, x_start, x_end],
//                                       P(i)), generalised to several runs per row
//   error-bounded quantisation ....... Sec. 4.2.3 contract |Q - D| <= E_abs, with the
//                                       Sz3-style linear quantiser of Sec. 4.3
//   prediction + entropy coding ...... Sec. 4.3 (Sz3: prediction-based), 1D Lorenzo
//                                       over the pixel section, canonical Huffman
//   reconstruction ................... Sec. 4.3, last paragraph (rows restored from
//                                       the geometry, background filled in)
//
// Floating point: compile with -O2 -ffp-contract=off and no fast-math, so that
// every float operation below is one IEEE-754 binary32 operation rounded to
// nearest-even and every double operation one binary64 operation.
//
// Parity pins (tests/test_oracle_*.py): brute-force nearest lattice point and
// the exact error bound for the quantiser; scipy.ndimage dilation and labelling
// for the mask; numpy boolean indexing for the compaction; the heap Huffman
// optimum, the Kraft equality and an independent bit reader for the codebook
// and packing; round trips for geometry, prediction and the whole container.
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <vector>
#include <algorithm>

namespace {

enum { DT_F32 = 1, DT_U16 = 2, DT_U8 = 3 };  // uint8: the normalised image (Sec. 4.1.2)
enum { ERR_OK = 0, ERR_INVAL = 1, ERR_CORRUPT = 4 };

const uint32_t kLMax = 24;          // longest Huffman code
const uint32_t kHeaderBytes = 256;  // fixed container header size

inline uint64_t align16(uint64_t v) { return (v + 15) & ~uint64_t(15); }

// Binary32 rounded toward zero from a binary64 value.
float f32_rz(double d) {
  float f = (float)d;
  if (std::fabs((double)f) > std::fabs(d)) f = std::nextafterf(f, 0.0f);
  return f;
}

int64_t floor_div(int64_t a, int64_t b) {  // b > 0
  return a >= 0 ? a / b : -((-a + b - 1) / b);
}

struct Buf {
  std::vector<uint8_t> b;
  template <class T> void put(uint64_t off, T v) { std::memcpy(&b[off], &v, sizeof(T)); }
};

}  // namespace

extern "C" {

// Parameters of one compression call (mirrors the container header fields).
struct OracleParams {
  int32_t dtype;         // 1 = float32, 2 = uint16
  int32_t eb_mode;       // 0 = absolute, 1 = relative to the ROI value range
  double eb_value;       // error bound (absolute) or factor (relative)
  int32_t cmp;           // 0: ROI where value > threshold, 1: value < threshold
  int32_t keep;          // 0: every thresholded voxel, 1: largest component only
  int32_t connectivity;  // 6 or 26 (2D: 4 or 8)
  int32_t dilate;        // dilation radius (cube), 0 or 1
  double threshold;
  double dark;           // constant background level B subtracted (uint16 only)
  double fill;           // value of non-ROI voxels after reconstruction
  uint32_t radius;       // R: symbol alphabet is 2R
  uint32_t chunk;        // C: symbols per independently decodable chunk
  uint32_t order;        // Lorenzo order along the pixel section: 1 (0 reads as 1) or 2
};

// Error-bound constants (Sec. 4.2.3: E_abs; relative mode as in Sz3, Sec. 4.3).
struct OracleEb {
  double eb_abs;
  double vmin, vmax;     // range of the finite retained values
  float two_eb, inv2eb, bound;
  int32_t eb_int;        // uint16 path: integer half-width
};

static uint32_t order_of(const OracleParams* p) { return p->order == 2 ? 2u : 1u; }

// ---------------------------------------------------------------- threshold
// Sec. 4.1.1 M = I - B (B constant = dark), Sec. 4.1.3-4.1.4: M(x,y) = 1 where
// the background-subtracted value lies above (cmp 0) or below (cmp 1) t.
int oracle_threshold(const void* in, const OracleParams* p, uint64_t nx,
                     uint64_t ny, uint64_t nz, uint8_t* T) {
  uint64_t N = nx * ny * nz;
  for (uint64_t i = 0; i < N; ++i) {
    double v;
    if (p->dtype == DT_F32) {
      v = (double)((const float*)in)[i];
    } else if (p->dtype == DT_U8) {
      v = (double)((int64_t)((const uint8_t*)in)[i] - (int64_t)p->dark);
    } else {
      v = (double)((int64_t)((const uint16_t*)in)[i] - (int64_t)p->dark);
    }
    bool on = p->cmp == 0 ? (v > p->threshold) : (v < p->threshold);
    T[i] = on ? 1 : 0;
  }
  return ERR_OK;
}

// ------------------------------------------------------- largest component
// Sec. 4.2.1 keeps the largest object. Components by breadth-first flood fill
// (the textbook definition) under 6- or 26-connectivity; the kept component is
// the one with the most voxels, ties to the one holding the smallest raster
// index. T is overwritten with that component.
int oracle_keep_largest(uint8_t* T, uint64_t nx, uint64_t ny, uint64_t nz,
                        int32_t conn) {
  uint64_t N = nx * ny * nz;
  if (N == 0) return ERR_OK;
  std::vector<int32_t> label(N, -1);
  std::vector<uint64_t> sizes;
  std::deque<uint64_t> queue;
  for (uint64_t s = 0; s < N; ++s) {
    if (!T[s] || label[s] >= 0) continue;
    int32_t id = (int32_t)sizes.size();
    sizes.push_back(0);
    label[s] = id;
    queue.push_back(s);
    while (!queue.empty()) {
      uint64_t v = queue.front();
      queue.pop_front();
      sizes[id]++;
      int64_t x = (int64_t)(v % nx), y = (int64_t)((v / nx) % ny),
              z = (int64_t)(v / (nx * ny));
      for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx) {
            int nonzero = (dx != 0) + (dy != 0) + (dz != 0);
            if (nonzero == 0) continue;
            if (conn == 6 && nonzero != 1) continue;
            int64_t X = x + dx, Y = y + dy, Z = z + dz;
            if (X < 0 || Y < 0 || Z < 0 || X >= (int64_t)nx ||
                Y >= (int64_t)ny || Z >= (int64_t)nz)
              continue;
            uint64_t u = (uint64_t)X + nx * ((uint64_t)Y + ny * (uint64_t)Z);
            if (T[u] && label[u] < 0) {
              label[u] = id;
              queue.push_back(u);
            }
          }
    }
  }
  if (sizes.empty()) return ERR_OK;
  int32_t best = 0;  // components are numbered by their smallest raster index
  for (int32_t c = 1; c < (int32_t)sizes.size(); ++c)
    if (sizes[c] > sizes[best]) best = c;
  for (uint64_t i = 0; i < N; ++i) T[i] = (label[i] == best) ? 1 : 0;
  return ERR_OK;
}

// ------------------------------------------------------------------ dilation
// D[v] = OR of T over the cube of half-width r around v, clipped to the volume.
int oracle_dilate(const uint8_t* T, uint64_t nx, uint64_t ny, uint64_t nz,
                  int32_t r, uint8_t* D) {
  for (uint64_t z = 0; z < nz; ++z)
    for (uint64_t y = 0; y < ny; ++y)
      for (uint64_t x = 0; x < nx; ++x) {
        uint8_t on = 0;
        for (int64_t dz = -r; dz <= r && !on; ++dz)
          for (int64_t dy = -r; dy <= r && !on; ++dy)
            for (int64_t dx = -r; dx <= r && !on; ++dx) {
              int64_t X = (int64_t)x + dx, Y = (int64_t)y + dy,
                      Z = (int64_t)z + dz;
              if (X < 0 || Y < 0 || Z < 0 || X >= (int64_t)nx ||
                  Y >= (int64_t)ny || Z >= (int64_t)nz)
                continue;
              if (T[(uint64_t)X + nx * ((uint64_t)Y + ny * (uint64_t)Z)]) on = 1;
            }
        D[x + nx * (y + ny * z)] = on;
      }
  return ERR_OK;
}

// ---------------------------------------------------------------- compaction
// Sec. 4.2.2: for every row i = (y, z) the geometry lists where the mask
// switches on or off (x_start, x_end pairs; x_end is one past the last ROI
// pixel, so n_i = x_end - x_start), and the pixel section P holds the ROI
// values row after row. Returns n = |D|; counts[r] = boundaries in row r.
int64_t oracle_compact(const void* in, int32_t dtype, uint64_t nx, uint64_t ny,
                       uint64_t nz, const uint8_t* D, void* P, uint16_t* counts,
                       uint16_t* bounds, uint64_t* n_bounds) {
  uint64_t n = 0, nb = 0;
  for (uint64_t r = 0; r < ny * nz; ++r) {
    const uint8_t* row = D + r * nx;
    uint16_t cnt = 0;
    uint8_t prev = 0;
    for (uint64_t x = 0; x <= nx; ++x) {
      uint8_t cur = x < nx ? row[x] : 0;
      if (cur != prev) {
        bounds[nb++] = (uint16_t)x;
        cnt++;
      }
      prev = cur;
      if (x < nx && cur) {
        if (dtype == DT_F32)
          ((float*)P)[n] = ((const float*)in)[r * nx + x];
        else if (dtype == DT_U8)
          ((uint8_t*)P)[n] = ((const uint8_t*)in)[r * nx + x];
        else
          ((uint16_t*)P)[n] = ((const uint16_t*)in)[r * nx + x];
        n++;
      }
    }
    counts[r] = cnt;
  }
  *n_bounds = nb;
  return (int64_t)n;
}

// ----------------------------------------------------------------- error bound
// Absolute mode: E_abs as given (Sec. 4.2.3). Relative mode: E_abs = factor x
// (max - min) of the finite values of the pixel section, the value-range
// convention of Sz3 (Sec. 4.3), which the paper applies to the extracted array.
void oracle_eb(const void* P, int32_t dtype, uint64_t n, int32_t mode,
               double value, OracleEb* e) {
  double vmin = INFINITY, vmax = -INFINITY;
  for (uint64_t k = 0; k < n; ++k) {
    double v;
    if (dtype == DT_F32) {
      float f = ((const float*)P)[k];
      if (!std::isfinite(f)) continue;
      v = (double)f;
    } else {
      v = (double)((const uint16_t*)P)[k];
    }
    if (v < vmin) vmin = v;
    if (v > vmax) vmax = v;
  }
  if (vmin == 0.0) vmin = 0.0;  // -0 and +0 are the same range end
  if (vmax == 0.0) vmax = 0.0;
  e->vmin = vmin;
  e->vmax = vmax;
  double eb;
  if (mode == 0) eb = value;
  else eb = (vmax >= vmin) ? value * (vmax - vmin) : 0.0;
  e->eb_abs = eb;
  float two = (float)(2.0 * eb);
  float inv = (eb > 0.0) ? (float)(1.0 / (2.0 * eb)) : 0.0f;
  bool ok = eb > 0.0 && std::isfinite(eb) && std::isfinite(two) && two > 0.0f &&
            std::isfinite(inv) && inv > 0.0f;
  if (ok) {
    e->two_eb = two;
    e->inv2eb = inv;
    // Margin so that |x - xh| <= E_abs holds exactly despite the rounding of
    // the binary32 subtraction used in the check (|rel. error| <= 2^-24).
    e->bound = f32_rz(eb * (1.0 - 0x1p-23));
  } else {  // degenerate bound: every retained value is kept verbatim
    e->two_eb = 0.0f;
    e->inv2eb = 0.0f;
    e->bound = -1.0f;
  }
  double ebi = std::floor(eb);
  if (!(ebi >= 0.0)) ebi = 0.0;
  if (ebi > 65535.0) ebi = 65535.0;
  e->eb_int = (int32_t)ebi;
}

// ---------------------------------------------------------------- quantiser
// Linear quantisation on the lattice 2*E_abs*Z (Sz3-style, Sec. 4.3) with the
// Sec. 4.2.3 contract |Q - D| <= E_abs. float32: q = rint(x / 2eb), checked
// reconstruction; values failing the check are outliers (q = 0, kept raw).
// uint16: exact integer arithmetic on v = raw - dark.
int oracle_quantize(const void* P, int32_t dtype, uint64_t n, const OracleEb* e,
                    double dark, int32_t* q, uint8_t* outl) {
  for (uint64_t k = 0; k < n; ++k) {
    if (dtype == DT_F32) {
      float x = ((const float*)P)[k];
      bool out = false;
      int32_t c = 0;
      if (!std::isfinite(x)) {
        out = true;
      } else {
        float y = x * e->inv2eb;
        if (!(std::fabs(y) < 1073741824.0f)) {
          out = true;
        } else {
          float r = rintf(y);  // round half to even
          c = (int32_t)r;
          float xh = (float)c * e->two_eb;
          float d = x - xh;
          out = !(std::fabs(d) <= e->bound);
        }
      }
      q[k] = out ? 0 : c;
      outl[k] = out ? 1 : 0;
    } else {
      int64_t v = (int64_t)((const uint16_t*)P)[k] - (int64_t)dark;
      int64_t c = e->eb_int == 0 ? v : floor_div(v + e->eb_int, 2 * (int64_t)e->eb_int);
      q[k] = (int32_t)c;
      outl[k] = 0;
    }
  }
  return ERR_OK;
}

// ---------------------------------------------------------------- prediction
// 1D Lorenzo over the pixel section (Sz3-style prediction, Sec. 4.3), in exact
// integer arithmetic. Order 1 predicts q[k-1]; order 2 (the two-layer
// Lorenzo) predicts 2 q[k-1] - q[k-2], i.e. extrapolates the last difference;
// q[-1] = q[-2] = 0 and an outlier counts as 0. The residual d = q[k] - pred
// is coded as symbol d + R when |d| < R, else as symbol 0 with a record
// (k | kind << 63, payload): kind 0 keeps q[k], kind 1 keeps the raw value
// bits. Returns the number of records.
uint64_t oracle_lorenzo(const int32_t* q, const uint8_t* outl, const void* P,
                        int32_t dtype, uint64_t n, uint32_t R, uint32_t order, uint16_t* sym,
                        uint64_t* rec_key, uint32_t* rec_val) {
  uint64_t m = 0;
  int64_t prev1 = 0, prev2 = 0;  // q[k-1], q[k-2]
  for (uint64_t k = 0; k < n; ++k) {
    int64_t c;
    if (outl[k]) {
      sym[k] = 0;
      rec_key[m] = k | (uint64_t(1) << 63);
      uint32_t bits = 0;
      if (dtype == DT_F32) std::memcpy(&bits, (const float*)P + k, 4);
      else bits = ((const uint16_t*)P)[k];
      rec_val[m] = bits;
      m++;
      c = 0;
    } else {
      c = q[k];
      const int64_t pred = order == 2 ? 2 * prev1 - prev2 : prev1;
      const int64_t d = c - pred;
      if (d > -(int64_t)R && d < (int64_t)R) {
        sym[k] = (uint16_t)(d + R);
      } else {
        sym[k] = 0;
        rec_key[m] = k;
        rec_val[m] = (uint32_t)q[k];
        m++;
      }
    }
    prev2 = prev1;
    prev1 = c;
  }
  return m;
}

void oracle_histogram(const uint16_t* sym, uint64_t n, uint32_t S, uint64_t* hist) {
  for (uint32_t s = 0; s < S; ++s) hist[s] = 0;
  for (uint64_t k = 0; k < n; ++k) hist[sym[k]]++;
}

// ------------------------------------------------------------------ codebook
// Canonical Huffman code (Huffman 1952) with lengths <= 24:
//  1. leaves = symbols with a nonzero count, sorted by (count, symbol);
//  2. two-queue construction (van Leeuwen 1976): repeatedly join the two
//     lightest of {front of leaf queue, front of internal-node queue}, the leaf
//     winning ties; leaf depth = code length;
//  3. lengths above 24 are folded back with the JPEG (ITU-T T.81 Annex K.3)
//     adjustment of the per-length counts;
//  4. the per-length counts are handed out shortest-first to the leaves in
//     decreasing (count, symbol) order;
//  5. canonical codes by (length, symbol), as in DEFLATE (RFC 1951 3.2.2).
int oracle_codebook(const uint64_t* hist, uint32_t S, uint8_t* len, uint32_t* code) {
  for (uint32_t s = 0; s < S; ++s) { len[s] = 0; code[s] = 0; }
  std::vector<uint32_t> leaves;
  for (uint32_t s = 0; s < S; ++s)
    if (hist[s] > 0) leaves.push_back(s);
  size_t m = leaves.size();
  if (m == 0) return ERR_OK;
  if (m == 1) {
    len[leaves[0]] = 1;
    return ERR_OK;
  }
  std::stable_sort(leaves.begin(), leaves.end(), [&](uint32_t a, uint32_t b) {
    return hist[a] < hist[b];
  });  // stable over increasing symbol: order (count, symbol)
  // nodes 0..m-1 leaves (sorted order), m..2m-2 internal in creation order
  std::vector<uint64_t> w(2 * m - 1);
  std::vector<int64_t> parent(2 * m - 1, -1);
  for (size_t i = 0; i < m; ++i) w[i] = hist[leaves[i]];
  size_t lf = 0, inf = m, created = m;
  auto take = [&]() -> size_t {
    bool leaf_ok = lf < m;
    bool int_ok = inf < created;
    if (leaf_ok && (!int_ok || w[lf] <= w[inf])) return lf++;
    return inf++;
  };
  for (size_t t = 0; t + 1 < m; ++t) {
    size_t a = take();
    size_t b = take();
    w[created] = w[a] + w[b];
    parent[a] = (int64_t)created;
    parent[b] = (int64_t)created;
    created++;
  }
  std::vector<uint32_t> depth(2 * m - 1, 0);
  for (size_t i = 2 * m - 2; i-- > 0;) depth[i] = depth[parent[i]] + 1;
  uint32_t maxl = 0;
  for (size_t i = 0; i < m; ++i) maxl = std::max(maxl, depth[i]);
  std::vector<uint64_t> bl(std::max<uint32_t>(maxl, kLMax) + 2, 0);
  for (size_t i = 0; i < m; ++i) bl[depth[i]]++;
  for (uint32_t l = maxl; l > kLMax; --l) {
    while (bl[l] > 0) {
      uint32_t j = l - 2;
      while (bl[j] == 0) j--;
      bl[l] -= 2;
      bl[l - 1] += 1;
      bl[j + 1] += 2;
      bl[j] -= 1;
    }
  }
  // shortest lengths to the most frequent leaves
  size_t idx = m;
  for (uint32_t l = 1; l <= kLMax; ++l)
    for (uint64_t c = 0; c < bl[l]; ++c) len[leaves[--idx]] = (uint8_t)l;
  // canonical codes
  uint32_t count[kLMax + 1] = {0};
  for (uint32_t s = 0; s < S; ++s) count[len[s]]++;
  count[0] = 0;
  uint32_t next[kLMax + 2] = {0};
  uint32_t c = 0;
  for (uint32_t l = 1; l <= kLMax; ++l) {
    c = (c + count[l - 1]) << 1;
    next[l] = c;
  }
  for (uint32_t s = 0; s < S; ++s)
    if (len[s]) code[s] = next[len[s]]++;
  return ERR_OK;
}

// ---------------------------------------------------------------------- pack
// Chunks of C symbols; each chunk starts on a fresh 32-bit word; codes are
// written most-significant bit first (first bit of a chunk = bit 31 of its
// first word); pad bits are 0. chunk_off[j] = word offset of chunk j.
// Returns the number of words; words may be null for a size query.
uint64_t oracle_pack(const uint16_t* sym, uint64_t n, const uint8_t* len,
                     const uint32_t* code, uint32_t C, uint64_t* chunk_off,
                     uint32_t* words) {
  uint64_t nchunks = (n + C - 1) / C;
  uint64_t w = 0;
  for (uint64_t j = 0; j < nchunks; ++j) {
    chunk_off[j] = w;
    uint64_t bitpos = 0;
    uint64_t end = std::min<uint64_t>(n, (j + 1) * (uint64_t)C);
    for (uint64_t k = j * (uint64_t)C; k < end; ++k) {
      uint32_t l = len[sym[k]], cw = code[sym[k]];
      for (uint32_t b = 0; b < l; ++b) {
        uint32_t bit = (cw >> (l - 1 - b)) & 1u;
        uint64_t p = bitpos + b;
        if (words) {
          if (p % 32 == 0) words[w + p / 32] = 0;
          words[w + p / 32] |= bit << (31 - p % 32);
        }
      }
      bitpos += l;
    }
    w += (bitpos + 31) / 32;
  }
  return w;
}

// ------------------------------------------------------------------ container
}  // extern "C"

namespace {

// Mask D of the whole volume: threshold -> (largest) -> dilation.
void full_mask(const void* in, const OracleParams* p, uint64_t nx, uint64_t ny, uint64_t nz,
               std::vector<uint8_t>& D) {
  uint64_t N = nx * ny * nz;
  std::vector<uint8_t> T(N);
  D.assign(N, 0);
  oracle_threshold(in, p, nx, ny, nz, T.data());
  if (p->keep) oracle_keep_largest(T.data(), nx, ny, nz, p->connectivity);
  oracle_dilate(T.data(), nx, ny, nz, p->dilate, D.data());
}

// Error-bound constants from the retained values of the volume under D.
void bound_of(const void* in, const OracleParams* p, uint64_t nx, uint64_t ny, uint64_t nz,
              const uint8_t* D, OracleEb* e) {
  uint64_t N = nx * ny * nz, rows = ny * nz;
  size_t esz = p->dtype == DT_F32 ? 4 : 2;
  std::vector<uint8_t> P(N * esz + 4);
  std::vector<uint16_t> counts(rows + 1), bounds(rows * (nx + 1) + 1);
  uint64_t nb = 0;
  uint64_t n = (uint64_t)oracle_compact(in, p->dtype, nx, ny, nz, D, P.data(), counts.data(),
                                        bounds.data(), &nb);
  oracle_eb(P.data(), p->dtype, n, p->eb_mode, p->eb_value, e);
}

// The container of the voxels of `in` (nx x ny x nz) retained by D, with the
// error-bound constants e: compact -> quantise -> predict -> histogram ->
// codebook -> pack -> container. *out is malloc'd.
int encode_container(const void* in, const OracleParams* p, uint64_t nx, uint64_t ny,
                     uint64_t nz, const uint8_t* D, const OracleEb& e, uint8_t** out,
                     uint64_t* out_size) {
  uint64_t N = nx * ny * nz, rows = ny * nz;
  uint32_t R = p->radius, S = 2 * R, C = p->chunk;
  size_t esz = p->dtype == DT_F32 ? 4 : 2;
  std::vector<uint8_t> P(N * esz + 4);
  std::vector<uint16_t> counts(rows + 1), bounds(rows * (nx + 1) + 1);
  uint64_t nb = 0;
  uint64_t n = (uint64_t)oracle_compact(in, p->dtype, nx, ny, nz, D, P.data(),
                                        counts.data(), bounds.data(), &nb);
  std::vector<int32_t> q(n + 1);
  std::vector<uint8_t> ol(n + 1);
  oracle_quantize(P.data(), p->dtype, n, &e, p->dark, q.data(), ol.data());
  std::vector<uint16_t> sym(n + 1);
  std::vector<uint64_t> rk(n + 1);
  std::vector<uint32_t> rv(n + 1);
  uint64_t nout = oracle_lorenzo(q.data(), ol.data(), P.data(), p->dtype, n, R, order_of(p),
                                 sym.data(), rk.data(), rv.data());
  std::vector<uint64_t> hist(S);
  oracle_histogram(sym.data(), n, S, hist.data());
  std::vector<uint8_t> len(S);
  std::vector<uint32_t> code(S);
  oracle_codebook(hist.data(), S, len.data(), code.data());
  uint64_t nchunks = (n + C - 1) / C;
  std::vector<uint64_t> coff(nchunks + 1);
  uint64_t nwords = oracle_pack(sym.data(), n, len.data(), code.data(), C, coff.data(), nullptr);
  std::vector<uint32_t> words(nwords + 1);
  oracle_pack(sym.data(), n, len.data(), code.data(), C, coff.data(), words.data());

  uint64_t off_lens = kHeaderBytes;
  uint64_t off_counts = align16(off_lens + S);
  uint64_t off_bounds = align16(off_counts + 2 * rows);
  uint64_t off_outk = align16(off_bounds + 2 * nb);
  uint64_t off_outv = align16(off_outk + 8 * nout);
  uint64_t off_chunks = align16(off_outv + 4 * nout);
  uint64_t off_payload = align16(off_chunks + 8 * nchunks);
  uint64_t total = align16(off_payload + 4 * nwords);

  Buf o;
  o.b.assign(total, 0);
  std::memcpy(&o.b[0], "ROIX", 4);
  o.put<uint16_t>(4, 1);
  o.put<uint8_t>(6, (uint8_t)p->dtype);
  o.put<uint8_t>(7, (uint8_t)p->eb_mode);
  o.put<uint32_t>(8, (uint32_t)nx);
  o.put<uint32_t>(12, (uint32_t)ny);
  o.put<uint32_t>(16, (uint32_t)nz);
  o.put<uint8_t>(20, (uint8_t)p->cmp);
  o.put<uint8_t>(21, (uint8_t)p->keep);
  o.put<uint8_t>(22, (uint8_t)p->connectivity);
  o.put<uint8_t>(23, (uint8_t)p->dilate);
  o.put<double>(24, p->threshold);
  o.put<double>(32, p->dark);
  o.put<double>(40, p->fill);
  o.put<double>(48, p->eb_value);
  o.put<double>(56, e.eb_abs);
  o.put<float>(64, e.two_eb);
  o.put<float>(68, e.inv2eb);
  o.put<float>(72, e.bound);
  o.put<int32_t>(76, e.eb_int);
  o.put<uint32_t>(80, R);
  o.put<uint32_t>(84, C);
  o.put<uint32_t>(88, kLMax);
  o.put<uint32_t>(92, order_of(p));
  o.put<uint64_t>(96, n);
  o.put<uint64_t>(104, nout);
  o.put<uint64_t>(112, nb);
  o.put<uint64_t>(120, nchunks);
  o.put<uint64_t>(128, nwords);
  o.put<double>(136, e.vmin);
  o.put<double>(144, e.vmax);
  o.put<uint64_t>(152, off_lens);
  o.put<uint64_t>(160, off_counts);
  o.put<uint64_t>(168, off_bounds);
  o.put<uint64_t>(176, off_outk);
  o.put<uint64_t>(184, off_outv);
  o.put<uint64_t>(192, off_chunks);
  o.put<uint64_t>(200, off_payload);
  o.put<uint64_t>(208, total);
  std::memcpy(&o.b[off_lens], len.data(), S);
  if (rows) std::memcpy(&o.b[off_counts], counts.data(), 2 * rows);
  if (nb) std::memcpy(&o.b[off_bounds], bounds.data(), 2 * nb);
  if (nout) {
    std::memcpy(&o.b[off_outk], rk.data(), 8 * nout);
    std::memcpy(&o.b[off_outv], rv.data(), 4 * nout);
  }
  if (nchunks) std::memcpy(&o.b[off_chunks], coff.data(), 8 * nchunks);
  if (nwords) std::memcpy(&o.b[off_payload], words.data(), 4 * nwords);

  *out = (uint8_t*)std::malloc(total);
  std::memcpy(*out, o.b.data(), total);
  *out_size = total;
  return ERR_OK;
}

}  // namespace

extern "C" {

// Whole compression path: mask, error bound, container. On success *out is a
// malloc'd buffer (free with oracle_free).
int oracle_compress(const void* in, const OracleParams* p, uint64_t nx,
                    uint64_t ny, uint64_t nz, uint8_t** out, uint64_t* out_size) {
  *out = nullptr;
  *out_size = 0;
  if (p->dtype != DT_F32 && p->dtype != DT_U16) return ERR_INVAL;  // linear quantiser only
  std::vector<uint8_t> D;
  full_mask(in, p, nx, ny, nz, D);
  OracleEb e;
  bound_of(in, p, nx, ny, nz, D.data(), &e);
  return encode_container(in, p, nx, ny, nz, D.data(), e, out, out_size);
}

// A volume in z-slabs of slab_z slices (the last may be shorter), one
// container per slab: the mask is the whole volume's (the dilation crosses
// slab borders), the error bound comes from the retained values of the whole
// volume, and each slab's stream starts afresh. keep = 1 is refused (a slab
// is not a volume of its own). outs[s] / sizes[s] for s < ceil(nz / slab_z).
int oracle_compress_slabs(const void* in, const OracleParams* p, uint64_t nx, uint64_t ny,
                          uint64_t nz, uint64_t slab_z, uint8_t** outs, uint64_t* sizes) {
  if (p->dtype != DT_F32 && p->dtype != DT_U16) return ERR_INVAL;
  if (p->keep || slab_z == 0) return ERR_INVAL;
  std::vector<uint8_t> D;
  full_mask(in, p, nx, ny, nz, D);
  OracleEb e;
  bound_of(in, p, nx, ny, nz, D.data(), &e);
  const uint64_t plane = nx * ny;
  const size_t esz = p->dtype == DT_F32 ? 4 : 2;
  for (uint64_t z0 = 0, s = 0; z0 < nz; z0 += slab_z, ++s) {
    const uint64_t dz = std::min(slab_z, nz - z0);
    int rc = encode_container((const uint8_t*)in + z0 * plane * esz, p, nx, ny, dz,
                              D.data() + z0 * plane, e, &outs[s], &sizes[s]);
    if (rc) return rc;
  }
  return ERR_OK;
}

// One z-slab of a larger volume (Sec. 4.2.2-4.3 per slab, as in
// oracle_compress_slabs) from the slab's slices alone: `in` holds nz_buf
// slices, the slab's dz slices starting at slice z0 of the buffer, with the
// volume's neighbouring slice before (z0 = 1) and after (z0 + dz < nz_buf)
// when the volume has them. The mask is threshold -> dilation over the buffer
// (the dilation of a slab voxel reads only its neighbouring slices, so these
// voxels get the whole volume's mask), the error-bound constants e are the
// whole volume's (its retained range), and the container is encoded from the
// slab's slices. keep = 1 is refused.
int oracle_encode_slab(const void* in, const OracleParams* p, uint64_t nx, uint64_t ny,
                       uint64_t nz_buf, uint64_t z0, uint64_t dz, const OracleEb* e,
                       uint8_t** out, uint64_t* out_size) {
  *out = nullptr;
  *out_size = 0;
  if (p->dtype != DT_F32 && p->dtype != DT_U16) return ERR_INVAL;
  if (p->keep || dz == 0 || z0 > 1 || z0 + dz > nz_buf || nz_buf > z0 + dz + 1) return ERR_INVAL;
  std::vector<uint8_t> D;
  full_mask(in, p, nx, ny, nz_buf, D);
  const uint64_t plane = nx * ny;
  const size_t esz = p->dtype == DT_F32 ? 4 : 2;
  return encode_container((const uint8_t*)in + z0 * plane * esz, p, nx, ny, dz,
                          D.data() + z0 * plane, *e, out, out_size);
}

void oracle_free(void* p) { std::free(p); }

// ----------------------------------------------------------------- decoding
// Sec. 4.3, decompression: rebuild the codes from the symbols (prefix sum of
// the deltas, records overriding), dequantise, restore every row from the
// geometry, and fill the rest with the background value. Every read is
// checked against the buffer; inconsistencies return ERR_CORRUPT.
int oracle_decode(const uint8_t* buf, uint64_t size, void* outv, int32_t dtype,
                  uint64_t nx, uint64_t ny, uint64_t nz) {
  auto get = [&](uint64_t off, void* dst, uint64_t bytes) -> bool {
    if (off > size || bytes > size - off) return false;
    std::memcpy(dst, buf + off, bytes);
    return true;
  };
  if (dtype != DT_F32 && dtype != DT_U16) return ERR_INVAL;
  if (size < kHeaderBytes || std::memcmp(buf, "ROIX", 4) != 0) return ERR_CORRUPT;
  uint16_t version; uint8_t dt;
  uint32_t hx, hy, hz, R, C, lmax;
  double dark, fill; float two_eb; int32_t eb_int;
  uint64_t n, nout, nb, nchunks, nwords, off_lens, off_counts, off_bounds,
      off_outk, off_outv, off_chunks, off_payload, total;
  get(4, &version, 2); get(6, &dt, 1);
  get(8, &hx, 4); get(12, &hy, 4); get(16, &hz, 4);
  get(32, &dark, 8); get(40, &fill, 8); get(64, &two_eb, 4); get(76, &eb_int, 4);
  uint32_t order = 0;
  get(80, &R, 4); get(84, &C, 4); get(88, &lmax, 4); get(92, &order, 4);
  get(96, &n, 8); get(104, &nout, 8); get(112, &nb, 8); get(120, &nchunks, 8);
  get(128, &nwords, 8);
  get(152, &off_lens, 8); get(160, &off_counts, 8); get(168, &off_bounds, 8);
  get(176, &off_outk, 8); get(184, &off_outv, 8); get(192, &off_chunks, 8);
  get(200, &off_payload, 8); get(208, &total, 8);
  if (version != 1 || dt != dtype || hx != nx || hy != ny || hz != nz) return ERR_CORRUPT;
  if (total > size || lmax != kLMax || R < 2 || R > 32768 || C == 0) return ERR_CORRUPT;
  if (order > 2) return ERR_CORRUPT;
  if (order == 0) order = 1;
  uint64_t N = nx * ny * nz, rows = ny * nz, S = 2ull * R;
  if (dtype == DT_U16 && !(fill >= 0.0 && fill <= 65535.0 && fill == std::floor(fill)))
    return ERR_CORRUPT;
  if (n > N || nout > n || nb > rows * (nx + 1)) return ERR_CORRUPT;
  if (nchunks != (n + C - 1) / C) return ERR_CORRUPT;
  std::vector<uint8_t> len(S);
  std::vector<uint16_t> counts(rows + 1), bounds(nb + 1);
  std::vector<uint64_t> rk(nout + 1), coff(nchunks + 1);
  std::vector<uint32_t> rv(nout + 1);
  if (!get(off_lens, len.data(), S) || !get(off_counts, counts.data(), 2 * rows) ||
      !get(off_bounds, bounds.data(), 2 * nb) || !get(off_outk, rk.data(), 8 * nout) ||
      !get(off_outv, rv.data(), 4 * nout) || !get(off_chunks, coff.data(), 8 * nchunks))
    return ERR_CORRUPT;
  if (off_payload > size || nwords > (size - off_payload) / 4) return ERR_CORRUPT;
  const uint8_t* payload = buf + off_payload;
  // canonical code table from the lengths
  uint32_t count[kLMax + 2] = {0};
  for (uint64_t s = 0; s < S; ++s) {
    if (len[s] > kLMax) return ERR_CORRUPT;
    count[len[s]]++;
  }
  count[0] = 0;
  uint32_t first[kLMax + 2] = {0}, index0[kLMax + 2] = {0};
  std::vector<uint32_t> by_code;  // symbols in canonical order
  for (uint32_t l = 1; l <= kLMax; ++l)
    for (uint64_t s = 0; s < S; ++s)
      if (len[s] == l) by_code.push_back((uint32_t)s);
  {
    uint32_t c = 0, idx = 0;
    for (uint32_t l = 1; l <= kLMax; ++l) {
      c = (c + count[l - 1]) << 1;
      first[l] = c;
      index0[l] = idx;
      idx += count[l];
    }
  }
  // symbols
  std::vector<uint16_t> sym(n + 1);
  for (uint64_t j = 0; j < nchunks; ++j) {
    uint64_t w0 = coff[j];
    uint64_t wend = (j + 1 < nchunks) ? coff[j + 1] : nwords;
    if (w0 > wend || wend > nwords) return ERR_CORRUPT;
    uint64_t bitpos = 0, nbits = 32 * (wend - w0);
    uint64_t end = std::min<uint64_t>(n, (j + 1) * (uint64_t)C);
    for (uint64_t k = j * (uint64_t)C; k < end; ++k) {
      uint32_t c = 0;
      bool found = false;
      for (uint32_t l = 1; l <= kLMax; ++l) {
        if (bitpos >= nbits) return ERR_CORRUPT;
        uint64_t p = bitpos++;
        uint32_t word;
        std::memcpy(&word, payload + 4 * (w0 + p / 32), 4);
        c = (c << 1) | ((word >> (31 - p % 32)) & 1u);
        if (count[l] && c >= first[l] && c - first[l] < count[l]) {
          sym[k] = (uint16_t)by_code[index0[l] + (c - first[l])];
          found = true;
          break;
        }
      }
      if (!found) return ERR_CORRUPT;
    }
  }
  // codes from the deltas; records override
  std::vector<int32_t> q(n + 1);
  std::vector<uint8_t> raw_kind(n + 1, 0);
  std::vector<uint32_t> raw_bits(n + 1, 0);
  uint64_t r = 0;
  int64_t prev1 = 0, prev2 = 0;
  for (uint64_t k = 0; k < n; ++k) {
    int64_t c;
    if (sym[k] != 0) {
      if (sym[k] >= S) return ERR_CORRUPT;
      const int64_t pred = order == 2 ? 2 * prev1 - prev2 : prev1;
      c = pred + (int64_t)sym[k] - (int64_t)R;
      if (c < INT32_MIN || c > INT32_MAX) return ERR_CORRUPT;
    } else {
      if (r >= nout || (rk[r] & ~(uint64_t(1) << 63)) != k) return ERR_CORRUPT;
      if (rk[r] >> 63) {
        c = 0;
        raw_kind[k] = 1;
        raw_bits[k] = rv[r];
      } else {
        c = (int32_t)rv[r];
      }
      r++;
    }
    q[k] = (int32_t)c;
    prev2 = prev1;
    prev1 = c;
  }
  if (r != nout) return ERR_CORRUPT;
  // rows from the geometry
  uint64_t k = 0, b = 0;
  for (uint64_t row = 0; row < rows; ++row) {
    uint16_t cnt = counts[row];
    if (cnt % 2 || b + cnt > nb) return ERR_CORRUPT;
    uint64_t x = 0;
    for (uint32_t i = 0; i <= cnt; i += 2) {
      uint64_t xs = i < cnt ? bounds[b + i] : nx;
      uint64_t xe = i < cnt ? bounds[b + i + 1] : nx;
      if (xs < x || xe < xs || xe > nx) return ERR_CORRUPT;
      for (; x < xs; ++x) {
        if (dtype == DT_F32) ((float*)outv)[row * nx + x] = (float)fill;
        else ((uint16_t*)outv)[row * nx + x] = (uint16_t)fill;
      }
      for (; x < xe; ++x, ++k) {
        if (k >= n) return ERR_CORRUPT;
        if (dtype == DT_F32) {
          float v;
          if (raw_kind[k]) std::memcpy(&v, &raw_bits[k], 4);
          else v = (float)q[k] * two_eb;
          ((float*)outv)[row * nx + x] = v;
        } else {
          int64_t v = (eb_int == 0 ? (int64_t)q[k] : 2 * (int64_t)eb_int * q[k]) + (int64_t)dark;
          v = std::min<int64_t>(65535, std::max<int64_t>(0, v));
          ((uint16_t*)outv)[row * nx + x] = (uint16_t)v;
        }
      }
    }
    b += cnt;
  }
  if (k != n || b != nb) return ERR_CORRUPT;
  return ERR_OK;
}

// ------------------------------------------- 8-bit normalisation (Sec. 4.1.2)
// I_n = I / I_max * 255 on the background-subtracted values (Sec. 4.1.1):
// v = x (float32) or raw - dark (uint16); negative and non-finite values are
// taken as 0; I_max = the largest v of the image (0 maps every pixel to 0).
// The paper leaves the arithmetic open. float32: the formula in its own order
// in binary32, fl(fl(v / I_max) * 255), rounded half to even; uint16: the exact
// rational 255 v / I_max rounded half to even (integer arithmetic). Returns
// I_max.
double oracle_normalize8(const void* in, int32_t dtype, uint64_t count, double dark,
                         uint8_t* out) {
  if (dtype == DT_F32) {
    const float* x = (const float*)in;
    auto value = [&](uint64_t i) -> float {
      const float f = x[i];
      return (std::isfinite(f) && f > 0.0f) ? f : 0.0f;
    };
    float imax = 0.0f;
    for (uint64_t i = 0; i < count; ++i) imax = std::max(imax, value(i));
    for (uint64_t i = 0; i < count; ++i) {
      float q = 0.0f;
      if (imax > 0.0f) {
        volatile float ratio = value(i) / imax;  // one rounding per operation
        volatile float scaled = ratio * 255.0f;
        q = std::nearbyint((float)scaled);
      }
      out[i] = (uint8_t)std::min(255.0f, q);
    }
    return (double)imax;
  }
  const uint16_t* raw = (const uint16_t*)in;
  const int64_t dk = (int64_t)dark;
  auto value = [&](uint64_t i) -> int64_t {
    const int64_t v = (int64_t)raw[i] - dk;
    return v > 0 ? v : 0;
  };
  int64_t imax = 0;
  for (uint64_t i = 0; i < count; ++i) imax = std::max(imax, value(i));
  for (uint64_t i = 0; i < count; ++i) {
    int64_t q = 0;
    if (imax > 0) {
      const int64_t num = 255 * value(i);
      q = num / imax;
      const int64_t r2 = 2 * (num - q * imax);
      if (r2 > imax || (r2 == imax && (q & 1))) ++q;  // half to even
    }
    out[i] = (uint8_t)q;
  }
  return (double)imax;
}

// ------------------------------------ greedy error-bounded quantiser (Sec. 4.2.3)
// The paper's steps on one pixel sequence D (Step 1 bounds, Step 2 init,
// Step 3 running intersection, Step 4 final group, Step 5 clip), with Q
// restricted to integers as it is stored in 8 bits: pixel k accepts the
// integers [ceil(D - E), floor(D + E)]; a group's value is floor((u + l) / 2)
// of its intersection [l, u], hence within every member's bound.
void oracle_greedy_seq(const uint8_t* D, uint64_t m, double eabs, uint8_t* Q) {
  const int64_t e = (int64_t)std::floor(eabs);
  int64_t l = 0, u = 0;
  uint64_t head = 0;
  bool open = false;
  for (uint64_t i = 0; i < m; ++i) {
    const int64_t lo = (int64_t)D[i] - e, hi = (int64_t)D[i] + e;
    if (!open) {
      l = lo;
      u = hi;
      head = i;
      open = true;
      continue;
    }
    const int64_t ln = std::max(l, lo), un = std::min(u, hi);
    if (un < ln) {  // no overlap: close the group
      const int64_t q = floor_div(u + l, 2);
      for (uint64_t j = head; j < i; ++j) Q[j] = (uint8_t)std::min<int64_t>(255, std::max<int64_t>(0, q));
      l = lo;
      u = hi;
      head = i;
    } else {
      l = ln;
      u = un;
    }
  }
  if (open) {
    const int64_t q = floor_div(u + l, 2);
    for (uint64_t j = head; j < m; ++j) Q[j] = (uint8_t)std::min<int64_t>(255, std::max<int64_t>(0, q));
  }
}

// Every row's retained pixels (mask D, one byte per voxel) form one sequence
// P(i) (Sec. 4.2.2); Q holds the quantised pixel section in voxel order.
uint64_t oracle_greedy_rows(const uint8_t* img, const uint8_t* mask, uint64_t nx, uint64_t ny,
                            uint64_t nz, double eabs, uint8_t* Q) {
  std::vector<uint8_t> seq(nx + 1);
  uint64_t n = 0;
  for (uint64_t r = 0; r < ny * nz; ++r) {
    uint64_t m = 0;
    for (uint64_t x = 0; x < nx; ++x)
      if (mask[r * nx + x]) seq[m++] = img[r * nx + x];
    oracle_greedy_seq(seq.data(), m, eabs, Q + n);
    n += m;
  }
  return n;
}

}  // extern "C"
