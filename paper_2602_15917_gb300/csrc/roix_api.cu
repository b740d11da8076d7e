// Host side of libroix: argument checks, workspace planning and the ordered
// kernel launches behind each entry point of include/roix.h.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "roix_internal.cuh"

using namespace roix;


namespace {

// ---------------------------------------------------------- device guard
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

roix_status fail(roix_ctx* ctx, roix_status s, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return s;
}

roix_status cuda_fail(roix_ctx* ctx, cudaError_t e, const char* where) {
  return fail(ctx, ROIX_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// --------------------------------------------------------------- arena
struct Arena {
  size_t off = 0;
  size_t take(size_t bytes, size_t align = 256) {
    off = (off + align - 1) / align * align;
    size_t o = off;
    off += bytes;
    return o;
  }
};

constexpr size_t kStateBytes = 256;
static_assert(sizeof(State) <= kStateBytes, "state fits its slot");

}  // namespace

void roix::borrow_ws(roix_ctx* ctx, char* ws, size_t bytes) {
  if (ctx->ws && !ctx->ws_borrowed) {
    cudaDeviceSynchronize();
    cudaFree(ctx->ws);
  }
  ctx->ws = ws;
  ctx->ws_bytes = bytes;
  ctx->ws_borrowed = true;
}

roix_status roix::ensure_ws(roix_ctx* ctx, size_t bytes, bool exact) {
  if (bytes <= ctx->ws_bytes) return ROIX_OK;
  if (ctx->ws_borrowed)
    return fail(ctx, ROIX_ENOMEM, "the borrowed workspace holds " +
                                      std::to_string(ctx->ws_bytes) + " bytes, " +
                                      std::to_string(bytes) + " needed");
  if (ctx->ws) {
    // keep an unread device status across the reallocation
    cudaDeviceSynchronize();
    u32 st = 0;
    cudaMemcpy(&st, ctx->ws, 4, cudaMemcpyDeviceToHost);
    if (!ctx->pending) ctx->pending = st;
    cudaFree(ctx->ws);
    ctx->ws = nullptr;
    ctx->ws_bytes = 0;
  }
  size_t want = exact ? bytes : bytes + (bytes >> 3);  // headroom against regrowth
  cudaError_t e = cudaMalloc(&ctx->ws, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    e = cudaMalloc(&ctx->ws, bytes);
    want = bytes;
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    ctx->ws = nullptr;
    return fail(ctx, ROIX_ENOMEM, "workspace allocation of " + std::to_string(bytes) + " bytes failed");
  }
  ctx->ws_bytes = want;
  cudaMemset(ctx->ws, 0, kStateBytes);
  return ROIX_OK;
}

namespace {

// ----------------------------------------------------------- parameters
float f32_round_down(double t) {
  float f = (float)t;
  if ((double)f > t) f = std::nextafterf(f, -INFINITY);
  return f;
}
float f32_round_up(double t) {
  float f = (float)t;
  if ((double)f < t) f = std::nextafterf(f, INFINITY);
  return f;
}

bool dims_ok(roix_dims d) {
  if (d.nx > 65534) return false;
  if (d.ny > 0xffffffffull || d.nz > 0xffffffffull) return false;
  const double N = (double)d.nx * (double)d.ny * (double)d.nz;
  return N < 1.1e12;
}

}  // namespace

// Validates the settings of a call and turns them into the kernel descriptor
// (thresholds converted once, on the host, to the comparisons the kernels do).
roix_status roix::make_desc(roix_ctx* ctx, roix_dtype dtype, roix_dims dims, const roix_roi* roi,
                            const roix_eb* eb, const roix_params* prm, Desc* d) {
  std::memset(d, 0, sizeof(*d));
  if (dtype != ROIX_F32 && dtype != ROIX_U16 && dtype != ROIX_U8)
    return fail(ctx, ROIX_EINVAL, "dtype must be ROIX_F32, ROIX_U16 or ROIX_U8");
  if (dtype == ROIX_U8 && (eb || prm))
    return fail(ctx, ROIX_EINVAL, "uint8 images go through roix_greedy_quantize, not the coder");
  if (!dims_ok(dims)) return fail(ctx, ROIX_EINVAL, "dims: nx <= 65534, ny, nz < 2^32, N < 1.1e12");
  d->nx = dims.nx;
  d->ny = dims.ny;
  d->nz = dims.nz;
  d->rows = dims.ny * dims.nz;
  d->W = (dims.nx + 31) / 32;
  d->N = dims.nx * dims.ny * dims.nz;
  d->dtype = dtype;
  d->front_words = ctx ? ctx->tune.front_words : 2048;
  d->spin_limit = ctx ? ctx->spin_limit : 0u;
  d->hold_scans = ctx ? (ctx->hold_scans ? 1u : 0u) : 0u;
  if (roi) {
    if (roi->cmp != 0 && roi->cmp != 1) return fail(ctx, ROIX_EINVAL, "roi.cmp must be 0 or 1");
    if (roi->keep != 0 && roi->keep != 1) return fail(ctx, ROIX_EINVAL, "roi.keep must be 0 or 1");
    if (roi->connectivity != 6 && roi->connectivity != 26)
      return fail(ctx, ROIX_EINVAL, "roi.connectivity must be 6 or 26");
    if (roi->dilate != 0 && roi->dilate != 1) return fail(ctx, ROIX_EINVAL, "roi.dilate must be 0 or 1");
    d->cmp = roi->cmp;
    d->keep = roi->keep;
    d->conn = roi->connectivity;
    d->dilate = roi->dilate;
    d->threshold = roi->threshold;
    d->dark_d = roi->dark;
    if (dtype == ROIX_F32) {
      if (roi->dark != 0.0) return fail(ctx, ROIX_EINVAL, "roi.dark must be 0 for float32 input");
      d->thr_never = std::isnan(roi->threshold);
      d->thr_f = roi->cmp == 0 ? f32_round_down(roi->threshold) : f32_round_up(roi->threshold);
    } else {
      if (!(roi->dark >= 0.0 && roi->dark <= 65535.0 && roi->dark == std::floor(roi->dark)))
        return fail(ctx, ROIX_EINVAL, "roi.dark must be an integer in [0, 65535]");
      d->dark = (int)roi->dark;
      const double t = roi->threshold;
      d->thr_never = std::isnan(t);
      double ti = roi->cmp == 0 ? std::floor(t) : std::ceil(t);
      if (ti < -1e6) ti = -1e6;
      if (ti > 1e6) ti = 1e6;
      d->thr_i = std::isnan(ti) ? 0 : (int)ti;
    }
  }
  if (eb) {
    if (eb->mode != 0 && eb->mode != 1) return fail(ctx, ROIX_EINVAL, "eb.mode must be 0 or 1");
    const bool lossless_u16 = dtype == ROIX_U16 && eb->mode == 0 && eb->value == 0.0;
    if (!(std::isfinite(eb->value) && (eb->value > 0.0 || lossless_u16)))
      return fail(ctx, ROIX_EINVAL, "eb.value must be finite and > 0");
    d->eb_mode = eb->mode;
    d->eb_value = eb->value;
  }
  if (prm) {
    if (prm->radius < 2 || prm->radius > kMaxRadius)
      return fail(ctx, ROIX_EINVAL, "params.radius must be in [2, 2048]");
    const u32 C = prm->chunk;
    if (C < 256 || C > 16384 || (C & (C - 1)))
      return fail(ctx, ROIX_EINVAL, "params.chunk must be a power of two in [256, 16384]");
    if (dtype == ROIX_U16 &&
        !(prm->fill >= 0.0 && prm->fill <= 65535.0 && prm->fill == std::floor(prm->fill)))
      return fail(ctx, ROIX_EINVAL, "params.fill must be an integer in [0, 65535] for uint16");
    if (prm->predictor > 2) return fail(ctx, ROIX_EINVAL, "params.predictor must be 0, 1 or 2");
    d->R = prm->radius;
    d->S = 2 * prm->radius;
    d->C = C;
    d->fill = prm->fill;
    d->order = prm->predictor == 2 ? 2u : 1u;
  }
  return ROIX_OK;
}

namespace {

bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

size_t dtype_bytes(int dt) { return dt == ROIX_F32 ? 4 : dt == ROIX_U16 ? 2 : 1; }

u32 front_rows_per_tile(const Desc& d) {
  const u64 target_words = d.front_words ? d.front_words : 2048;
  u64 rpt = d.W ? target_words / d.W : 1;
  if (rpt < 1) rpt = 1;
  if (rpt > kMaxTileRows) rpt = kMaxTileRows;
  if (rpt > d.rows) rpt = d.rows ? d.rows : 1;
  return (u32)rpt;
}

// ----------------------------------------------------- compress workspace
// Layout of a batch's workspace: State[n] at offset 0 (state 0's first word is
// the context status), then one zeroed region (look-back flags, histograms of
// every item), then every item's data (look-back values, mask, pixel section,
// symbols, records, code tables).
struct ItemPlan {
  size_t crec, hist, sff, sfp;  // zeroed
  size_t sfa, spa;
  u64 stf, stp;  // scan tiles of the compaction and of the pack
  size_t ftn, ftb, ftno, ftbo, rno, rbo, Dm, cw, cwoff, crecoff, rbits, T, P, sym, lens, codes;
  // largest-component scratch (keep = 1): zeroed flags and counters, then data
  size_t cf, cvars, ca, crr, cro, cxs, cxe, cpar, csize, T2;
  u64 ctiles;
  u64 ftiles, qtiles, pchunks, pranges, rec_cap, n_cap;
  u32 rpt;
};

struct BatchPlan {
  size_t zero_begin = 0, zero_end = 0, total = 0;
  std::vector<ItemPlan> items;
  u64 qtiles = 0, pranges = 0;  // symbol segments, pack chunks
};

BatchPlan plan_batch(const Desc& c, const roix_dims* dims, const u64* n_caps, const u64* caps,
                     u32 n, bool need_T, bool need_P) {
  BatchPlan bp;
  bp.items.resize(n);
  Arena a;
  a.take(sizeof(State) * (n ? n : 1));
  bp.zero_begin = a.take(0);
  const size_t esz = dtype_bytes(c.dtype);
  for (u32 i = 0; i < n; ++i) {
    ItemPlan& p = bp.items[i];
    Desc d = c;
    d.nx = dims[i].nx;
    d.ny = dims[i].ny;
    d.nz = dims[i].nz;
    d.rows = d.ny * d.nz;
    d.W = (d.nx + 31) / 32;
    p.n_cap = n_caps[i];
    p.rpt = front_rows_per_tile(d);
    p.ftiles = d.rows ? (d.rows + p.rpt - 1) / p.rpt : 0;
    p.qtiles = (p.n_cap + kQuantTile - 1) / kQuantTile;
    p.pchunks = c.C ? (p.n_cap + c.C - 1) / c.C : 0;
    p.pranges = (p.pchunks + kPackRange - 1) / kPackRange;
    p.rec_cap = umin(p.n_cap, caps[i] / 12 + 1);
    p.crec = a.take(4 * (p.pchunks + 1));
    p.hist = a.take(8 * (size_t)c.S);
    p.stf = (p.ftiles + kScanTile - 1) / kScanTile;
    p.stp = (p.pchunks + kScanTile - 1) / kScanTile;
    p.sff = a.take(4 * (p.stf + 1));
    p.sfp = a.take(4 * (p.stp + 1));
    if (c.keep) {
      const u64 rows = dims[i].ny * dims[i].nz;
      p.ctiles = (rows + 2047) / 2048;
      p.cf = a.take(4 * (p.ctiles + 1));
      p.cvars = a.take(64);  // total, best, best_root, tickets
    }
    bp.qtiles += p.qtiles;
    bp.pranges += p.pranges;
  }
  bp.zero_end = a.take(0);
  for (u32 i = 0; i < n; ++i) {
    ItemPlan& p = bp.items[i];
    const u64 rows = dims[i].ny * dims[i].nz, W = (dims[i].nx + 31) / 32;
    p.sfa = a.take(8 * 2 * 2 * (p.stf + 1));
    p.spa = a.take(8 * 2 * 2 * (p.stp + 1));
    p.ftn = a.take(4 * (p.ftiles + 1));
    p.ftb = a.take(4 * (p.ftiles + 1));
    p.ftno = a.take(8 * (p.ftiles + 1));
    p.ftbo = a.take(8 * (p.ftiles + 1));
    p.Dm = c.dilate ? a.take(4 * rows * W + 16) : 0;
    p.rno = a.take(4 * rows + 16);
    p.rbo = a.take(4 * rows + 16);
    p.cw = a.take(4 * (p.pchunks + 1));
    p.cwoff = a.take(8 * (p.pchunks + 1));
    p.crecoff = a.take(8 * (p.pchunks + 1));
    p.rbits = a.take(4 * (p.n_cap / 32 + 2));
    p.T = need_T ? a.take(4 * rows * W + 16) : 0;
    p.P = need_P ? a.take(esz * p.n_cap + 16) : 0;
    p.sym = a.take(2 * p.n_cap + 16);
    p.lens = a.take(c.S + 16);
    p.codes = a.take(4 * (size_t)c.S + 16);  // (copied in 16-byte units)
    if (c.keep) {
      Desc di = c;
      di.nx = dims[i].nx;
      di.rows = rows;
      const u64 maxr = ccl_max_runs(di);
      p.ca = a.take(8 * 2 * (p.ctiles + 1));
      p.crr = a.take(4 * rows + 16);
      p.cro = a.take(8 * rows + 16);
      p.cxs = a.take(2 * maxr + 16);
      p.cxe = a.take(2 * maxr + 16);
      p.cpar = a.take(4 * maxr + 16);
      p.csize = a.take(8 * maxr + 16);
      p.T2 = a.take(4 * rows * W + 16);
    }
  }
  bp.total = a.take(0);
  return bp;
}

template <int NV>
LookBack<NV> lb_at(char* ws, size_t flags, size_t data, u64 tiles) {
  LookBack<NV> lb;
  lb.flags = (u32*)(ws + flags);
  lb.agg = (u64*)(ws + data);
  lb.inc = (u64*)(ws + data) + NV * (tiles + 1);
  return lb;
}

bool rows_vector_aligned(const void* in, roix_dtype dt, u64 nx) {
  if (((uintptr_t)in & 15) != 0) return false;
  return (nx * dtype_bytes(dt)) % 16 == 0;
}

// Fills the batch structure for items [first, first + n) of the plan;
// pointers into `ws`. Item fields for outputs and inputs are set by the
// caller. The batch's work tickets live in the state of its first item (all
// states but the context status word are zeroed per call).
void fill_batch(Batch& B, const Desc& c, const BatchPlan& bp, const roix_dims* dims, char* ws,
                u32 n, u32 first = 0) {
  std::memset(&B, 0, sizeof(B));
  B.c = c;
  B.n = n;
  State* st = (State*)ws;
  B.status = &st[0].status;
  B.ctr = &st[first].ctr_front;
  u64 seg = 0, ft = 0, rw = 0;
  for (u32 i = 0; i < n; ++i) {
    const ItemPlan& p = bp.items[first + i];
    Item& I = B.it[i];
    I.nx = dims[first + i].nx;
    I.ny = dims[first + i].ny;
    I.nz = dims[first + i].nz;
    I.rows = I.ny * I.nz;
    I.W = (I.nx + 31) / 32;
    I.N = p.n_cap;
    I.st = st + first + i;
    I.rst = I.st;
    I.T = p.T ? (u32*)(ws + p.T) : nullptr;
    I.P = p.P ? (void*)(ws + p.P) : nullptr;
    I.sym = (uint16_t*)(ws + p.sym);
    I.rec_cap = p.rec_cap;
    I.hist = (unsigned long long*)(ws + p.hist);
    I.lens = (uint8_t*)(ws + p.lens);
    I.codes = (u32*)(ws + p.codes);
    I.sizes = &I.st->n;
    I.lbsf = lb_at<2>(ws, p.sff, p.sfa, p.stf);
    I.lbsp = lb_at<2>(ws, p.sfp, p.spa, p.stp);
    I.ftn = (u32*)(ws + p.ftn);
    I.ftb = (u32*)(ws + p.ftb);
    I.ftno = (u64*)(ws + p.ftno);
    I.ftbo = (u64*)(ws + p.ftbo);
    I.D = p.Dm ? (u32*)(ws + p.Dm) : nullptr;
    I.rno = (u32*)(ws + p.rno);
    I.rbo = (u32*)(ws + p.rbo);
    I.crec = (u32*)(ws + p.crec);
    I.cw = (u32*)(ws + p.cw);
    I.cwoff = (u64*)(ws + p.cwoff);
    I.crecoff = (u64*)(ws + p.crecoff);
    I.rbits = (u32*)(ws + p.rbits);
    I.rpt = p.rpt;
    I.m_rpt = recip64(p.rpt);
    I.m_ny = recip64(I.ny);
    I.ftiles = p.ftiles;
    I.fscan = p.ftiles <= kInScanMax ? 1u : 0u;
    I.pscan = p.pchunks <= kInScanMax ? 1u : 0u;
    B.seg0[i] = seg;
    B.ftile0[i] = ft;
    B.row0[i] = rw;
    seg += I.rows * ((I.nx + 1023) / 1024);
    ft += p.ftiles;
    rw += I.rows;
  }
  B.seg0[n] = seg;
  B.ftile0[n] = ft;
  B.row0[n] = rw;
}

}  // namespace

// Binarisation work units: 1024-voxel row segments when the rows are 16-byte
// aligned and fill whole segments (nx a multiple of 1024) or are short (nx <
// 256); kFlatSpan-voxel steps of the flat array for any other 16-byte aligned
// volume.
void roix::set_threshold_units(Batch& B) {
  constexpr u64 kFlatSpanHost = 1024;
  u64 seg = 0, fseg = 0;
  for (u32 i = 0; i < B.n; ++i) {
    Item& I = B.it[i];
    const roix_dtype dt = (roix_dtype)B.c.dtype;
    I.vec = rows_vector_aligned(I.in, dt, I.nx) ? 1u : 0u;
    I.flat = (!(I.vec && I.nx % 1024 == 0) && I.nx >= 256 && aligned(I.in, 16)) ? 1u : 0u;
    I.m_nx = recip64(I.nx);
    I.m_spr = recip64((I.nx + 1023) / 1024);
    B.seg0[i] = seg;
    B.fseg0[i] = fseg;
    const u64 N = I.nx * I.ny * I.nz;
    if (I.flat) fseg += (N + kFlatSpanHost - 1) / kFlatSpanHost;
    else seg += I.rows * ((I.nx + 1023) / 1024);
  }
  B.seg0[B.n] = seg;
  B.fseg0[B.n] = fseg;
}

// One-item batch for the binarisation kernel alone.
void roix::make_threshold_batch(Batch& B, const Desc& d, const void* in, u32* T) {
  std::memset(&B, 0, sizeof(B));
  B.c = d;
  B.n = 1;
  Item& I = B.it[0];
  I.nx = d.nx;
  I.ny = d.ny;
  I.nz = d.nz;
  I.rows = d.rows;
  I.W = d.W;
  I.N = d.N;
  I.in = in;
  I.T = T;
  set_threshold_units(B);
}

namespace {

CclWs ccl_ws(char* ws, const ItemPlan& p, u32* status) {
  CclWs w;
  w.row_runs = (u32*)(ws + p.crr);
  w.row_off = (u64*)(ws + p.cro);
  w.xs = (uint16_t*)(ws + p.cxs);
  w.xe = (uint16_t*)(ws + p.cxe);
  w.par = (u32*)(ws + p.cpar);
  w.size = (unsigned long long*)(ws + p.csize);
  w.total = (u64*)(ws + p.cvars);
  w.best = (unsigned long long*)(ws + p.cvars + 8);
  w.best_root = (u32*)(ws + p.cvars + 16);
  w.ctr = (u32*)(ws + p.cvars + 20);
  w.lb = lb_at<1>(ws, p.cf, p.ca, p.ctiles);
  w.status = status;
  return w;
}

bool ccl_fits(const Desc& d) { return ccl_max_runs(d) < 0xffffffffull; }

Desc item_desc(const Desc& c, const Item& I) {
  Desc d = c;
  d.nx = I.nx;
  d.ny = I.ny;
  d.nz = I.nz;
  d.rows = I.rows;
  d.W = I.W;
  d.N = I.N;
  return d;
}

// Output side of a fused item: geometry written straight into the container.
void set_container(Item& I, const Desc& c, void* out, u64 cap, u64* size_dev) {
  const Layout lo = make_layout(c.S, I.rows, 0, 0, 0, 0);
  uint8_t* o = (uint8_t*)out;
  I.out = o;
  I.cap = cap;
  I.size_dev = size_dev;
  I.counts = (uint16_t*)(o + lo.off_counts);
  I.counts_cap = cap > lo.off_counts ? (cap - lo.off_counts) / 2 : 0;
  I.bounds = (uint16_t*)(o + lo.off_bounds);
  I.bounds_cap = cap > lo.off_bounds ? (cap - lo.off_bounds) / 2 : 0;
}

// profiling marks: an event after each stage when profiling is on
void mark(roix_ctx* ctx, cudaStream_t s) {
  if (!ctx->profile || ctx->nev >= 16) return;
  if (!ctx->ev[ctx->nev]) cudaEventCreate(&ctx->ev[ctx->nev]);
  cudaEventRecord(ctx->ev[ctx->nev], s);
  ctx->nev++;
}

}  // namespace


extern "C" {

const char* roix_status_string(roix_status s) {
  switch (s) {
    case ROIX_OK: return "ok";
    case ROIX_EINVAL: return "invalid argument";
    case ROIX_ENOMEM: return "out of device memory";
    case ROIX_ECAPACITY: return "output buffer too small";
    case ROIX_ECORRUPT: return "corrupt container";
    case ROIX_ETIMEOUT: return "inter-block wait timed out";
    case ROIX_ECUDA: return "CUDA error";
    case ROIX_EBUSY: return "busy";
  }
  return "unknown status";
}

roix_status roix_ctx_create(int device, roix_ctx** out) {
  if (!out) return ROIX_EINVAL;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
    cudaGetLastError();
    return ROIX_ECUDA;
  }
  roix_ctx* c = new roix_ctx();
  c->device = device;
  DeviceGuard g(device);
  cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device);
  if (c->sms <= 0) c->sms = 1;
  *out = c;
  return ROIX_OK;
}

roix_status roix_ctx_destroy(roix_ctx* ctx) {
  if (!ctx) return ROIX_EINVAL;
  DeviceGuard g(ctx->device);
  if (ctx->ws && !ctx->ws_borrowed) {
    cudaDeviceSynchronize();
    cudaFree(ctx->ws);
  }
  for (auto& e : ctx->ev)
    if (e) cudaEventDestroy(e);
  delete ctx;
  return ROIX_OK;
}

roix_status roix_reserve(roix_ctx* ctx, size_t bytes) {
  if (!ctx) return ROIX_EINVAL;
  DeviceGuard g(ctx->device);
  return ensure_ws(ctx, bytes < kStateBytes ? kStateBytes : bytes, true);
}

const char* roix_last_error(const roix_ctx* ctx) { return ctx ? ctx->err.c_str() : ""; }

uint64_t roix_mask_words(roix_dims d) { return d.ny * d.nz * ((d.nx + 31) / 32); }

uint64_t roix_compress_bound(roix_dtype dtype, roix_dims dims, const roix_params* prm) {
  (void)dtype;
  const u32 R = prm ? prm->radius : 512, C = prm && prm->chunk ? prm->chunk : 4096;
  const u64 N = dims.nx * dims.ny * dims.nz, rows = dims.ny * dims.nz;
  const u64 nch = (N + C - 1) / C;
  const u64 nw = (N * kLMax + 31) / 32 + nch;
  return make_layout(2ull * R, rows, rows * (dims.nx + 1), N, nch, nw).total;
}

size_t roix_workspace_size(roix_dtype dtype, roix_dims dims, const roix_roi* roi,
                           const roix_params* params, uint64_t cap) {
  Desc d;
  if (make_desc(nullptr, dtype, dims, roi, nullptr, params, &d) != ROIX_OK) return 0;
  const u64 ncap = d.N, cap64 = cap;
  return plan_batch(d, &dims, &ncap, &cap64, 1, true, true).total;
}

roix_status roix_sync(roix_ctx* ctx, void* stream) {
  if (!ctx) return ROIX_EINVAL;
  DeviceGuard g(ctx->device);
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "stream synchronize");
  u32 st = ctx->pending;
  ctx->pending = 0;
  if (ctx->ws) {
    u32 dev = 0;
    e = cudaMemcpy(&dev, ctx->ws, 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "status read");
    if (dev) {
      const u32 zero = 0;
      cudaMemcpy(ctx->ws, &zero, 4, cudaMemcpyHostToDevice);
    }
    if (!st) st = dev;
  }
  if (st) {
    ctx->err = std::string("device reported: ") + roix_status_string((roix_status)st);
    return (roix_status)st;
  }
  return ROIX_OK;
}

roix_status roix_set_wait_limit(roix_ctx* ctx, uint32_t polls) {
  if (!ctx) return ROIX_EINVAL;
  ctx->spin_limit = polls;
  return ROIX_OK;
}

roix_status roix_debug_hold_scans(roix_ctx* ctx, int on) {
  if (!ctx) return ROIX_EINVAL;
  ctx->hold_scans = on ? 1 : 0;
  return ROIX_OK;
}

// Profiling: when on, the fused path records an event after every stage; the
// stage durations of the last call are read with roix_profile_read.
roix_status roix_profile(roix_ctx* ctx, int on) {
  if (!ctx) return ROIX_EINVAL;
  ctx->profile = on;
  return ROIX_OK;
}

int roix_profile_read(roix_ctx* ctx, float* ms, int max) {
  if (!ctx || ctx->nev < 2) return 0;
  DeviceGuard g(ctx->device);
  int k = 0;
  for (int i = 1; i < ctx->nev && k < max; ++i, ++k) {
    cudaEventSynchronize(ctx->ev[i]);
    cudaEventElapsedTime(&ms[k], ctx->ev[i - 1], ctx->ev[i]);
  }
  return k;
}

roix_status roix_extract_roi(roix_ctx* ctx, const void* in, roix_dtype dtype, roix_dims dims,
                             const roix_roi* roi, uint32_t* mask_out, uint64_t* popcount_dev,
                             void* stream) {
  if (!ctx || !roi) return fail(ctx, ROIX_EINVAL, "null context or roi");
  Desc d;
  roix_status s = make_desc(ctx, dtype, dims, roi, nullptr, nullptr, &d);
  if (s) return s;
  if (d.keep && !ccl_fits(d)) return fail(ctx, ROIX_EINVAL, "too many rows x runs for keep = 1");
  if (d.N && (!in || !mask_out)) return fail(ctx, ROIX_EINVAL, "null buffer");
  if (!popcount_dev) return fail(ctx, ROIX_EINVAL, "null popcount_dev");
  DeviceGuard g(ctx->device);
  // the mask T lives in the item plan (with the largest-component scratch)
  const u64 ncap = 0, cap = 0;
  Desc dp = d;
  dp.S = 2;
  BatchPlan bp = plan_batch(dp, &dims, &ncap, &cap, 1, true, false);
  if ((s = ensure_ws(ctx, bp.total))) return s;
  cudaStream_t cs = (cudaStream_t)stream;
  Launch L{cs, ctx->sms, ctx->tune};
  u32* T = (u32*)(ctx->ws + bp.items[0].T);
  launch_init(L, (State*)ctx->ws, 1, ctx->ws + bp.zero_begin, bp.zero_end - bp.zero_begin);
  cudaMemsetAsync(popcount_dev, 0, 8, cs);
  static thread_local Batch B;  // 22 KB: kept off the stack
  make_threshold_batch(B, d, in, T);
  launch_threshold(L, B);
  if (d.keep) {
    u32* T2 = (u32*)(ctx->ws + bp.items[0].T2);
    launch_keep_largest(L, d, T, T2, ccl_ws(ctx->ws, bp.items[0], &((State*)ctx->ws)->status));
    T = T2;
  }
  launch_dilate(L, d, T, mask_out, (u64*)popcount_dev);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ROIX_OK : cuda_fail(ctx, e, "extract_roi launch");
}

roix_status roix_compact(roix_ctx* ctx, const void* in, roix_dtype dtype, roix_dims dims,
                         const uint32_t* mask, void* pixels_out, uint16_t* counts_out,
                         uint16_t* bounds_out, uint64_t bounds_cap, uint64_t* sizes_dev,
                         void* stream) {
  if (!ctx) return ROIX_EINVAL;
  Desc d;
  roix_status s = make_desc(ctx, dtype, dims, nullptr, nullptr, nullptr, &d);
  if (s) return s;
  if (d.N && (!in || !mask || !pixels_out || !counts_out || (!bounds_out && bounds_cap)))
    return fail(ctx, ROIX_EINVAL, "null buffer");
  if (!sizes_dev) return fail(ctx, ROIX_EINVAL, "null sizes_dev");
  if (!aligned(pixels_out, 4)) return fail(ctx, ROIX_EINVAL, "pixels_out must be 4-byte aligned");
  DeviceGuard g(ctx->device);
  d.dilate = 0;  // the mask is used as given
  d.S = 2;       // no coder settings: one histogram bin pair reserved, unused
  const u64 ncap = d.N, cap = 0;
  BatchPlan bp = plan_batch(d, &dims, &ncap, &cap, 1, false, false);
  if ((s = ensure_ws(ctx, bp.total))) return s;
  cudaStream_t cs = (cudaStream_t)stream;
  Launch L{cs, ctx->sms, ctx->tune};
  static thread_local Batch B;
  fill_batch(B, d, bp, &dims, ctx->ws, 1);
  Item& I = B.it[0];
  I.in = in;
  I.T = const_cast<uint32_t*>(mask);
  I.P = pixels_out;
  I.counts = counts_out;
  I.counts_cap = d.rows;
  I.bounds = bounds_out;
  I.bounds_cap = bounds_cap;
  I.sizes = (u64*)sizes_dev;
  launch_init(L, (State*)ctx->ws, 1, ctx->ws + bp.zero_begin, bp.zero_end - bp.zero_begin);
  cudaMemsetAsync(sizes_dev, 0, 16, cs);
  launch_front(L, B);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ROIX_OK : cuda_fail(ctx, e, "compact launch");
}

roix_status roix_quantize(roix_ctx* ctx, const void* pixels, roix_dtype dtype, uint64_t n_cap,
                          const uint64_t* n_dev, const roix_eb* eb, double dark, int32_t* q_out,
                          uint32_t* outlier_bits_out, roix_eb_info* info_dev, void* stream) {
  if (!ctx || !eb) return fail(ctx, ROIX_EINVAL, "null context or eb");
  Desc d;
  if (n_cap > (1ull << 40)) return fail(ctx, ROIX_EINVAL, "n_cap too large");
  const roix_dims dims{1, 1, 1};
  roix_status s = make_desc(ctx, dtype, dims, nullptr, eb, nullptr, &d);
  if (s) return s;
  if (dtype == ROIX_U16 && !(dark >= 0.0 && dark <= 65535.0 && dark == std::floor(dark)))
    return fail(ctx, ROIX_EINVAL, "dark must be an integer in [0, 65535]");
  if (dtype == ROIX_F32 && dark != 0.0) return fail(ctx, ROIX_EINVAL, "dark must be 0 for float32");
  d.dark = (int)dark;
  d.dark_d = dark;
  if (n_cap && (!pixels || !q_out || !outlier_bits_out))
    return fail(ctx, ROIX_EINVAL, "null buffer");
  if (!info_dev) return fail(ctx, ROIX_EINVAL, "null info_dev");
  DeviceGuard g(ctx->device);
  Arena a;
  const size_t st_off = a.take(kStateBytes);
  if ((s = ensure_ws(ctx, a.take(0)))) return s;
  cudaStream_t cs = (cudaStream_t)stream;
  Launch L{cs, ctx->sms, ctx->tune};
  State* st = (State*)(ctx->ws + st_off);
  launch_init(L, st, 1, nullptr, 0);
  launch_quantize_stage(L, d, pixels, n_cap, (const u64*)n_dev, q_out, outlier_bits_out,
                        info_dev, st);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ROIX_OK : cuda_fail(ctx, e, "quantize launch");
}

roix_status roix_encode(roix_ctx* ctx, const int32_t* q, const uint32_t* outlier_bits,
                        const void* pixels, uint64_t n_cap, const uint64_t* sizes_dev,
                        const uint16_t* counts, const uint16_t* bounds,
                        const roix_eb_info* info_dev, roix_dtype dtype, roix_dims dims,
                        const roix_roi* roi, const roix_eb* eb, const roix_params* params,
                        void* out, uint64_t cap, uint64_t* size_dev, void* stream) {
  if (!ctx || !roi || !eb || !params) return fail(ctx, ROIX_EINVAL, "null parameter struct");
  Desc d;
  roix_status s = make_desc(ctx, dtype, dims, roi, eb, params, &d);
  if (s) return s;
  if (n_cap > d.N) return fail(ctx, ROIX_EINVAL, "n_cap exceeds the voxel count");
  if (!sizes_dev || !info_dev || !out || !size_dev) return fail(ctx, ROIX_EINVAL, "null buffer");
  if (n_cap && (!q || !outlier_bits || !pixels)) return fail(ctx, ROIX_EINVAL, "null buffer");
  if (d.rows && !counts) return fail(ctx, ROIX_EINVAL, "null counts");
  if (!aligned(out, 16)) return fail(ctx, ROIX_EINVAL, "out must be 16-byte aligned");
  if (!aligned(q, 8)) return fail(ctx, ROIX_EINVAL, "q must be 8-byte aligned");
  DeviceGuard g(ctx->device);
  const u64 ncap64 = n_cap, cap64 = cap;
  BatchPlan bp = plan_batch(d, &dims, &ncap64, &cap64, 1, false, false);
  if ((s = ensure_ws(ctx, bp.total))) return s;
  cudaStream_t cs = (cudaStream_t)stream;
  Launch L{cs, ctx->sms, ctx->tune};
  static thread_local Batch B;
  fill_batch(B, d, bp, &dims, ctx->ws, 1);
  Item& I = B.it[0];
  I.out = (uint8_t*)out;
  I.cap = cap;
  I.size_dev = (u64*)size_dev;
  I.P = const_cast<void*>(pixels);
  I.q = q ? q : (const int32_t*)ctx->ws;  // non-null selects the staged-code kernels
  I.obits = outlier_bits;
  I.info_in = info_dev;
  I.sizes = const_cast<u64*>((const u64*)sizes_dev);
  I.counts_src = counts;
  I.bounds_src = bounds;
  launch_init(L, (State*)ctx->ws, 1, ctx->ws + bp.zero_begin, bp.zero_end - bp.zero_begin);
  launch_symbols(L, B, bp.qtiles);
  launch_codebook(L, B);
  launch_pack(L, B, bp.pranges);
  launch_finalize(L, B);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ROIX_OK : cuda_fail(ctx, e, "encode launch");
}

}  // extern "C"

namespace {

// The fused path for one group of at most kMaxBatch items sharing `c`.
roix_status enqueue_group(roix_ctx* ctx, const Desc& c, const roix_item* items, u32 n,
                          cudaStream_t cs, bool profile) {
  std::vector<roix_dims> dims(n);
  std::vector<u64> ncaps(n), caps(n);
  for (u32 i = 0; i < n; ++i) {
    dims[i] = items[i].dims;
    ncaps[i] = items[i].dims.nx * items[i].dims.ny * items[i].dims.nz;
    caps[i] = items[i].cap;
  }
  BatchPlan bp = plan_batch(c, dims.data(), ncaps.data(), caps.data(), n, true, true);
  roix_status s = ensure_ws(ctx, bp.total);
  if (s) return s;
  Launch L{cs, ctx->sms, ctx->tune};
  static thread_local Batch B;
  fill_batch(B, c, bp, dims.data(), ctx->ws, n);
  for (u32 i = 0; i < n; ++i) {
    Item& I = B.it[i];
    I.in = items[i].in;
    set_container(I, c, items[i].out, items[i].cap, (u64*)items[i].size_dev);
  }
  set_threshold_units(B);
  if (profile) {
    ctx->nev = 0;
    mark(ctx, cs);
  }
  launch_init(L, (State*)ctx->ws, n, ctx->ws + bp.zero_begin, bp.zero_end - bp.zero_begin);
  if (profile) mark(ctx, cs);
  launch_threshold(L, B);
  if (c.keep) {  // largest component of each item's mask, then compact from that mask
    for (u32 i = 0; i < n; ++i) {
      Item& I = B.it[i];
      const Desc di = item_desc(c, I);
      launch_keep_largest(L, di, I.T, (u32*)(ctx->ws + bp.items[i].T2),
                          ccl_ws(ctx->ws, bp.items[i], B.status));
      I.T = (u32*)(ctx->ws + bp.items[i].T2);
    }
  }
  if (profile) mark(ctx, cs);
  launch_front(L, B);
  if (profile) mark(ctx, cs);
  launch_symbols(L, B, bp.qtiles);
  if (profile) mark(ctx, cs);
  launch_codebook(L, B);
  if (profile) mark(ctx, cs);
  launch_pack(L, B, bp.pranges);
  if (profile) mark(ctx, cs);
  launch_finalize(L, B);
  if (profile) mark(ctx, cs);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ROIX_OK : cuda_fail(ctx, e, "compress launch");
}

}  // namespace

size_t roix::batch_workspace(const Desc& c, const roix_item* items, u32 n) {
  std::vector<roix_dims> dims(n);
  std::vector<u64> ncaps(n), caps(n);
  for (u32 i = 0; i < n; ++i) {
    dims[i] = items[i].dims;
    ncaps[i] = items[i].dims.nx * items[i].dims.ny * items[i].dims.nz;
    caps[i] = items[i].cap;
  }
  return plan_batch(c, dims.data(), ncaps.data(), caps.data(), n, true, true).total;
}

namespace {

roix_status check_item(roix_ctx* ctx, const roix_item& it, roix_dtype dtype) {
  if (!dims_ok(it.dims)) return fail(ctx, ROIX_EINVAL, "dims: nx <= 65534, ny, nz < 2^32");
  const u64 N = it.dims.nx * it.dims.ny * it.dims.nz;
  if ((N && !it.in) || !it.out || !it.size_dev) return fail(ctx, ROIX_EINVAL, "null buffer");
  if (!aligned(it.out, 16)) return fail(ctx, ROIX_EINVAL, "out must be 16-byte aligned");
  if (!aligned(it.in, dtype == ROIX_F32 ? 4 : 2)) return fail(ctx, ROIX_EINVAL, "misaligned input");
  return ROIX_OK;
}

}  // namespace

extern "C" {

roix_status roix_compress(roix_ctx* ctx, const void* in, roix_dtype dtype, roix_dims dims,
                          const roix_roi* roi, const roix_eb* eb, const roix_params* params,
                          void* out, uint64_t cap, uint64_t* size_dev, void* stream) {
  if (!ctx || !roi || !eb || !params) return fail(ctx, ROIX_EINVAL, "null parameter struct");
  Desc d;
  roix_status s = make_desc(ctx, dtype, dims, roi, eb, params, &d);
  if (s) return s;
  if (d.keep && !ccl_fits(d)) return fail(ctx, ROIX_EINVAL, "too many rows x runs for keep = 1");
  const roix_item it{in, dims, out, cap, size_dev};
  if ((s = check_item(ctx, it, dtype))) return s;
  DeviceGuard g(ctx->device);
  return enqueue_group(ctx, d, &it, 1, (cudaStream_t)stream, ctx->profile != 0);
}

roix_status roix_compress_batch(roix_ctx* ctx, uint32_t n, const roix_item* items,
                                roix_dtype dtype, const roix_roi* roi, const roix_eb* eb,
                                const roix_params* params, void* stream) {
  if (!ctx || !roi || !eb || !params || (n && !items))
    return fail(ctx, ROIX_EINVAL, "null argument");
  Desc d;
  const roix_dims one{1, 1, 1};
  roix_status s = make_desc(ctx, dtype, one, roi, eb, params, &d);
  if (s) return s;
  for (u32 i = 0; i < n; ++i) {
    if ((s = check_item(ctx, items[i], dtype))) return s;
    Desc di = d;
    di.nx = items[i].dims.nx;
    di.rows = items[i].dims.ny * items[i].dims.nz;
    if (d.keep && !ccl_fits(di)) return fail(ctx, ROIX_EINVAL, "too many rows x runs for keep = 1");
  }
  DeviceGuard g(ctx->device);
  for (u32 i0 = 0; i0 < n; i0 += kMaxBatch) {
    const u32 m = n - i0 < (u32)kMaxBatch ? n - i0 : (u32)kMaxBatch;
    if ((s = enqueue_group(ctx, d, items + i0, m, (cudaStream_t)stream, ctx->profile != 0)))
      return s;
  }
  return ROIX_OK;
}

}  // extern "C"

namespace {

// ------------------------------------------------------------- z-slabs
// A volume cut into z-slabs of slab_z slices, each slab an item of its own
// (own container, stream, histogram and codebook) while the mask and the
// error bound are the whole volume's: one binarisation of the whole volume
// into one contiguous T, slab items whose T points at their first plane with
// the neighbouring planes marked as present (the dilation crosses the slab
// borders), and one value range shared by every slab.
struct SlabPlan {
  std::vector<roix_dims> dims;
  std::vector<u64> ncaps, caps;
  BatchPlan bp;
  size_t T_off = 0, total = 0;
};

SlabPlan plan_slabs(const Desc& d, u64 slab_z, const uint64_t* caps, u64 cap_all) {
  SlabPlan sp;
  const u64 ns = d.nz ? (d.nz + slab_z - 1) / slab_z : 0;
  sp.dims.resize(ns);
  sp.ncaps.resize(ns);
  sp.caps.resize(ns);
  for (u64 s = 0; s < ns; ++s) {
    const u64 dz = umin(slab_z, d.nz - s * slab_z);
    sp.dims[s] = roix_dims{d.nx, d.ny, dz};
    sp.ncaps[s] = d.nx * d.ny * dz;
    sp.caps[s] = caps ? caps[s] : cap_all;
  }
  sp.bp = plan_batch(d, sp.dims.data(), sp.ncaps.data(), sp.caps.data(), (u32)ns, false, true);
  Arena a;
  a.off = sp.bp.total;
  sp.T_off = a.take(4 * d.rows * d.W + 16);
  sp.total = a.take(0);
  return sp;
}

roix_status slab_desc(roix_ctx* ctx, roix_dtype dtype, roix_dims dims, uint64_t slab_z,
                      const roix_roi* roi, const roix_eb* eb, const roix_params* params,
                      Desc* d) {
  if (!roi || !eb || !params) return fail(ctx, ROIX_EINVAL, "null parameter struct");
  if (dtype != ROIX_F32 && dtype != ROIX_U16)
    return fail(ctx, ROIX_EINVAL, "slabs: float32 or uint16 only");
  roix_status s = make_desc(ctx, dtype, dims, roi, eb, params, d);
  if (s) return s;
  if (d->keep) return fail(ctx, ROIX_EINVAL, "slabs: keep = 1 is refused (a slab is not a volume)");
  if (slab_z == 0) return fail(ctx, ROIX_EINVAL, "slab_z must be >= 1");
  return ROIX_OK;
}

}  // namespace

extern "C" {

size_t roix_slabs_workspace_size(roix_dtype dtype, roix_dims dims, uint64_t slab_z,
                                 const roix_roi* roi, const roix_params* params, uint64_t cap) {
  Desc d;
  const roix_eb eb{0, 1.0};
  if (slab_desc(nullptr, dtype, dims, slab_z, roi, &eb, params, &d) != ROIX_OK) return 0;
  return plan_slabs(d, slab_z, nullptr, cap).total;
}

roix_status roix_compress_slabs(roix_ctx* ctx, const void* in, roix_dtype dtype, roix_dims dims,
                                uint64_t slab_z, const roix_roi* roi, const roix_eb* eb,
                                const roix_params* params, void* const* outs,
                                const uint64_t* caps, uint64_t* sizes_dev, void* stream) {
  if (!ctx) return ROIX_EINVAL;
  Desc d;
  roix_status s = slab_desc(ctx, dtype, dims, slab_z, roi, eb, params, &d);
  if (s) return s;
  const u64 ns = d.nz ? (d.nz + slab_z - 1) / slab_z : 0;
  if (ns == 0) return ROIX_OK;
  if (!outs || !caps || !sizes_dev) return fail(ctx, ROIX_EINVAL, "null outs, caps or sizes_dev");
  if (d.N && !in) return fail(ctx, ROIX_EINVAL, "null input");
  const size_t esz = dtype_bytes(dtype);
  if (!aligned(in, esz)) return fail(ctx, ROIX_EINVAL, "misaligned input");
  for (u64 k = 0; k < ns; ++k)
    if (!outs[k] || !aligned(outs[k], 16))
      return fail(ctx, ROIX_EINVAL, "every slab output must be a 16-byte aligned buffer");
  DeviceGuard g(ctx->device);
  const SlabPlan sp = plan_slabs(d, slab_z, caps, 0);
  if ((s = ensure_ws(ctx, sp.total))) return s;
  cudaStream_t cs = (cudaStream_t)stream;
  Launch L{cs, ctx->sms, ctx->tune};
  char* ws = ctx->ws;
  State* st = (State*)ws;
  u32* T = (u32*)(ws + sp.T_off);
  const u64 plane_words = d.ny * d.W;
  const bool profile = ctx->profile != 0;
  if (profile) {
    ctx->nev = 0;
    mark(ctx, cs);
  }
  launch_init(L, st, (u32)ns, ws + sp.bp.zero_begin, sp.bp.zero_end - sp.bp.zero_begin);
  if (profile) mark(ctx, cs);
  {
    static thread_local Batch Bt;
    make_threshold_batch(Bt, d, in, T);
    launch_threshold(L, Bt);
  }
  if (profile) mark(ctx, cs);
  // groups of up to kMaxBatch slabs, all sharing the range kept in state 0
  const u32 ngroups = (u32)((ns + kMaxBatch - 1) / kMaxBatch);
  std::vector<Batch> G(ngroups);
  std::vector<u64> gq(ngroups, 0), gp(ngroups, 0);
  for (u32 gi = 0; gi < ngroups; ++gi) {
    const u32 first = gi * kMaxBatch;
    const u32 m = (u32)umin(kMaxBatch, ns - first);
    Batch& B = G[gi];
    fill_batch(B, d, sp.bp, sp.dims.data(), ws, m, first);
    for (u32 i = 0; i < m; ++i) {
      const u64 k = first + i;
      const u64 z0 = k * slab_z;
      Item& I = B.it[i];
      I.in = (const char*)in + z0 * d.ny * d.nx * esz;
      I.T = T + z0 * plane_words;
      I.zhalo = (z0 > 0 ? 1u : 0u) | (z0 + I.nz < d.nz ? 2u : 0u);
      I.rst = st;
      set_container(I, d, outs[k], caps[k], (u64*)sizes_dev + k);
      gq[gi] += sp.bp.items[k].qtiles;
      gp[gi] += sp.bp.items[k].pranges;
    }
  }
  for (u32 gi = 0; gi < ngroups; ++gi) launch_front(L, G[gi]);
  if (profile) mark(ctx, cs);
  for (u32 gi = 0; gi < ngroups; ++gi) launch_symbols(L, G[gi], gq[gi]);
  if (profile) mark(ctx, cs);
  for (u32 gi = 0; gi < ngroups; ++gi) launch_codebook(L, G[gi]);
  if (profile) mark(ctx, cs);
  for (u32 gi = 0; gi < ngroups; ++gi) launch_pack(L, G[gi], gp[gi]);
  if (profile) mark(ctx, cs);
  for (u32 gi = 0; gi < ngroups; ++gi) launch_finalize(L, G[gi]);
  if (profile) mark(ctx, cs);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ROIX_OK : cuda_fail(ctx, e, "compress_slabs launch");
}

roix_status roix_decode(roix_ctx* ctx, const void* in, uint64_t size, void* out,
                        roix_dtype dtype, roix_dims dims, void* stream) {
  if (!ctx) return ROIX_EINVAL;
  Desc d;
  roix_status s = make_desc(ctx, dtype, dims, nullptr, nullptr, nullptr, &d);
  if (s) return s;
  if (dtype == ROIX_U8) return fail(ctx, ROIX_EINVAL, "containers hold float32 or uint16");
  if (!in || (d.N && !out)) return fail(ctx, ROIX_EINVAL, "null buffer");
  if (!aligned(in, 16)) return fail(ctx, ROIX_EINVAL, "in must be 16-byte aligned");
  DeviceGuard g(ctx->device);
  const u64 max_chunks = (d.N + 255) / 256;
  const u64 row_tiles = (d.rows + kDecRowTile - 1) / kDecRowTile;
  const size_t esz = dtype == ROIX_F32 ? 4 : 2;
  Arena a;
  const size_t st_off = a.take(kStateBytes);
  const size_t plan = a.take(8 * kPlanWords);
  const size_t zb = a.take(0);
  const size_t table = a.take(dec_table_bytes());
  const size_t fb = a.take(4 * (row_tiles + 1));
  const size_t fv = a.take(4 * (row_tiles + 1));
  const size_t ctr = a.take(16);
  const size_t ze = a.take(0);
  const size_t db = a.take(8 * 2 * (row_tiles + 1));
  const size_t dv = a.take(8 * 2 * (row_tiles + 1));
  const size_t sym = a.take(2 * d.N + 16);
  const size_t agg = a.take(48 * (max_chunks + 1));    // order 1: 2 words a chunk, order 2: 6
  const size_t carry = a.take(16 * (max_chunks + 1));  // order 1: 1 word a chunk, order 2: 2
  const size_t vals = a.take(esz * d.N + 16);
  const size_t rb = a.take(8 * (d.rows + 1));
  const size_t rv = a.take(8 * (d.rows + 1));
  if ((s = ensure_ws(ctx, a.take(0)))) return s;
  cudaStream_t cs = (cudaStream_t)stream;
  Launch L{cs, ctx->sms, ctx->tune};
  char* ws = ctx->ws;
  State* st = (State*)(ws + st_off);
  launch_init(L, st, 1, ws + zb, ze - zb);
  DecodeWs w;
  w.status = &st->status;
  w.plan = (u64*)(ws + plan);
  w.table = ws + table;
  w.sym = (uint16_t*)(ws + sym);
  w.agg = (u64*)(ws + agg);
  w.carry = (u64*)(ws + carry);
  w.vals = ws + vals;
  w.row_boff = (u64*)(ws + rb);
  w.row_voff = (u64*)(ws + rv);
  w.lb_rows_b = lb_at<1>(ws, fb, db, row_tiles);
  w.lb_rows_v = lb_at<1>(ws, fv, dv, row_tiles);
  w.row_ctr = (u32*)(ws + ctr);
  launch_decode(L, d, (const uint8_t*)in, size, out, w, max_chunks);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ROIX_OK : cuda_fail(ctx, e, "decode launch");
}

}  // extern "C"

// ------------------------------------------------ 8-bit preprocessor path
roix_status roix_normalize8(roix_ctx* ctx, const void* in, roix_dtype dtype, roix_dims dims,
                            double dark, uint8_t* out, double* imax_dev, void* stream) {
  if (!ctx) return ROIX_EINVAL;
  if (dtype != ROIX_F32 && dtype != ROIX_U16)
    return fail(ctx, ROIX_EINVAL, "normalize8 takes float32 or uint16 input");
  Desc d;
  roix_status s = make_desc(ctx, dtype, dims, nullptr, nullptr, nullptr, &d);
  if (s) return s;
  if (dtype == ROIX_U16 && !(dark >= 0.0 && dark <= 65535.0 && dark == std::floor(dark)))
    return fail(ctx, ROIX_EINVAL, "dark must be an integer in [0, 65535]");
  if (dtype == ROIX_F32 && dark != 0.0) return fail(ctx, ROIX_EINVAL, "dark must be 0 for float32");
  if (d.N && (!in || !out)) return fail(ctx, ROIX_EINVAL, "null buffer");
  if (d.N && !aligned(in, dtype_bytes(dtype))) return fail(ctx, ROIX_EINVAL, "misaligned input");
  DeviceGuard g(ctx->device);
  Arena a;
  a.take(kStateBytes);
  const size_t key = a.take(16);
  if ((s = ensure_ws(ctx, a.take(0)))) return s;
  cudaStream_t cs = (cudaStream_t)stream;
  Launch L{cs, ctx->sms, ctx->tune};
  cudaMemsetAsync(ctx->ws + key, 0, 4, cs);
  if (d.N == 0) {
    if (imax_dev) cudaMemsetAsync(imax_dev, 0, 8, cs);
  } else {
    launch_normalize8(L, dtype, in, d.N, (int)dark, out, (u32*)(ctx->ws + key), imax_dev);
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ROIX_OK : cuda_fail(ctx, e, "normalize8 launch");
}

roix_status roix_greedy_quantize_batch(roix_ctx* ctx, uint32_t n, const roix_greedy_item* items,
                                       double eabs, void* stream) {
  if (!ctx) return ROIX_EINVAL;
  if (n && !items) return fail(ctx, ROIX_EINVAL, "null items");
  if (!(std::isfinite(eabs) && eabs >= 0.0))
    return fail(ctx, ROIX_EINVAL, "eabs must be finite and >= 0");
  u64 rows_all = 0, tiles_all = 0, rows_max = 0, tiles_max = 0;
  for (u32 k = 0; k < n; ++k) {
    Desc d;
    roix_status s = make_desc(ctx, ROIX_U8, items[k].dims, nullptr, nullptr, nullptr, &d);
    if (s) return s;
    if (d.N && (!items[k].pixels || !items[k].mask || !items[k].q_out))
      return fail(ctx, ROIX_EINVAL, "null buffer");
    rows_all += d.rows;
    tiles_all += (d.rows + 31) / 32;
  }
  DeviceGuard g(ctx->device);
  // workspace for the largest group of up to kGreedyMaxItems items
  for (u32 k0 = 0; k0 < n; k0 += kGreedyMaxItems) {
    u64 r = 0, t = 0;
    for (u32 k = k0; k < n && k < k0 + kGreedyMaxItems; ++k) {
      const u64 rows = items[k].dims.ny * items[k].dims.nz;
      r += rows;
      t += (rows + 31) / 32;
    }
    rows_max = r > rows_max ? r : rows_max;
    tiles_max = t > tiles_max ? t : tiles_max;
  }
  (void)rows_all;
  (void)tiles_all;
  Arena a;
  a.take(kStateBytes);
  const size_t lens = a.take(4 * rows_max + 16);
  const size_t rpre = a.take(4 * rows_max + 16);
  const size_t ctr = a.take(16 * ((n + kGreedyMaxItems - 1) / kGreedyMaxItems + 1));
  const size_t tsum = a.take(4 * tiles_max + 16);
  const size_t toff = a.take(8 * (tiles_max + 1));
  roix_status s;
  if ((s = ensure_ws(ctx, a.take(0)))) return s;
  cudaStream_t cs = (cudaStream_t)stream;
  Launch L{cs, ctx->sms, ctx->tune};
  static thread_local GreedyBatch B;
  const double ef = std::floor(eabs);
  for (u32 k0 = 0; k0 < n; k0 += kGreedyMaxItems) {
    std::memset(&B, 0, sizeof(B));
    B.n = n - k0 < kGreedyMaxItems ? n - k0 : kGreedyMaxItems;
    B.e2 = (u32)(2.0 * (ef > 255.0 ? 255.0 : ef));
    B.lens = (u32*)(ctx->ws + lens);
    B.tsum = (u32*)(ctx->ws + tsum);
    B.toff = (u64*)(ctx->ws + toff);
    B.rpre = (u32*)(ctx->ws + rpre);
    B.rowctr = (u64*)(ctx->ws + ctr) + 2 * (k0 / kGreedyMaxItems);
    cudaMemsetAsync(B.rowctr, 0, 8, cs);
    for (u32 k = 0; k < B.n; ++k) {
      const roix_greedy_item& it = items[k0 + k];
      GreedyItem& I = B.it[k];
      I.P = it.pixels;
      I.mask = it.mask;
      I.Q = it.q_out;
      I.n_out = (u64*)it.n_dev;
      I.rows = it.dims.ny * it.dims.nz;
      I.W = (it.dims.nx + 31) / 32;
      I.inplace = it.q_out == it.pixels ? 1u : 0u;
      if (it.dims.nx == 0) I.rows = 0;  // no voxels: no rows to scan
      B.tile0[k + 1] = B.tile0[k] + (I.rows + 31) / 32;
      B.row0[k + 1] = B.row0[k] + I.rows;
    }
    launch_greedy(L, B);
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ROIX_OK : cuda_fail(ctx, e, "greedy launch");
}

roix_status roix_greedy_quantize(roix_ctx* ctx, const uint8_t* pixels, const uint32_t* mask,
                                 roix_dims dims, double eabs, uint8_t* q_out, uint64_t* n_dev,
                                 void* stream) {
  const roix_greedy_item it{pixels, mask, dims, q_out, n_dev};
  return roix_greedy_quantize_batch(ctx, 1, &it, eabs, stream);
}

// ------------------------------------------------------ evaluation metrics
roix_status roix_roi_quality(roix_ctx* ctx, const uint32_t* pred_mask, const uint32_t* truth_mask,
                             roix_dims dims, int distances, roix_roi_metrics* out_dev,
                             void* stream) {
  if (!ctx) return ROIX_EINVAL;
  Desc d;
  roix_status s = make_desc(ctx, ROIX_U8, dims, nullptr, nullptr, nullptr, &d);
  if (s) return s;
  if (distances != 0 && distances != 1) return fail(ctx, ROIX_EINVAL, "distances must be 0 or 1");
  if (!out_dev || (d.N && (!pred_mask || !truth_mask))) return fail(ctx, ROIX_EINVAL, "null buffer");
  if (distances) {
    const double a = (double)(dims.nx ? dims.nx - 1 : 0), b = (double)(dims.ny ? dims.ny - 1 : 0),
                 c = (double)(dims.nz ? dims.nz - 1 : 0);
    if (a * a + b * b + c * c >= 4294967295.0)
      return fail(ctx, ROIX_EINVAL, "volume too large for 32-bit squared distances");
  }
  DeviceGuard g(ctx->device);
  Arena ar;
  ar.take(kStateBytes);
  const size_t off = ar.take(roi_quality_ws_bytes(dims.nx, dims.ny, dims.nz, distances));
  if ((s = ensure_ws(ctx, ar.take(0)))) return s;
  Launch L{(cudaStream_t)stream, ctx->sms, ctx->tune};
  launch_roi_quality(L, pred_mask, truth_mask, dims.nx, dims.ny, dims.nz, distances,
                     ctx->ws + off, out_dev);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ROIX_OK : cuda_fail(ctx, e, "roi_quality launch");
}

roix_status roix_ssim(roix_ctx* ctx, const void* x, const void* y, roix_dtype dtype,
                      roix_dims dims, double data_range, double* ssim_dev, void* stream) {
  if (!ctx) return ROIX_EINVAL;
  Desc d;
  roix_status s = make_desc(ctx, dtype, dims, nullptr, nullptr, nullptr, &d);
  if (s) return s;
  if (!(std::isfinite(data_range) && data_range > 0.0))
    return fail(ctx, ROIX_EINVAL, "data_range must be finite and > 0");
  if (!ssim_dev || (d.N && (!x || !y))) return fail(ctx, ROIX_EINVAL, "null buffer");
  if (d.N && (!aligned(x, dtype_bytes(dtype)) || !aligned(y, dtype_bytes(dtype))))
    return fail(ctx, ROIX_EINVAL, "misaligned input");
  DeviceGuard g(ctx->device);
  Arena ar;
  ar.take(kStateBytes);
  const size_t off = ar.take(64);
  if ((s = ensure_ws(ctx, ar.take(0)))) return s;
  Launch L{(cudaStream_t)stream, ctx->sms, ctx->tune};
  launch_ssim(L, dtype, x, y, dims.nx, dims.ny, dims.nz, data_range, ctx->ws + off, ssim_dev);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ROIX_OK : cuda_fail(ctx, e, "ssim launch");
}

// ---------------------------------------------------- paper-mode ROI
roix_status roix_extract_roi_paper(roix_ctx* ctx, const uint8_t* img, roix_dims dims,
                                   uint32_t* mask_out, uint64_t* popcount_dev,
                                   uint32_t* thresholds_dev, void* stream) {
  if (!ctx) return ROIX_EINVAL;
  Desc d;
  roix_status s = make_desc(ctx, ROIX_U8, dims, nullptr, nullptr, nullptr, &d);
  if (s) return s;
  if (!popcount_dev || (d.N && (!img || !mask_out))) return fail(ctx, ROIX_EINVAL, "null buffer");
  if (!ccl_fits(d)) return fail(ctx, ROIX_EINVAL, "too many rows x runs");
  DeviceGuard g(ctx->device);
  const u64 rows = d.rows, W = d.W, nz = dims.nz, maxr = ccl_max_runs(d);
  const u64 ctiles = (rows + 2047) / 2048;
  Arena a;
  const size_t st_off = a.take(kStateBytes);
  const size_t zb = a.take(0);
  const size_t cf = a.take(4 * (ctiles + 1));  // look-back flags of the run-count scan
  const size_t cv = a.take(32);                 // total, scan tickets
  const size_t ze = a.take(0);
  const size_t best = a.take(8 * nz + 16);
  const size_t broot = a.take(4 * nz + 16);
  const size_t ca = a.take(8 * 2 * (ctiles + 1));
  const size_t hist = a.take(4 * 256 * nz + 16);
  const size_t thr = a.take(8 * nz + 16);
  const size_t T = a.take(4 * rows * W + 16);
  const size_t BB = a.take(4 * rows * W + 16);
  const size_t K = a.take(4 * rows * W + 16);
  const size_t rr = a.take(4 * rows + 16);
  const size_t ro = a.take(8 * rows + 16);
  const size_t xs = a.take(2 * maxr + 16);
  const size_t xe = a.take(2 * maxr + 16);
  const size_t par = a.take(4 * maxr + 16);
  const size_t sz = a.take(8 * maxr + 16);
  if ((s = ensure_ws(ctx, a.take(0)))) return s;
  cudaStream_t cs = (cudaStream_t)stream;
  Launch L{cs, ctx->sms, ctx->tune};
  State* st = (State*)(ctx->ws + st_off);
  char* ws = ctx->ws;
  cudaMemsetAsync(popcount_dev, 0, 8, cs);
  if (d.N == 0) {
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? ROIX_OK : cuda_fail(ctx, e, "paper roi launch");
  }
  u32* th = thresholds_dev ? thresholds_dev : (u32*)(ws + thr);
  launch_paper_hist_otsu(L, img, dims.nx, dims.ny, nz, (u32*)(ws + hist), th);
  launch_paper_binarize(L, img, dims.nx, dims.ny, nz, th, (u32*)(ws + T));
  CclWs w;
  w.row_runs = (u32*)(ws + rr);
  w.row_off = (u64*)(ws + ro);
  w.xs = (uint16_t*)(ws + xs);
  w.xe = (uint16_t*)(ws + xe);
  w.par = (u32*)(ws + par);
  w.size = (unsigned long long*)(ws + sz);
  w.total = (u64*)(ws + cv);
  w.ctr = (u32*)(ws + cv + 8);
  w.best = (unsigned long long*)(ws + best);
  w.best_root = (u32*)(ws + broot);
  w.lb = lb_at<1>(ws, cf, ca, ctiles);
  w.status = &st->status;
  // background reaching the slice border (4-connected), from the complement of M
  Desc d4 = d;
  d4.conn = 4;
  launch_init(L, st, 1, ws + zb, ze - zb);
  launch_ccl_planar(L, d4, (const u32*)(ws + T), ~0u, 1, (u32*)(ws + BB), w);
  // the filled mask is its complement; its largest 8-connected object per slice
  Desc d8 = d;
  d8.conn = 8;
  cudaMemsetAsync(ws + zb, 0, ze - zb, cs);
  cudaMemsetAsync(ws + best, 0, 8 * nz, cs);
  cudaMemsetAsync(ws + broot, 0, 4 * nz, cs);
  launch_ccl_planar(L, d8, (const u32*)(ws + BB), ~0u, 0, (u32*)(ws + K), w);
  launch_paper_spans(L, (const u32*)(ws + K), rows, W, mask_out, (u64*)popcount_dev);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ROIX_OK : cuda_fail(ctx, e, "paper roi launch");
}
