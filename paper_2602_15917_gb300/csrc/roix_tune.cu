// Autotuner of the compression kernels' launch shapes (roix_tune).
//
// None of the tuned values changes an output byte: they set the compaction
// tile size and the number of resident blocks per SM of the binarisation,
// symbol and pack kernels. The tuner times roix_compress_batch on the
// caller's own items (CUDA events around whole calls, median of `reps`), one
// parameter at a time over a fixed candidate list (coordinate descent, in
// pipeline order), keeps the fastest value of each and leaves the result in
// the context. Results can be kept in a small JSON file keyed by device name,
// dtype and shape class, so that a later process applies them without timing.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "roix_internal.cuh"

using namespace roix;

namespace {

struct Param {
  const char* name;
  u32 Tuning::*field;
  std::vector<u32> candidates;
};

std::vector<Param> params_list() {
  return {
      {"thr_blocks_per_sm", &Tuning::thr_blocks_per_sm, {2, 4, 8, 16}},
      {"flat_blocks_per_sm", &Tuning::flat_blocks_per_sm, {2, 3, 4, 8}},
      {"front_words", &Tuning::front_words, {512, 1024, 2048, 4096, 8192}},
      {"sym_blocks_per_sm", &Tuning::sym_blocks_per_sm, {0, 1, 2, 3}},
      {"pack_blocks_per_sm", &Tuning::pack_blocks_per_sm, {0, 1, 2, 4}},
      {"front_kernel", &Tuning::front_kernel, {0, 1}},
  };
}

u32 ceil_log2(u64 v) {
  u32 l = 0;
  while ((1ull << l) < v) ++l;
  return l;
}

// Cache key: device name, dtype, and a shape class (x extent and voxels per
// item rounded up to powers of two, item count bucket, dilation, keep).
std::string cache_key(int device, roix_dtype dtype, u32 n, const roix_item* items,
                      const roix_roi* roi) {
  cudaDeviceProp prop;
  std::string dev = "device";
  if (cudaGetDeviceProperties(&prop, device) == cudaSuccess) dev = prop.name;
  u64 nx = 1, N = 0;
  for (u32 i = 0; i < n; ++i) {
    nx = std::max<u64>(nx, items[i].dims.nx);
    N += items[i].dims.nx * items[i].dims.ny * items[i].dims.nz;
  }
  const u64 per = n ? (N + n - 1) / n : 0;
  std::ostringstream k;
  k << dev << "|" << (dtype == ROIX_F32 ? "f32" : "u16") << "|nx" << (1ull << ceil_log2(nx))
    << "|N" << ceil_log2(per ? per : 1) << "|n" << ceil_log2(n ? n : 1) << "|d" << roi->dilate
    << "|k" << roi->keep;
  return k.str();
}

bool cache_load(const char* path, const std::string& key, Tuning* t) {
  std::ifstream f(path);
  if (!f) return false;
  const std::string quoted = "\"" + key + "\"";
  std::string line;
  while (std::getline(f, line)) {
    if (line.find(quoted) == std::string::npos) continue;
    Tuning r;
    for (const Param& p : params_list()) {
      const std::string field = "\"" + std::string(p.name) + "\":";
      const size_t at = line.find(field);
      if (at == std::string::npos) return false;
      r.*(p.field) = (u32)std::strtoul(line.c_str() + at + field.size(), nullptr, 10);
    }
    *t = r;
    return true;
  }
  return false;
}

// One line per entry; the entry for `key` is replaced, the others kept.
void cache_store(const char* path, const std::string& key, const Tuning& t, double ms) {
  std::vector<std::string> keep;
  {
    std::ifstream f(path);
    std::string line;
    const std::string quoted = "\"" + key + "\"";
    while (f && std::getline(f, line)) {
      if (line.find(": {") == std::string::npos || line.find(quoted) != std::string::npos)
        continue;
      while (!line.empty() && (line.back() == ',' || line.back() == ' ')) line.pop_back();
      keep.push_back(line);
    }
  }
  std::ostringstream e;
  e << "  \"" << key << "\": {";
  bool first = true;
  for (const Param& p : params_list()) {
    e << (first ? "" : ", ") << "\"" << p.name << "\": " << t.*(p.field);
    first = false;
  }
  char buf[64];
  std::snprintf(buf, sizeof buf, ", \"ms\": %.4f}", ms);
  e << buf;
  keep.push_back(e.str());
  const std::string tmp = std::string(path) + ".tmp";
  {
    std::ofstream o(tmp);
    o << "{\n";
    for (size_t i = 0; i < keep.size(); ++i) o << keep[i] << (i + 1 < keep.size() ? ",\n" : "\n");
    o << "}\n";
  }
  std::rename(tmp.c_str(), path);
}

bool tuning_ok(const Tuning& t) {
  return t.front_words >= 256 && t.front_words <= 16384 && t.thr_blocks_per_sm >= 1 &&
         t.thr_blocks_per_sm <= 32 && t.flat_blocks_per_sm >= 1 && t.flat_blocks_per_sm <= 32 &&
         t.sym_blocks_per_sm <= 32 && t.pack_blocks_per_sm <= 32 && t.front_kernel <= 1;
}

}  // namespace

extern "C" {

roix_status roix_get_tuning(const roix_ctx* ctx, roix_tuning* out) {
  if (!ctx || !out) return ROIX_EINVAL;
  out->front_words = ctx->tune.front_words;
  out->thr_blocks_per_sm = ctx->tune.thr_blocks_per_sm;
  out->flat_blocks_per_sm = ctx->tune.flat_blocks_per_sm;
  out->sym_blocks_per_sm = ctx->tune.sym_blocks_per_sm;
  out->pack_blocks_per_sm = ctx->tune.pack_blocks_per_sm;
  out->front_kernel = ctx->tune.front_kernel;
  return ROIX_OK;
}

roix_status roix_set_tuning(roix_ctx* ctx, const roix_tuning* t) {
  if (!ctx || !t) return ROIX_EINVAL;
  Tuning r;
  r.front_words = t->front_words;
  r.thr_blocks_per_sm = t->thr_blocks_per_sm;
  r.flat_blocks_per_sm = t->flat_blocks_per_sm;
  r.sym_blocks_per_sm = t->sym_blocks_per_sm;
  r.pack_blocks_per_sm = t->pack_blocks_per_sm;
  r.front_kernel = t->front_kernel;
  if (!tuning_ok(r)) {
    ctx->err = "tuning values out of range";
    return ROIX_EINVAL;
  }
  ctx->tune = r;
  return ROIX_OK;
}

roix_status roix_tune(roix_ctx* ctx, uint32_t n, const roix_item* items, roix_dtype dtype,
                      const roix_roi* roi, const roix_eb* eb, const roix_params* params,
                      uint32_t reps, const char* cache_path, roix_tuning* out, void* stream) {
  if (!ctx || !items || n == 0 || !roi || !eb || !params) return ROIX_EINVAL;
  if (!cache_path) cache_path = std::getenv("ROIX_TUNE_CACHE");
  if (cache_path && !*cache_path) cache_path = nullptr;
  if (reps == 0) reps = 5;
  const std::string key = cache_key(ctx->device, dtype, n, items, roi);
  Tuning cached;
  if (cache_path && cache_load(cache_path, key, &cached) && tuning_ok(cached)) {
    ctx->tune = cached;
    if (out) roix_get_tuning(ctx, out);
    return ROIX_OK;
  }
  cudaStream_t cs = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    return ROIX_ECUDA;
  }
  const int was_profiling = ctx->profile;
  ctx->profile = 0;
  roix_status st = ROIX_OK;
  // median device time of one call under the current tuning
  auto measure = [&](double* ms_out) -> roix_status {
    roix_status s = roix_compress_batch(ctx, n, items, dtype, roi, eb, params, stream);  // warm-up
    if (s) return s;
    if ((s = roix_sync(ctx, stream))) return s;
    std::vector<float> t(reps);
    for (u32 r = 0; r < reps; ++r) {
      cudaEventRecord(e0, cs);
      if ((s = roix_compress_batch(ctx, n, items, dtype, roi, eb, params, stream))) return s;
      cudaEventRecord(e1, cs);
      if ((s = roix_sync(ctx, stream))) return s;
      cudaEventElapsedTime(&t[r], e0, e1);
    }
    std::nth_element(t.begin(), t.begin() + reps / 2, t.end());
    *ms_out = t[reps / 2];
    return ROIX_OK;
  };
  Tuning best = ctx->tune;
  double best_ms = 0.0;
  if ((st = measure(&best_ms)) == ROIX_OK) {
    for (const Param& p : params_list()) {
      for (u32 c : p.candidates) {
        if (best.*(p.field) == c) continue;
        Tuning trial = best;
        trial.*(p.field) = c;
        ctx->tune = trial;
        double ms = 0.0;
        if ((st = measure(&ms))) break;
        if (ms < best_ms * 0.99) {  // keep a change only when it is clearly faster
          best = trial;
          best_ms = ms;
        }
      }
      if (st) break;
    }
  }
  ctx->tune = best;
  ctx->profile = was_profiling;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st) return st;
  if (cache_path) cache_store(cache_path, key, best, best_ms);
  if (out) roix_get_tuning(ctx, out);
  return ROIX_OK;
}

}  // extern "C"
