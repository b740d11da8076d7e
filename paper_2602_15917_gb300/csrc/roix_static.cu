// Allocation-free ROI extraction: roix_extract_roi_static.
//
// Some callers cannot allocate device memory at the moment they need a mask:
// acquisition loops that must never stall on the implicit device
// synchronisation of cudaMalloc/cudaFree, and processes whose device memory is
// entirely handed out by another allocator or a fixed HBM budget. This entry
// point serves them: it keeps its scratch (the thresholded bit mask before
// dilation) in one file-scope device array instead of a context workspace,
// and allocates nothing.
//
// The array is kStaticScratchBytes = 32 MiB on every GPU that loads the
// library, held until the process exits. It fits the mask of a volume with at
// most 2^23 mask words (rows * ceil(nx/32)), e.g. 512^3 voxels or sixteen
// 4096 x 4096 images; larger volumes are rejected with ROIX_EINVAL before
// anything is enqueued. All calls share the array and it keeps the last
// call's contents; the threshold kernel overwrites every word it later reads,
// so nothing needs clearing except the caller's popcount output. Calls whose
// work overlaps on the GPU (different streams, or different host threads on
// the same device) race on the array and must be serialised by the caller.
#include <mutex>

#include "roix_internal.cuh"

using namespace roix;

namespace {

constexpr size_t kStaticScratchBytes = size_t(32) << 20;
constexpr u64 kStaticMaxWords = kStaticScratchBytes / 4;

__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void* g_scratch_addr[kMaxDevices] = {};
int g_scratch_sms[kMaxDevices] = {};

// Device address of the array on the current device. In host code the
// array's name is only a host-side stand-in, so the address is looked up with
// that device current. The lookup is repeated on every call whose stream is
// not capturing (a device reset reloads the module, possibly elsewhere); a
// call on a capturing stream uses the address of the last lookup on that
// device, and the first call on a device must come before any stream capture.
cudaError_t scratch_for_current_device(cudaStream_t stream, void** addr, int* sms) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  const bool capturing =
      cudaStreamIsCapturing(stream, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone;
  if (capturing) cudaGetLastError();  // clear a refusal of the query itself
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!capturing || !g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    int n = 0;
    e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    g_scratch_sms[dev] = n > 0 ? n : 1;
    g_scratch_addr[dev] = p;
  }
  *addr = g_scratch_addr[dev];
  *sms = g_scratch_sms[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" roix_status roix_extract_roi_static(const void* in, roix_dtype dtype, roix_dims dims,
                                               const roix_roi* roi, uint32_t* mask_out,
                                               uint64_t* popcount_dev, void* stream) {
  if (!roi) return ROIX_EINVAL;
  Desc d;
  if (make_desc(nullptr, dtype, dims, roi, nullptr, nullptr, &d) != ROIX_OK) return ROIX_EINVAL;
  if (d.rows * d.W > kStaticMaxWords) return ROIX_EINVAL;  // beyond the static scratch
  if (d.keep) return ROIX_EINVAL;
  if ((d.N && (!in || !mask_out)) || !popcount_dev) return ROIX_EINVAL;
  cudaStream_t cs = (cudaStream_t)stream;
  void* scratch = nullptr;
  int sms = 0;
  if (scratch_for_current_device(cs, &scratch, &sms) != cudaSuccess) {
    cudaGetLastError();
    return ROIX_ECUDA;
  }
  Launch L{cs, sms};
  if (cudaMemsetAsync(popcount_dev, 0, 8, cs) != cudaSuccess) {
    cudaGetLastError();
    return ROIX_ECUDA;
  }
  u32* T = reinterpret_cast<u32*>(scratch);
  static thread_local Batch B;  // kernel argument, built on the host
  make_threshold_batch(B, d, in, T);
  launch_threshold(L, B);
  launch_dilate(L, d, T, mask_out, (u64*)popcount_dev);
  return cudaGetLastError() == cudaSuccess ? ROIX_OK : ROIX_ECUDA;
}
