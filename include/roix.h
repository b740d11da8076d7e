/* libroix: GB300 (sm_103a) implementation of the ROIX-Comp hot path.
 *
 * ROIX-Comp (arXiv 2602.15917) compresses X-ray CT data by keeping only the
 * region of interest: background subtraction and binarisation (Sec. 4.1),
 * extraction of the object as row geometry plus a pixel section (Sec. 4.2.1-
 * 4.2.2), error-bounded quantisation of the pixels (Sec. 4.2.3) and an
 * error-bounded prediction + entropy coder in the role of Sz3 (Sec. 4.3), with
 * the matching reconstruction (Sec. 4.3, decompression).
 *
 * Conventions for every call:
 *  - Volumes are (nx, ny, nz) with x fastest: voxel (x, y, z) sits at index
 *    x + nx * (y + ny * z); row r = y + ny * z holds nx voxels. 1 <= nx <= 65534.
 *    A 2D image is nz = 1. Any of nx, ny, nz may be 0 only for an empty volume.
 *  - Every data pointer is DEVICE memory owned by the caller (e.g. a tensor's
 *    data pointer), unless the name ends in _host. Pointers to parameter structs
 *    are host memory and are read before the call returns.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Calls only enqueue work on it and return; outputs are valid once the
 *    stream has reached that point. Counts produced on the device are written
 *    to *_dev outputs (device memory), never returned on the host.
 *  - Argument errors are returned at once (ROIX_EINVAL) and nothing is
 *    enqueued. Errors found on the device (a container that does not fit its
 *    buffer, a corrupt container, a wait that ran out) are recorded in the
 *    context's status word; roix_sync() returns the first one and clears it.
 *    No call traps the GPU on any input; outputs are unspecified after an error.
 *  - A context is used from one host thread and one stream at a time: its
 *    workspace is shared by the calls made on it. Use one context per stream
 *    for concurrent work. Workspace grows on demand (cudaMalloc, which
 *    synchronises the device); roix_reserve() pre-sizes it.
 */
#ifndef ROIX_H_
#define ROIX_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  ROIX_OK = 0,
  ROIX_EINVAL = 1,     /* bad argument: nothing was enqueued */
  ROIX_ENOMEM = 2,     /* device workspace could not be allocated */
  ROIX_ECAPACITY = 3,  /* output buffer too small; *size_dev holds the size needed */
  ROIX_ECORRUPT = 4,   /* container inconsistent with itself or with size/dims/dtype */
  ROIX_ETIMEOUT = 5,   /* a bounded inter-block wait ran out (results invalid) */
  ROIX_ECUDA = 6,      /* a CUDA runtime call failed (see roix_last_error) */
  ROIX_EBUSY = 7
} roix_status;

/* ROIX_U8 is the 8-bit normalised image of Sec. 4.1.2 (roix_normalize8). It is
 * accepted by the region and compaction stages (roix_extract_roi,
 * roix_extract_roi_static, roix_compact), where it behaves like uint16 (v =
 * raw - dark, integer comparisons), and its pixel section is quantised by
 * roix_greedy_quantize; the linear quantiser, the coder and the container
 * (roix_quantize, roix_encode, roix_compress*, roix_decode) refuse it. */
typedef enum { ROIX_F32 = 1, ROIX_U16 = 2, ROIX_U8 = 3 } roix_dtype;

typedef struct {
  uint64_t nx, ny, nz;
} roix_dims;

/* Region of interest (Sec. 4.1.1, 4.1.3-4.1.4, 4.2.1):
 *   v = value (float32) or raw - dark (uint16, exact integer: M = I - B with a
 *       constant background level B);
 *   T = [v > threshold] (cmp 0) or [v < threshold] (cmp 1), comparison of the
 *       exact value against the binary64 threshold; NaN is never in T;
 *   keep = 1: T is reduced to its largest connected component (most voxels,
 *       ties to the component holding the smallest voxel index) under 6- or
 *       26-connectivity (4 or 8 in 2D): the paper's "largest object" step;
 *   D = T dilated by the (2*dilate+1)^3 cube (3x3 in 2D), clipped at the
 *       borders; D is the set of retained voxels. */
typedef struct {
  int32_t cmp;           /* 0: v > threshold, 1: v < threshold */
  int32_t keep;          /* 0: all of T, 1: largest component of T */
  int32_t connectivity;  /* 6 or 26 */
  int32_t dilate;        /* 0 or 1 */
  double threshold;
  double dark;           /* uint16: integer in [0, 65535]; float32: must be 0 */
} roix_roi;

/* Error bound (Sec. 4.2.3: E_abs with |Q - D| <= E_abs on every retained voxel).
 * mode 0: E_abs = value. mode 1: E_abs = value * (max - min) over the finite
 * retained values (the value-range convention of Sz3, applied to the pixel
 * section as in ROIX-Sz3). value must be finite and > 0 (uint16 mode 0: >= 0,
 * integer part used; 0 = lossless). */
typedef struct {
  int32_t mode;
  double value;
} roix_eb;

/* Entropy-coder settings and the reconstruction fill value. */
typedef struct {
  uint32_t radius;  /* R: deltas with |d| < R are coded as symbol d + R;
                       2 <= R <= 2048 (default 512) */
  uint32_t chunk;   /* C: symbols per independently decodable chunk; a power of
                       two in [256, 16384] (default 4096) */
  double fill;      /* value of non-retained voxels after decoding (uint16:
                       integer in [0, 65535]) */
  uint32_t predictor; /* 1D Lorenzo order along the pixel section: 0 or 1 = first
                       order (predict q[k-1]), 2 = two-layer Lorenzo (predict
                       2 q[k-1] - q[k-2]); stored in the container header */
} roix_params;

/* Error-bound constants as computed on the device (written by roix_quantize,
 * read by roix_encode). Layout is fixed: 40 bytes. */
typedef struct {
  double eb_abs;            /* E_abs */
  double vmin, vmax;        /* finite range of the retained values */
  float two_eb, inv2eb;     /* float32 lattice step and its reciprocal */
  float bound;              /* acceptance bound of |x - x_hat| (< E_abs) */
  int32_t eb_int;           /* uint16: integer half-width */
} roix_eb_info;

typedef struct roix_ctx roix_ctx;
typedef struct roix_server roix_server;

/* ----------------------------------------------------------- context */
roix_status roix_ctx_create(int device, roix_ctx** out);
roix_status roix_ctx_destroy(roix_ctx* ctx);
/* Pre-sizes the workspace to at least `bytes` (call before graph capture). */
roix_status roix_reserve(roix_ctx* ctx, size_t bytes);
/* Workspace bytes roix_compress needs for this volume. */
size_t roix_workspace_size(roix_dtype dtype, roix_dims dims, const roix_roi* roi,
                           const roix_params* params, uint64_t cap);
/* Waits for `stream`, returns the first device-side error since the last call
 * (or ROIX_ECUDA) and clears it. */
roix_status roix_sync(roix_ctx* ctx, void* stream);

/* Bounded device waits. Some kernels wait on another block of the same launch
 * (the look-back of the tile scans of compaction and packing, the decoder's
 * row scans, the run scan of the largest-component step). Each wait gives up
 * after `polls` polls (0: the default, 2^22, several hundred milliseconds),
 * records ROIX_ETIMEOUT in the context status and lets its launch end; the
 * later kernels of the same call then do nothing, so no output is formed from
 * the missing prefix. roix_sync returns ROIX_ETIMEOUT and clears it, and the
 * context stays usable. Not in the paper: it is how the library keeps a GPU
 * from hanging. */
roix_status roix_set_wait_limit(roix_ctx* ctx, uint32_t polls);
/* Test hook for the bounded waits (no paper counterpart). While `on` is
 * nonzero, the first tile of every tile scan that the context launches
 * (compaction and pack scans of the first item of a batch, decoder row scans)
 * never publishes its prefix: a flag that nobody sets, so the tile after it
 * waits until its limit runs out. Off by default. */
roix_status roix_debug_hold_scans(roix_ctx* ctx, int on);
const char* roix_last_error(const roix_ctx* ctx);
const char* roix_status_string(roix_status s);
/* Words of a bit mask: rows = ny*nz rows of ceil(nx/32) uint32 words; voxel x
 * of a row is bit (x % 32) of word (x / 32); bits at x >= nx are 0. */
uint64_t roix_mask_words(roix_dims dims);
/* Upper bound of a container's size in bytes for this volume (worst case:
 * every voxel retained, every value an outlier). */
uint64_t roix_compress_bound(roix_dtype dtype, roix_dims dims, const roix_params* params);

/* ------------------------------------------------------------- stages
 * Chained, the four stages give the bytes of roix_compress:
 *   extract_roi -> compact -> quantize -> encode. */

/* Sec. 4.1-4.2.1: retained-voxel mask D (layout of roix_mask_words) and its
 * voxel count (*popcount_dev, uint64). */
roix_status roix_extract_roi(roix_ctx* ctx, const void* in, roix_dtype dtype, roix_dims dims,
                             const roix_roi* roi, uint32_t* mask_out, uint64_t* popcount_dev,
                             void* stream);

/* Sec. 4.2.2: geometry and pixel section of the voxels set in `mask`.
 *  pixels_out: the retained values in voxel order (dtype; room for every voxel
 *              of the volume, nx*ny*nz values);
 *  counts_out: per row, the number of boundaries (uint16, ny*nz entries);
 *  bounds_out: the boundaries, row after row: x positions where the mask turns
 *              on (x_start) or off (x_end, one past the last voxel), so a row's
 *              runs are [b0, b1), [b2, b3), ...; room for bounds_cap entries;
 *  sizes_dev:  [0] = n retained voxels, [1] = number of boundaries (uint64).
 *  More than bounds_cap boundaries sets ROIX_ECAPACITY. */
roix_status roix_compact(roix_ctx* ctx, const void* in, roix_dtype dtype, roix_dims dims,
                         const uint32_t* mask, void* pixels_out, uint16_t* counts_out,
                         uint16_t* bounds_out, uint64_t bounds_cap, uint64_t* sizes_dev,
                         void* stream);

/* Sec. 4.2.3: error-bounded quantisation of a pixel sequence D[0..n-1] into
 * codes Q with |Q*2E_abs - D| <= E_abs (float32: reconstruction checked in
 * binary32; values that fail, and non-finite ones, are outliers: bit k of
 * outlier_bits_out set, q_out[k] = 0). n = *n_dev when n_dev is not NULL (it
 * must not exceed n_cap), else n_cap. Writes the constants to *info_dev. */
roix_status roix_quantize(roix_ctx* ctx, const void* pixels, roix_dtype dtype, uint64_t n_cap,
                          const uint64_t* n_dev, const roix_eb* eb, double dark,
                          int32_t* q_out, uint32_t* outlier_bits_out,
                          roix_eb_info* info_dev, void* stream);

/* Sec. 4.3: prediction (1D Lorenzo over the pixel section), canonical Huffman
 * coding and the container. Inputs are the outputs of the three calls above
 * (sizes_dev of roix_compact). Writes at most `cap` bytes to `out` and the
 * container size to *size_dev (uint64; the size needed if it exceeds cap,
 * with ROIX_ECAPACITY). */
roix_status roix_encode(roix_ctx* ctx, const int32_t* q, const uint32_t* outlier_bits,
                        const void* pixels, uint64_t n_cap, const uint64_t* sizes_dev,
                        const uint16_t* counts, const uint16_t* bounds,
                        const roix_eb_info* info_dev, roix_dtype dtype, roix_dims dims,
                        const roix_roi* roi, const roix_eb* eb, const roix_params* params,
                        void* out, uint64_t cap, uint64_t* size_dev, void* stream);

/* Sec. 4.3, decompression: rebuilds the volume (dtype, dims must match the
 * container) from `size` bytes at `in`. Retained voxels get their
 * error-bounded value, the others params.fill. */
roix_status roix_decode(roix_ctx* ctx, const void* in, uint64_t size, void* out,
                        roix_dtype dtype, roix_dims dims, void* stream);

/* Sec. 4.1.2: 8-bit intensity normalisation I_n = I / I_max * 255 of the
 * background-subtracted image (Sec. 4.1.1): v = x for float32 input (negative
 * and non-finite values count as 0), v = max(raw - dark, 0) for uint16 (dark an
 * integer in [0, 65535]). I_max is the largest v of the count = nx*ny*nz
 * values at `in`; I_max = 0 maps every voxel to 0.
 *  float32: I_n = rint(fl(fl(v / I_max) * 255)) in binary32, round half to
 *           even, at most 255;
 *  uint16:  I_n = the exact rational 255 v / I_max rounded half to even.
 * out: count uint8 values (device). imax_dev: I_max as a double (device, may
 * be NULL). Buffers are the caller's; `in` and `out` may not overlap. Two
 * passes over the input (the maximum, then the scaling). */
roix_status roix_normalize8(roix_ctx* ctx, const void* in, roix_dtype dtype, roix_dims dims,
                            double dark, uint8_t* out, double* imax_dev, void* stream);

/* Sec. 4.2.3: the greedy absolute-error-bounded quantiser over the pixel
 * section of an 8-bit image. Every row's retained pixels (the bits of `mask`
 * in that row, layout of roix_mask_words) form one pixel sequence P(i) of
 * Sec. 4.2.2; `pixels` holds the sequences row after row (the pixel section
 * roix_compact writes for a ROIX_U8 image). Each sequence is cut greedily into
 * groups whose acceptable sets [D - E_abs, D + E_abs] share an integer; a
 * group's value is floor((u + l) / 2) of that shared interval [l, u], so
 * |Q - D| <= E_abs for every pixel and Q is in [0, 255]. Q is integer (it is
 * stored in 8 bits), so only floor(E_abs) matters; eabs must be finite and
 * >= 0 (eabs < 1 returns Q = D).
 *  q_out: n uint8 values (device), n = popcount of the mask; n_dev (device,
 *  uint64, may be NULL) receives n. `pixels` must hold n values; q_out may
 *  equal pixels (in place) but may not overlap it otherwise. */
roix_status roix_greedy_quantize(roix_ctx* ctx, const uint8_t* pixels, const uint32_t* mask,
                                 roix_dims dims, double eabs, uint8_t* q_out,
                                 uint64_t* n_dev, void* stream);

/* roix_greedy_quantize over several images in one call (same E_abs): their
 * rows are scanned together, so that small images fill the device. Items are
 * independent; n_dev of each (may be NULL) receives its pixel count. */
typedef struct {
  const uint8_t* pixels;
  const uint32_t* mask;
  roix_dims dims;
  uint8_t* q_out;
  uint64_t* n_dev;
} roix_greedy_item;
roix_status roix_greedy_quantize_batch(roix_ctx* ctx, uint32_t n, const roix_greedy_item* items,
                                       double eabs, void* stream);

/* Paper-mode region of interest of an 8-bit image (Sec. 4.1.3-4.2.2), every
 * 2D slice (z) on its own:
 *  1. multi-Otsu with three classes [0, t1], (t1, t2], (t2, 255] on the
 *     slice's 256-bin histogram: the pair t1 < t2 of [0, 254] maximising the
 *     sum over the classes of (sum of values)^2 / count (the between-class
 *     variance up to constants; binary64, empty classes add 0), ties to the
 *     smallest (t1, t2);
 *  2. M = [I_n > t1];
 *  3. holes filled: background 4-connected to no slice border becomes object
 *     (the region inside the external contours);
 *  4. the largest 8-connected object of the filled mask by pixel count, ties
 *     to the one holding the smallest raster index;
 *  5. one span per row: [x_start, x_end) from its leftmost to its rightmost
 *     pixel, gaps included.
 * mask_out: the spans in the layout of roix_mask_words; *popcount_dev: their
 * pixel count (uint64); thresholds_dev (may be NULL): (t1, t2) per slice as
 * uint32. Workspace about 50 bytes per row and 14 per pixel. */
roix_status roix_extract_roi_paper(roix_ctx* ctx, const uint8_t* img, roix_dims dims,
                                   uint32_t* mask_out, uint64_t* popcount_dev,
                                   uint32_t* thresholds_dev, void* stream);

/* ------------------------------------------------ evaluation metrics */
/* Sec. 5.2: quality of a predicted ROI A against a ground truth B, both bit
 * masks in the layout of roix_mask_words. Counts TP = |A and B|, FP = |A and
 * not B|, FN = |B and not A|, TN = the rest; the ratios are the section's
 * equations in binary64, one IEEE operation at a time in their printed order:
 *   DSC = 2TP / ((TP + FP) + (TP + FN)),  IoU = TP / (TP + FP + FN),
 *   sensitivity = TP / (TP + FN),  specificity = TN / (TN + FP),
 *   accuracy = (TP + TN) / (TP + TN + FP + FN),
 *   f_c = ((TN + FN)(TN + FP) + (FP + TP)(FN + TP)) / (TP + TN + FN + FP),
 *   kappa = ((TP + TN) - f_c) / ((TP + TN + FN + FP) - f_c),
 *   AUC = 1 - (FP / (FP + TN) + FN / (FN + TP)) / 2;
 * a zero denominator gives NaN or inf as IEEE division does. With distances =
 * 1 also the average Hausdorff distance AHD = max(sum_ab / |A|, sum_ba / |B|),
 * sum_ab = sum over a in A of the Euclidean distance (voxel units) to the
 * nearest voxel of B (exact distance transform), sum_ba the reverse; NaN when
 * A or B is empty. The sums are accumulated with binary64 atomics (order not
 * fixed). Distances need (nx-1)^2 + (ny-1)^2 + (nz-1)^2 < 2^32 - 1 and a
 * workspace of about 8 bytes per voxel. out_dev: one roix_roi_metrics on the
 * device. */
typedef struct {
  uint64_t tp, fp, fn, tn;
  double dsc, iou, sensitivity, specificity, accuracy, kappa, auc, ahd;
  double sum_ab, sum_ba;
} roix_roi_metrics;
roix_status roix_roi_quality(roix_ctx* ctx, const uint32_t* pred_mask, const uint32_t* truth_mask,
                             roix_dims dims, int distances, roix_roi_metrics* out_dev,
                             void* stream);

/* Sec. 5.6: structural similarity of x and y (same dtype and dims; float32,
 * uint16 or uint8), in the form of Wang, Bovik, Sheikh and Simoncelli (2004):
 * Gaussian weights (sigma 1.5, 11 x 11, normalised), population moments,
 * C1 = (0.01 L)^2, C2 = (0.03 L)^2 with L = data_range, evaluated on every 2D
 * slice (z) at every position where the window lies inside the slice, and
 * averaged over all those positions (binary64; sums by atomics, order not
 * fixed). Slices smaller than 11 x 11 give NaN. ssim_dev: one double. */
roix_status roix_ssim(roix_ctx* ctx, const void* x, const void* y, roix_dtype dtype,
                      roix_dims dims, double data_range, double* ssim_dev, void* stream);

/* Allocation-free variant of roix_extract_roi, for callers that cannot
 * allocate device memory when they need a mask: acquisition loops that must
 * never block on the device synchronisation that cudaMalloc/cudaFree imply,
 * and processes whose device memory all belongs to another allocator or a
 * fixed budget. The paper has no counterpart; this is an interface choice.
 * Same inputs, outputs and results as roix_extract_roi, without a context: it
 * runs on the calling thread's current CUDA device. Its scratch (the mask
 * before dilation) is a 32 MiB device array in the library itself, present on
 * every GPU that loads the library until the process exits; volumes needing
 * more than 2^23 mask words (ny*nz*ceil(nx/32)) return ROIX_EINVAL before
 * anything is enqueued. The array's device address is looked up on every call
 * whose stream is not capturing (so a device reset, which may move the array,
 * is followed); a call on a capturing stream reuses the last address found on
 * that device, so make the first call on a device before any stream capture.
 * All calls share the array: calls that overlap on the GPU (other streams or
 * host threads on the same device) race and must be serialised by the caller.
 * Nothing is allocated: no cudaMalloc, no cudaFree. */
roix_status roix_extract_roi_static(const void* in, roix_dtype dtype, roix_dims dims,
                                    const roix_roi* roi, uint32_t* mask_out,
                                    uint64_t* popcount_dev, void* stream);

/* Per-stage timing: with profiling on, roix_compress records a CUDA event on
 * its stream after each stage; roix_profile_read waits for them and writes up
 * to `max` stage durations (ms) of the last call, returning their number. The
 * stages are: reset, binarisation, compaction, symbols, codebook, pack,
 * finalise. */
roix_status roix_profile(roix_ctx* ctx, int on);
int roix_profile_read(roix_ctx* ctx, float* ms, int max);

/* One volume or image of a batch (device pointers, caller-owned). */
typedef struct {
  const void* in;      /* input values (dtype of the batch), nx*ny*nz of them */
  roix_dims dims;
  void* out;           /* container buffer, 16-byte aligned */
  uint64_t cap;        /* its size in bytes */
  uint64_t* size_dev;  /* container size (uint64, device), as for roix_compress */
} roix_item;

/* Batched fused path (no paper counterpart; a throughput form of
 * roix_compress): n independent items sharing dtype and settings are
 * compressed together, 64 items per group of 7 kernel launches whose work
 * tickets run over all items of the group; each item's container is the one
 * roix_compress would write for it alone. Enqueued on `stream`, capturable in
 * a CUDA graph once the workspace is reserved (roix_reserve with
 * roix_workspace_size of the largest group). */
roix_status roix_compress_batch(roix_ctx* ctx, uint32_t n, const roix_item* items,
                                roix_dtype dtype, const roix_roi* roi, const roix_eb* eb,
                                const roix_params* params, void* stream);

/* A volume in z-slabs (no paper counterpart; the streaming form of
 * roix_compress for volumes of tens of GB, e.g. 2048^3 float32 in 64-slice
 * slabs). The volume is cut into ns = ceil(nz / slab_z) slabs of slab_z slices
 * (the last may be shorter); slab s (slices [s*slab_z, s*slab_z + dz_s)) gets a
 * container of its own, decodable alone by roix_decode as an nx x ny x dz_s
 * volume. What makes the slabs one volume:
 *  - the mask D is the whole volume's: the dilation of a slab's border slices
 *    sees the neighbouring slab's T (Sec. 4.1.4 binarisation of the whole scan);
 *  - the error bound is the whole volume's: with a relative bound, E_abs =
 *    value * (max - min) over the finite retained values of all slabs, and
 *    every container carries that E_abs and that range;
 *  - each slab's pixel section, prediction (q[-1] = 0), histogram, codebook and
 *    payload are its own, so the slabs decode independently.
 * The slabs' decodes, stacked, equal the decode of roix_compress's container
 * for the whole volume voxel for voxel; with slab_z >= nz the single container
 * is roix_compress's, byte for byte. keep = 1 is refused (ROIX_EINVAL): the
 * largest object of a slab is not the volume's. float32 and uint16 only.
 *  outs, caps: HOST arrays of ns entries: 16-byte aligned device buffers and
 *              their sizes in bytes;
 *  sizes_dev:  ns uint64 on the device: each container's size (the size needed
 *              with ROIX_ECAPACITY when it exceeds its cap).
 * Workspace: roix_slabs_workspace_size (cap = the largest slab cap); about
 * (esz + 2) bytes per voxel plus the whole volume's bit mask. */
roix_status roix_compress_slabs(roix_ctx* ctx, const void* in, roix_dtype dtype, roix_dims dims,
                                uint64_t slab_z, const roix_roi* roi, const roix_eb* eb,
                                const roix_params* params, void* const* outs,
                                const uint64_t* caps, uint64_t* sizes_dev, void* stream);
/* Workspace bytes roix_compress_slabs needs when every slab's cap is `cap`
 * (0 for invalid arguments). */
size_t roix_slabs_workspace_size(roix_dtype dtype, roix_dims dims, uint64_t slab_z,
                                 const roix_roi* roi, const roix_params* params, uint64_t cap);

/* --------------------------------------------------------------- serving
 * A serving loop for compression requests that arrive over time (no paper
 * counterpart; a deployment form of roix_compress_batch). The server holds
 * one device arena of hbm_budget bytes (allocated at creation) and `lanes`
 * contexts, each with its own stream. A batch's workspace, the device state
 * (masks, pixel sections, symbols, records, code tables) of the requests it
 * holds, is taken from the arena when the batch is admitted and returned
 * when it completes. A scheduler thread batches continuously: when a lane is
 * free and the oldest pending request's workspace fits the largest free
 * region of the arena, that request opens a batch and later pending requests
 * with the same dtype and settings join it, in arrival order, while the batch
 * has fewer than max_batch items and its workspace still fits the region;
 * otherwise the oldest request (and the queue behind it) waits until memory
 * is returned. Batches on different lanes run concurrently. Each request's
 * container is the one roix_compress writes for it alone. Requests reference
 * caller-owned device buffers that must stay valid until their completion is
 * polled. */
typedef struct {
  uint64_t hbm_budget;  /* bytes of the workspace arena the batches share */
  uint32_t lanes;       /* batches in flight at once (>= 1) */
  uint32_t max_batch;   /* requests per batch, 1..64 */
} roix_server_config;

typedef struct {
  uint64_t tag;         /* returned in the completion */
  const void* in;
  roix_dtype dtype;
  roix_dims dims;
  roix_roi roi;
  roix_eb eb;
  roix_params params;
  void* out;            /* container buffer, 16-byte aligned */
  uint64_t cap;
} roix_request;

typedef struct {
  uint64_t tag;
  int32_t status;       /* roix_status of the request */
  uint64_t size;        /* container size (bytes) */
  double t_submit, t_admit, t_done;  /* seconds since the server was created */
} roix_completion;

typedef struct {
  uint64_t submitted, completed, batches, bytes_in, max_queue, pending;
  uint64_t budget_bytes;  /* the arena */
  uint64_t in_use_bytes;  /* workspace of the batches in flight */
} roix_server_stats;

roix_status roix_server_create(int device, const roix_server_config* cfg, roix_server** out);
/* Thread-safe. ROIX_ENOMEM: the request's workspace alone exceeds the budget. */
roix_status roix_server_submit(roix_server* s, const roix_request* req);
/* Non-blocking: moves up to `max` completions to `out`, returns how many. */
uint32_t roix_server_poll(roix_server* s, roix_completion* out, uint32_t max);
/* Waits until every submitted request has completed (ROIX_ETIMEOUT otherwise). */
roix_status roix_server_drain(roix_server* s, double timeout_s);
roix_status roix_server_get_stats(roix_server* s, roix_server_stats* out);
/* Finishes the pending requests, then releases the lanes. */
roix_status roix_server_destroy(roix_server* s);

/* ------------------------------------------------------------ autotuner
 * Launch shapes of the compression kernels (no paper counterpart). None of
 * them changes an output byte: they set the compaction tile size and counting
 * kernel and how many blocks of the binarisation, symbol and pack kernels are
 * resident per SM. */
typedef struct {
  uint32_t front_words;         /* mask words per compaction tile, 256..16384 (2048) */
  uint32_t thr_blocks_per_sm;   /* binarisation, row form, 1..32 (8) */
  uint32_t flat_blocks_per_sm;  /* binarisation, flat form, 1..32 (4) */
  uint32_t sym_blocks_per_sm;   /* symbols, 0..32, 0 = as many as fit (0) */
  uint32_t pack_blocks_per_sm;  /* pack, 0..32, 0 = as many as fit (0) */
  uint32_t front_kernel;        /* compaction counts: 0 = a block per tile, its rows staged
                                   in shared memory; 1 = a warp per tile, rows walked with a
                                   register window (0) */
} roix_tuning;
roix_status roix_get_tuning(const roix_ctx* ctx, roix_tuning* out);
/* ROIX_EINVAL for values out of range (nothing changed). */
roix_status roix_set_tuning(roix_ctx* ctx, const roix_tuning* t);
/* Picks the context's launch shapes for a workload: times roix_compress_batch
 * on the caller's items (real inputs and output buffers; containers are
 * overwritten) for the candidates of one parameter at a time, in pipeline
 * order, keeping a value only when the median of `reps` calls (0 = 5) is at
 * least 1 % faster. cache_path (NULL: the ROIX_TUNE_CACHE environment
 * variable, if set): a JSON file of tuned shapes keyed by device name, dtype
 * and shape class (x extent and voxels per item rounded up to powers of two,
 * item count bucket, dilation, keep); an entry found there is applied without
 * timing and a new result is written back. Synchronises `stream`; the
 * workspace may grow (do it before capturing graphs). *out (may be NULL)
 * receives the result. */
roix_status roix_tune(roix_ctx* ctx, uint32_t n, const roix_item* items, roix_dtype dtype,
                      const roix_roi* roi, const roix_eb* eb, const roix_params* params,
                      uint32_t reps, const char* cache_path, roix_tuning* out, void* stream);

/* The fused path: the same bytes as the four stages, in fewer passes. */
roix_status roix_compress(roix_ctx* ctx, const void* in, roix_dtype dtype, roix_dims dims,
                          const roix_roi* roi, const roix_eb* eb, const roix_params* params,
                          void* out, uint64_t cap, uint64_t* size_dev, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* ROIX_H_ */
