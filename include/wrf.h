/*
 * wrf.h - C ABI of the B300 (sm_103a) spectrum-synthesis library.
 *
 * Implements the spectrum-synthesis path of SwiftWRF, "Deformable 2D Gaussian
 * Splatting for Efficient Wireless Radiance Field Rendering" (arXiv 2506.12787):
 * the problem F: R^3 -> spectrum (Sec. 3.3.2) solved by a deformation MLP over
 * 2D Gaussians (Sec. 4.2, Eqs. 12-15) followed by tile rasterisation of the
 * order-free Gaussian sum (Sec. 4.1, Eqs. 8-9, 13).
 *
 * Conventions shared by every entry point
 *   - Pointers named *device* are CUDA device pointers; they are owned by the
 *     caller and must stay valid until the work queued on `stream` finishes.
 *     Scratch space is passed in as `ws` (size from the matching
 *     *_workspace_size call), 256-byte aligned; no call on the path
 *     allocates device memory (only the wrf_measure_alu_peaks diagnostic
 *     does, a 4-byte sink, and the host-to-host pipeline, which owns its
 *     buffers: see wrf_pipeline_create).
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Every call
 *     only enqueues work and returns; nothing synchronises the host (except
 *     wrf_status_read and the pipeline's step and wait, as documented).
 *   - Host buffers: every array argument is a device pointer, except in the
 *     host-to-host pipeline (wrf_pipeline_*), which takes TX positions and
 *     returns spectra in host memory, overlapping one step's copies with the
 *     next step's compute.
 *   - Argument errors are detected on the host and returned before any work
 *     is queued (WRF_EINVAL / WRF_EUNSUPPORTED).  A failed launch returns
 *     WRF_ECUDA.  Conditions only the device can see (key-capacity overflow,
 *     a bounded wait that ran out) are recorded in a library-global device
 *     status word that wrf_status_read() returns (and clears).
 *   - wrf_last_error() returns a thread-local message for the last non-OK
 *     status returned on the calling thread.
 *   - Spectrum layout: FP32 [Q][H][W] row-major; row y = elevation index,
 *     column x = azimuth index (Sec. 3.1, Eq. 5: 90 rows x 360 columns at
 *     1 degree).  Pixel (x, y) is sampled at integer coordinates (x, y).
 *   - Channels: one (C = 1, the scalar signal response) everywhere; two
 *     (real and imaginary amplitude, Sec. 6.1) for the forward calls, with
 *     wrf_render_complex giving magnitude and phase.  The backward calls take
 *     one channel.
 */
#ifndef WRF_H
#define WRF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    WRF_OK = 0,
    WRF_EINVAL = -1,       /* bad argument (null pointer, size, alignment)       */
    WRF_ENOSPC = -2,       /* key capacity too small; required count reported    */
    WRF_ECUDA = -3,        /* a CUDA launch or runtime call failed               */
    WRF_ETIMEOUT = -4,     /* a bounded device-side wait gave up                 */
    WRF_EUNSUPPORTED = -5  /* valid request outside what the kernels implement   */
} wrf_status;

/* Network precision.  WRF_BF16X3: every FP32 operand split into BF16
 * hi + lo = bf16(x) + bf16(x - bf16(x)) and every product taken as
 * hi hi + hi lo + lo hi on the tensor cores with FP32 accumulation
 * (relative error ~2^-17 per product). */
enum { WRF_FP32 = 0, WRF_BF16 = 1, WRF_BF16X3 = 2 };
enum { WRF_MAX_LAYERS = 8, WRF_HIDDEN = 128, WRF_OUT = 5 };

/* Reference-frame Gaussians G^0 (Sec. 4.2, Eq. 10-12), structure of arrays,
 * FP32, device.  Per Gaussian: centre mean[2] in pixels (x, y); log_scale[2]
 * = natural log of the two principal standard deviations in pixels; rot =
 * angle of the first principal axis (radians); opacity_logit a with
 * attenuation delta = sigmoid(a) (Sec. 4.1); amp = scalar response psi. */
typedef struct {
    int32_t n;                   /* number of Gaussians N (>= 0)              */
    int32_t channels;            /* 1, or 2: real and imaginary amplitude     */
    const float *mean;           /* [N][2] device                             */
    const float *log_scale;      /* [N][2] device                             */
    const float *rot;            /* [N]    device                             */
    const float *opacity_logit;  /* [N]    device                             */
    const float *amp;            /* [N][channels] device                      */
} wrf_scene;

/* Deformation MLP F_theta (Sec. 4.2, Eq. 14): input [gamma(mean/(W,H)),
 * gamma((tx - room_min)/room_size)] with gamma from Eq. 15 (L_mean and L_tx
 * frequency bands), n_layers Linear layers with ReLU between them, output
 * (dx, dy, drot, dlog_scale1, dlog_scale2).  Weights are FP32, device,
 * W[l] is [dims[l+1]][dims[l]] row-major, b[l] is [dims[l+1]].
 * Supported: dims[0] = 2(2 L_mean + 1) + 3(2 L_tx + 1), hidden widths 128,
 * 2 <= n_layers <= 8, output width 5.  precision = WRF_BF16 runs the hidden
 * layers on tcgen05 tensor cores with BF16 operands and FP32 accumulation;
 * WRF_BF16X3 runs the hidden and output layers on the tensor cores with
 * three BF16 products per FP32 product (FP32-level results; the first
 * layer stays in FP32 on the CUDA cores); WRF_FP32 runs everything in FP32
 * on the CUDA cores.  Both tensor-core precisions take n_layers <= 5 (the
 * weights stay resident in shared memory). */
typedef struct {
    int32_t n_layers;
    int32_t dims[WRF_MAX_LAYERS + 1];
    const float *W[WRF_MAX_LAYERS];
    const float *b[WRF_MAX_LAYERS];
    int32_t L_mean, L_tx;
    float room_min[3], room_size[3];
    int32_t precision;           /* WRF_FP32, WRF_BF16 or WRF_BF16X3          */
} wrf_mlp;

/* Spectrum grid and tiling.  A Gaussian contributes to pixel p only where
 * q = d^T Sigma^-1 d <= q_cut (d = p - centre); q_cut = +inf disables the
 * cutoff.  Tiles are tile_w x tile_h pixels, numbered row-major; the last
 * tile row/column may be partial.  Supported tile shapes: 8x8, 16x8, 16x16,
 * 32x8, 32x16 (w x h); H, W <= 65536 and at most 3000 tiles (else
 * WRF_EUNSUPPORTED / WRF_EINVAL).
 * wrap_x = 1 makes the azimuth axis periodic (columns 0 and W the same
 * direction, as for a 0-360 degree spectrum): every Gaussian also acts through
 * its images centre + k W, tile lists cover columns modulo W, and each tile is
 * rendered with the image nearest to it; this needs q_cut finite and every
 * footprint narrower than W - tile_w pixels (2 rx < W - tile_w), else the
 * device status word records WRF_EUNSUPPORTED.  wrap_x = 0: a flat plane
 * clipped at the edges.
 * Rasteriser knobs (they change how the work is laid out, not the result
 * beyond FP32 summation order, which they keep: each pixel sums its
 * Gaussians in the same ascending order whatever the knobs):
 *   px_per_thread  pixels one thread accumulates: 2 (default) or 4 (needs
 *                  tile_w >= 16);
 *   batch_factor   Gaussian records each thread stages per shared-memory
 *                  batch: 1 (default) or 2 (a batch then holds 2 x threads
 *                  records);
 *   tma_staging    how the records reach shared memory: 0 (default) each
 *                  thread copies the records it sets up with cp.async; 1 TMA
 *                  gathers (cp.async.bulk.tensor tile::gather4, four records
 *                  per copy, completion on an mbarrier).  The same bytes land
 *                  in the same slots either way.
 * 0 selects the default.  Both renderers (wrf_render, wrf_render_complex)
 * take every combination. */
typedef struct {
    int32_t H, W;
    int32_t tile_w, tile_h;
    float q_cut;
    int32_t wrap_x;
    int32_t px_per_thread;
    int32_t batch_factor;
    int32_t tma_staging;
} wrf_grid;

/* Projected record of one deformed Gaussian for one query: 8 floats, 32-byte
 * aligned, [Q][N][8]:
 *   [0] mx, [1] my     deformed centre (pixels)
 *   [2] a, [3] b, [4] c  inverse covariance scaled by log2(e)/2, so that
 *                      exp(-q/2) = exp2(-(a dx^2 + 2 b dx dy + c dy^2))
 *   [5] w              sigmoid(opacity_logit) * amp (amp[n][0])
 *   [6] rx, [7] ry     sqrt(q_cut Sigma_xx), sqrt(q_cut Sigma_yy): axis
 *                      half-widths of the q <= q_cut ellipse
 * With a 2-channel scene (real and imaginary amplitude, Sec. 6.1) the record
 * buffer holds Q x N x 8 floats followed by Q x N imaginary weights
 * sigmoid(opacity_logit) * amp[n][1] ([Q][N]): the writers (wrf_project,
 * wrf_deform_project) fill both and the caller allocates Q x N x 9 floats;
 * wrf_bin reads the records only, wrf_render_complex both parts.            */
enum { WRF_REC_FLOATS = 8 };

/* ---------------------------------------------------------------------- */
/* Deformation: residuals for every (query, Gaussian) row, Sec. 4.2 Eq. 14
 * (with the positional encoding of Eq. 15).
 *   tx     [Q][3] device, TX positions in metres.
 *   resid  [Q][N][5] device output (dx, dy, drot, dls1, dls2).
 *   ws     workspace of wrf_deform_workspace_size(N, Q, mlp) bytes.        */
size_t wrf_deform_workspace_size(int32_t n, int32_t Q, const wrf_mlp *mlp);
wrf_status wrf_deform(const wrf_scene *scene, const wrf_mlp *mlp, const wrf_grid *grid,
                      const float *tx, int32_t Q, float *resid, void *ws, size_t ws_bytes,
                      void *stream);

/* As wrf_deform, and also stores every hidden activation for the backward
 * (training): acts [n_layers - 1][Q][N][128] FP32 device, row-major, layer l
 * = the output of hidden layer l + 1 after its ReLU (the first entry is the
 * first layer's output).  mlp->precision must be WRF_FP32 or WRF_BF16X3
 * (else WRF_EUNSUPPORTED).  Needs (n_layers - 1) x Q x N x 512 bytes.     */
wrf_status wrf_deform_acts(const wrf_scene *scene, const wrf_mlp *mlp, const wrf_grid *grid,
                           const float *tx, int32_t Q, float *resid, float *acts, void *ws,
                           size_t ws_bytes, void *stream);

/* Deform + project: Eq. 12-13 applied to every (query, Gaussian) row, giving
 * the projected record (layout above) and, if tile_count is non-NULL, the
 * number of tiles its footprint rectangle covers.
 *   resid      [Q][N][5] device, or NULL for no deformation (Q copies of G^0).
 *   rec        [Q][N][8] device output, 32-byte aligned.
 *   tile_count [Q][N] device output or NULL.                                */
wrf_status wrf_project(const wrf_scene *scene, const float *resid, int32_t Q,
                       const wrf_grid *grid, float *rec, uint32_t *tile_count, void *stream);

/* Fused deformation + projection: the MLP epilogue writes records directly
 * (no [Q][N][5] residual round trip through HBM).  Same outputs as
 * wrf_deform followed by wrf_project, up to FP32 rounding order.            */
wrf_status wrf_deform_project(const wrf_scene *scene, const wrf_mlp *mlp, const wrf_grid *grid,
                              const float *tx, int32_t Q, float *rec, uint32_t *tile_count,
                              void *ws, size_t ws_bytes, void *stream);

/* Tile binning (Sec. 4.1: the spectrum is partitioned into tiles processed
 * in parallel).  For every query q and tile t, lists the ids n of the
 * Gaussians whose footprint rectangle covers t, ascending in n: a stable
 * one-digit radix (counting) sort of keys (q, t, n) on the digit (q, t).
 * The footprint rectangle of a record covers pixels ceil(mx - rx) ..
 * floor(mx + rx) (x) and ceil(my - ry) .. floor(my + ry) (y), clipped to the
 * grid, computed in FP32.
 *   gids          [key_capacity] device output: n of every key, (q,t)-major.
 *   n_keys_out    device int64: total number of keys (always written).
 *   tile_offsets  [Q*T + 1] device output (CSR): keys of (q, t) are
 *                 gids[tile_offsets[q*T+t] .. tile_offsets[q*T+t+1]).
 * If the total exceeds key_capacity (or 2^32-1) no gids are written, the
 * device status word records WRF_ENOSPC and *n_keys_out holds the required
 * count; wrf_render then produces zeros for those queries.                */
size_t wrf_bin_workspace_size(int32_t n, int32_t Q, const wrf_grid *grid);
wrf_status wrf_bin(const float *rec, int32_t n, int32_t Q, const wrf_grid *grid, uint32_t *gids,
                   int64_t key_capacity, int64_t *n_keys_out, uint32_t *tile_offsets, void *ws,
                   size_t ws_bytes, void *stream);

/* wrf_bin without a caller workspace (no counterpart in the paper: it is a
 * convenience for callers that cannot allocate device memory -- for example
 * code embedded in a host application that owns the device's memory pool, or
 * a latency-critical loop where a cudaMalloc, which may synchronise the
 * device, is not allowed).  It behaves exactly like wrf_bin, with the
 * scratch space taken from a fixed 4 MiB array in device memory that the
 * library holds on every device that loads it until the process exits.
 *   - Calls whose scratch need (wrf_bin_workspace_size) exceeds 4 MiB are
 *     rejected with WRF_EINVAL before any work is queued; at 16 x 16 tiles
 *     on a 360 x 90 grid (138 tiles, so binning chunks of 512 Gaussians;
 *     grids of more than 256 tiles use chunks of 1024) that admits
 *     Q * ceil(N / 512) up to about 7,500.
 *   - The function allocates nothing (no cudaMalloc, cudaFree or allocating
 *     library call).  Its first call on a device looks the array's device
 *     address up once (cudaGetSymbolAddress) and caches it with the context's
 *     id; make that first call outside any stream capture.  After a device
 *     reset the next call looks the address up again in the new context
 *     (again outside capture).
 *   - Every call shares the one array: calls that may run at the same time
 *     on the GPU (different streams, or overlapping work on one device)
 *     race on it.  Serialise them.  The array keeps the last call's
 *     contents; binning overwrites everything it reads, so nothing needs
 *     clearing between calls.
 * Arguments and outputs are those of wrf_bin.                               */
wrf_status wrf_bin_noalloc(const float *rec, int32_t n, int32_t Q, const wrf_grid *grid,
                           uint32_t *gids, int64_t key_capacity, int64_t *n_keys_out,
                           uint32_t *tile_offsets, void *stream);

/* ---------------------------------------------------------------------- */
/* Multi-scene batches.  Each scene is its own reference frame G^0 with its
 * own deformation network (Sec. 4.2); a batch may hold queries of several
 * resident scenes, and one launch sequence serves all of them:
 *   wrf_multi_set_prepare (once)  ->  per batch: wrf_deform_project_multi,
 *   wrf_bin_multi, wrf_render_multi.
 * A query's records, tile lists and spectrum are exactly those of a
 * single-scene launch of that query (wrf_deform_project with BF16, wrf_bin,
 * wrf_render), whatever else the batch holds.
 * Scenes: 1 <= S <= 16, one channel each; every network BF16 (tensor
 * cores) with the same n_layers, bands and room (their weights differ).    */
enum { WRF_MAX_SCENES = 16 };

/* The prepared scene set: per scene the BF16 gamma(mean) rows and weight
 * images of the tensor-core network, and a device table of the scenes, in
 * `set` (device, 256-byte aligned, wrf_multi_set_size bytes).  The scenes'
 * and networks' arrays must stay valid and unchanged while the set is used
 * (prepare again after changing weights). */
size_t wrf_multi_set_size(const wrf_scene *scenes, const wrf_mlp *mlps, int32_t S);
wrf_status wrf_multi_set_prepare(const wrf_scene *scenes, const wrf_mlp *mlps, int32_t S,
                                 const wrf_grid *grid, void *set, size_t set_bytes,
                                 void *stream);

/* Deform + project a batch of Q queries: query q is TX position tx[q] in
 * scene scene_of[q] (device int32 [Q]; an index outside [0, S) gives the
 * query no Gaussians: it renders zeros).  Writes query_base (device int64
 * [Q+1]): query q's records are rows query_base[q] .. query_base[q+1]-1 of
 * rec (device, 16-byte aligned, room for rec_capacity records of 8 floats),
 * in the order of its scene's Gaussians.  The offsets are computed on the
 * device, so a captured graph serves any mix of scenes.  If the batch needs
 * more than rec_capacity records, every query is emptied (no records) and
 * the status word records WRF_ENOSPC.  rec_capacity < 2^31 (record rows are
 * addressed with 32-bit coordinates; else WRF_EUNSUPPORTED).  wrf_render_multi
 * reads only rows below query_base[Q].  scenes / mlps / S: the host arrays
 * the set was prepared from.  ws: wrf_multi_workspace_size(Q) bytes.     */
size_t wrf_multi_workspace_size(int32_t Q);
wrf_status wrf_deform_project_multi(const wrf_scene *scenes, const wrf_mlp *mlps, int32_t S,
                                    const void *set, const int32_t *scene_of, const float *tx,
                                    int32_t Q, const wrf_grid *grid, float *rec,
                                    int64_t rec_capacity, int64_t *query_base, void *ws,
                                    size_t ws_bytes, void *stream);

/* wrf_bin over a multi-scene batch: query q's records are rows
 * query_base[q] .. query_base[q+1]-1 of rec (at most n_max of them: the
 * largest scene); gids index those rows (0 = query_base[q]).  Workspace:
 * wrf_bin_workspace_size(n_max, Q, grid).  Other arguments as wrf_bin.     */
wrf_status wrf_bin_multi(const float *rec, const int64_t *query_base, int32_t n_max, int32_t Q,
                         const wrf_grid *grid, uint32_t *gids, int64_t key_capacity,
                         int64_t *n_keys_out, uint32_t *tile_offsets, void *ws, size_t ws_bytes,
                         void *stream);

/* wrf_render over a multi-scene batch (records located by query_base). */
wrf_status wrf_render_multi(const float *rec, const int64_t *query_base, const uint32_t *gids,
                            const uint32_t *tile_offsets, const int64_t *n_keys,
                            int64_t key_capacity, int32_t Q, const wrf_grid *grid, float *spectra,
                            void *stream);

/* Rasterisation, Eq. 9 / Eq. 13: A_q(y, x) = sum over the Gaussians listed
 * for the pixel's tile, ascending n, of [q <= q_cut] w exp(-q/2).  No depth
 * order, no transmittance, no clamping (order-free accumulation).
 *   spectra  [Q][H][W] device output (fully overwritten).
 *   n_keys / key_capacity as produced/used by wrf_bin.                     */
wrf_status wrf_render(const float *rec, const uint32_t *gids, const uint32_t *tile_offsets,
                      const int64_t *n_keys, int64_t key_capacity, int32_t n, int32_t Q,
                      const wrf_grid *grid, float *spectra, void *stream);

/* Training loss of Sec. 4.4, Eq. 16, over a batch of Q maps:
 *   L = lambda1 mean|pred - target| + (1 - lambda1) (1 - mean_q SSIM(pred_q, target_q)),
 * the SSIM index in its standard form (local means, variances and covariance
 * under an 11 x 11 Gaussian window with sigma 1.5 and weights summing to 1,
 * zero outside the map; C1 = 0.01^2, C2 = 0.03^2, i.e. data range 1; the
 * per-pixel index averaged over the map).  The paper uses lambda1 = 0.7.
 *   pred, target  [Q][H][W] device FP32.
 *   out           [1 + Q] device output: L, then SSIM of each map.
 *   d_pred        [Q][H][W] device output dL/dpred (sign(0) = 0 for the L1
 *                 term), or NULL to compute the loss only.
 *   ws            wrf_loss_workspace_size(Q, H, W) bytes, 256-byte aligned.
 * Sums run in a fixed order: results do not vary from run to run.          */
size_t wrf_loss_workspace_size(int32_t Q, int32_t H, int32_t W);
wrf_status wrf_loss(const float *pred, const float *target, int32_t Q, int32_t H, int32_t W,
                    float lambda1, float *out, float *d_pred, void *ws, size_t ws_bytes,
                    void *stream);

/* One Adam step (Kingma & Ba; the paper trains with PyTorch's Adam, learning
 * rates in its Table I: 1e-2 for the Gaussians, 8e-3 for the MLP) over up to
 * 32 parameter tensors in one launch:
 *   m = b1 m + (1 - b1) g,  v = b2 v + (1 - b2) g^2,
 *   param -= lr (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps).
 * groups is a host array; every pointer in it is a device FP32 array of n
 * elements, m and v the caller's optimizer state (zero before step 1).
 * step >= 1.                                                               */
typedef struct {
    float *param;
    const float *grad;
    float *m;
    float *v;
    int64_t n;
    float lr;
} wrf_adam_group;
wrf_status wrf_adam(const wrf_adam_group *groups, int32_t n_groups, int32_t step, float beta1,
                    float beta2, float eps, void *stream);

/* Anneal smoothing of the fine stage (Sec. 4.4, Eq. 17-18): the MLP's TX
 * input at fine-stage iteration i carries the noise
 *   n_i = gamma N3(0,1) (2 / cbrt(N_s)) (1 - i / tau)   for i < tau, else 0
 * on the position normalised to the room's unit cube, i.e. room_size * n_i
 * in metres:
 *   tx_out[q] = tx[idx[q]] + room_size * normals[q] * gamma (2 / cbrt(N_s)) (1 - i / tau).
 *   tx       [n_positions][3] device, the training positions (metres).
 *   idx      [Q] device row indices into tx (the minibatch), or NULL (row q).
 *   normals  [Q][3] device N(0,1) draws (the caller's generator).
 *   room_size host float[3] (> 0); gamma >= 0 (Table I: 1); tau >= 1 (Table I:
 *            10k); iter >= 0; n_positions = N_s.
 *   tx_out   [Q][3] device output.                                          */
wrf_status wrf_anneal_tx(const float *tx, const int32_t *idx, int32_t n_positions,
                         const float *normals, int32_t Q, int32_t iter, float gamma, int32_t tau,
                         const float room_size[3], float *tx_out, void *stream);

/* RSSI head (Sec. 7.2): for each query the map of wrf_deform_project +
 * wrf_render, reduced by a global average pool of its magnitude,
 *   rssi[q] = (1 / (H W)) sum_pixels |A_q(pixel)|
 * (Sec. 6.6 defines RSSI as the spectrum magnitude averaged over azimuth and
 * elevation).  The paper's setting is 50 Gaussians on a 16 x 16 map, a
 * latency-bound size, so the whole path runs fused, one CTA per query, with
 * the MLP in FP32 (mlp->precision is ignored) and every pixel tested against
 * every Gaussian (the tile fields of grid are ignored).
 *   scene  n <= 64 Gaussians (WRF_EUNSUPPORTED above).
 *   grid   H W <= 65536 pixels, q_cut as for wrf_render.
 *   tx     [Q][3] device, TX positions in metres.
 *   rssi   [Q] device output.
 *   map    [Q][H][W] device output of the un-pooled map, or NULL.
 *   ws     workspace of wrf_deform_workspace_size(n, Q, mlp) bytes, 256-byte
 *          aligned (the factorised layer-1 terms and FP32 weight images).
 * n == 0 gives rssi = 0.  Pooling sums in a fixed order, so a query's value
 * does not depend on the other queries of the call.                        */
wrf_status wrf_rssi(const wrf_scene *scene, const wrf_mlp *mlp, const wrf_grid *grid,
                    const float *tx, int32_t Q, float *rssi, float *map, void *ws,
                    size_t ws_bytes, void *stream);

/* Two-channel rasterisation (Sec. 6.1: the real and imaginary parts of the
 * spectrum are rasterised as separate channels and decomposed into magnitude
 * and phase): per pixel re = the sum of wrf_render with the records' w, im =
 * the same sum with the imaginary weights that follow the records (see the
 * record layout), one exp per pixel and Gaussian for both; out
 * [Q][2][H][W] = |re + i im|, arg(re + i im) (atan2, arg 0 = 0).  Other
 * arguments as wrf_render.  The backward entry points take one channel.    */
wrf_status wrf_render_complex(const float *rec, const uint32_t *gids,
                              const uint32_t *tile_offsets, const int64_t *n_keys,
                              int64_t key_capacity, int32_t n, int32_t Q, const wrf_grid *grid,
                              float *out, void *stream);

/* ---------------------------------------------------------------------- */
/* The paper's own primitive and deformation head (Sec. 4.1-4.2, Sec. 6.1).
 * Primitive n, FP32, device, structure of arrays:
 *   mu[n]         raw angular centre (u, v); the reference centre in pixels
 *                 is x = W (tanh u + 1) / 2 (azimuth), y = H (tanh v + 1) / 2
 *                 (elevation);
 *   chol[n]       Cholesky entries (l1, l2, l3) of the covariance in pixels,
 *                 Sigma = L L^T with L = [[l1, 0], [l2, l3]] (Sec. 3.2);
 *                 l1 l3 != 0;
 *   attn_logit[n] attenuation delta = sigmoid(a);
 *   psi[n]        complex response (re, im).                                */
typedef struct {
    int32_t n;
    const float *mu;          /* [N][2] device, 8-byte aligned               */
    const float *chol;        /* [N][3] device                               */
    const float *attn_logit;  /* [N]    device                               */
    const float *psi;         /* [N][2] device, 8-byte aligned               */
} wrf_paper_scene;

/* Deformation network F (Eq. 14) of the paper's head: n_hidden Linear+ReLU
 * layers of width `width`, the encoded input e = [gamma((x/W, y/H)) with
 * L_mean bands, gamma((tx - room_min)/room_size) with L_tx bands] (Eq. 15)
 * entering layer 0 and concatenated after the activations entering hidden
 * layers 2, 4 and 6 (a skip every two layers), then a Linear output of width
 * 5 = (dmu_x, dmu_y, dpsi_re, dpsi_im, ddelta).  W[l] is [out][in] row-major
 * FP32 device with in = dim(e) for l = 0, width + dim(e) for a skip layer,
 * width otherwise; W[n_hidden] is the output layer [5][width].  The paper's
 * network: n_hidden 8, width 156, L_mean 10, L_tx 6.
 * Supported: 1 <= n_hidden <= 8, 1 <= width <= 160, bands in [0, 15]
 * (L_mean <= 15 in FP32, <= 15 with 2(2 L_mean + 1) <= 64 in BF16).
 * precision = WRF_FP32: every product in FP32 on the CUDA cores.
 * precision = WRF_BF16: the hidden and output layers on the tcgen05 tensor
 * cores with BF16 weights, activations and gamma(mean), FP32 accumulation;
 * the query's part of the encoding, W_s gamma(s) + b, stays FP32.
 * precision = WRF_BF16X3: the same on the tensor cores with weights,
 * activations and gamma(mean) each as BF16 hi + lo and three products per
 * multiply (FP32-level results at about three times the tensor work).     */
enum { WRF_PAPER_MAX_LAYERS = 9, WRF_PAPER_MAX_WIDTH = 160 };
typedef struct {
    int32_t n_hidden, width;
    const float *W[WRF_PAPER_MAX_LAYERS];
    const float *b[WRF_PAPER_MAX_LAYERS];
    int32_t L_mean, L_tx;
    float room_min[3], room_size[3];
    int32_t precision;           /* WRF_FP32 or WRF_BF16 (see below)          */
} wrf_paper_mlp;

/* Deform + project with the paper's head: the frame at TX s is
 * (mu + dmu, Sigma, psi + dpsi, delta + ddelta) (Eq. 12, no covariance
 * residual), written as two-channel records (layout above: w = (delta +
 * ddelta)(psi_re + dpsi_re), the imaginary weights (delta + ddelta)(psi_im +
 * dpsi_im) after them; the caller allocates Q x N x 9 floats) for wrf_bin
 * and wrf_render_complex, which give magnitude and phase (Sec. 6.1).
 *   mlp   NULL: no deformation (Q copies of the reference frame).
 *   tx    [Q][3] device, TX positions in metres (unused when mlp is NULL).
 *   rec   device output, 16-byte aligned.
 *   ws    wrf_paper_workspace_size(N, Q) bytes, 256-byte aligned (the
 *         per-Gaussian and per-query terms of the layers that read the
 *         encoding, and padded weight images).                              */
size_t wrf_paper_workspace_size(int32_t n, int32_t Q);
wrf_status wrf_paper_deform_project(const wrf_paper_scene *scene, const wrf_paper_mlp *mlp,
                                    const wrf_grid *grid, const float *tx, int32_t Q, float *rec,
                                    void *ws, size_t ws_bytes, void *stream);

/* Measurement helper (no paper counterpart): the device's FP32 FMA rate in
 * FLOP/s with one-lane fma and with two-lane fma.rn.f32x2, and its MUFU ex2
 * rate in results per second, each timed with CUDA events over one launch of
 * 8 x SMs x 1024 threads (after one warm-up launch) on `stream`.  These are
 * the denominators of the rooflines of the CUDA-core kernels.  Blocks the
 * calling thread until the probes finish.                                  */
wrf_status wrf_measure_alu_peaks(double *fma_flops, double *fma2_flops, double *ex2_per_s,
                                 void *stream);

/* Backward of wrf_render: from dL/dA [Q][H][W] to d_rec [Q][N][6] =
 * dL/d(mx, my, A, B, C, w) where (A, B, C) is the unscaled inverse
 * covariance (Eq. 8).  Per-pixel weights are recomputed from the records
 * and tile lists (nothing is stored by the forward).  d_rec is accumulated
 * with atomic adds and must be zeroed by the caller.                        */
wrf_status wrf_render_backward(const float *rec, const uint32_t *gids,
                               const uint32_t *tile_offsets, const int64_t *n_keys,
                               int64_t key_capacity, int32_t n, int32_t Q, const wrf_grid *grid,
                               const float *dL_dspectra, float *d_rec, void *stream);

/* Backward of wrf_project: from d_rec [Q][N][6] to d_resid [Q][N][5] and the
 * reference-frame gradients summed over queries.  Outputs are overwritten
 * (d_mean [N][2], d_log_scale [N][2], d_rot, d_opacity, d_amp [N]);
 * d_resid may be NULL when resid is NULL.                                   */
wrf_status wrf_project_backward(const wrf_scene *scene, const float *resid, int32_t Q,
                                const float *d_rec, float *d_resid, float *d_mean,
                                float *d_log_scale, float *d_rot, float *d_opacity, float *d_amp,
                                void *stream);

/* Backward of wrf_deform (MLP back-propagation, Sec. 4.4): from d_resid
 * [Q][N][5] to dW[l], db[l] (same shapes as the weights; overwritten) and,
 * unless stop_grad_mean is non-zero, adds the derivative through
 * gamma(mean) into d_mean [N][2] (the paper freezes position gradients in
 * its fine stage; the flag reproduces that).  The dense products over rows
 * (the delta chain D_{l-1} = (D_l W_l) * [H_l > 0] and the weight gradients
 * D_l^T H_l) run on the tcgen05 tensor cores with every FP32 operand split
 * into BF16 hi + lo and three products hi*hi + hi*lo + lo*hi (relative error
 * ~2^-17 of |a||b|), FP32 accumulation; the output layer (5 units) runs on
 * the CUDA cores in FP32.  The weight and bias gradients are reduced in a
 * fixed order (bit-reproducible); d_mean is accumulated with FP32 atomics
 * over queries (order not fixed).  A bounded device-side wait that runs out
 * records WRF_ETIMEOUT and leaves the outputs undefined.
 *   acts  the hidden activations saved by wrf_deform_acts for the same
 *         scene, MLP and tx, or NULL: then the forward is recomputed.      */
size_t wrf_deform_backward_workspace_size(int32_t n, int32_t Q, const wrf_mlp *mlp);
wrf_status wrf_deform_backward(const wrf_scene *scene, const wrf_mlp *mlp, const wrf_grid *grid,
                               const float *tx, int32_t Q, const float *d_resid, const float *acts, float *const *dW,
                               float *const *db, float *d_mean, int32_t stop_grad_mean, void *ws,
                               size_t ws_bytes, void *stream);

/* Host-to-host forward pipeline (the problem as Sec. 4.1-4.2 state it: the
 * Gaussian parameters and the network stay on the device, TX positions come
 * in, spectra go out; Eq. 9 / Eq. 13 per query).  It owns everything a step
 * needs: records, workspaces, tile lists and two slots of device TX and
 * spectrum buffers, each slot with a CUDA graph of wrf_deform_project +
 * wrf_bin + wrf_render (wrf_render_complex for two channels), and its own
 * two streams.  A step copies its TX positions into pinned staging, uploads
 * them, replays the slot's graph and copies the spectra back to the caller's
 * host buffer on the second stream, so one step's read-back overlaps the next
 * step's compute.  The library allocates at create and at a key-capacity
 * growth, never in a step otherwise.
 *   wrf_pipeline_create  scene / mlp / grid as for the calls above (device
 *                        arrays the caller keeps alive and unchanged until
 *                        destroy; the structs themselves are copied), Q >= 1
 *                        queries per step, on the current device.
 *                        key_margin >= 1: the key capacity is the first
 *                        step's key count x key_margin + 1024 (0 = 1.25).
 *   wrf_pipeline_step    tx_host [Q][3] host FP32 (read before the call
 *                        returns); spectra_host host FP32, [Q][H][W] (one
 *                        channel) or [Q][2][H][W] (two: magnitude, phase),
 *                        written when the step completes: it must stay valid
 *                        until then.  Pinned memory (cudaHostAlloc /
 *                        cudaHostRegister) keeps the read-back asynchronous.
 *                        A step first waits (on the host) for the step two
 *                        before it, which used the same slot.  The first step
 *                        runs synchronously: it sizes the key capacity and
 *                        captures the graphs.
 *   wrf_pipeline_wait    blocks until every enqueued step has completed.
 *   wrf_pipeline_destroy waits, then frees everything; NULL is a no-op.
 * A step whose keys did not fit (the device records WRF_ENOSPC) is detected
 * when its slot is next waited on: the pipeline grows the capacity, captures
 * its graphs again, recomputes that step synchronously into the same host
 * buffer and clears the status word, so every completed step holds the
 * spectra of its own TX positions.  Errors: WRF_EINVAL / WRF_EUNSUPPORTED
 * (arguments, as the calls above), WRF_ECUDA (a failed CUDA call; the
 * pipeline should then be destroyed).  One pipeline is used by one host
 * thread at a time.                                                         */
typedef struct wrf_pipeline wrf_pipeline;
wrf_status wrf_pipeline_create(const wrf_scene *scene, const wrf_mlp *mlp, const wrf_grid *grid,
                               int32_t Q, float key_margin, wrf_pipeline **out);
wrf_status wrf_pipeline_step(wrf_pipeline *p, const float *tx_host, float *spectra_host);
wrf_status wrf_pipeline_wait(wrf_pipeline *p);
wrf_status wrf_pipeline_destroy(wrf_pipeline *p);

/* Diagnostic of the bounded device-side waits (no paper counterpart): one
 * GPU thread waits, with the same bounded wait the kernels use, on an
 * mbarrier phase that nothing completes.  The wait gives up after limit_ns
 * (0 < limit_ns <= 2e9) and records WRF_ETIMEOUT in the status word; the
 * kernel then returns normally and *completed (device int) is set to 0.
 * Read the outcome with wrf_status_read.                                      */
wrf_status wrf_selftest_wait(int64_t limit_ns, int32_t *completed, void *stream);

/* Device status word: returns the first device-side error recorded since the
 * last call (WRF_OK if none) after synchronising `stream`, and clears it.    */
wrf_status wrf_status_read(void *stream);

const char *wrf_last_error(void);
int32_t wrf_version(void);

#ifdef __cplusplus
}
#endif
#endif /* WRF_H */
