// Internal launcher declarations shared by the kernel files and the C ABI.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace wrf {

// Weight images prepared once per call from the caller's FP32 weights.
struct MlpView {
    int n_layers;          // Linear layers (>= 2)
    int dm, dt;            // widths of gamma(mean) and gamma(tx)
    int L_mean, L_tx;
    float room_min[3], room_size[3];
    const float *W0;       // [128][dm+dt] (caller's first layer)
    const float *b0;       // [128]
    const float *Wh[8];    // hidden layers 1..n_layers-2: [128][128]
    const float *bh[8];
    const float *Wo;       // output layer [5][128]
    const float *bo;       // [5]
};

// Workspace carve-up for deformation (all offsets 256-byte aligned).
struct DeformWs {
    float *U;              // [N][128]  W0[:, :dm] gamma(mean_n)            (FP32 path;
                           // BF16X3: blocked [N/128][32][128][4], see prep.cu)
    uint16_t *G;           // [N][k1]   gamma(mean_n) in BF16, zero-padded  (BF16 path)
    float *V;              // [Q][128]  W0[:, dm:] gamma(tx_q) + b0
    float *wt_f32;         // hidden layers transposed [l][k=128][j=128], FP32
    float *wo_f32;         // output layer transposed [k=128][8] (cols 5..7 zero)
    uint16_t *w_bf16;      // tcgen05 operand images: W1m, hidden layers, output,
                           // bias image, bias selectors
    uint16_t *w_x3;        // FP32-level tcgen05 images (hi and lo of every weight):
                           // hidden layers, output layer, bias image, selectors
};

// Biases enter the tensor-core MLP as one extra K = 16 MMA per layer.  The
// bias image is a no-swizzle K-major B operand of 128 rows x 8 BF16 columns
// (16 row groups of 8 rows x 16 B, 128 B apart; row n at (n/8)*128 + (n%8)*16):
// columns 2l, 2l+1 hold hidden layer l's bias b split as hi = bf16(b),
// lo = bf16(b - hi); columns 6, 7 the output bias.  A selector is an A
// operand whose every row has ones in columns 2p, 2p+1 (one 8-row core
// matrix, repeated with row-group stride 0, and a zero core matrix for
// K = 8..15), so A_sel(p) B_bias adds hi + lo of pair p to every row.
constexpr size_t kBiasImageBytes = 2048;
constexpr size_t kSelImageBytes = 4 * 256;

// The three-product image (precision WRF_BF16X3): per hidden layer four
// 128 x 64 K-major 128-byte-swizzled panels (hi K 0-63, hi K 64-127, lo K
// 0-63, lo K 64-127; hi = bf16(w), lo = bf16(w - hi)), the output layer the
// same way as 16-row panels, then the bias image and the selectors.
constexpr size_t kX3PanelBytes = 128 * 128;
constexpr size_t kX3OutPanelBytes = 16 * 128;
inline __host__ __device__ constexpr size_t mlp_x3_image_bytes(int nh) {
    return static_cast<size_t>(nh) * 4 * kX3PanelBytes + 4 * kX3OutPanelBytes + kBiasImageBytes +
           kSelImageBytes;
}

// K of the tensor-core layer-1 MMA: gamma(mean) width dm padded to 32 or 64.
inline __host__ __device__ int mlp_k1(int dm) { return dm <= 32 ? 32 : 64; }

size_t deform_ws_layout(int n, int Q, int n_layers, DeformWs *ws, char *base);

// A resident scene of a multi-scene batch: its Gaussians, its BF16
// gamma(mean) rows and weight images (prepared once), and its first layer in
// FP32 (for the per-query term).
struct SceneEntry {
    SceneView s;
    const uint16_t *G;       // [n][k1]
    const uint16_t *w_img;   // W1m, hidden layers, output, bias image, selectors
    const float *W0, *b0;
};
constexpr int kMaxScenes = 16;

// images: WRF_FP32 (U, V, FP32 transposes), WRF_BF16 (BF16 gamma(mean) rows
// instead of U, V, BF16 images) or WRF_BF16X3 (U, V, three-product images)
cudaError_t launch_prep(const SceneView &s, const MlpView &m, const GridView &g, const float *tx,
                        int Q, const DeformWs &ws, int images, cudaStream_t st);

// mode 0: write residuals [Q][N][5]; mode 1: project and write records.
cudaError_t launch_mlp_f32(const SceneView &s, const MlpView &m, const GridView &g, int Q,
                           const DeformWs &ws, int mode, float *resid, float4 *rec,
                           uint32_t *count, float *acts, cudaStream_t st);
cudaError_t launch_mlp_tc(const SceneView &s, const MlpView &m, const GridView &g, int Q,
                          const DeformWs &ws, int mode, float *resid, float4 *rec,
                          uint32_t *count, int *status, cudaStream_t st);
// FP32-level tensor-core MLP (three BF16 products per FP32 product); acts
// (or NULL) receives the hidden activations like launch_mlp_f32.
cudaError_t launch_mlp_x3(const SceneView &s, const MlpView &m, const GridView &g, int Q,
                          const DeformWs &ws, int mode, float *resid, float4 *rec,
                          uint32_t *count, float *acts, int *status, cudaStream_t st);

// Multi-scene batches (multi.cu): query q of scene scene_of[q] (-1: none).
struct MultiSet {           // a prepared scene set (caller-owned device memory)
    SceneEntry *table;      // [kMaxScenes]
    float *wt_scratch, *wo_scratch;
    uint16_t *G[kMaxScenes], *img[kMaxScenes];
};
struct MultiWs {            // per-batch scratch
    int *tstart;            // [Q+1] 128-row MLP tile ranges
    float *V;               // [Q][128] per-query layer-1 terms
};
size_t multi_set_layout(const SceneView *s, int S, int n_layers, int k1, MultiSet *ms, char *base);
cudaError_t launch_multi_prepare(const SceneView *s, const MlpView *m, int S, const GridView &g,
                                 const MultiSet &ms, cudaStream_t st);
size_t multi_ws_layout(int Q, MultiWs *mw, char *base);
cudaError_t launch_deform_project_multi(const MultiSet &ms, int S, const MlpView &m,
                                        const GridView &g, const int *scene_of, const float *tx,
                                        int Q, float4 *rec, long long rec_capacity,
                                        long long *qbase, const MultiWs &w, int *status,
                                        cudaStream_t st);
cudaError_t launch_mlp_tc_multi(const SceneEntry *table, const MlpView &m, const GridView &g,
                                int Q, const int *scene_of, const long long *qbase,
                                const int *tstart, const float *V, float4 *rec, int *status,
                                cudaStream_t st);

cudaError_t launch_project(const SceneView &s, const float *resid, int Q, const GridView &g,
                           float4 *rec, uint32_t *count, cudaStream_t st);

// FP32 FMA (one- and two-lane) and MUFU ex2 rate probes (peaks.cu): out3 = FLOP/s, FLOP/s, ex2/s.
cudaError_t measure_alu_peaks(double *out3, cudaStream_t st);

// The paper's primitive and deformation head (paper.cu).
constexpr int kPaperMaxWidth = 160;
constexpr int kPaperMaxLayers = 9;  // <= 8 hidden + output
struct PaperSceneView {
    int n;
    const float *mu, *chol, *attn_logit, *psi;
};
struct PaperMlpView {
    int n_hidden, width, L_mean, L_tx;
    float room_min[3], room_size[3];
    const float *W[kPaperMaxLayers], *b[kPaperMaxLayers];
};
struct PaperWs {
    float *U, *V, *Wt, *bh, *Wo;  // FP32 network (paper.cu)
    uint16_t *G, *img;            // tensor-core network (paper_tc.cu): BF16 gamma rows, panels
    float *vec;                   //   per-query FP32 layer terms [Q][8][160]
};
size_t paper_ws_layout(int n, int Q, PaperWs *ws, char *base);
cudaError_t launch_paper(const PaperSceneView &s, const PaperMlpView *m, const GridView &g,
                         const float *tx, int Q, const PaperWs &ws, float4 *rec, cudaStream_t st);
size_t paper_tc_image_bytes(int n_hidden);
// precision WRF_BF16 or WRF_BF16X3 (three BF16 products per FP32 product)
cudaError_t launch_paper_tc(const PaperSceneView &s, const PaperMlpView &m, const GridView &g,
                            const float *tx, int Q, const PaperWs &ws, float4 *rec, int *status,
                            int precision, cudaStream_t st);

// Training protocol (train.cu): Eq. 16 loss with SSIM, and Adam.
size_t loss_ws_layout(int Q, int H, int W, float **coef, float **part);
cudaError_t launch_loss(const float *pred, const float *target, int Q, int H, int W, float lam,
                        float *out, float *d_pred, char *ws, cudaStream_t st);
struct AdamGroup {
    float *param;
    const float *grad;
    float *m, *v;
    long long n;
    float lr;
};
constexpr int kAdamGroups = 32;
cudaError_t launch_adam(const AdamGroup *groups, int n, int step, float beta1, float beta2,
                        float eps, cudaStream_t st);
cudaError_t launch_anneal(const float *tx, const int *idx, const float *normals, int Q, int iter,
                          int n_pos, float gamma, int tau, const float *room_size, float *out,
                          cudaStream_t st);

// RSSI head: one CTA per query, whole path fused (rssi.cu); U, V and the
// FP32 weight images come from launch_prep(..., want_bf16 = false).
constexpr int kRssiMaxN = 64;
constexpr int kRssiMaxPixels = 65536;
cudaError_t launch_rssi(const SceneView &s, const MlpView &m, const GridView &g, int Q,
                        const DeformWs &ws, float *rssi, float *map, cudaStream_t st);

// Binning.
struct BinWs {
    uint32_t *chunk_counts;  // [Q][T][C]
    unsigned long long *block_sums;
    int C;                   // chunks of Gaussians per query (512 or 1024 each)
    long long M;             // Q*T*C
    int nblocks;
};
size_t bin_ws_layout(int n, int Q, const GridView &g, BinWs *ws, char *base);
// qbase (multi-scene batches, else NULL): query q's records start at
// qbase[q] and number qbase[q+1] - qbase[q] (<= n, the chunked maximum).
cudaError_t launch_bin(const float4 *rec, int n, int Q, const GridView &g, uint32_t *gids,
                       long long cap, long long *n_keys, uint32_t *offsets, const BinWs &ws,
                       int *status, cudaStream_t st, const long long *qbase = nullptr);

// Rasteriser.
cudaError_t launch_render(const float4 *rec, const uint32_t *gids, const uint32_t *offsets,
                          const long long *n_keys, long long cap, int n, int Q,
                          const GridView &g, float *out, int *status, cudaStream_t st,
                          const long long *qbase = nullptr);
// Two channels (records followed by [Q][N] imaginary weights): out
// [Q][2][H][W] = magnitude, phase.
cudaError_t launch_render_complex(const float4 *rec, const uint32_t *gids,
                                  const uint32_t *offsets, const long long *n_keys, long long cap,
                                  int n, int Q, const GridView &g, float *out, int *status,
                                  cudaStream_t st);
cudaError_t launch_render_bwd(const float4 *rec, const uint32_t *gids, const uint32_t *offsets,
                              const long long *n_keys, long long cap, int n, int Q,
                              const GridView &g, const float *dA, float *d_rec, int *status,
                              cudaStream_t st);
cudaError_t launch_project_bwd(const SceneView &s, const float *resid, int Q, const float *d_rec,
                               float *d_resid, float *d_mean, float *d_ls, float *d_rot,
                               float *d_op, float *d_amp, cudaStream_t st);

// MLP backward on the tensor cores (mlp_bwd.cu).
struct DeformBwdWs {
    char *wimg;          // BF16 hi / lo W^T panels of the hidden layers
    char *gimg;          // BF16 hi / lo gamma(mean) tiles (two term images)
    long long gterm;     // bytes per term image
    float *gam_t;        // [Q][dt] gamma(tx) in FP32
    float *pdw, *pdb, *pdwo, *pdw0;  // per-CTA partial sums
    float *tilesum;      // [Q * tiles per query][128] per-tile sums of D_0
    float *colsum;       // [Q][128]
    float *acts;         // recomputed hidden activations of a chunk of queries
    float *resid;        // the recompute's residuals (unused)
    float *d0;           // [chunk rows][128] D_0, for the gradient through gamma(mean)
    int qc;              // queries per chunk
};
size_t deform_bwd_ws_layout(int n, int Q, const MlpView &m, DeformWs *fw, DeformBwdWs *bw,
                            char *base);
cudaError_t launch_mlp_bwd(const SceneView &s, const MlpView &m, const GridView &g,
                           const float *tx, int Q, const DeformWs &fw, const DeformBwdWs &bw,
                           const float *d_resid, const float *acts, float *const *dW, float *const *db,
                           float *d_mean, int stop_grad_mean, int *status, cudaStream_t st);

bool render_config_supported(int tw, int th);

// cuTensorMapEncodeTiled from the driver (NULL if unavailable); render.cu.
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                   const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                   const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled();


// For the library's host code outside the C ABI file (the forward pipeline):
// the forward calls' argument checks (scene, network, grid, Q >= 1), and the
// thread-local message that wrf_last_error returns (with the CUDA error's
// text when e is not cudaSuccess).  Both return their status argument or
// the check's result.
wrf_status check_forward(const wrf_scene *scene, const wrf_mlp *mlp, const wrf_grid *grid, int Q);
wrf_status set_error(wrf_status s, const char *where, cudaError_t e = cudaSuccess);

}  // namespace wrf
