// Preparation for the deformation MLP (Sec. 4.2, Eqs. 14-15).
//
// The first Linear layer acts on [gamma(mean_n), gamma(tx_q)], so its
// pre-activation splits exactly into a per-Gaussian part and a per-query
// part:  W0 [gamma(mu_n); gamma(s_q)] + b0 = U[n] + V[q] with
//   U[n] = W0[:, :dm] gamma(mu_n),   V[q] = W0[:, dm:] gamma(s_q) + b0.
// U costs N*128*dm FMAs and V Q*128*dt, instead of Q*N*128*(dm+dt); the MLP
// kernels then start every row from ReLU(U[n] + V[q]).
//
// This file also builds the weight images the MLP kernels read: FP32
// transposed copies for the CUDA-core path, BF16 K-major 128-byte-swizzled
// operand images for the tcgen05 path, and the hi / lo pairs of the same
// images for the three-product (FP32-level) tcgen05 path.
#include <cuda_bf16.h>

#include "kernels.h"

namespace wrf {

namespace {

constexpr int kMaxPe = 3 * (2 * 15 + 1);  // d(2L+1) for d <= 3, L <= 15
constexpr size_t kW1ImageBytes = WRF_HIDDEN * 128;  // 128 rows x 64 BF16 columns


// Per-Gaussian part of layer 1 for 32 Gaussians per block.  FP32 path:
// U[n][j] = W0[j, :dm] . gamma(mean_n), thread j owns column j; row-major
// [N][128], or (blocked, for the three-product tensor-core kernel) in
// 128-Gaussian blocks of [32 column quads][128 rows][4], so that the 128
// threads of a tile, one row each, read a column quad as one contiguous
// 2 KB run.  BF16 path: the row gamma(mean_n) itself in BF16, zero-padded to
// k1 columns, which the tensor-core kernel multiplies by the W1m image.
__device__ __forceinline__ void pe_mean_block(int blk, const SceneView &s, const MlpView &m,
                                              const GridView &g, float *U, uint16_t *G, int k1,
                                              bool blocked) {
    __shared__ float gam[32][kMaxPe];
    const int n0 = blk * 32;
    const int din = m.dm + m.dt;
    if (threadIdx.x < 32) {
        int n = n0 + threadIdx.x;
        if (n < s.n) {
            float2 mu = reinterpret_cast<const float2 *>(s.mean)[n];
            const PeArg x[2] = {pe_arg(mu.x, 0.f, static_cast<float>(g.W)),
                                pe_arg(mu.y, 0.f, static_cast<float>(g.H))};
            pe_encode(x, 2, m.L_mean, gam[threadIdx.x]);
        }
    }
    __syncthreads();
    if (G) {
        for (int e = threadIdx.x; e < 32 * k1; e += blockDim.x) {
            const int r = e / k1, k = e % k1, n = n0 + r;
            if (n < s.n)
                reinterpret_cast<__nv_bfloat16 *>(G)[static_cast<size_t>(n) * k1 + k] =
                    __float2bfloat16_rn(k < m.dm ? gam[r][k] : 0.f);
        }
        return;
    }
    // thread j: 32 independent row sums, each over k in ascending order
    const int j = threadIdx.x;
    const float *wrow = m.W0 + static_cast<size_t>(j) * din;
    float acc[32];
#pragma unroll
    for (int r = 0; r < 32; ++r) acc[r] = 0.f;
#pragma unroll 8
    for (int k = 0; k < m.dm; ++k) {
        const float w = __ldg(wrow + k);
#pragma unroll
        for (int r = 0; r < 32; ++r) acc[r] = fmaf(w, gam[r][k], acc[r]);
    }
#pragma unroll
    for (int r = 0; r < 32; ++r) {
        const int n = n0 + r;
        if (n >= s.n) continue;
        const size_t at = blocked ? ((static_cast<size_t>(n >> 7) * 32 + (j >> 2)) * 128 +
                                     (n & 127)) * 4 + (j & 3)
                                  : static_cast<size_t>(n) * WRF_HIDDEN + j;
        U[at] = acc[r];
    }
}

// V[q][j] for 4 queries per block: the 4 x dt features of Eq. 15 are
// computed one per thread, then thread j forms output column j of each query.
constexpr int kTxPerBlock = 4;
__device__ __forceinline__ void pe_tx_block(int blk, const MlpView &m, const float *tx, int Q,
                                            float *V) {
    __shared__ float gam[kTxPerBlock][kMaxPe];
    const int q0 = blk * kTxPerBlock;
    const int din = m.dm + m.dt;
    const int L = m.L_tx;
    for (int e = threadIdx.x; e < kTxPerBlock * m.dt; e += blockDim.x) {
        const int r = e / m.dt, f = e % m.dt, q = q0 + r;
        if (q >= Q) continue;
        // feature f: [x (3), sin band k (3 each), cos band k (3 each)]
        const int i = f % 3, grp = f / 3;
        const PeArg x = pe_arg(tx[3 * q + i], m.room_min[i], m.room_size[i]);
        float val = pe_value(x);
        if (grp >= 1) {
            float sn, cs;
            pe_band(x, (grp - 1) % L, sn, cs);
            val = grp <= L ? sn : cs;
        }
        gam[r][f] = val;
    }
    __syncthreads();
    const int j = threadIdx.x;
    const float *wrow = m.W0 + static_cast<size_t>(j) * din + m.dm;
    const float bj = m.b0[j];
    float acc[kTxPerBlock];
#pragma unroll
    for (int r = 0; r < kTxPerBlock; ++r) acc[r] = 0.f;
    #pragma unroll 16
    for (int k = 0; k < m.dt; ++k) {
        const float w = wrow[k];
#pragma unroll
        for (int r = 0; r < kTxPerBlock; ++r) acc[r] = fmaf(w, gam[r][k], acc[r]);
    }
#pragma unroll
    for (int r = 0; r < kTxPerBlock; ++r)
        if (q0 + r < Q) V[static_cast<size_t>(q0 + r) * WRF_HIDDEN + j] = acc[r] + bj;
}

// Byte offset of element (row n, col k) in a K-major, 128-byte-swizzled
// tcgen05 operand image with `rows` rows and 128 columns of BF16: two
// 64-column halves of rows x 128 B; inside a row the 16-byte chunk index
// (k % 64) / 8 is XORed with n % 8.
__device__ __forceinline__ uint32_t sw128_offset(int n, int k, int rows) {
    int half = k >> 6, kk = k & 63;
    return static_cast<uint32_t>(half * rows * 128 + n * 128 + ((((kk >> 3) ^ (n & 7))) << 4) +
                                 ((kk & 7) << 1));
}

// Element e of the bias image (e < 1024) or of the four selectors (e >= 1024)
// at `aug` (layout in kernels.h).
__device__ __forceinline__ void aug_element(int e, const MlpView &m, int nh, char *aug) {
    float v = 0.f;
    if (e < 1024) {
        const int n = e >> 3, col = e & 7, pair = col >> 1;
        float b = 0.f;
        if (pair < 3 && pair < nh) b = m.bh[pair][n];
        if (pair == 3 && n < WRF_OUT) b = m.bo[n];
        const float hi = __bfloat162float(__float2bfloat16_rn(b));
        v = (col & 1) ? b - hi : hi;
        *reinterpret_cast<__nv_bfloat16 *>(aug + (n >> 3) * 128 + (n & 7) * 16 + col * 2) =
            __float2bfloat16_rn(v);
    } else {
        const int s2 = e - 1024, p = s2 >> 7, within = s2 & 127;  // 128 elements each
        const int col = within & 7;                                // core 0: rows x 8
        if (within < 64 && (col >> 1) == p) v = 1.f;
        *reinterpret_cast<__nv_bfloat16 *>(aug + kBiasImageBytes + p * 256 + within * 2) =
            __float2bfloat16_rn(v);
    }
}

// One thread per (layer, row, col) of every hidden layer and the output
// layer: FP32 transposes and BF16 swizzled images.  The BF16 image starts
// with W1m = W0[:, :dm] as a 128 x 64 K-major image (columns >= dm zero) and
// ends with the bias image and the four bias selectors (layout in kernels.h).
__device__ __forceinline__ void weights_block(int blk, int nblk, const MlpView &m,
                                              const DeformWs &ws, int want_bf16) {
    const int nh = m.n_layers - 2;
    const long long per = WRF_HIDDEN * WRF_HIDDEN;
    const long long w1 = want_bf16 ? WRF_HIDDEN * 64 : 0;
    const long long mats = w1 + nh * per + 16 * WRF_HIDDEN;
    const long long total = mats + (want_bf16 ? (kBiasImageBytes + kSelImageBytes) / 2 : 0);
    char *img = reinterpret_cast<char *>(ws.w_bf16);
    const int din = m.dm + m.dt;
    const size_t aug_off = kW1ImageBytes + static_cast<size_t>(nh) * per * 2 + 16 * WRF_HIDDEN * 2;
    for (long long i = blk * static_cast<long long>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<long long>(nblk) * blockDim.x) {
        if (i >= mats) {
            aug_element(static_cast<int>(i - mats), m, nh, img + aug_off);
            continue;
        }
        if (i < w1) {
            const int j = static_cast<int>(i / 64), k = static_cast<int>(i % 64);
            const float v = k < m.dm ? m.W0[static_cast<size_t>(j) * din + k] : 0.f;
            *reinterpret_cast<__nv_bfloat16 *>(img + sw128_offset(j, k, WRF_HIDDEN)) =
                __float2bfloat16_rn(v);
            continue;
        }
        const long long ii = i - w1;
        if (ii < nh * per) {
            int l = static_cast<int>(ii / per);
            int r = static_cast<int>(ii % per);
            int j = r / WRF_HIDDEN, k = r % WRF_HIDDEN;  // W[j][k]
            float v = m.Wh[l][r];
            ws.wt_f32[l * per + k * WRF_HIDDEN + j] = v;
            if (want_bf16)
                *reinterpret_cast<__nv_bfloat16 *>(img + kW1ImageBytes + l * per * 2 +
                                                   sw128_offset(j, k, WRF_HIDDEN)) =
                    __float2bfloat16_rn(v);
        } else {
            int r = static_cast<int>(ii - nh * per);
            int j = r / WRF_HIDDEN, k = r % WRF_HIDDEN;  // output row j (< 16)
            float v = j < WRF_OUT ? m.Wo[j * WRF_HIDDEN + k] : 0.f;
            if (j < 8) ws.wo_f32[k * 8 + j] = v;
            if (want_bf16)
                *reinterpret_cast<__nv_bfloat16 *>(img + kW1ImageBytes + nh * per * 2 +
                                                   sw128_offset(j, k, 16)) =
                    __float2bfloat16_rn(v);
        }
    }
}

// The three-product image (layout in kernels.h): one thread per weight
// writes its hi = bf16(w) into the hi panel and lo = bf16(w - hi) into the
// lo panel; then the bias image and the selectors.
__device__ __forceinline__ void weights_block_x3(int blk, int nblk, const MlpView &m,
                                                 const DeformWs &ws) {
    const int nh = m.n_layers - 2;
    const long long per = WRF_HIDDEN * WRF_HIDDEN;
    const long long mats = nh * per + 16 * WRF_HIDDEN;
    const long long total = mats + (kBiasImageBytes + kSelImageBytes) / 2;
    char *img = reinterpret_cast<char *>(ws.w_x3);
    const size_t out_off = static_cast<size_t>(nh) * 4 * kX3PanelBytes;
    const size_t aug_off = out_off + 4 * kX3OutPanelBytes;
    for (long long i = blk * static_cast<long long>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<long long>(nblk) * blockDim.x) {
        if (i >= mats) {
            aug_element(static_cast<int>(i - mats), m, nh, img + aug_off);
            continue;
        }
        float v;
        size_t hi_off, lo_off;
        if (i < nh * per) {
            const int l = static_cast<int>(i / per), r = static_cast<int>(i % per);
            const int j = r / WRF_HIDDEN, k = r % WRF_HIDDEN;  // W[j][k]
            v = m.Wh[l][r];
            hi_off = l * 4 * kX3PanelBytes + sw128_offset(j, k, WRF_HIDDEN);
            lo_off = hi_off + 2 * kX3PanelBytes;
        } else {
            const int r = static_cast<int>(i - nh * per);
            const int j = r / WRF_HIDDEN, k = r % WRF_HIDDEN;  // output row j (< 16)
            v = j < WRF_OUT ? m.Wo[j * WRF_HIDDEN + k] : 0.f;
            hi_off = out_off + sw128_offset(j, k, 16);
            lo_off = hi_off + 2 * kX3OutPanelBytes;
        }
        const __nv_bfloat16 hi = __float2bfloat16_rn(v);
        *reinterpret_cast<__nv_bfloat16 *>(img + hi_off) = hi;
        *reinterpret_cast<__nv_bfloat16 *>(img + lo_off) =
            __float2bfloat16_rn(v - __bfloat162float(hi));
    }
}

// The three independent preparation jobs in one launch, so that they run
// side by side: blocks [0, nb_mean) encode 32 Gaussians each, the next nb_tx
// blocks 4 queries each, the rest build the weight images (grid-stride).
// Every block runs exactly one job, so each job's barriers see all 128
// threads of its block.
__global__ void __launch_bounds__(128) prep_kernel(SceneView s, MlpView m, GridView g,
                                                   const float *tx, int Q, DeformWs ws,
                                                   int images, int k1, int nb_mean,
                                                   int nb_tx) {
    int b = blockIdx.x;
    if (b < nb_mean) {
        pe_mean_block(b, s, m, g, ws.U, images == WRF_BF16 ? ws.G : nullptr, k1,
                      images == WRF_BF16X3);
        return;
    }
    b -= nb_mean;
    if (b < nb_tx) {
        pe_tx_block(b, m, tx, Q, ws.V);
        return;
    }
    b -= nb_tx;
    const int nblk = static_cast<int>(gridDim.x) - nb_mean - nb_tx;
    if (images == WRF_BF16X3)
        weights_block_x3(b, nblk, m, ws);
    else
        weights_block(b, nblk, m, ws, images == WRF_BF16);
}

inline size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

}  // namespace

size_t deform_ws_layout(int n, int Q, int n_layers, DeformWs *ws, char *base) {
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char *p = base ? base + off : nullptr;
        off = align256(off + bytes);
        return p;
    };
    int nh = n_layers - 2 > 0 ? n_layers - 2 : 0;
    DeformWs w{};
    // rows rounded up to whole 128-Gaussian blocks (the blocked layout)
    w.U = reinterpret_cast<float *>(take(static_cast<size_t>((n + 127) & ~127) * WRF_HIDDEN * 4));
    w.G = reinterpret_cast<uint16_t *>(take(static_cast<size_t>(n) * 64 * 2));
    w.V = reinterpret_cast<float *>(take(static_cast<size_t>(Q) * WRF_HIDDEN * 4));
    w.wt_f32 = reinterpret_cast<float *>(take(static_cast<size_t>(nh) * WRF_HIDDEN * WRF_HIDDEN * 4));
    w.wo_f32 = reinterpret_cast<float *>(take(WRF_HIDDEN * 8 * 4));
    w.w_bf16 = reinterpret_cast<uint16_t *>(
        take(kW1ImageBytes + static_cast<size_t>(nh) * WRF_HIDDEN * WRF_HIDDEN * 2 +
             16 * WRF_HIDDEN * 2 + kBiasImageBytes + kSelImageBytes));
    w.w_x3 = reinterpret_cast<uint16_t *>(take(mlp_x3_image_bytes(nh)));
    if (ws) *ws = w;
    return off;
}

cudaError_t launch_prep(const SceneView &s, const MlpView &m, const GridView &g, const float *tx,
                        int Q, const DeformWs &ws, int images, cudaStream_t st) {
    if (images != WRF_FP32 && images != WRF_BF16 && images != WRF_BF16X3)
        return cudaErrorInvalidValue;
    const int nb_mean = s.n > 0 ? (s.n + 31) / 32 : 0;
    const int nb_tx = Q > 0 ? (Q + kTxPerBlock - 1) / kTxPerBlock : 0;
    const bool bf16 = images == WRF_BF16, tc = images != WRF_FP32;
    const long long total = (bf16 ? WRF_HIDDEN * 64 : 0) +
                            static_cast<long long>(m.n_layers - 2) * WRF_HIDDEN * WRF_HIDDEN +
                            16 * WRF_HIDDEN +
                            (tc ? (kBiasImageBytes + kSelImageBytes) / 2 : 0);
    long long nb_w = (total + 127) / 128;
    if (nb_w > 2368) nb_w = 2368;
    const long long blocks = nb_mean + nb_tx + nb_w;
    if (blocks >= (1ll << 31)) return cudaErrorInvalidValue;
    prep_kernel<<<static_cast<unsigned>(blocks), 128, 0, st>>>(
        s, m, g, tx, Q, ws, images, mlp_k1(m.dm), nb_mean, nb_tx);
    return cudaGetLastError();
}

}  // namespace wrf
