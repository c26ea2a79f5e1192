// Deformation MLP (Sec. 4.2, Eq. 14) at FP32-level accuracy on the
// 5th-generation tensor cores (precision WRF_BF16X3).
//
// Every FP32 operand x of a hidden or output layer (weights, activations) is
// split into BF16 hi = bf16(x) and lo = bf16(x - hi), and every product is
// taken as hi hi + hi lo + lo hi (relative error ~2^-17 of |a||b|), with FP32
// accumulation in tensor memory; biases enter as one K = 16 MMA of a
// selector against an image holding each bias as BF16 hi + lo.  Layer 1 is
// exact FP32 on the CUDA cores: its pre-activation is U[n] + V[q] (the
// per-Gaussian and per-query parts of Eq. 14's first layer, prep.cu).
//
// Rows are the (query, Gaussian) pairs; a tile is 128 consecutive Gaussians
// of one query (TMEM lane = row).  A CTA runs two warpgroups, each owning one
// tile at a time, so the tensor core works on one warpgroup's layer while the
// other converts its accumulator.  Per warpgroup the tensor memory holds the
// FP32 accumulator (128 columns) and the next layer's A operand as BF16 hi
// pairs (64 columns) and lo pairs (64 columns); every MMA takes A from tensor
// memory and B (the weights) from shared memory.  All weight images (hidden
// layers and output layer as hi and lo panels, the bias image and the
// selectors; <= 203 KB for three hidden layers) stay resident in shared
// memory, copied once per CTA with bulk copies.  Per tile:
//   1. layer 1: thread n reads its row of U (FP32; U is stored in
//      128-Gaussian blocks of column quads, so the tile's 128 threads read
//      contiguous 2 KB runs, the next 32 columns in flight while the current
//      ones convert, the first 32 fetched during the previous tile), adds
//      V[q], applies ReLU, stores the activations (if requested) and writes
//      its hi / lo pairs;
//   2. hidden layer l: bias MMA, then 8 K-steps x 3 products, committed to
//      an mbarrier; the conversion reads the accumulator (tcgen05.ld),
//      applies ReLU, stores the activations (if requested) and writes the
//      hi / lo pairs of the next layer's A operand (tcgen05.st);
//   3. output layer (N = 16, 5 used) the same way, then the residual row or
//      the deformed and projected record (Eq. 12-13).
// Saved activations leave through a 2 KB staging area per warp (16 columns
// of its 32 rows) by TMA tensor stores: the conversion waits only until the
// previous box has been read out of the staging area, not for the writes,
// and no thread writes 32 scattered 16-byte pieces.
// Every wait is bounded (WRF_ETIMEOUT on the status word).
#include <cstring>

#include "kernels.h"
#include "tc.cuh"

namespace wrf {

namespace {

constexpr int kTileRows = 128;
constexpr int kWG = 2;                           // tiles in flight per CTA
constexpr int kThreads = 128 * kWG;
constexpr uint32_t kPanel = static_cast<uint32_t>(kX3PanelBytes);        // 128 rows x 64 K
constexpr uint32_t kOutPanel = static_cast<uint32_t>(kX3OutPanelBytes);  // 16 rows x 64 K
constexpr uint32_t kWgCols = 256;                // TMEM columns per warpgroup
constexpr uint32_t kTmemCols = 512;

// activation staging: per warp 32 rows x 16 FP32 columns (2 KB)
constexpr int kStageCols = 16;
constexpr size_t kStageBytes = static_cast<size_t>(kThreads) * kStageCols * 4;

constexpr size_t smem_bytes(int nh) {
    return 1024 + mlp_x3_image_bytes(nh) + kStageBytes + kWG * WRF_HIDDEN * 4 + (1 + kWG) * 8 +
           16;
}
static_assert(smem_bytes(3) <= 227 * 1024, "shared memory of one CTA");

struct X3Args {
    SceneView s;
    GridView g;
    const float *U;          // FP32 per-Gaussian layer-1 term, blocked [N/128][32][128][4]
    const float *V;          // [Q][128] FP32 per-query layer-1 term (incl. b1)
    const uint16_t *w_img;   // X3 weight image (mlp_x3_image_bytes)
    int nh;                  // hidden 128x128 layers after the first (0..3)
    int Q, N, tpq, ntiles;
    int mode;                // 0: residuals, 1: records
    float *resid;
    float4 *rec;
    uint32_t *count;
    float *rec_im;
    float *acts;             // [nh + 1][Q N][128] (stored through the tensor map) or NULL
    int *status;
};

// TMA tensor store of a 3-D box from shared memory (bulk group), and the
// bulk-group waits: `read` until the sources have been read, else until the
// writes are done.
__device__ __forceinline__ void tma_store_3d(const CUtensorMap *map, const void *src, int x, int y,
                                             int z) {
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%2, %3, %4}], [%1];"
                 ::"l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(src)), "r"(x), "r"(y),
                 "r"(z)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() {
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_read_all() {
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_all() {
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// hi / lo BF16 pairs of 32 consecutive FP32 values (ReLU already applied)
__device__ __forceinline__ void split_pairs(const float *v, uint32_t *hi, uint32_t *lo) {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const uint32_t h = pack_bf16(v[2 * j], v[2 * j + 1]);
        const float h0 = __uint_as_float(h << 16), h1 = __uint_as_float(h & 0xFFFF0000u);
        hi[j] = h;
        lo[j] = pack_bf16(__fsub_rn(v[2 * j], h0), __fsub_rn(v[2 * j + 1], h1));
    }
}

// amap: the activations as a 3-D tensor [(nh + 1) Q][N][128] FP32, box 16
// columns x 32 rows, 64-byte swizzle (used only when a.acts is set).
__global__ void __launch_bounds__(kThreads, 1) mlp_x3_kernel(X3Args a,
                                                             const __grid_constant__ CUtensorMap amap) {
    extern __shared__ uint8_t smem_raw[];
    // 1024-byte aligned base (128-byte swizzle atoms must be 1024-aligned)
    const uint32_t raw = smem_u32(smem_raw);
    uint8_t *base = smem_raw + (((raw + 1023u) & ~1023u) - raw);
    const uint32_t w_bytes = static_cast<uint32_t>(mlp_x3_image_bytes(a.nh));
    uint8_t *wsm = base;
    float *stage0 = reinterpret_cast<float *>(base + w_bytes);               // [warp][32][16]
    float *vsm0 = stage0 + kThreads * kStageCols;                            // [kWG][128]
    uint64_t *bars = reinterpret_cast<uint64_t *>(vsm0 + kWG * WRF_HIDDEN);  // wbar, mbar[kWG]
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 1 + kWG);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int wg = warp >> 2, wq = warp & 3;
    const int wt = tid & 127;

    if (tid == 0) {
        for (int i = 0; i < 1 + kWG; ++i) mbar_init(&bars[i], 1);
        fence_mbar_init();
        *abort_flag = 0;
    }
    if (warp == 0) tmem_alloc(tmem_slot, kTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    if (tid == 0) {
        mbar_arrive_expect_tx(&bars[0], w_bytes);
        const uint8_t *src = reinterpret_cast<const uint8_t *>(a.w_img);
        for (uint32_t off = 0; off < w_bytes; off += 16384u) {
            const uint32_t len = w_bytes - off < 16384u ? w_bytes - off : 16384u;
            bulk_g2s(wsm + off, src + off, len, &bars[0]);
        }
    }
    wait_or_abort(&bars[0], 0, abort_flag, a.status);
    __syncthreads();

    uint64_t *mbar = &bars[1 + wg];
    uint32_t phase = 0;
    float *vsm = vsm0 + wg * WRF_HIDDEN;
    const uint32_t t_acc = tmem_base + static_cast<uint32_t>(wg) * kWgCols;
    const uint32_t t_hi = t_acc + 128u, t_lo = t_acc + 192u;
    const uint32_t lane_off = static_cast<uint32_t>(wq * 32) << 16;
    const int my_row = wq * 32 + lane;
    const bool leader = wt == 0;
    const uint32_t id128 = idesc_bf16(128, 128), id16 = idesc_bf16(128, 16);
    // image: hidden layer l at l * 4 panels (hi K 0-63, hi K 64-127, lo K
    // 0-63, lo K 64-127), the output layer (hi 2 panels, lo 2 panels), the
    // bias image, the selectors
    const uint32_t w_addr = smem_u32(wsm);
    const uint32_t o_addr = w_addr + static_cast<uint32_t>(a.nh) * 4u * kPanel;
    const uint32_t aug_addr = o_addr + 4u * kOutPanel;
    const uint64_t d_w = sw128_desc(w_addr), d_o = sw128_desc(o_addr);
    const uint64_t d_bias = plain_desc(aug_addr, 0u, 128u);
    const uint64_t d_sel = plain_desc(aug_addr + static_cast<uint32_t>(kBiasImageBytes), 128u, 0u);
    const int stride = gridDim.x * kWG;

    // The activations of a warp's 32 rows: each lane writes 16 values of its
    // own row into the warp's staging rows (16-byte chunk k of row r at chunk
    // k ^ ((r >> 1) & 3): the map's 64-byte swizzle, and conflict-free), then
    // lane 0 stores the 32 x 16 box at (column col0, row n0 + 32 wq, layer
    // plane z) once the previous box has been read out.  Rows past the
    // query's N are clipped by the map; a warp without valid rows stores
    // nothing.
    float *stage = stage0 + warp * 32 * kStageCols;
    auto stage_out = [&](const float *v, int z, int n0, int col0, bool any) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (lane == 0) bulk_wait_read_all();
            __syncwarp();
#pragma unroll
            for (int k = 0; k < 4; ++k)
                *reinterpret_cast<float4 *>(stage + lane * kStageCols +
                                            ((k ^ ((lane >> 1) & 3)) << 2)) =
                    make_float4(v[16 * h + 4 * k], v[16 * h + 4 * k + 1], v[16 * h + 4 * k + 2],
                                v[16 * h + 4 * k + 3]);
            fence_async_smem();
            __syncwarp();
            if (lane == 0 && any) {
                tma_store_3d(&amap, stage, col0 + 16 * h, n0 + wq * 32, z);
                bulk_commit();
            }
        }
    };
    // converts 32 activations (columns 32c ..) of this thread's row into the
    // activation plane z (z < 0: none) and the hi / lo pairs
    auto store_act = [&](int c, const float *v, int z, int n0, bool any) {
        if (z >= 0) stage_out(v, z, n0, 32 * c, any);
        uint32_t hi[16], lo[16];
        split_pairs(v, hi, lo);
        tmem_st16(t_hi + lane_off + static_cast<uint32_t>(c * 16), hi);
        tmem_st16(t_lo + lane_off + static_cast<uint32_t>(c * 16), lo);
    };
    // one layer's MMAs (N = 128 hidden or N = 16 output) from the hi / lo
    // pairs in tensor memory: bias, then 8 K-steps x (hi hi, hi lo, lo hi)
    auto layer_mmas = [&](bool out, int l) {
        tc_fence_after();
        const uint32_t id = out ? id16 : id128;
        mma_bf16(t_acc, desc_adv(d_sel, static_cast<uint32_t>(out ? 3 : l) * 256u), d_bias, id, 0u);
        const uint64_t bh = out ? d_o : desc_adv(d_w, static_cast<uint32_t>(l) * 4u * kPanel);
        const uint32_t pan = out ? kOutPanel : kPanel;
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
            const uint32_t ko = static_cast<uint32_t>(kk >> 2) * pan + static_cast<uint32_t>(kk & 3) * 32u;
            const uint64_t b_hi = desc_adv(bh, ko), b_lo = desc_adv(bh, 2u * pan + ko);
            const uint32_t ca = static_cast<uint32_t>(kk * 8);
            mma_bf16_ts(t_acc, t_hi + ca, b_hi, id, 1u);
            mma_bf16_ts(t_acc, t_hi + ca, b_lo, id, 1u);
            mma_bf16_ts(t_acc, t_lo + ca, b_hi, id, 1u);
        }
        mma_commit(mbar);
    };

    // U column quad j4 of this thread's row in 128-Gaussian block b
    auto u_quad = [&](int b, int j4) {
        return __ldg(reinterpret_cast<const float4 *>(a.U) +
                     (static_cast<size_t>(b) * 32 + j4) * kTileRows + my_row);
    };
    // operands of the next tile, fetched while the current one finishes: its
    // V[q] column, its Gaussian (projection epilogue) and U columns 0..31
    float vpre = 0.f;
    GaussParams ppre{};
    float4 u0[8];
    auto prefetch = [&](int t) {
        const int q = t / a.tpq, n0 = (t % a.tpq) * kTileRows;
        vpre = __ldg(a.V + static_cast<size_t>(q) * WRF_HIDDEN + wt);
        if (a.mode == 1 && n0 + my_row < a.N) ppre = load_params(a.s, n0 + my_row);
#pragma unroll
        for (int j = 0; j < 8; ++j) u0[j] = u_quad(n0 / kTileRows, j);
    };
    int tile = blockIdx.x * kWG + wg;
    if (tile < a.ntiles) prefetch(tile);
    for (; tile < a.ntiles; tile += stride) {
        if (wg_bar_any(1 + wg, *abort_flag != 0)) break;
        const int q = tile / a.tpq, n0 = (tile % a.tpq) * kTileRows;
        const int n = n0 + my_row;
        const bool ok = n < a.N;
        const bool any = wq * 32 < a.N - n0;  // this warp has rows to store
        const size_t row = static_cast<size_t>(q) * a.N + (ok ? n : 0);
        const bool save = a.acts != nullptr;
        const GaussParams pcur = ppre;
        vsm[wt] = vpre;
        named_bar(1 + wg, 128);
        // ---- layer 1: ReLU(U[n] + V[q]), exact FP32; U columns 32(c+1) ..
        // are in flight while columns 32c .. are converted
        {
            float4 ub[2][8];
#pragma unroll
            for (int j = 0; j < 8; ++j) ub[0][j] = u0[j];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                if (c < 3) {
#pragma unroll
                    for (int j = 0; j < 8; ++j) ub[(c + 1) & 1][j] = u_quad(n0 / kTileRows, (c + 1) * 8 + j);
                }
                float v[32];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const float4 u = ub[c & 1][j];
                    const float4 b = *reinterpret_cast<const float4 *>(vsm + c * 32 + 4 * j);
                    v[4 * j] = fmaxf(__fadd_rn(u.x, b.x), 0.f);
                    v[4 * j + 1] = fmaxf(__fadd_rn(u.y, b.y), 0.f);
                    v[4 * j + 2] = fmaxf(__fadd_rn(u.z, b.z), 0.f);
                    v[4 * j + 3] = fmaxf(__fadd_rn(u.w, b.w), 0.f);
                }
                store_act(c, v, save ? q : -1, n0, any);
            }
        }
        tmem_wait_st();
        tc_fence_before();
        named_bar(1 + wg, 128);
        // ---- hidden layers
        for (int l = 0; l < a.nh; ++l) {
            if (leader) layer_mmas(false, l);
            wait_or_abort(mbar, phase, abort_flag, a.status);
            phase ^= 1u;
            tc_fence_after();
            const int z = save ? (l + 1) * a.Q + q : -1;
#pragma unroll 1
            for (int c = 0; c < 4; ++c) {
                float v[32];
                tmem_ld32(t_acc + lane_off + static_cast<uint32_t>(c * 32), v);
#pragma unroll
                for (int j = 0; j < 32; ++j) v[j] = fmaxf(v[j], 0.f);
                store_act(c, v, z, n0, any);
            }
            tmem_wait_st();
            tc_fence_before();
            named_bar(1 + wg, 128);
        }
        // ---- output layer (the next tile's operands load meanwhile)
        if (leader) layer_mmas(true, 0);
        if (tile + stride < a.ntiles) prefetch(tile + stride);
        wait_or_abort(mbar, phase, abort_flag, a.status);
        phase ^= 1u;
        tc_fence_after();
        float o[16];
        tmem_ld16(t_acc + lane_off, o);
        tc_fence_before();
        if (ok && !*abort_flag) {
            if (a.mode == 0) {
                float *dst = a.resid + row * WRF_OUT;
#pragma unroll
                for (int j = 0; j < WRF_OUT; ++j) dst[j] = o[j];
            } else {
                float4 r0, r1;
                project_geom(pcur, o[0], o[1], o[2], o[3], o[4], a.g, r0, r1);
                a.rec[2 * row] = r0;
                a.rec[2 * row + 1] = r1;
                if (a.rec_im) a.rec_im[row] = weight_im(pcur);
                if (a.count) a.count[row] = record_tiles(r0, r1, a.g);
            }
        }
        named_bar(1 + wg, 128);  // TMEM columns and the V row are free again
    }
    if (lane == 0) bulk_wait_all();  // this warp's activation stores are done
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem_base, kTmemCols);
    }
}

}  // namespace

cudaError_t launch_mlp_x3(const SceneView &s, const MlpView &m, const GridView &g, int Q,
                          const DeformWs &ws, int mode, float *resid, float4 *rec,
                          uint32_t *count, float *acts, int *status, cudaStream_t st) {
    const long long rows = static_cast<long long>(Q) * s.n;
    if (rows == 0) return cudaSuccess;
    const int nh = m.n_layers - 2;
    if (nh < 0 || nh > 3) return cudaErrorInvalidValue;
    X3Args a{};
    a.s = s;
    a.g = g;
    a.U = ws.U;
    a.V = ws.V;
    a.w_img = ws.w_x3;
    a.nh = nh;
    a.Q = Q;
    a.N = s.n;
    a.tpq = (s.n + kTileRows - 1) / kTileRows;
    const long long nt = static_cast<long long>(a.tpq) * Q;
    if (nt >= (1ll << 31)) return cudaErrorInvalidValue;
    a.ntiles = static_cast<int>(nt);
    a.mode = mode;
    a.resid = resid;
    a.rec = rec;
    a.count = count;
    a.rec_im = (mode == 1 && s.channels == 2) ? reinterpret_cast<float *>(rec + 2 * rows) : nullptr;
    a.acts = acts;
    a.status = status;
    // the activations as [(nh + 1) Q][N][128], a box of 16 columns x 32 rows
    CUtensorMap amap;
    std::memset(&amap, 0, sizeof(amap));
    if (acts) {
        EncodeTiledFn f = encode_tiled();
        if (!f) return cudaErrorSymbolNotFound;
        const cuuint64_t dims[3] = {WRF_HIDDEN, static_cast<cuuint64_t>(s.n),
                                    static_cast<cuuint64_t>(nh + 1) * static_cast<cuuint64_t>(Q)};
        const cuuint64_t strides[2] = {WRF_HIDDEN * 4,
                                       static_cast<cuuint64_t>(s.n) * WRF_HIDDEN * 4};
        const cuuint32_t box[3] = {static_cast<cuuint32_t>(kStageCols), 32, 1};
        const cuuint32_t elem[3] = {1, 1, 1};
        if (f(&amap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, acts, dims, strides, box, elem,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
              CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    const size_t smem = smem_bytes(nh);
    cudaError_t e = cudaFuncSetAttribute(mlp_x3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int grid = (a.ntiles + kWG - 1) / kWG;
    if (grid > sms) grid = sms;
    mlp_x3_kernel<<<grid, kThreads, smem, st>>>(a, amap);
    return cudaGetLastError();
}

}  // namespace wrf
