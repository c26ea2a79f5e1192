// Deformation MLP on the 5th-generation tensor cores (tcgen05), BF16
// operands with FP32 accumulation in tensor memory (Sec. 4.2, Eq. 14).
//
// Rows are the (query, Gaussian) pairs.  A tile is 128 consecutive Gaussians
// of one query (one tcgen05 M=128 tile; TMEM lane = row); the last tile of a
// query is partial.  A CTA runs three warpgroups that each own one tile at a
// time and run independently, so the tensor core works on one warpgroup's
// layer while the others run their epilogues on the CUDA cores.  Per tile:
//   1. layer 1 splits exactly into a per-Gaussian and a per-query part:
//      W1 [gamma(mean_n); gamma(s_q)] + b1 = W1m gamma(mean_n) + V[q], with
//      V[q] = W1s gamma(s_q) + b1 computed once per query in FP32
//      (prep.cu).  The per-Gaussian part runs on the tensor core: the
//      thread of row n copies the BF16 row gamma(mean_n) (K = 32 or 64
//      columns; it, V[q] and the row's Gaussian parameters for the
//      projection epilogue are prefetched during the previous tile) into
//      the A tile, and
//      one thread issues the K/16 MMAs against the resident W1m image;
//   2. biases are added by the tensor core: every layer starts with one
//      K = 16 MMA of a selector A (ones in two columns) against a bias
//      image B holding the bias split into BF16 hi + lo (kernels.h); for
//      layer 1 the bias image is the warpgroup's own 128 x 8 image of V[q]
//      (hi, lo), written by the 128 threads with the tile's other operand;
//   3. every layer's epilogue: the 128 threads read their row from TMEM
//      (tcgen05.ld 32x32b, 64 columns per load), apply ReLU and round to
//      BF16 in one cvt.rn.relu.bf16x2 per pair, into the 128x128 K-major,
//      128-byte-swizzled A tile of the next layer;
//   4. hidden layers: bias MMA + 8 MMAs of 128x128x16, committed to an
//      mbarrier;
//   5. the output layer is one 128x16x128 MMA chain (5 useful columns)
//      whose epilogue either stores the residual row or deforms and
//      projects the Gaussian (fused Eq. 12-13) into its record.
// All weights (W1m, <= 3 hidden layers, output, bias image and selectors;
// <= 119 KB of BF16) are copied into shared memory once per CTA with bulk
// (TMA) copies.
#include "kernels.h"
#include "tc.cuh"

namespace wrf {

namespace {

constexpr int kTileRows = 128;
constexpr int kWG = 3;                    // warpgroups per CTA
constexpr int kThreads = 128 * kWG;
constexpr uint32_t kLayerBytes = 128 * 128 * 2;
constexpr uint32_t kW1Bytes = 128 * 128;  // W1m image: 128 rows x 128 B (K <= 64)
constexpr uint32_t kOutBytes = 16 * 128 * 2;
constexpr uint32_t kActBytes = 128 * 128 * 2;
constexpr uint32_t kAugBytes = static_cast<uint32_t>(kBiasImageBytes + kSelImageBytes);
constexpr uint32_t kVImgBytes = 2048;     // per warpgroup: V[q] hi/lo, 128 rows x 16 B
constexpr uint32_t kTmemCols = 512;       // kWG x 128 accumulator columns, power of 2

struct TcArgs {
    SceneView s;
    GridView g;
    const uint16_t *G;       // [N][k1] BF16 gamma(mean) rows, zero-padded
    const float *V;          // [Q][128] FP32 per-query layer-1 term (incl. b1)
    const uint16_t *w_img;   // BF16 images: W1m, hidden layers, output layer
    int nh;                  // hidden 128x128 layers (0..3)
    int k1;                  // layer-1 K: 32 or 64
    int Q, N, tpq;           // tiles per query
    int ntiles;
    int mode;
    float *resid;
    float4 *rec;
    uint32_t *count;
    float *rec_im;           // two channels: imaginary weights after the records
    int *status;
    // multi-scene batches (MULTI): query q belongs to scene scene_of[q] of the
    // table; its records start at qbase[q]; its 128-row tiles are
    // tstart[q] .. tstart[q+1]-1 of the launch (tstart[Q] tiles in all)
    const SceneEntry *table;
    const int *scene_of;
    const long long *qbase;
    const int *tstart;
};

constexpr size_t smem_bytes(int nh) {
    return 1024 + kW1Bytes + nh * kLayerBytes + kOutBytes + kAugBytes + kWG * kActBytes +
           kWG * kVImgBytes + (1 + kWG) * 8 + 16;
}
static_assert(smem_bytes(3) <= 227 * 1024, "shared memory of one CTA");

// The tile of a launch: query q, Gaussians n0 .. n0+127 of its scene, the
// scene's Gaussians and gamma(mean) rows, and where its records go.
struct TcTile {
    int q, n0, nq;
    long long rbase;  // record index of (q, Gaussian 0)
    SceneView s;
    const uint16_t *G;
};

// Query of tile t (MULTI): the last q with tstart[q] <= t.
__device__ __forceinline__ int tile_query(const int *tstart, int Q, int t) {
    int lo = 0, hi = Q - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(tstart + mid) <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <bool MULTI>
__device__ __forceinline__ TcTile tile_info(const TcArgs &a, int tile) {
    TcTile t;
    if (!MULTI) {
        t.q = tile / a.tpq;
        t.n0 = (tile % a.tpq) * kTileRows;
        t.nq = a.N;
        t.rbase = static_cast<long long>(t.q) * a.N;
        t.s = a.s;
        t.G = a.G;
    } else {
        t.q = tile_query(a.tstart, a.Q, tile);
        t.n0 = (tile - __ldg(a.tstart + t.q)) * kTileRows;
        const SceneEntry &e = a.table[__ldg(a.scene_of + t.q)];
        t.s = e.s;
        t.nq = e.s.n;
        t.rbase = __ldg(a.qbase + t.q);
        t.G = e.G;
    }
    return t;
}

template <bool MULTI>
__global__ void __launch_bounds__(kThreads, 1) mlp_tc_kernel(TcArgs a) {
    extern __shared__ uint8_t smem_raw[];
    // 1024-byte aligned base (128-byte swizzle atoms must be 1024-aligned)
    const uint32_t raw = smem_u32(smem_raw);
    uint8_t *base = smem_raw + (((raw + 1023u) & ~1023u) - raw);
    // weights (W1m, hidden, output, bias image, selectors): a multiple of
    // 1024 bytes, so the activation tiles after them stay 1024-aligned
    const uint32_t w_bytes = kW1Bytes + a.nh * kLayerBytes + kOutBytes + kAugBytes;
    uint8_t *wsm = base;
    uint8_t *act0 = base + w_bytes;
    uint8_t *vimg0 = act0 + kWG * kActBytes;                               // [kWG][2048]
    uint64_t *bars = reinterpret_cast<uint64_t *>(vimg0 + kWG * kVImgBytes);  // wbar, mbar[kWG]
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 1 + kWG);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int wg = warp >> 2, wq = warp & 3;  // warpgroup, warp within warpgroup
    const int wt = tid & 127;                 // thread within the warpgroup

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
    // the weights (and bias images) into shared memory; every thread waits
    uint32_t wphase = 0;
    auto load_weights = [&](const uint16_t *img) {
        if (tid == 0) {
            mbar_arrive_expect_tx(&bars[0], w_bytes);
            const uint8_t *src = reinterpret_cast<const uint8_t *>(img);
            for (uint32_t off = 0; off < w_bytes; off += 16384u) {
                uint32_t len = w_bytes - off < 16384u ? w_bytes - off : 16384u;
                bulk_g2s(wsm + off, src + off, len, &bars[0]);
            }
        }
        wait_or_abort(&bars[0], wphase, abort_flag, a.status);
        wphase ^= 1u;
        __syncthreads();
    };
    if (!MULTI) load_weights(a.w_img);

    uint64_t *mbar = &bars[1 + wg];
    uint32_t phase = 0;
    uint8_t *A = act0 + wg * kActBytes;
    uint8_t *vimg = vimg0 + wg * kVImgBytes;
    const uint32_t a_addr = smem_u32(A);
    const uint32_t w1_addr = smem_u32(wsm);
    const uint32_t wh_addr = w1_addr + kW1Bytes;
    const uint32_t aug_addr = wh_addr + a.nh * kLayerBytes + kOutBytes;
    const uint32_t sel_addr = aug_addr + static_cast<uint32_t>(kBiasImageBytes);
    // bias operands: B = bias image (row groups 128 B apart, K 8..15 repeat
    // K 0..7 and meet the selector's zero core matrix); A = selector p
    const uint64_t d_bias = plain_desc(aug_addr, 0u, 128u);
    const uint64_t d_vimg = plain_desc(smem_u32(vimg), 0u, 128u);
    // descriptor bases; each MMA advances them by a constant (desc_adv)
    const uint64_t d_a = sw128_desc(a_addr), d_w1 = sw128_desc(w1_addr);
    const uint64_t d_wh = sw128_desc(wh_addr), d_sel = plain_desc(sel_addr, 128u, 0u);
    const uint32_t t_acc = tmem_base + static_cast<uint32_t>(wg * 128);
    const uint32_t lane_off = static_cast<uint32_t>(wq * 32) << 16;  // TMEM lane field
    const int my_row = wq * 32 + lane;                               // row within the tile
    const bool leader = wt == 0;
    const uint32_t id128 = idesc_bf16(128, 128), id16 = idesc_bf16(128, 16);
    const int nch = a.k1 >> 3;  // 16-byte chunks of a gamma(mean) row (4 or 8)
    const int stride = gridDim.x * kWG;

    // prefetch of this thread's gamma(mean) row for its next tile
    uint4 gpre[8];
    float vpre = 0.f;     // this thread's column of V[q] for the next tile
    GaussParams ppre{};  // this thread's Gaussian for the next tile (projection epilogue)
    auto load_g = [&](int tile, bool have) {
        if (!have) return;
        const TcTile ti = tile_info<MULTI>(a, tile);
        const int n = ti.n0 + my_row;
        const bool ok = n < ti.nq;
        vpre = __ldg(a.V + static_cast<size_t>(ti.q) * 128 + wt);
        if (ok && a.mode == 1) ppre = load_params(ti.s, n);
        const uint4 *src =
            reinterpret_cast<const uint4 *>(ti.G + static_cast<size_t>(ok ? n : 0) * a.k1);
#pragma unroll
        for (int c = 0; c < 8; ++c)
            gpre[c] = (ok && c < nch) ? __ldg(src + c) : make_uint4(0u, 0u, 0u, 0u);
    };

    // one tile: layer 1 from the prefetched operands, the hidden layers, the
    // output layer and its epilogue; prefetches tile `next` (if has_next)
    auto run_tile = [&](int tile, int next, bool has_next) {
        const TcTile ti = tile_info<MULTI>(a, tile);
        const int q = ti.q;
        const int n = ti.n0 + my_row;
        // ---- layer 1 operand: gamma(mean_n) row -> A columns 0..k1-1
#pragma unroll
        for (int c = 0; c < 8; ++c)
            if (c < nch)
                *reinterpret_cast<uint4 *>(A + my_row * 128 + ((c ^ (my_row & 7)) << 4)) = gpre[c];
        {
            // V[q] column wt as BF16 hi + lo, K columns 0 and 1 of row wt
            const uint32_t hi = pack_bf16(vpre, 0.f) & 0xFFFFu;
            const float hif = __uint_as_float(hi << 16);
            const uint32_t lo = pack_bf16(__fsub_rn(vpre, hif), 0.f) & 0xFFFFu;
            *reinterpret_cast<uint4 *>(vimg + (wt >> 3) * 128 + (wt & 7) * 16) =
                make_uint4(hi | (lo << 16), 0u, 0u, 0u);
        }
        const GaussParams pcur = ppre;
        load_g(next, has_next);
        fence_async_smem();
        named_bar(1 + wg, 128);

        // ---- layers: 0 = layer 1 (K = k1, bias V[q]), 1..nh = hidden
        for (int l = 0; l <= a.nh; ++l) {
            if (leader) {
                tc_fence_after();
                if (l == 0) {
                    // D = V[q] (hi + lo), then += W1m gamma(mean)
                    mma_bf16(t_acc, d_sel, d_vimg, id128, 0u);
                    mma_bf16(t_acc, d_a, d_w1, id128, 1u);
                    mma_bf16(t_acc, desc_adv(d_a, 32u), desc_adv(d_w1, 32u), id128, 1u);
                    if (a.k1 == 64) {
                        mma_bf16(t_acc, desc_adv(d_a, 64u), desc_adv(d_w1, 64u), id128, 1u);
                        mma_bf16(t_acc, desc_adv(d_a, 96u), desc_adv(d_w1, 96u), id128, 1u);
                    }
                } else {
                    // D = b_l (hi + lo, selector pair l-1), then += W_l h
                    mma_bf16(t_acc, desc_adv(d_sel, (l - 1) * 256u), d_bias, id128, 0u);
                    const uint64_t d_wl = desc_adv(d_wh, (l - 1) * kLayerBytes);
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const uint32_t koff = (k >> 2) * 16384u + (k & 3) * 32u;
                        mma_bf16(t_acc, desc_adv(d_a, koff), desc_adv(d_wl, koff), id128, 1u);
                    }
                }
                mma_commit(mbar);
            }
            wait_or_abort(mbar, phase, abort_flag, a.status);
            phase ^= 1u;
            tc_fence_after();
            {
                // 16 columns at a time; the next chunk's load is in flight
                // while this one is converted and stored
                uint32_t ra[16], rb[16];
                auto convert16 = [&](const uint32_t (&r)[16], int c) {
#pragma unroll
                    for (int j = 0; j < 2; ++j) {
                        const uint32_t *v = r + j * 8;
                        uint4 p;
                        p.x = pack_bf16_relu(__uint_as_float(v[0]), __uint_as_float(v[1]));
                        p.y = pack_bf16_relu(__uint_as_float(v[2]), __uint_as_float(v[3]));
                        p.z = pack_bf16_relu(__uint_as_float(v[4]), __uint_as_float(v[5]));
                        p.w = pack_bf16_relu(__uint_as_float(v[6]), __uint_as_float(v[7]));
                        const int kc = c * 2 + j;  // 16-byte chunk 0..15 along K
                        *reinterpret_cast<uint4 *>(A + (kc >> 3) * 16384 + my_row * 128 +
                                                   (((kc & 7) ^ (my_row & 7)) << 4)) = p;
                    }
                };
                tmem_ld16_issue(t_acc + lane_off, ra);
                tmem_ld16_wait(ra);
#pragma unroll
                for (int c = 0; c < 8; c += 2) {
                    tmem_ld16_issue(t_acc + lane_off + (c + 1) * 16, rb);
                    convert16(ra, c);
                    tmem_ld16_wait(rb);
                    if (c + 2 < 8) tmem_ld16_issue(t_acc + lane_off + (c + 2) * 16, ra);
                    convert16(rb, c + 1);
                    if (c + 2 < 8) tmem_ld16_wait(ra);
                }
            }
            tc_fence_before();
            fence_async_smem();
            named_bar(1 + wg, 128);
        }

        // ---- output layer (N = 16, columns 0..4 used), into the same columns
        if (leader) {
            tc_fence_after();
            const uint64_t d_wo = desc_adv(d_wh, a.nh * kLayerBytes);
            // D = b_out (selector pair 3), then += W_out h
            mma_bf16(t_acc, desc_adv(d_sel, 3 * 256u), d_bias, id16, 0u);
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const uint32_t ka = (k >> 2) * 16384u + (k & 3) * 32u;
                const uint32_t kb = (k >> 2) * 2048u + (k & 3) * 32u;
                mma_bf16(t_acc, desc_adv(d_a, ka), desc_adv(d_wo, kb), id16, 1u);
            }
            mma_commit(mbar);
        }
        wait_or_abort(mbar, phase, abort_flag, a.status);
        phase ^= 1u;
        tc_fence_after();
        float o[16];
        tmem_ld16(t_acc + lane_off, o);
        tc_fence_before();
        if (n < ti.nq && !*abort_flag) {
            const long long row = ti.rbase + n;
            const float d0 = o[0], d1 = o[1], d2 = o[2], d3 = o[3], d4 = o[4];
            if (a.mode == 0) {
                float *dst = a.resid + row * WRF_OUT;
                dst[0] = d0;
                dst[1] = d1;
                dst[2] = d2;
                dst[3] = d3;
                dst[4] = d4;
            } else {
                float4 r0, r1;
                project_geom(pcur, d0, d1, d2, d3, d4, a.g, r0, r1);
                a.rec[2 * row] = r0;
                a.rec[2 * row + 1] = r1;
                if (a.rec_im) a.rec_im[row] = weight_im(pcur);
                if (a.count) a.count[row] = record_tiles(r0, r1, a.g);
            }
        }
        named_bar(1 + wg, 128);  // TMEM columns, A tile and V image are free again
    };

    if (!MULTI) {
        int tile = blockIdx.x * kWG + wg;
        load_g(tile, tile < a.ntiles);
        for (; tile < a.ntiles; tile += stride) {
            // uniform per warpgroup: a timed-out wait anywhere ends the loop for
            // all 128 threads together (no thread is left at a named barrier)
            if (wg_bar_any(1 + wg, *abort_flag != 0)) break;
            run_tile(tile, tile + stride, tile + stride < a.ntiles);
        }
    } else {
        // a contiguous range of tiles per CTA, in segments of one scene: the
        // scene's weights are loaded at a segment start (all threads wait),
        // then the warpgroups take the segment's tiles in turn
        const int ntiles = __ldg(a.tstart + a.Q);
        const int t0 = static_cast<int>(static_cast<long long>(ntiles) * blockIdx.x / gridDim.x);
        const int t1 =
            static_cast<int>(static_cast<long long>(ntiles) * (blockIdx.x + 1) / gridDim.x);
        int cur = -1;
        for (int seg = t0; seg < t1;) {
            int q = tile_query(a.tstart, a.Q, seg);
            const int sc = __ldg(a.scene_of + q);
            while (q + 1 < a.Q && __ldg(a.scene_of + q + 1) == sc) ++q;
            const int seg_end = min(t1, __ldg(a.tstart + q + 1));
            if (sc != cur) {
                // uniform over the CTA: a timed-out wait ends the loop for all
                if (wg_bar_any(4, *abort_flag != 0, kThreads)) break;
                load_weights(a.table[sc].w_img);
                cur = sc;
            }
            int tile = seg + wg;
            load_g(tile, tile < seg_end);
            for (; tile < seg_end; tile += kWG) {
                if (wg_bar_any(1 + wg, *abort_flag != 0)) break;
                run_tile(tile, tile + kWG, tile + kWG < seg_end);
            }
            seg = seg_end;
            __syncthreads();  // every warpgroup is done with the segment's weights
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem_base, kTmemCols);
    }
}

}  // namespace

cudaError_t launch_mlp_tc(const SceneView &s, const MlpView &m, const GridView &g, int Q,
                          const DeformWs &ws, int mode, float *resid, float4 *rec,
                          uint32_t *count, int *status, cudaStream_t st) {
    const long long rows = static_cast<long long>(Q) * s.n;
    if (rows == 0) return cudaSuccess;
    const int nh = m.n_layers - 2;
    if (nh < 0 || nh > 3 || m.dm > 64) return cudaErrorInvalidValue;
    TcArgs a{};
    a.s = s;
    a.g = g;
    a.G = ws.G;
    a.V = ws.V;
    a.w_img = ws.w_bf16;
    a.nh = nh;
    a.k1 = mlp_k1(m.dm);
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
    a.status = status;
    const size_t smem = smem_bytes(nh);
    cudaError_t e = cudaFuncSetAttribute(mlp_tc_kernel<false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int grid = (a.ntiles + kWG - 1) / kWG;
    if (grid > sms) grid = sms;
    mlp_tc_kernel<false><<<grid, kThreads, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_mlp_tc_multi(const SceneEntry *table, const MlpView &m, const GridView &g,
                                int Q, const int *scene_of, const long long *qbase,
                                const int *tstart, const float *V, float4 *rec, int *status,
                                cudaStream_t st) {
    if (Q == 0) return cudaSuccess;
    const int nh = m.n_layers - 2;
    if (nh < 0 || nh > 3 || m.dm > 64) return cudaErrorInvalidValue;
    TcArgs a{};
    a.g = g;
    a.V = V;
    a.nh = nh;
    a.k1 = mlp_k1(m.dm);
    a.Q = Q;
    a.mode = 1;
    a.rec = rec;
    a.status = status;
    a.table = table;
    a.scene_of = scene_of;
    a.qbase = qbase;
    a.tstart = tstart;
    const size_t smem = smem_bytes(nh);
    cudaError_t e = cudaFuncSetAttribute(mlp_tc_kernel<true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // persistent: the tile count is on the device (it depends on the batch)
    mlp_tc_kernel<true><<<sms, kThreads, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace wrf
