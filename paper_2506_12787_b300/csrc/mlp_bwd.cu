// Back-propagation through the deformation MLP (Sec. 4.2 Eq. 14-15; the
// paper fits all parameters by gradient descent, Sec. 4.4), on the
// 5th-generation tensor cores.
//
// Notation: layer l maps H_l -> Z_l, H_{l+1} = ReLU(Z_l); H_0 = [gamma(mean_n),
// gamma(tx_q)] (Eq. 15), the output layer is l = L-1 and D_l = dL/dZ_l:
//   D_{L-1} = d_resid,   dW_l += D_l^T H_l,   db_l += sum_rows D_l,
//   D_{l-1} = (D_l W_l) * [H_l > 0].
// The forward's hidden activations H_1 .. H_{L-1} are read from `acts`
// (saved by wrf_deform_acts, or recomputed here by the FP32 forward kernel in
// chunks of queries).
//
// Tiles and layouts.  A tile is 64 consecutive Gaussians (rows) of one query.
// TMEM lanes are hidden units, not rows: everything a row-sum or a mask needs
// is then thread-local.  Per tile and layer:
//   * D_l^T is a 128-unit x 64-row shared tile (K-major, 128-byte swizzle:
//     unit u's 64 rows in one 128-byte line), written by thread u;
//   * H_l^T is a 128-unit x 64-row shared tile laid out like D^T, written by
//     thread u from a coalesced column load;
//   * delta:  D_{l-1}^T = W_l^T D_l^T   (M = 128 units, N = 64 rows, K = 128):
//             A = W_l^T panels (K-major), B = the D^T tile read MN-major;
//   * weight gradient:  dW_l^T += H_l^T D_l   (M = 128 in units, N = 128 out
//             units, K = 64 rows): A = the H^T tile, B = the D^T tile (both
//             K-major), accumulated in TMEM over many tiles;
//   * the epilogue (thread u = TMEM lane u) reads its unit's 64 deltas,
//     applies the ReLU mask of H_l (bits kept from the load), sums them into
//     db, and writes D_{l-1}^T back to the tile.
// The output layer (K = 5) runs on the CUDA cores in FP32: D_{L-2} =
// (d_resid W_{L-1}) * mask, dW_{L-1} and db_{L-1} in registers.  Layer 0: the
// gamma(mean) part of dW_0 is one more MMA (A = D_0^T, B = a 64-row x 64-
// feature tile of gamma(mean) rows); the gamma(tx) part is rank one per
// query, gamma(tx_q) x (sum over the query's rows of D_0), and db_0 is that
// row sum: per-tile column sums are stored and reduced per query at the end.
//
// Precision.  Every FP32 operand x is split into BF16 hi = bf16(x) and lo =
// bf16(x - hi); each product is hi*hi + hi*lo + lo*hi (relative error ~2^-17
// of |a||b|), accumulated in FP32 by the tensor core.  The weight gradients
// sum over a million rows: each CTA's TMEM accumulators are added into an
// FP32 partial in global memory every kFlush tile pairs (a bounded number of
// tensor-core accumulations per FP32 value), and the partials of all CTAs are
// reduced in a fixed order.
//
// A CTA runs two compute warpgroups (a tile each) that share the three dW
// accumulators, and one producer warp that streams the hidden layers' W^T
// panels (16 KB each, 4 per layer) through a ring of shared slots with bulk
// copies; a slot is refilled once both warpgroups' MMAs reading it are done.
// A model with more than three hidden layers runs in passes of at most three
// weight-gradient layers (the delta chain is recomputed from the top in each).
#include <cuda_bf16.h>

#include "kernels.h"
#include "tc.cuh"

namespace wrf {

namespace {

constexpr int kR = 64;                    // rows per tile
constexpr int kWG = 2;                    // compute warpgroups
constexpr int kThreads = kWG * 128 + 32;  // + producer warp
constexpr int kRing = 5;                  // weight panel slots
constexpr uint32_t kPanel = 128 * 128;    // W^T panel: 128 rows x 64 K x BF16
constexpr uint32_t kDt = 128 * 128;       // D^T tile, one term: 128 units x 64 rows x BF16
constexpr uint32_t kHt = 128 * 128;       // H^T tile, one term: 128 units x 64 rows x BF16
constexpr uint32_t kGt = 64 * 128;        // gamma(mean) tile, one term: 64 rows x 64 features
constexpr uint32_t kMnLbo = 8192;         // MN-major B with N = 64: one swizzle atom, LBO unused
constexpr int kSlots = 3;                 // dW accumulators (hidden layers per pass)
constexpr int kFlush = 8;                 // tile pairs between flushes of the accumulators
constexpr int kGp = 8;                    // floats per staged d_resid row
constexpr int kGammaF = 64;               // gamma(mean) features per row, zero-padded
constexpr uint32_t kTmemCols = 512;       // 3 x 128 dW + 2 x 64 delta
constexpr int kMaxGrid = 256;             // CTAs with partial-sum slots

constexpr size_t smem_bytes() {
    return 1024 + kRing * kPanel + kWG * (2 * kDt + 2 * kHt) + kWG * kR * kGp * 4 +
           8 * WRF_HIDDEN * 4 + (2 * kRing + kWG) * 8 + 16;
}
static_assert(smem_bytes() <= 227 * 1024, "shared memory of one CTA");

// Shared-memory descriptor with both byte offsets (MN-major operands: lbo =
// stride between 64-element swizzle atoms along M/N, sbo = stride between
// 8-row groups along K), 128-byte swizzle.
__device__ __forceinline__ uint64_t sw128_desc_lbo(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);
    d |= static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16;
    d |= static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32;
    d |= static_cast<uint64_t>(1) << 46;
    d |= static_cast<uint64_t>(2) << 61;
    return d;
}
// kind::f16 instruction descriptor with B read MN-major (A K-major).
__host__ __device__ constexpr uint32_t idesc_bf16_bmn(int M, int N) {
    return idesc_bf16(M, N) | (1u << 16);
}

// dst[0..3] += (a, b, c, d) at the L2 (a vector atomic whose result is unused).
__device__ __forceinline__ void red_add_v4(float4 *dst, float a, float b, float c, float d) {
    atomicAdd(dst, make_float4(a, b, c, d));
}

// BF16 hi / lo of a pair (x0 in the low half).
__device__ __forceinline__ void split2(float x0, float x1, uint32_t &hi, uint32_t &lo) {
    hi = pack_bf16(x0, x1);
    const float h0 = __uint_as_float(hi << 16), h1 = __uint_as_float(hi & 0xFFFF0000u);
    lo = pack_bf16(__fsub_rn(x0, h0), __fsub_rn(x1, h1));
}
__device__ __forceinline__ void split1(float x, uint16_t &hi, uint16_t &lo) {
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    const __nv_bfloat16 l = __float2bfloat16_rn(__fsub_rn(x, __bfloat162float(h)));
    hi = *reinterpret_cast<const uint16_t *>(&h);
    lo = *reinterpret_cast<const uint16_t *>(&l);
}

// Byte offset of (row m, column k < 64) in a K-major 128-byte-swizzled panel.
__host__ __device__ inline uint32_t panel_off(int m, int k) {
    return static_cast<uint32_t>((m >> 3) * 1024 + (m & 7) * 128 + ((((k >> 3) ^ (m & 7))) << 4) +
                                 (k & 7) * 2);
}


struct BwdArgs {
    int N, Qc, tpq, ntiles, npairs;
    int nh;                 // hidden layers (W_1 .. W_nh)
    int lo, hi;             // hidden layers whose dW this pass accumulates (none if hi < lo)
    int dlo;                // lowest layer of the delta chain this pass (>= 1)
    int first_pass, last_pass;
    int dm;
    const float *acts;      // [L-1][Qc N][128]; acts + (l-1) stride = H_l
    long long act_stride;
    const float *dres;      // [Qc N][5]
    const float *Wo;        // [5][128]
    const uint8_t *wimg;    // W^T panels [nh][4][kPanel]
    const uint8_t *gimg;    // gamma(mean) tiles [2 terms][Npad / 64][kGt]
    long long gterm;        // bytes per term image
    float *pdw;             // [grid][kSlots][128][128]
    float *pdb;             // [grid][kWG][8][128]  db of hidden layer l at [l]
    float *pdwo;            // [grid][kWG][8][128]  rows 0..4 dW_out, row 5 db_out (lanes < 5)
    float *pdw0;            // [grid][kWG][64][128] dW_0 gamma(mean) part, [feature][unit]
    float *tilesum;         // [ntiles][128]
    float *d0;              // [Qc N][128] or NULL
    int *status;
};

// 9 warps: the SM's four register sub-files hold up to 3 warps each, so at
// most 168 registers per thread; a single 64-float column buffer (prefetch)
// keeps the kernel within that.
__global__ void __launch_bounds__(kThreads, 1) mlp_bwd_tc_kernel(BwdArgs a) {
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    uint8_t *base = smem_raw + (((raw + 1023u) & ~1023u) - raw);
    uint8_t *ring = base;
    uint8_t *tiles = ring + kRing * kPanel;                       // [kWG][Dt 2 terms, Ht 2 terms]
    float *gstage = reinterpret_cast<float *>(tiles + kWG * (2 * kDt + 2 * kHt));  // [kWG][kR][kGp]
    float *wo_s = gstage + kWG * kR * kGp;                        // [8][128]
    uint64_t *bars = reinterpret_cast<uint64_t *>(wo_s + 8 * WRF_HIDDEN);
    uint64_t *full = bars, *empty = bars + kRing, *accb = bars + 2 * kRing;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * kRing + kWG);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int i = 0; i < kRing; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], kWG);
        }
        for (int i = 0; i < kWG; ++i) mbar_init(&accb[i], 1);
        fence_mbar_init();
        *abort_flag = 0;
    }
    for (int i = tid; i < 8 * WRF_HIDDEN; i += blockDim.x)
        wo_s[i] = i < WRF_OUT * WRF_HIDDEN ? a.Wo[i] : 0.f;
    if (warp == 0) tmem_alloc(tmem_slot, kTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    const int rounds = blockIdx.x < a.npairs
                           ? (a.npairs - static_cast<int>(blockIdx.x) + gridDim.x - 1) / gridDim.x
                           : 0;
    const bool have_dw = a.hi >= a.lo;
    // per round, in order: W^T panels of the delta layers nh .. dlo (4 each),
    // then (last pass) the gamma(mean) tiles of the two warpgroups' tiles

    if (warp == kWG * 4) {
        // ------------------------------------------------------ producer warp
        if (lane == 0) {
            uint32_t g = 0;
            bool ok = true;
            auto acquire = [&](int &slot) {
                slot = static_cast<int>(g % kRing);
                if (g >= kRing &&
                    !wait_or_abort(&empty[slot], ((g / kRing) - 1) & 1u, abort_flag, a.status))
                    return false;
                return true;
            };
            for (int r = 0; r < rounds && ok; ++r) {
                for (int l = a.nh; l >= a.dlo && ok; --l)
                    for (int p = 0; p < 4; ++p) {
                        int slot;
                        if (!(ok = acquire(slot))) break;
                        mbar_arrive_expect_tx(&full[slot], kPanel);
                        bulk_g2s(ring + slot * kPanel,
                                 a.wimg + (static_cast<size_t>(l - 1) * 4 + p) * kPanel, kPanel,
                                 &full[slot]);
                        ++g;
                    }
                if (!a.last_pass) continue;
                const int pr = static_cast<int>(blockIdx.x) + r * static_cast<int>(gridDim.x);
                for (int w2 = 0; w2 < kWG && ok; ++w2) {
                    int slot;
                    if (!(ok = acquire(slot))) break;
                    const int tile = 2 * pr + w2;
                    // a warpgroup without a tile this round multiplies zeros: any
                    // gamma tile will do
                    const size_t t0 =
                        static_cast<size_t>(tile < a.ntiles ? (tile % a.tpq) : 0) * kGt;
                    mbar_arrive_expect_tx(&full[slot], 2 * kGt);
                    bulk_g2s(ring + slot * kPanel, a.gimg + t0, kGt, &full[slot]);
                    bulk_g2s(ring + slot * kPanel + kGt, a.gimg + a.gterm + t0, kGt, &full[slot]);
                    ++g;
                }
            }
            // copies still in flight land before the CTA exits (bounded waits)
            for (uint32_t i = 0; i < kRing && i < g; ++i) {
                const uint32_t gg = g - 1 - i;
                mbar_wait(&full[gg % kRing], (gg / kRing) & 1u, a.status, kWaitLimitNs);
            }
        }
    } else {
        // ---------------------------------------------------- compute groups
        const int wg = warp >> 2, wq = warp & 3;
        const int u = tid & 127;  // hidden unit = TMEM lane
        const bool leader = u == 0, mma_warp = u < 32;
        uint8_t *Dt = tiles + wg * (2 * kDt + 2 * kHt);
        uint8_t *Ht = Dt + 2 * kDt;
        float *gs = gstage + wg * kR * kGp;
        const uint32_t dt_a = smem_u32(Dt), ht_a = smem_u32(Ht), ring_a = smem_u32(ring);
        const uint32_t lane_off = static_cast<uint32_t>(wq * 32) << 16;
        const uint32_t t_dw = tmem_base;                                   // + 128 s
        const uint32_t t_dl = tmem_base + 384u + static_cast<uint32_t>(64 * wg);
        const uint32_t id_dw = idesc_bf16(128, 128), id_dl = idesc_bf16_bmn(128, 64);

        // zero this warpgroup's half (64 columns) of every dW accumulator
        auto zero_dw = [&]() {
            uint32_t z[32];
#pragma unroll
            for (int i = 0; i < 32; ++i) z[i] = 0u;
            for (int s = 0; s < kSlots; ++s)
                for (int c = 0; c < 2; ++c)
                    tmem_st32(t_dw + lane_off + static_cast<uint32_t>(128 * s + 64 * wg + 32 * c), z);
            tmem_wait_st();
        };
        // add this warpgroup's half of every dW accumulator of the pass into
        // the CTA's FP32 partial, then zero it
        auto flush_dw = [&]() {
            float *pd = a.pdw + static_cast<size_t>(blockIdx.x) * kSlots * 128 * 128;
            for (int s = 0; s <= a.hi - a.lo; ++s)
                for (int c = 0; c < 2; ++c) {
                    float v[32];
                    tmem_ld32(t_dw + lane_off + static_cast<uint32_t>(128 * s + 64 * wg + 32 * c), v);
                    float4 *dst = reinterpret_cast<float4 *>(
                        pd + (static_cast<size_t>(s) * 128 + u) * 128 + 64 * wg + 32 * c);
                    // fire-and-forget vector reductions: the CTA owns its
                    // partial, and one thread's reductions to an address are
                    // applied in order, so every element is still the sum of
                    // its flushes in flush order
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        red_add_v4(dst + j, v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
                }
            zero_dw();
        };
        if (have_dw) zero_dw();
        float db_acc[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) db_acc[i] = 0.f;
        float dwo[WRF_OUT] = {0.f, 0.f, 0.f, 0.f, 0.f}, dbo = 0.f;
        uint32_t g = 0, phase = 0;
        tc_fence_before();
        named_bar(1, kWG * 128);
        tc_fence_after();

        struct TileRef {
            int tile, q, n0, nvalid;
            bool tv;
            long long row0;
        };
        auto tile_at = [&](int round) {
            TileRef t{};
            const int p = static_cast<int>(blockIdx.x) + round * static_cast<int>(gridDim.x);
            t.tile = 2 * p + wg;
            t.tv = round < rounds && t.tile < a.ntiles;
            t.q = t.tv ? t.tile / a.tpq : 0;
            t.n0 = t.tv ? (t.tile % a.tpq) * kR : 0;
            t.nvalid = t.tv ? min(kR, a.N - t.n0) : 0;
            t.row0 = static_cast<long long>(t.q) * a.N + t.n0;
            return t;
        };
        // this unit's column of an activation tile: h[r] = H[row0 + r][u]
        auto load_col = [&](const float *H, const TileRef &t, float *h) {
#pragma unroll
            for (int r = 0; r < kR; ++r)
                h[r] = r < t.nvalid ? __ldg(H + (t.row0 + r) * WRF_HIDDEN + u) : 0.f;
        };
        // this thread's share of the tile's d_resid rows (kR x 5 values)
        auto load_g = [&](const TileRef &t, float *gp) {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const int e = u + 128 * k, r = e / WRF_OUT;
                gp[k] = (e < kR * WRF_OUT && r < t.nvalid) ? __ldg(a.dres + t.row0 * WRF_OUT + e)
                                                           : 0.f;
            }
        };
        // rows 16 qt .. 16 qt + 15 of D^T row u (hi and lo terms)
        auto write_dt_q = [&](const float *t, int qt) {
#pragma unroll
            for (int c4 = 0; c4 < 2; ++c4) {
                const int c = 2 * qt + c4;
                uint4 h4, l4;
                split2(t[8 * c4 + 0], t[8 * c4 + 1], h4.x, l4.x);
                split2(t[8 * c4 + 2], t[8 * c4 + 3], h4.y, l4.y);
                split2(t[8 * c4 + 4], t[8 * c4 + 5], h4.z, l4.z);
                split2(t[8 * c4 + 6], t[8 * c4 + 7], h4.w, l4.w);
                const uint32_t off = static_cast<uint32_t>(u * 128 + ((c ^ (u & 7)) << 4));
                *reinterpret_cast<uint4 *>(Dt + off) = h4;
                *reinterpret_cast<uint4 *>(Dt + kDt + off) = l4;
            }
        };
        auto write_d0_q = [&](const float *t, int qt, const TileRef &ti) {
            if (!a.d0) return;
#pragma unroll
            for (int r = 0; r < 16; ++r)
                if (16 * qt + r < ti.nvalid)
                    a.d0[(ti.row0 + 16 * qt + r) * WRF_HIDDEN + u] = t[r];
        };

        // h: one 64-row column of activations, always the next one needed
        // (loaded a step ahead); gacc: the gamma(mean) part of dW_0 for
        // features < 32 (the rest, when L_mean > 7, read-modify-written per tile)
        float h[kR], gpre[3], gacc[32];
#pragma unroll
        for (int f = 0; f < 32; ++f) gacc[f] = 0.f;
        {
            const TileRef t0 = tile_at(0);
            load_col(a.acts + static_cast<size_t>(a.nh) * a.act_stride, t0, h);
            load_g(t0, gpre);
        }
        for (int round = 0; round < rounds; ++round) {
            const TileRef ti = tile_at(round), tn = tile_at(round + 1);
            // ---- output layer (K = 5) on the CUDA cores; h = H_{nh+1}
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const int e = u + 128 * k;
                if (e < kR * WRF_OUT) gs[(e / WRF_OUT) * kGp + e % WRF_OUT] = gpre[k];
            }
            named_bar(2 + wg, 128);
            // what this step needs from h: the ReLU mask and dW of the output layer
            uint64_t mask_o = 0;
#pragma unroll
            for (int r = 0; r < kR; ++r) {
                if (h[r] > 0.f) mask_o |= 1ull << r;
                if (a.first_pass) {
                    const float4 g0 = *reinterpret_cast<const float4 *>(gs + r * kGp);
                    const float g4 = gs[r * kGp + 4];
                    dwo[0] = fmaf(g0.x, h[r], dwo[0]);
                    dwo[1] = fmaf(g0.y, h[r], dwo[1]);
                    dwo[2] = fmaf(g0.z, h[r], dwo[2]);
                    dwo[3] = fmaf(g0.w, h[r], dwo[3]);
                    dwo[4] = fmaf(g4, h[r], dwo[4]);
                }
            }
            // the first delta layer's activations, in flight during the rest of the step
            if (a.nh >= a.dlo) {
                load_col(a.acts + static_cast<size_t>(a.nh - 1) * a.act_stride, ti, h);
            } else {
                // no delta layer: the next round's inputs
                load_col(a.acts + static_cast<size_t>(a.nh) * a.act_stride, tn, h);
                load_g(tn, gpre);
            }
            float dsum = 0.f;
#pragma unroll
            for (int qt = 0; qt < 4; ++qt) {
                float t[16];
#pragma unroll
                for (int r = 0; r < 16; ++r) {
                    const int rr = 16 * qt + r;
                    const float4 g0 = *reinterpret_cast<const float4 *>(gs + rr * kGp);
                    const float g4 = gs[rr * kGp + 4];
                    float dv = g0.x * wo_s[u];
                    dv = fmaf(g0.y, wo_s[WRF_HIDDEN + u], dv);
                    dv = fmaf(g0.z, wo_s[2 * WRF_HIDDEN + u], dv);
                    dv = fmaf(g0.w, wo_s[3 * WRF_HIDDEN + u], dv);
                    dv = fmaf(g4, wo_s[4 * WRF_HIDDEN + u], dv);
                    t[r] = ((mask_o >> rr) & 1ull) ? dv : 0.f;
                    dsum += t[r];
                }
                if (a.nh == 0) write_d0_q(t, qt, ti);
                write_dt_q(t, qt);
            }
            if (a.first_pass && u < WRF_OUT)
                for (int r = 0; r < kR; ++r) dbo += gs[r * kGp + u];
#pragma unroll
            for (int i = 1; i < 8; ++i)
                if (i == a.nh && i >= a.lo && i <= a.hi) db_acc[i] += dsum;

            // ---- hidden layers l = nh .. dlo: delta chain and dW; d = H_l
            for (int l = a.nh; l >= a.dlo; --l) {
                uint64_t mask = 0;
#pragma unroll
                for (int r = 0; r < kR; ++r)
                    if (h[r] > 0.f) mask |= 1ull << r;
                const bool dw_here = l >= a.lo && l <= a.hi;
                if (dw_here) {
                    // H_l^T row u (64 rows of unit u), hi and lo terms
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        uint4 h4, l4;
                        split2(h[8 * c + 0], h[8 * c + 1], h4.x, l4.x);
                        split2(h[8 * c + 2], h[8 * c + 3], h4.y, l4.y);
                        split2(h[8 * c + 4], h[8 * c + 5], h4.z, l4.z);
                        split2(h[8 * c + 6], h[8 * c + 7], h4.w, l4.w);
                        const uint32_t off = static_cast<uint32_t>(u * 128 + ((c ^ (u & 7)) << 4));
                        *reinterpret_cast<uint4 *>(Ht + off) = h4;
                        *reinterpret_cast<uint4 *>(Ht + kHt + off) = l4;
                    }
                }
                fence_async_smem();
                tc_fence_before();
                named_bar(2 + wg, 128);
                if (leader) {
                    tc_fence_after();
                    if (dw_here) {
                        // dW_l^T += H_l^T D_l (lanes = input units, columns = output units)
                        const uint32_t acc = t_dw + static_cast<uint32_t>(128 * (a.hi - l));
                        const uint64_t dh = sw128_desc(ht_a), dd = sw128_desc(dt_a);
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {
                            const uint32_t ko = kk * 32u;
                            const uint64_t ah = desc_adv(dh, ko), al = desc_adv(dh, kHt + ko);
                            const uint64_t bh = desc_adv(dd, ko), bl = desc_adv(dd, kDt + ko);
                            mma_bf16(acc, ah, bh, id_dw, 1u);
                            mma_bf16(acc, ah, bl, id_dw, 1u);
                            mma_bf16(acc, al, bh, id_dw, 1u);
                        }
                    }
                    // D_{l-1}^T = W_l^T D_l^T: panels (hi, K 0-63), (hi, K 64-127),
                    // (lo, K 0-63), (lo, K 64-127)
                    for (int pn = 0; pn < 4; ++pn, ++g) {
                        const int slot = static_cast<int>(g % kRing);
                        wait_or_abort(&full[slot], (g / kRing) & 1u, abort_flag, a.status);
                        tc_fence_after();
                        const uint32_t wa = ring_a + static_cast<uint32_t>(slot) * kPanel;
                        const uint64_t dwa = sw128_desc(wa);
                        const uint64_t dmn = sw128_desc_lbo(dt_a, kMnLbo, 1024u);
#pragma unroll
                        for (int k4 = 0; k4 < 4; ++k4) {
                            const int kk = (pn & 1) * 4 + k4;
                            const uint64_t aw = desc_adv(dwa, k4 * 32u);
                            const uint64_t bh = desc_adv(dmn, kk * 2048u);
                            if (pn < 2) {
                                const uint64_t bl = desc_adv(dmn, kDt + kk * 2048u);
                                mma_bf16(t_dl, aw, bh, id_dl, (pn == 0 && k4 == 0) ? 0u : 1u);
                                mma_bf16(t_dl, aw, bl, id_dl, 1u);
                            } else {
                                mma_bf16(t_dl, aw, bh, id_dl, 1u);
                            }
                        }
                        mma_commit(&empty[slot]);
                    }
                    mma_commit(&accb[wg]);
                }
                if (mma_warp) __syncwarp();
                // in flight during the MMAs and the epilogue: the next layer's
                // activations, or the next round's inputs after the last layer
                if (l - 1 >= a.dlo) {
                    load_col(a.acts + static_cast<size_t>(l - 2) * a.act_stride, ti, h);
                } else {
                    load_col(a.acts + static_cast<size_t>(a.nh) * a.act_stride, tn, h);
                    load_g(tn, gpre);
                }
                wait_or_abort(&accb[wg], phase, abort_flag, a.status);
                phase ^= 1u;
                tc_fence_after();
                // epilogue: D_{l-1}^T row u = mask * (W_l^T D_l^T) row u
                dsum = 0.f;
#pragma unroll
                for (int qt = 0; qt < 4; ++qt) {
                    float t[16];
                    tmem_ld16(t_dl + lane_off + static_cast<uint32_t>(16 * qt), t);
#pragma unroll
                    for (int r = 0; r < 16; ++r) {
                        t[r] = ((mask >> (16 * qt + r)) & 1ull) ? t[r] : 0.f;
                        dsum += t[r];
                    }
                    if (l - 1 == 0) write_d0_q(t, qt, ti);
                    if (l - 1 >= a.dlo || a.last_pass) write_dt_q(t, qt);
                }
#pragma unroll
                for (int i = 1; i < 8; ++i)
                    if (i == l - 1 && i >= a.lo && i <= a.hi) db_acc[i] += dsum;
                tc_fence_before();
            }

            // ---- layer 0: the gamma(mean) part of dW_0 and per-tile sums of D_0
            if (a.last_pass) {
                if (ti.tv) a.tilesum[static_cast<size_t>(ti.tile) * WRF_HIDDEN + u] = dsum;
                fence_async_smem();
                tc_fence_before();
                named_bar(2 + wg, 128);
                if (leader) {
                    for (int w2 = 0; w2 < kWG; ++w2, ++g) {
                        const int slot = static_cast<int>(g % kRing);
                        wait_or_abort(&full[slot], (g / kRing) & 1u, abort_flag, a.status);
                        if (w2 != wg) {
                            mbar_arrive(&empty[slot]);  // the other warpgroup's tile
                            continue;
                        }
                        tc_fence_after();
                        const uint32_t ga = ring_a + static_cast<uint32_t>(slot) * kPanel;
                        const uint64_t dd = sw128_desc(dt_a), dg = sw128_desc_lbo(ga, kMnLbo, 1024u);
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {
                            const uint64_t ah = desc_adv(dd, kk * 32u), al = desc_adv(dd, kDt + kk * 32u);
                            const uint64_t bh = desc_adv(dg, kk * 2048u);
                            const uint64_t bl = desc_adv(dg, kGt + kk * 2048u);
                            mma_bf16(t_dl, ah, bh, id_dl, kk == 0 ? 0u : 1u);
                            mma_bf16(t_dl, ah, bl, id_dl, 1u);
                            mma_bf16(t_dl, al, bh, id_dl, 1u);
                        }
                        mma_commit(&empty[slot]);
                    }
                    mma_commit(&accb[wg]);
                }
                if (mma_warp) __syncwarp();
                wait_or_abort(&accb[wg], phase, abort_flag, a.status);
                phase ^= 1u;
                tc_fence_after();
#pragma unroll
                for (int qt = 0; qt < 2; ++qt) {
                    float t[16];
                    tmem_ld16(t_dl + lane_off + static_cast<uint32_t>(16 * qt), t);
#pragma unroll
                    for (int f = 0; f < 16; ++f) gacc[16 * qt + f] += t[f];
                }
                if (a.dm > 32) {
                    float *pw =
                        a.pdw0 + (static_cast<size_t>(blockIdx.x) * kWG + wg) * kGammaF * 128;
                    for (int qt = 2; qt < 4; ++qt) {
                        float t[16];
                        tmem_ld16(t_dl + lane_off + static_cast<uint32_t>(16 * qt), t);
                        if (!*abort_flag) {
#pragma unroll
                            for (int f = 0; f < 16; ++f)
                                if (16 * qt + f < a.dm) pw[(16 * qt + f) * 128 + u] += t[f];
                        }
                    }
                }
                tc_fence_before();
            }
            named_bar(2 + wg, 128);  // tiles and TMEM columns are free for the next round
            // Every kFlush rounds both warpgroups meet: the dW accumulators are
            // added into the CTA's partial, and a timed-out wait anywhere (after
            // which every wait returns at once) ends the loop for all threads
            // together.
            if ((round + 1) % kFlush == 0 || round + 1 == rounds) {
                // every MMA into the dW accumulators is complete past this point
                const bool stop = wg_bar_any(1, *abort_flag != 0, kWG * 128);
                tc_fence_after();
                if (!stop && have_dw) flush_dw();
                tc_fence_before();
                named_bar(1, kWG * 128);
                tc_fence_after();
                if (stop) break;
            }
        }
        // per-thread sums of this warpgroup
        if (!*abort_flag) {
            const size_t cw = static_cast<size_t>(blockIdx.x) * kWG + wg;
#pragma unroll
            for (int l = 1; l < 8; ++l)
                if (l >= a.lo && l <= a.hi) a.pdb[(cw * 8 + l) * 128 + u] += db_acc[l];
            if (a.first_pass) {
                for (int o = 0; o < WRF_OUT; ++o) a.pdwo[(cw * 8 + o) * 128 + u] += dwo[o];
                if (u < WRF_OUT) a.pdwo[(cw * 8 + 5) * 128 + u] += dbo;
            }
            if (a.last_pass) {
                float *pw = a.pdw0 + cw * kGammaF * 128;
#pragma unroll
                for (int f = 0; f < 32; ++f)
                    if (f < a.dm) pw[f * 128 + u] += gacc[f];
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem_base, kTmemCols);
    }
}

// ------------------------------------------------------------ preparation
// Jobs in one launch: [0, nb_w) W^T panels of the hidden layers (element
// grid-stride), then one thread per gamma(mean) row (BF16 hi and lo images,
// pre-swizzled for the MN-major B operand: 8-row groups of 1024 bytes,
// 16-byte chunks XOR row % 8), then one thread per query for gamma(tx) in FP32.
__global__ void __launch_bounds__(128) bwd_prep_kernel(SceneView s, MlpView m, GridView g,
                                                       const float *tx, int Q, int nb_w,
                                                       int nb_g, uint8_t *wimg, uint8_t *gimg,
                                                       long long gterm, int npad, float *gam_t) {
    int b = blockIdx.x;
    if (b < nb_w) {
        const long long total = static_cast<long long>(m.n_layers - 2) * 4 * 128 * 64;
        for (long long i = b * 128LL + threadIdx.x; i < total; i += 128LL * nb_w) {
            const int l = static_cast<int>(i / (4 * 128 * 64));  // hidden layer l+1
            const int pn = static_cast<int>((i / (128 * 64)) % 4);
            const int mrow = static_cast<int>((i / 64) % 128), k = static_cast<int>(i % 64);
            const int o = (pn & 1) * 64 + k;  // W[o][mrow] at (row mrow, K o)
            const float w = m.Wh[l][o * WRF_HIDDEN + mrow];
            uint16_t hi, lo;
            split1(w, hi, lo);
            *reinterpret_cast<uint16_t *>(wimg + (static_cast<size_t>(l) * 4 + pn) * kPanel +
                                          panel_off(mrow, k)) = (pn < 2) ? hi : lo;
        }
        return;
    }
    b -= nb_w;
    if (b < nb_g) {
        const int n = b * 128 + threadIdx.x;
        if (n >= npad) return;
        float gam[kGammaF];
#pragma unroll
        for (int f = 0; f < kGammaF; ++f) gam[f] = 0.f;
        if (n < s.n) {
            const float2 mu = reinterpret_cast<const float2 *>(s.mean)[n];
            const PeArg x[2] = {pe_arg(mu.x, 0.f, static_cast<float>(g.W)),
                                pe_arg(mu.y, 0.f, static_cast<float>(g.H))};
            pe_encode(x, 2, m.L_mean, gam);
        }
        const size_t tbase = static_cast<size_t>(n >> 6) * kGt;
        const int r = n & 63;
        for (int c = 0; c < kGammaF / 8; ++c) {
            uint4 h4, l4;
            split2(gam[8 * c + 0], gam[8 * c + 1], h4.x, l4.x);
            split2(gam[8 * c + 2], gam[8 * c + 3], h4.y, l4.y);
            split2(gam[8 * c + 4], gam[8 * c + 5], h4.z, l4.z);
            split2(gam[8 * c + 6], gam[8 * c + 7], h4.w, l4.w);
            const size_t off =
                tbase + static_cast<size_t>((r >> 3) * 1024 + (r & 7) * 128 + ((c ^ (r & 7)) << 4));
            *reinterpret_cast<uint4 *>(gimg + off) = h4;
            *reinterpret_cast<uint4 *>(gimg + gterm + off) = l4;
        }
        return;
    }
    b -= nb_g;
    const int q = b * 128 + threadIdx.x;
    if (q >= Q) return;
    PeArg x[3];
    for (int c = 0; c < 3; ++c) x[c] = pe_arg(tx[3 * q + c], m.room_min[c], m.room_size[c]);
    pe_encode(x, 3, m.L_tx, gam_t + static_cast<size_t>(q) * m.dt);
}

// ------------------------------------------------------------ reductions
// The caller's gradient arrays, by value (device pointers).
struct GradPtrs {
    float *dW[WRF_MAX_LAYERS];
    float *db[WRF_MAX_LAYERS];
};

// Partials of all CTAs into the caller's gradients, in a fixed order (one
// thread per output element): hidden dW and db of the pass, the output layer
// (first pass) and the gamma(mean) part of dW_0 (last pass).
__global__ void bwd_reduce_kernel(MlpView m, int grid, int lo, int hi, int first, int last,
                                  const float *pdw, const float *pdb, const float *pdwo,
                                  const float *pdw0, GradPtrs gp) {
    float *const *dW = gp.dW;
    float *const *db = gp.db;
    const int nslot = hi >= lo ? hi - lo + 1 : 0;
    const long long n_dw = static_cast<long long>(nslot) * 128 * 128;
    const long long n_db = static_cast<long long>(nslot) * 128;
    const long long n_o = first ? 6 * 128 : 0;
    const long long n_0 = last ? static_cast<long long>(m.dm) * 128 : 0;
    const long long total = n_dw + n_db + n_o + n_0;
    const int din = m.dm + m.dt;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        if (e < n_dw) {
            const int s = static_cast<int>(e / (128 * 128));
            const int oi = static_cast<int>(e % (128 * 128));
            float acc = 0.f;
            for (int c = 0; c < grid; ++c) acc += pdw[(static_cast<size_t>(c) * kSlots + s) * 128 * 128 + oi];
            // the partial holds dW_l^T [128 in][128 out]; W_l is [128 out][128 in]
            dW[hi - s][(oi % 128) * 128 + oi / 128] += acc;
            continue;
        }
        long long f = e - n_dw;
        if (f < n_db) {
            const int l = lo + static_cast<int>(f / 128), uu = static_cast<int>(f % 128);
            float acc = 0.f;
            for (int c = 0; c < grid * kWG; ++c) acc += pdb[(static_cast<size_t>(c) * 8 + l) * 128 + uu];
            db[l][uu] += acc;
            continue;
        }
        f -= n_db;
        if (f < n_o) {
            const int o = static_cast<int>(f / 128), uu = static_cast<int>(f % 128);
            if (o == 5 && uu >= WRF_OUT) continue;
            float acc = 0.f;
            for (int c = 0; c < grid * kWG; ++c) acc += pdwo[(static_cast<size_t>(c) * 8 + o) * 128 + uu];
            const int L = m.n_layers;
            if (o < WRF_OUT)
                dW[L - 1][o * WRF_HIDDEN + uu] += acc;
            else
                db[L - 1][uu] += acc;
            continue;
        }
        f -= n_o;
        {
            const int ft = static_cast<int>(f / 128), uu = static_cast<int>(f % 128);
            float acc = 0.f;
            for (int c = 0; c < grid * kWG; ++c)
                acc += pdw0[(static_cast<size_t>(c) * kGammaF + ft) * 128 + uu];
            dW[0][static_cast<size_t>(uu) * din + ft] += acc;
        }
    }
}

// Per-query sums of D_0 over the query's tiles: colsum[q][u] (fixed order).
__global__ void bwd_colsum_kernel(const float *tilesum, int Qc, int tpq, float *colsum) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Qc * 128) return;
    const int q = i / 128, uu = i % 128;
    float acc = 0.f;
    for (int t = 0; t < tpq; ++t) acc += tilesum[(static_cast<size_t>(q) * tpq + t) * 128 + uu];
    colsum[i] = acc;
}

// The gamma(tx) part of dW_0 (rank one per query) and db_0:
// dW_0[u][dm + f] += sum_q colsum[q][u] gamma(tx_q)[f];  db_0[u] += sum_q colsum[q][u].
__global__ void bwd_tx_part_kernel(MlpView m, int Qc, const float *colsum, const float *gam_t,
                                   float *dW0, float *db0) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int din = m.dm + m.dt;
    if (i >= 128 * (m.dt + 1)) return;
    const int uu = i % 128, f = i / 128;
    float acc = 0.f;
    if (f < m.dt) {
        for (int q = 0; q < Qc; ++q)
            acc = fmaf(colsum[q * 128 + uu], gam_t[static_cast<size_t>(q) * m.dt + f], acc);
        dW0[static_cast<size_t>(uu) * din + m.dm + f] += acc;
    } else {
        for (int q = 0; q < Qc; ++q) acc += colsum[q * 128 + uu];
        db0[uu] += acc;
    }
}

// d_mean[n] += dgamma(mean_n) . d gamma / d (mean / (W, H)) / (W, H), with
// dgamma(mean) = D_0 W_0[:, :dm] for every row of the chunk (FP32, one thread
// per row; W_0's gamma(mean) columns staged in shared memory).
__global__ void __launch_bounds__(128) bwd_dmean_kernel(SceneView s, MlpView m, GridView g,
                                                        int N, long long rows, const float *d0,
                                                        float *d_mean) {
    __shared__ float w0m[62 * WRF_HIDDEN];  // [feature][unit]
    const int din = m.dm + m.dt;
    for (int i = threadIdx.x; i < m.dm * WRF_HIDDEN; i += blockDim.x) {
        const int f = i / WRF_HIDDEN, j = i % WRF_HIDDEN;
        w0m[i] = m.W0[static_cast<size_t>(j) * din + f];
    }
    __syncthreads();
    const long long r = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (r >= rows) return;
    const int n = static_cast<int>(r % N);
    float dg[62];
    for (int f = 0; f < m.dm; ++f) dg[f] = 0.f;
    const float4 *row = reinterpret_cast<const float4 *>(d0 + r * WRF_HIDDEN);
    for (int j4 = 0; j4 < WRF_HIDDEN / 4; ++j4) {
        const float4 v = row[j4];
        for (int f = 0; f < m.dm; ++f) {
            const float *w = w0m + f * WRF_HIDDEN + 4 * j4;
            dg[f] = fmaf(v.x, w[0], fmaf(v.y, w[1], fmaf(v.z, w[2], fmaf(v.w, w[3], dg[f]))));
        }
    }
    const float2 mu = reinterpret_cast<const float2 *>(s.mean)[n];
    const PeArg x[2] = {pe_arg(mu.x, 0.f, static_cast<float>(g.W)),
                        pe_arg(mu.y, 0.f, static_cast<float>(g.H))};
    const int Lm = m.L_mean;
    float gx[2] = {0.f, 0.f};
    for (int f = 0; f < m.dm; ++f) {
        const int i = f % 2, grp = f / 2;
        float dgv = 1.f;
        if (grp >= 1) {
            const int k = (grp - 1) % Lm;
            float sn, cs;
            pe_band(x[i], k, sn, cs);
            const float w = ldexpf(3.14159265358979f, k);
            dgv = grp <= Lm ? w * cs : -w * sn;
        }
        gx[i] = fmaf(dg[f], dgv, gx[i]);
    }
    atomicAdd(d_mean + 2 * n, gx[0] / static_cast<float>(g.W));
    atomicAdd(d_mean + 2 * n + 1, gx[1] / static_cast<float>(g.H));
}

inline size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

// Queries per launch: everything when the forward saved its activations and
// positions are stop-gradded; otherwise chunks whose recomputed activations
// and D_0 rows fit in about 1 GiB.
constexpr size_t kChunkBudget = size_t(1) << 30;
inline int chunk_queries(int n, int Q, int n_layers) {
    const size_t per_q = static_cast<size_t>(n > 0 ? n : 1) * WRF_HIDDEN * 4 * n_layers;
    size_t qc = kChunkBudget / per_q;
    if (qc < 1) qc = 1;
    return static_cast<int>(qc < static_cast<size_t>(Q) ? qc : Q);
}

inline int grid_size() {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

}  // namespace

size_t deform_bwd_ws_layout(int n, int Q, const MlpView &m, DeformWs *fw, DeformBwdWs *bw,
                            char *base) {
    size_t off = align256(deform_ws_layout(n, Q, m.n_layers, fw, base));
    auto take = [&](size_t bytes) {
        char *p = base ? base + off : nullptr;
        off = align256(off + bytes);
        return p;
    };
    DeformBwdWs w{};
    const int nh = m.n_layers - 2 > 0 ? m.n_layers - 2 : 0;
    const int qc = chunk_queries(n, Q > 0 ? Q : 1, m.n_layers);
    const int npad = ((n > 0 ? n : 1) + kR - 1) / kR * kR;
    const size_t grid = kMaxGrid;
    w.wimg = take(static_cast<size_t>(nh > 0 ? nh : 1) * 4 * kPanel);
    w.gterm = static_cast<long long>(npad) * 128;
    w.gimg = take(2 * static_cast<size_t>(w.gterm));
    w.gam_t = reinterpret_cast<float *>(take(static_cast<size_t>(Q > 0 ? Q : 1) * m.dt * 4));
    w.pdw = reinterpret_cast<float *>(take(grid * kSlots * 128 * 128 * 4));
    w.pdb = reinterpret_cast<float *>(take(grid * kWG * 8 * 128 * 4));
    w.pdwo = reinterpret_cast<float *>(take(grid * kWG * 8 * 128 * 4));
    w.pdw0 = reinterpret_cast<float *>(take(grid * kWG * kGammaF * 128 * 4));
    const size_t tpq = static_cast<size_t>(npad / kR);
    const size_t qall = static_cast<size_t>(Q > 0 ? Q : 1);
    w.tilesum = reinterpret_cast<float *>(take(qall * tpq * 128 * 4));
    w.colsum = reinterpret_cast<float *>(take(qall * 128 * 4));
    const size_t chunk_rows = static_cast<size_t>(qc) * (n > 0 ? n : 1);
    w.acts = reinterpret_cast<float *>(
        take(static_cast<size_t>(m.n_layers - 1) * chunk_rows * WRF_HIDDEN * 4));
    w.resid = reinterpret_cast<float *>(take(chunk_rows * WRF_OUT * 4));
    w.d0 = reinterpret_cast<float *>(take(chunk_rows * WRF_HIDDEN * 4));
    w.qc = qc;
    if (bw) *bw = w;
    return off;
}

cudaError_t launch_mlp_bwd(const SceneView &s, const MlpView &m, const GridView &g,
                           const float *tx, int Q, const DeformWs &fw, const DeformBwdWs &bw,
                           const float *d_resid, const float *acts, float *const *dW,
                           float *const *db, float *d_mean, int stop_grad_mean, int *status,
                           cudaStream_t st) {
    const int L = m.n_layers, nh = L - 2;
    const int din = m.dm + m.dt;
    for (int l = 0; l < L; ++l) {
        const int dout = l == L - 1 ? WRF_OUT : WRF_HIDDEN;
        const int dinl = l == 0 ? din : WRF_HIDDEN;
        cudaError_t e = cudaMemsetAsync(dW[l], 0, static_cast<size_t>(dout) * dinl * 4, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(db[l], 0, static_cast<size_t>(dout) * 4, st);
        if (e != cudaSuccess) return e;
    }
    const long long rows = static_cast<long long>(Q) * s.n;
    if (rows == 0) return cudaGetLastError();
    if (m.dm > kGammaF || m.dm > 62) return cudaErrorInvalidValue;
    const int N = s.n;
    const int npad = (N + kR - 1) / kR * kR;
    {
        const int nb_w = nh > 0 ? 256 : 0;
        const int nb_g = (npad + 127) / 128;
        const int nb_t = (Q + 127) / 128;
        bwd_prep_kernel<<<nb_w + nb_g + nb_t, 128, 0, st>>>(
            s, m, g, tx, Q, nb_w, nb_g, reinterpret_cast<uint8_t *>(bw.wimg),
            reinterpret_cast<uint8_t *>(bw.gimg), bw.gterm, npad, bw.gam_t);
    }
    cudaError_t e = cudaFuncSetAttribute(mlp_bwd_tc_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem_bytes()));
    if (e != cudaSuccess) return e;
    int sms = grid_size();
    if (sms > kMaxGrid) sms = kMaxGrid;
    GradPtrs gp{};
    for (int l = 0; l < L; ++l) {
        gp.dW[l] = dW[l];
        gp.db[l] = db[l];
    }
    const int tpq = npad / kR;
    // passes of at most kSlots weight-gradient layers, from the top
    int npass = nh > 0 ? (nh + kSlots - 1) / kSlots : 1;
    // queries per launch
    const bool need_chunks = !acts || !stop_grad_mean;
    const int qc = need_chunks ? bw.qc : Q;
    const size_t pdw_bytes = static_cast<size_t>(kMaxGrid) * kSlots * 128 * 128 * 4;
    const size_t small_bytes = static_cast<size_t>(kMaxGrid) * kWG * 8 * 128 * 4;
    const size_t pdw0_bytes = static_cast<size_t>(kMaxGrid) * kWG * kGammaF * 128 * 4;
    for (int q0 = 0; q0 < Q; q0 += qc) {
        const int Qc = Q - q0 < qc ? Q - q0 : qc;
        const long long crows = static_cast<long long>(Qc) * N;
        const float *cacts = acts ? acts + static_cast<size_t>(q0) * N * WRF_HIDDEN : bw.acts;
        const long long astride = acts ? rows * WRF_HIDDEN : crows * WRF_HIDDEN;
        if (!acts) {
            // recompute this chunk's hidden activations with the FP32 forward
            DeformWs cw = fw;
            cw.V = fw.V + static_cast<size_t>(q0) * WRF_HIDDEN;
            e = launch_mlp_f32(s, m, g, Qc, cw, 0, bw.resid, nullptr, nullptr, bw.acts, st);
            if (e != cudaSuccess) return e;
        }
        const int ntiles = Qc * tpq;
        const int npairs = (ntiles + 1) / 2;
        const int grid = npairs < sms ? npairs : sms;
        for (int pass = 0; pass < npass; ++pass) {
            BwdArgs a{};
            a.N = N;
            a.Qc = Qc;
            a.tpq = tpq;
            a.ntiles = ntiles;
            a.npairs = npairs;
            a.nh = nh;
            a.hi = nh - pass * kSlots;
            a.lo = a.hi - kSlots + 1 > 1 ? a.hi - kSlots + 1 : 1;
            if (nh == 0) {
                a.hi = 0;
                a.lo = 1;
            }
            a.first_pass = pass == 0;
            a.last_pass = pass == npass - 1;
            a.dlo = a.last_pass ? 1 : a.lo;
            a.dm = m.dm;
            a.acts = cacts;
            a.act_stride = astride;
            a.dres = d_resid + static_cast<size_t>(q0) * N * WRF_OUT;
            a.Wo = m.Wo;
            a.wimg = reinterpret_cast<const uint8_t *>(bw.wimg);
            a.gimg = reinterpret_cast<const uint8_t *>(bw.gimg);
            a.gterm = bw.gterm;
            a.pdw = bw.pdw;
            a.pdb = bw.pdb;
            a.pdwo = bw.pdwo;
            a.pdw0 = bw.pdw0;
            a.tilesum = bw.tilesum;
            a.d0 = (!stop_grad_mean && a.last_pass) ? bw.d0 : nullptr;
            a.status = status;
            if ((e = cudaMemsetAsync(bw.pdw, 0, pdw_bytes, st)) != cudaSuccess) return e;
            if ((e = cudaMemsetAsync(bw.pdb, 0, small_bytes, st)) != cudaSuccess) return e;
            if ((e = cudaMemsetAsync(bw.pdwo, 0, small_bytes, st)) != cudaSuccess) return e;
            if ((e = cudaMemsetAsync(bw.pdw0, 0, pdw0_bytes, st)) != cudaSuccess) return e;
            mlp_bwd_tc_kernel<<<grid, kThreads, smem_bytes(), st>>>(a);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            bwd_reduce_kernel<<<256, 256, 0, st>>>(m, grid, a.lo, a.hi, a.first_pass, a.last_pass,
                                                   bw.pdw, bw.pdb, bw.pdwo, bw.pdw0, gp);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        bwd_colsum_kernel<<<(Qc * 128 + 255) / 256, 256, 0, st>>>(bw.tilesum, Qc, tpq, bw.colsum);
        bwd_tx_part_kernel<<<(128 * (m.dt + 1) + 255) / 256, 256, 0, st>>>(
            m, Qc, bw.colsum, bw.gam_t + static_cast<size_t>(q0) * m.dt, dW[0], db[0]);
        if (!stop_grad_mean)
            bwd_dmean_kernel<<<static_cast<unsigned>((crows + 127) / 128), 128, 0, st>>>(
                s, m, g, N, crows, bw.d0, d_mean);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

}  // namespace wrf
