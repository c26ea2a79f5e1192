// The paper's deformation network (Sec. 4.2, Sec. 6.1) on the 5th-generation
// tensor cores: BF16 operands, FP32 accumulation in tensor memory.
//
// Rows are (query, Gaussian) pairs; a tile is 128 consecutive Gaussians of
// one query (TMEM lane = row).  A CTA runs two compute warpgroups, each with
// its own tile, and one producer warp.  Per tile the A operand lives in
// shared memory as 128 rows x 224 K columns (BF16, K-major, 128-byte
// swizzle, four 64-column panels):
//   K 0..159    the previous layer's activations (width <= 160, zero-padded),
//               rewritten by every epilogue;
//   K 160..223  gamma(mean_n) of Eq. 15 (42 values, zero-padded), written once
//               per tile: the encoding part that depends on the Gaussian.
// Layer l runs over the K range its input holds: layer 0 K 160..223 (the
// encoding alone), a skip layer K 0..223 (activations and encoding),
// another hidden layer K 0..159.  The encoding part that depends on the
// query, W_s gamma(s_q), is the same for the 128 rows of a tile: it is
// computed once per query in FP32 together with the bias (vec[q][l]) and
// added, like the bias of the other layers, by the tensor core: each layer
// starts with one K = 16 MMA of a selector A (ones in K columns 0 and 1) by
// a per-warpgroup B image holding the layer's term as BF16 hi + lo, written
// by the previous epilogue.  N = 160 output columns per MMA (M = 128, K = 16
// per instruction).
//
// The hidden weights (up to 4 panels of 160 rows x 64 K per layer, 20 KB
// each, 26 panels for the paper's network) do not fit in shared memory
// together, so the producer warp streams them with bulk copies through a
// ring of four panel slots, in the order the layers consume them; both
// warpgroups consume every panel (their tiles are at most four panels
// apart), and a slot is refilled once the MMAs of both have completed
// (tcgen05.commit to the slot's empty barrier, arrival count 2).  Every
// epilogue reads its row's 160 accumulators from TMEM, applies ReLU and
// rounds to BF16 into the A tile (and writes the next layer's term image).
// The output layer (N = 16, 5 used, bias by the same selector MMA) runs on
// resident weights; its epilogue projects the Gaussian into its two-channel
// record.
// Every wait is bounded (WRF_ETIMEOUT on the status word).
#include <cuda_bf16.h>

#include "kernels.h"
#include "paper.cuh"
#include "tc.cuh"

namespace wrf {

namespace {

constexpr int kPW = kPaperMaxWidth;          // 160
constexpr int kTile = 128;
constexpr int kWGs = 2;
constexpr int kTcThreads = kWGs * 128 + 32;  // + producer warp
constexpr uint32_t kAPanel = 128 * 128;      // 128 rows x 64 K x BF16
constexpr uint32_t kATile = 4 * kAPanel;
constexpr uint32_t kBPanel = kPW * 128;      // 160 rows x 64 K x BF16
constexpr int kRing = 4;
constexpr uint32_t kOutPanel = 16 * 128;     // 16 rows x 64 K x BF16
constexpr uint32_t kOutImg = 3 * kOutPanel;  // K 0..191 (0..159 used)
constexpr int kGammaK0 = 160;
constexpr int kGammaCols = 64;
constexpr uint32_t kTmemCols = 512;          // two accumulators of 160 columns, at 0 and 256
constexpr uint32_t kTermImg = kPW * 16;      // per-layer term image: 160 rows x 16 B (hi, lo)
constexpr uint32_t kSelImg = 256;            // selector: two 8 x 16 B core matrices

constexpr size_t tc_smem_bytes() {
    return 1024 + kWGs * kATile + kRing * kBPanel + kOutImg + kWGs * kTermImg + kSelImg +
           (2 * kRing + kWGs + 1) * 8 + 16;
}
static_assert(tc_smem_bytes() <= 227 * 1024, "shared memory of one CTA");

// K range of layer l's input in A-tile columns.
__host__ __device__ inline int k_begin(int l) { return l == 0 ? kGammaK0 : 0; }
__host__ __device__ inline int k_end(int l) {
    return (l == 0 || is_skip(l)) ? kGammaK0 + kGammaCols : kPW;
}
__host__ __device__ inline int panels_of(int l) { return (k_end(l) - 1) / 64 - k_begin(l) / 64 + 1; }
__host__ __device__ inline int seq_len(int nh) {
    int s = 0;
    for (int l = 0; l < nh; ++l) s += panels_of(l);
    return s;
}

// Byte offset of element (row r, column k < 64) in a 128-byte-swizzled
// K-major panel (8-row groups of 1024 bytes, 16-byte chunks XOR row % 8).
__host__ __device__ inline uint32_t sw128_off(int r, int k) {
    return static_cast<uint32_t>((r >> 3) * 1024 + (r & 7) * 128 + ((((k >> 3) ^ (r & 7))) << 4) +
                                 (k & 7) * 2);
}

struct PaperNetTc {
    int n_hidden, width, dm, dt, L_mean, L_tx;
    float room_min[3], room_size[3];
    const float *W[kPaperMaxLayers], *b[kPaperMaxLayers];
};

// W_l's input index for A-tile column k (-1: no weight there).
__device__ inline int input_index(const PaperNetTc &m, int l, int k) {
    if (l == 0) return (k >= kGammaK0 && k - kGammaK0 < m.dm) ? k - kGammaK0 : -1;
    if (k < kPW) return k < m.width ? k : -1;
    if (is_skip(l) && k - kGammaK0 < m.dm) return m.width + (k - kGammaK0);
    return -1;
}
__device__ inline int in_dim_tc(const PaperNetTc &m, int l) {
    return (l == 0 ? 0 : m.width) + (l == 0 || is_skip(l) ? m.dm + m.dt : 0);
}

// BF16 panels of every hidden layer in consumption order, and the output
// layer's three panels (rows = output units, K-major, 128-byte swizzle).
__global__ void paper_tc_weights_kernel(PaperNetTc m, int nseq, uint16_t *wimg, uint16_t *oimg) {
    const long long per = static_cast<long long>(kPW) * 64;
    const long long total = nseq * per + 3LL * 16 * 64;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        if (i < nseq * per) {
            const int s = static_cast<int>(i / per);
            const int r = static_cast<int>((i % per) / 64), kl = static_cast<int>(i % 64);
            int l = 0, p = 0, acc = 0;
            for (l = 0; l < m.n_hidden; ++l) {
                const int np = panels_of(l);
                if (s < acc + np) {
                    p = k_begin(l) / 64 + (s - acc);
                    break;
                }
                acc += np;
            }
            const int k = 64 * p + kl;
            float v = 0.f;
            if (k >= k_begin(l) && k < k_end(l) && r < m.width) {
                const int j = input_index(m, l, k);
                if (j >= 0) v = m.W[l][static_cast<size_t>(r) * in_dim_tc(m, l) + j];
            }
            const __nv_bfloat16 bv = __float2bfloat16_rn(v);
            wimg[(static_cast<size_t>(s) * kBPanel + sw128_off(r, kl)) / 2] =
                *reinterpret_cast<const uint16_t *>(&bv);
        } else {
            const long long e = i - nseq * per;
            const int p = static_cast<int>(e / (16 * 64));
            const int r = static_cast<int>((e % (16 * 64)) / 64), kl = static_cast<int>(e % 64);
            const int k = 64 * p + kl;
            const float v = (r < WRF_OUT && k < m.width)
                                ? m.W[m.n_hidden][static_cast<size_t>(r) * m.width + k]
                                : 0.f;
            const __nv_bfloat16 bv = __float2bfloat16_rn(v);
            oimg[(static_cast<size_t>(p) * kOutPanel + sw128_off(r, kl)) / 2] =
                *reinterpret_cast<const uint16_t *>(&bv);
        }
    }
}

// gamma(mean_n) rows [N][64] BF16 (42 values of Eq. 15 at L_mean = 10, zeros
// after them): the encoding input on the unit square (tanh u + 1) / 2.
__global__ void paper_tc_gamma_kernel(PaperView s, int L_mean, int dm, uint16_t *G) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= s.n) return;
    const float2 mu = reinterpret_cast<const float2 *>(s.mu)[n];
    const PeArg a[2] = {unit_centre(mu.x), unit_centre(mu.y)};
    float gam[2 * (2 * 15 + 1)];
    encode_vec(a, 2, L_mean, gam);
    uint32_t *dst = reinterpret_cast<uint32_t *>(G + static_cast<size_t>(n) * kGammaCols);
    for (int i = 0; i < kGammaCols / 2; ++i) {
        const float x0 = 2 * i < dm ? gam[2 * i] : 0.f;
        const float x1 = 2 * i + 1 < dm ? gam[2 * i + 1] : 0.f;
        dst[i] = pack_bf16(x0, x1);
    }
}

// vec[q][l][j] (FP32): W_s gamma(s_q) + b for the layers whose input holds
// the encoding, b for the others, zero past the width.
__global__ void __launch_bounds__(kPW) paper_tc_vec_kernel(PaperNetTc m, const float *tx, float *vec) {
    __shared__ float gam[3 * (2 * 15 + 1)];
    const int q = blockIdx.x, j = threadIdx.x;
    if (j == 0) {
        PeArg a[3];
        for (int c = 0; c < 3; ++c) a[c] = pe_arg(tx[3 * q + c], m.room_min[c], m.room_size[c]);
        encode_vec(a, 3, m.L_tx, gam);
    }
    __syncthreads();
    for (int l = 0; l < kPaperMaxLayers - 1; ++l) {
        float acc = 0.f;
        if (l < m.n_hidden && j < m.width) {
            if (l == 0 || is_skip(l)) {
                const float *wr = m.W[l] + static_cast<size_t>(j) * in_dim_tc(m, l) +
                                  (l == 0 ? 0 : m.width) + m.dm;
                for (int k = 0; k < m.dt; ++k) acc = fmaf(__ldg(wr + k), gam[k], acc);
            }
            acc += m.b[l][j];
        }
        vec[(static_cast<size_t>(q) * (kPaperMaxLayers - 1) + l) * kPW + j] = acc;
    }
}

struct PaperTcArgs {
    PaperView s;
    GridView g;
    const uint16_t *G, *wimg, *oimg;
    const float *vec, *bout;
    int nh, nseq, Q, N, tpq, ntiles, npairs;
    float4 *rec;
    float *rec_im;
    int *status;
};

__device__ __forceinline__ uint32_t a_chunk_off(int row, int kc) {
    // 16-byte chunk kc (0..27) of A-tile row `row`
    return static_cast<uint32_t>((kc >> 3) * kAPanel + row * 128 + (((kc & 7) ^ (row & 7)) << 4));
}

__global__ void __launch_bounds__(kTcThreads, 1) paper_tc_kernel(PaperTcArgs a) {
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    uint8_t *base = smem_raw + (((raw + 1023u) & ~1023u) - raw);
    uint8_t *atile0 = base;
    uint8_t *ring = base + kWGs * kATile;
    uint8_t *oimg = ring + kRing * kBPanel;
    uint8_t *term0 = oimg + kOutImg;         // [kWGs][160 rows x 16 B]
    uint8_t *sel = term0 + kWGs * kTermImg;   // selector A
    uint64_t *bars = reinterpret_cast<uint64_t *>(sel + kSelImg);
    uint64_t *full = bars, *empty = bars + kRing, *accb = bars + 2 * kRing;
    uint64_t *wbar = bars + 2 * kRing + kWGs;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(wbar + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid < 16) {
        // selector: rows 0..7 of core matrix 0 hold (1, 1, 0 ...) in K 0..7,
        // core matrix 1 (K 8..15) is zero; every 8-row group repeats it
        const uint32_t one2 = 0x3F803F80u;  // BF16 1.0 twice
        reinterpret_cast<uint4 *>(sel)[tid] =
            tid < 8 ? make_uint4(one2, 0u, 0u, 0u) : make_uint4(0u, 0u, 0u, 0u);
    }
    if (tid == 0) {
        for (int i = 0; i < kRing; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], kWGs);
        }
        for (int i = 0; i < kWGs; ++i) mbar_init(&accb[i], 1);
        mbar_init(wbar, 1);
        fence_mbar_init();
        *abort_flag = 0;
    }
    if (warp == 0) tmem_alloc(tmem_slot, kTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == kWGs * 4) {
        // ---------------------------------------------------- producer warp
        if (lane == 0) {
            mbar_arrive_expect_tx(wbar, kOutImg);
            bulk_g2s(oimg, a.oimg, kOutImg, wbar);
            uint32_t g = 0;  // panels issued
            bool ok = true;
            for (int p = blockIdx.x; p < a.npairs && ok; p += gridDim.x) {
                for (int s = 0; s < a.nseq; ++s) {
                    const int slot = static_cast<int>(g % kRing);
                    if (g >= kRing &&
                        !wait_or_abort(&empty[slot], ((g / kRing) - 1) & 1u, abort_flag, a.status)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(&full[slot], kBPanel);
                    bulk_g2s(ring + slot * kBPanel,
                             reinterpret_cast<const uint8_t *>(a.wimg) + static_cast<size_t>(s) * kBPanel,
                             kBPanel, &full[slot]);
                    ++g;
                }
            }
            // the copies still in flight land before the CTA exits (bounded)
            for (uint32_t i = 0; i < kRing && i < g; ++i) {
                const uint32_t gg = g - 1 - i;
                mbar_wait(&full[gg % kRing], (gg / kRing) & 1u, a.status, kWaitLimitNs);
            }
            mbar_wait(wbar, 0, a.status, kWaitLimitNs);
        }
    } else {
        // ---------------------------------------------- compute warpgroups
        const int wg = warp >> 2, wq = warp & 3, wt = tid & 127;
        uint8_t *A = atile0 + wg * kATile;
        const uint32_t a_addr = smem_u32(A), ring_addr = smem_u32(ring), o_addr = smem_u32(oimg);
        const uint32_t t_acc = tmem_base + static_cast<uint32_t>(wg * 256);
        const uint32_t lane_off = static_cast<uint32_t>(wq * 32) << 16;
        const int my_row = wq * 32 + lane;
        const bool leader = wt == 0;
        const uint32_t id_h = idesc_bf16(128, kPW), id_o = idesc_bf16(128, 16);
        uint8_t *term = term0 + wg * kTermImg;
        const uint64_t d_sel = plain_desc(smem_u32(sel), 128u, 0u);
        const uint64_t d_term = plain_desc(smem_u32(term), 0u, 128u);
        // the term image of layer l (vec[q][l], or the output bias when l ==
        // nh): rows wt and 128 + wt as BF16 hi + lo in K columns 0 and 1
        auto write_term = [&](int q, int l) {
            for (int j = wt; j < kPW; j += 128) {
                float v = 0.f;
                if (l < a.nh)
                    v = __ldg(a.vec + (static_cast<size_t>(q) * (kPaperMaxLayers - 1) + l) * kPW + j);
                else if (j < WRF_OUT)
                    v = __ldg(a.bout + j);
                const uint32_t hi = pack_bf16(v, 0.f) & 0xFFFFu;
                const uint32_t lo = pack_bf16(__fsub_rn(v, __uint_as_float(hi << 16)), 0.f) & 0xFFFFu;
                *reinterpret_cast<uint4 *>(term + j * 16) = make_uint4(hi | (lo << 16), 0u, 0u, 0u);
            }
        };
        uint32_t phase = 0, g = 0;
        wait_or_abort(wbar, 0, abort_flag, a.status);
        for (int p = blockIdx.x; p < a.npairs; p += gridDim.x) {
            if (wg_bar_any(1 + wg, *abort_flag != 0)) break;
            const int tile = 2 * p + wg;
            const bool tv = tile < a.ntiles;
            const int q = tv ? tile / a.tpq : 0;
            const int n = tv ? (tile % a.tpq) * kTile + my_row : a.N;
            const bool rv = n < a.N;
            // gamma(mean_n) -> A columns 160..223 (chunks 20..27)
            {
                const uint4 *src = reinterpret_cast<const uint4 *>(
                    a.G + static_cast<size_t>(rv ? n : 0) * kGammaCols);
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const uint4 v = rv ? __ldg(src + c) : make_uint4(0u, 0u, 0u, 0u);
                    *reinterpret_cast<uint4 *>(A + a_chunk_off(my_row, kGammaK0 / 8 + c)) = v;
                }
            }
            write_term(q, 0);
            fence_async_smem();
            named_bar(1 + wg, 128);
            for (int l = 0; l < a.nh; ++l) {
                if (leader) {
                    tc_fence_after();
                    const int kb = k_begin(l), ke = k_end(l);
                    // D = vec[q][l] (hi + lo), then += W_l x
                    mma_bf16(t_acc, d_sel, d_term, id_h, 0u);
                    uint32_t acc_flag = 1u;
                    for (int pn = kb / 64; pn <= (ke - 1) / 64; ++pn, ++g) {
                        const int slot = static_cast<int>(g % kRing);
                        wait_or_abort(&full[slot], (g / kRing) & 1u, abort_flag, a.status);
                        tc_fence_after();
                        const int k0 = kb > pn * 64 ? kb : pn * 64;
                        const int k1 = ke < pn * 64 + 64 ? ke : pn * 64 + 64;
                        const uint32_t b_addr = ring_addr + static_cast<uint32_t>(slot) * kBPanel;
                        for (int k = k0; k < k1; k += 16) {
                            const uint32_t kin = static_cast<uint32_t>((k & 63) >> 4) * 32u;
                            mma_bf16(t_acc, sw128_desc(a_addr + static_cast<uint32_t>(pn) * kAPanel + kin),
                                     sw128_desc(b_addr + kin), id_h, acc_flag);
                            acc_flag = 1u;
                        }
                        mma_commit(&empty[slot]);
                    }
                    mma_commit(&accb[wg]);
                } else {
                    g += static_cast<uint32_t>(panels_of(l));
                }
                wait_or_abort(&accb[wg], phase, abort_flag, a.status);
                phase ^= 1u;
                tc_fence_after();
                write_term(q, l + 1);  // the layer-l MMAs that read the image are complete
#pragma unroll 1
                for (int c = 0; c < kPW / 32; ++c) {
                    float v[32];
                    tmem_ld32(t_acc + lane_off + c * 32, v);
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        uint4 pk;
                        pk.x = pack_bf16_relu(v[8 * j + 0], v[8 * j + 1]);
                        pk.y = pack_bf16_relu(v[8 * j + 2], v[8 * j + 3]);
                        pk.z = pack_bf16_relu(v[8 * j + 4], v[8 * j + 5]);
                        pk.w = pack_bf16_relu(v[8 * j + 6], v[8 * j + 7]);
                        *reinterpret_cast<uint4 *>(A + a_chunk_off(my_row, c * 4 + j)) = pk;
                    }
                }
                tc_fence_before();
                fence_async_smem();
                named_bar(1 + wg, 128);
            }
            // output layer: N = 16 (5 used), K 0..159, resident weights
            if (leader) {
                tc_fence_after();
                mma_bf16(t_acc, d_sel, d_term, id_o, 0u);  // D = output bias (hi + lo)
#pragma unroll
                for (int k = 0; k < kPW; k += 16) {
                    const uint32_t kin = static_cast<uint32_t>((k & 63) >> 4) * 32u;
                    mma_bf16(t_acc, sw128_desc(a_addr + static_cast<uint32_t>(k >> 6) * kAPanel + kin),
                             sw128_desc(o_addr + static_cast<uint32_t>(k >> 6) * kOutPanel + kin), id_o,
                             1u);
                }
                mma_commit(&accb[wg]);
            }
            wait_or_abort(&accb[wg], phase, abort_flag, a.status);
            phase ^= 1u;
            tc_fence_after();
            float o[16];
            tmem_ld16(t_acc + lane_off, o);
            tc_fence_before();
            if (tv && rv && !*abort_flag) {
                float d[5];
#pragma unroll
                for (int i = 0; i < WRF_OUT; ++i) d[i] = o[i];
                paper_project(a.s, n, q, d, a.g, a.rec, a.rec_im);
            }
            named_bar(1 + wg, 128);  // TMEM columns and the A tile are free again
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

size_t paper_tc_image_bytes(int n_hidden) {
    return static_cast<size_t>(seq_len(n_hidden)) * kBPanel + kOutImg;
}

cudaError_t launch_paper_tc(const PaperSceneView &sv, const PaperMlpView &mv, const GridView &g,
                            const float *tx, int Q, const PaperWs &ws, float4 *rec, int *status,
                            cudaStream_t st) {
    const long long rows = static_cast<long long>(Q) * sv.n;
    if (rows == 0) return cudaSuccess;
    PaperNetTc m{};
    m.n_hidden = mv.n_hidden;
    m.width = mv.width;
    m.L_mean = mv.L_mean;
    m.L_tx = mv.L_tx;
    m.dm = 2 * (2 * mv.L_mean + 1);
    m.dt = 3 * (2 * mv.L_tx + 1);
    if (m.dm > kGammaCols) return cudaErrorInvalidValue;
    for (int i = 0; i < 3; ++i) {
        m.room_min[i] = mv.room_min[i];
        m.room_size[i] = mv.room_size[i];
    }
    for (int l = 0; l <= mv.n_hidden; ++l) {
        m.W[l] = mv.W[l];
        m.b[l] = mv.b[l];
    }
    PaperView s{sv.n, sv.mu, sv.chol, sv.attn_logit, sv.psi};
    const int nseq = seq_len(m.n_hidden);
    uint16_t *wimg = ws.img;
    uint16_t *oimg = ws.img + static_cast<size_t>(nseq) * kBPanel / 2;
    paper_tc_weights_kernel<<<148 * 2, 256, 0, st>>>(m, nseq, wimg, oimg);
    paper_tc_gamma_kernel<<<(sv.n + 127) / 128, 128, 0, st>>>(s, m.L_mean, m.dm, ws.G);
    paper_tc_vec_kernel<<<Q, kPW, 0, st>>>(m, tx, ws.vec);
    PaperTcArgs a{};
    a.s = s;
    a.g = g;
    a.G = ws.G;
    a.wimg = wimg;
    a.oimg = oimg;
    a.vec = ws.vec;
    a.bout = mv.b[mv.n_hidden];
    a.nh = m.n_hidden;
    a.nseq = nseq;
    a.Q = Q;
    a.N = sv.n;
    a.tpq = (sv.n + kTile - 1) / kTile;
    const long long nt = static_cast<long long>(a.tpq) * Q;
    if (nt >= (1ll << 30)) return cudaErrorInvalidValue;
    a.ntiles = static_cast<int>(nt);
    a.npairs = (a.ntiles + 1) / 2;
    a.rec = rec;
    a.rec_im = reinterpret_cast<float *>(rec + 2 * rows);
    a.status = status;
    const size_t smem = tc_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(paper_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = a.npairs < sms ? a.npairs : sms;
    paper_tc_kernel<<<grid, kTcThreads, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace wrf
