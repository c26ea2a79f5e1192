// The paper's deformation network (Sec. 4.2, Sec. 6.1) on the 5th-generation
// tensor cores: BF16 operands, FP32 accumulation in tensor memory.
//
// Rows are (query, Gaussian) pairs; a tile is 128 consecutive Gaussians of
// one query (TMEM lane = row).  A CTA runs two compute groups of eight warps,
// each group with its own tile (the two warps of a TMEM lane quarter split
// the 160 columns of every epilogue), and one producer warp.
//
// A layer's input is split in two operands:
//   * the previous layer's activations (K 0..159, width <= 160 zero-padded)
//     stay in tensor memory as BF16 pairs (lane = row, column j = elements
//     2j, 2j+1): each epilogue reads the FP32 accumulator, applies ReLU,
//     rounds to BF16 and writes the pairs back (tcgen05.st), where the next
//     layer's MMAs read their A operand;
//   * gamma(mean_n) of Eq. 15 (42 values, zero-padded to 64) sits in shared
//     memory (one 128-byte-swizzled 128 x 64 panel per tile, written once per
//     tile): the encoding part that depends on the Gaussian, read by layer 0
//     and by the skip layers.
// The encoding part that depends on the query, W_s gamma(s_q), is the same
// for the 128 rows of a tile: it is computed once per query in FP32 together
// with the bias (vec[q][l]) and added, like the bias of the other layers, by
// the tensor core: each layer starts with one K = 16 MMA of a selector A
// (ones in K columns 0 and 1) by a per-group B image holding the layer's term
// as BF16 hi + lo, written by the previous epilogue.  N = 160 output columns
// per MMA (M = 128, K = 16 per instruction).
//
// The weights arrive as 160-row x 64-K panels (20 KB, 128-byte swizzle):
// activations K 0..63, 64..127, 128..159 (half used) and the gamma(mean)
// block, 25 panels for the paper's network in the order the layers consume
// them.  They do not fit in shared memory together, so the producer warp
// streams them with bulk copies through a ring of nine slots (two layers and
// more); both groups consume every panel, a slot is refilled once the MMAs of
// both have completed (tcgen05.commit to the slot's empty barrier, arrival
// count 2), and the ring is deep enough for one group to run a layer ahead of
// the other, so one group's epilogue overlaps the other's MMAs.  The output
// layer (N = 16, 5 used, bias by the same selector MMA) runs on resident
// weights; its epilogue projects the Gaussian into its two-channel record.
// Every wait is bounded (WRF_ETIMEOUT on the status word).
#include <cuda_bf16.h>

#include "kernels.h"
#include "paper.cuh"
#include "tc.cuh"

namespace wrf {

namespace {

constexpr int kPW = kPaperMaxWidth;          // 160
constexpr int kTile = 128;
constexpr int kGroup = 256;                  // threads per compute group (8 warps)
constexpr uint32_t kGPanel = 128 * 128;      // gamma(mean) A panel: 128 rows x 64 K x BF16
constexpr uint32_t kBPanel = kPW * 128;      // weight panel: 160 rows x 64 K x BF16
constexpr uint32_t kOutPanel = 16 * 128;     // 16 rows x 64 K x BF16
constexpr uint32_t kOutImg = 3 * kOutPanel;  // K 0..191 (0..159 used)
constexpr int kGammaCols = 64;
constexpr int kGammaPanel = 3;               // panel id of the gamma(mean) block
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kTermImg = kPW * 16;      // per-layer term image: 160 rows x 16 B (hi, lo)
constexpr uint32_t kSelImg = 256;            // selector: two 8 x 16 B core matrices

// Precision X: 1 = BF16 operands; 3 = every FP32 operand (weights,
// activations, gamma(mean)) as BF16 hi + lo and each product as the three
// BF16 products hi hi + hi lo + lo hi.
//   X = 1: two compute groups (two tiles per CTA); TMEM: accumulators at 0
//          and 256 (160 columns each), BF16 activation pairs (80 columns) at
//          160 and 416; a ring of nine weight panels.
//   X = 3: one compute group; TMEM: accumulator at 0 (160 columns),
//          activation hi pairs at 160, lo pairs at 240; every weight panel
//          comes as a hi and a lo panel; a ring of eight panels.
template <int X>
struct TcCfg {
    static constexpr int WGs = X == 3 ? 1 : 2;
    static constexpr int Terms = X == 3 ? 2 : 1;
    static constexpr int Threads = WGs * kGroup + 32;  // + producer warp
    static constexpr int Ring = X == 3 ? 8 : 9;
    static constexpr size_t smem = 1024 + WGs * Terms * kGPanel + Ring * kBPanel +
                                   Terms * kOutImg + WGs * kTermImg + kSelImg +
                                   (2 * Ring + WGs + 1) * 8 + 16;
};
static_assert(TcCfg<1>::smem <= 227 * 1024, "shared memory of one CTA");
static_assert(TcCfg<3>::smem <= 227 * 1024, "shared memory of one CTA");

// Panels layer l consumes, in order: activation panels 0, 1, 2 (l >= 1), then
// the gamma(mean) panel (layer 0 and the skip layers).
__host__ __device__ inline int panels_of(int l) {
    return (l == 0 ? 0 : 3) + ((l == 0 || is_skip(l)) ? 1 : 0);
}
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

// W_l's input index for column k of panel pid (-1: no weight there).
__device__ inline int input_index(const PaperNetTc &m, int l, int pid, int k) {
    if (pid == kGammaPanel) {
        if (k >= m.dm) return -1;
        return l == 0 ? k : m.width + k;
    }
    const int j = 64 * pid + k;
    return j < m.width ? j : -1;
}
__device__ inline int in_dim_tc(const PaperNetTc &m, int l) {
    return (l == 0 ? 0 : m.width) + (l == 0 || is_skip(l) ? m.dm + m.dt : 0);
}

// BF16 panels of every hidden layer in consumption order, and the output
// layer's three panels (rows = output units, K-major, 128-byte swizzle).
// terms = 2: panel s of the sequence becomes physical panels 2s (hi) and
// 2s + 1 (lo = BF16 of the remainder), the output image its three hi panels
// then its three lo panels.
__device__ __forceinline__ void store_terms(uint16_t *img, size_t hi_index, size_t lo_index,
                                            float v, int terms) {
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    img[hi_index] = *reinterpret_cast<const uint16_t *>(&h);
    if (terms == 2) {
        const __nv_bfloat16 l = __float2bfloat16_rn(__fsub_rn(v, __bfloat162float(h)));
        img[lo_index] = *reinterpret_cast<const uint16_t *>(&l);
    }
}

__device__ __forceinline__ void paper_tc_weights_block(int blk, int nblk, const PaperNetTc &m,
                                                       int nseq, uint16_t *wimg, uint16_t *oimg,
                                                       int terms) {
    const long long per = static_cast<long long>(kPW) * 64;
    const long long total = nseq * per + 3LL * 16 * 64;
    for (long long i = blk * static_cast<long long>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<long long>(nblk) * blockDim.x) {
        if (i < nseq * per) {
            const int s = static_cast<int>(i / per);
            const int r = static_cast<int>((i % per) / 64), kl = static_cast<int>(i % 64);
            int l = 0, pid = 0, acc = 0;
            for (l = 0; l < m.n_hidden; ++l) {
                const int np = panels_of(l);
                if (s < acc + np) {
                    const int idx = s - acc;
                    pid = (l == 0 || idx == 3) ? kGammaPanel : idx;
                    break;
                }
                acc += np;
            }
            float v = 0.f;
            if (r < m.width) {
                const int j = input_index(m, l, pid, kl);
                if (j >= 0) v = m.W[l][static_cast<size_t>(r) * in_dim_tc(m, l) + j];
            }
            const size_t o = sw128_off(r, kl) / 2;
            store_terms(wimg, static_cast<size_t>(terms * s) * kBPanel / 2 + o,
                        static_cast<size_t>(terms * s + 1) * kBPanel / 2 + o, v, terms);
        } else {
            const long long e = i - nseq * per;
            const int p = static_cast<int>(e / (16 * 64));
            const int r = static_cast<int>((e % (16 * 64)) / 64), kl = static_cast<int>(e % 64);
            const int k = 64 * p + kl;
            const float v = (r < WRF_OUT && k < m.width)
                                ? m.W[m.n_hidden][static_cast<size_t>(r) * m.width + k]
                                : 0.f;
            const size_t o = (static_cast<size_t>(p) * kOutPanel + sw128_off(r, kl)) / 2;
            store_terms(oimg, o, o + kOutImg / 2, v, terms);
        }
    }
}

// gamma(mean_n) rows [N][64] BF16 (42 values of Eq. 15 at L_mean = 10, zeros
// after them): the encoding input on the unit square (tanh u + 1) / 2.
__device__ __forceinline__ void paper_tc_gamma_block(int blk, const PaperView &s, int L_mean,
                                                     int dm, uint16_t *G, int terms) {
    const int n = blk * blockDim.x + threadIdx.x;
    if (n >= s.n) return;
    const float2 mu = reinterpret_cast<const float2 *>(s.mu)[n];
    const PeArg a[2] = {unit_centre(mu.x), unit_centre(mu.y)};
    float gam[2 * (2 * 15 + 1)];
    pe_encode(a, 2, L_mean, gam);
    uint32_t *dst = reinterpret_cast<uint32_t *>(G + static_cast<size_t>(n) * kGammaCols);
    // terms = 2: the lo rows [N][64] follow the hi rows
    uint32_t *dlo = reinterpret_cast<uint32_t *>(G + (static_cast<size_t>(s.n) + n) * kGammaCols);
    for (int i = 0; i < kGammaCols / 2; ++i) {
        const float x0 = 2 * i < dm ? gam[2 * i] : 0.f;
        const float x1 = 2 * i + 1 < dm ? gam[2 * i + 1] : 0.f;
        const uint32_t h = pack_bf16(x0, x1);
        dst[i] = h;
        if (terms == 2)
            dlo[i] = pack_bf16(__fsub_rn(x0, __uint_as_float(h << 16)),
                               __fsub_rn(x1, __uint_as_float(h & 0xFFFF0000u)));
    }
}

// vec[q][l][j] (FP32): W_s gamma(s_q) + b for the layers whose input holds
// the encoding, b for the others, zero past the width; one block per (q, l).
__device__ __forceinline__ void paper_tc_vec_block(int q, int l, const PaperNetTc &m,
                                                   const float *tx, float *vec) {
    __shared__ float gam[3 * (2 * 15 + 1)];
    const int j = threadIdx.x;
    const bool enc = l < m.n_hidden && (l == 0 || is_skip(l));
    if (enc && j == 0) {
        PeArg a[3];
        for (int c = 0; c < 3; ++c) a[c] = pe_arg(tx[3 * q + c], m.room_min[c], m.room_size[c]);
        pe_encode(a, 3, m.L_tx, gam);
    }
    __syncthreads();
    float acc = 0.f;
    if (l < m.n_hidden && j < m.width) {
        if (enc) {
            const float *wr = m.W[l] + static_cast<size_t>(j) * in_dim_tc(m, l) +
                              (l == 0 ? 0 : m.width) + m.dm;
            for (int k = 0; k < m.dt; ++k) acc = fmaf(__ldg(wr + k), gam[k], acc);
        }
        acc += m.b[l][j];
    }
    vec[(static_cast<size_t>(q) * (kPaperMaxLayers - 1) + l) * kPW + j] = acc;
}

// The three independent preparation jobs of the network in one launch of
// kPW-thread blocks, so that they run side by side: blocks [0, nb_vec) form
// vec for one (query, layer) each, the next nb_gamma blocks encode kPW
// Gaussians each, the rest build the weight panels (grid-stride).  Every
// block runs exactly one job, so the vec job's barrier sees all its threads.
__global__ void __launch_bounds__(kPW) paper_tc_prep_kernel(PaperNetTc m, int nseq, uint16_t *wimg,
                                                            uint16_t *oimg, PaperView s,
                                                            uint16_t *G, const float *tx,
                                                            float *vec, int nb_vec, int nb_gamma,
                                                            int terms) {
    int b = blockIdx.x;
    if (b < nb_vec) {
        paper_tc_vec_block(b / (kPaperMaxLayers - 1), b % (kPaperMaxLayers - 1), m, tx, vec);
        return;
    }
    b -= nb_vec;
    if (b < nb_gamma) {
        paper_tc_gamma_block(b, s, m.L_mean, m.dm, G, terms);
        return;
    }
    b -= nb_gamma;
    paper_tc_weights_block(b, static_cast<int>(gridDim.x) - nb_vec - nb_gamma, m, nseq, wimg,
                           oimg, terms);
}

struct PaperTcArgs {
    PaperView s;
    GridView g;
    const uint16_t *G, *wimg, *oimg;
    const float *vec, *bout;
    int nh, nseq, Q, N, tpq, ntiles;
    float4 *rec;
    float *rec_im;
    int *status;
};

template <int X>
__global__ void __launch_bounds__(TcCfg<X>::Threads, 1) paper_tc_kernel(PaperTcArgs a) {
    using Cfg = TcCfg<X>;
    constexpr int kWGs = Cfg::WGs, kRing = Cfg::Ring, kTerms = Cfg::Terms;
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    uint8_t *base = smem_raw + (((raw + 1023u) & ~1023u) - raw);
    uint8_t *gp0 = base;                       // [kWGs][kTerms] gamma(mean) panels
    uint8_t *ring = base + kWGs * kTerms * kGPanel;
    uint8_t *oimg = ring + kRing * kBPanel;    // [kTerms] output images
    uint8_t *term0 = oimg + kTerms * kOutImg;  // [kWGs][160 rows x 16 B]
    uint8_t *sel = term0 + kWGs * kTermImg;    // selector A
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
    const int rounds_total = (a.ntiles + kWGs - 1) / kWGs;  // tiles per round: one per group

    if (warp == kWGs * (kGroup / 32)) {
        // ---------------------------------------------------- producer warp
        if (lane == 0) {
            mbar_arrive_expect_tx(wbar, kTerms * kOutImg);
            bulk_g2s(oimg, a.oimg, kTerms * kOutImg, wbar);
            uint32_t g = 0;  // panels issued
            bool ok = true;
            for (int p = blockIdx.x; p < rounds_total && ok; p += gridDim.x) {
                for (int s = 0; s < kTerms * a.nseq; ++s) {
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
        // ---------------------------------------------- compute groups
        // group, TMEM lane quarter, column half, thread within the group
        const int wg = warp / (kGroup / 32), wq = warp & 3, half = (warp >> 2) & 1;
        const int wt = tid & (kGroup - 1);
        uint8_t *G = gp0 + wg * kTerms * kGPanel;
        const uint32_t g_addr = smem_u32(G), ring_addr = smem_u32(ring), o_addr = smem_u32(oimg);
        const uint32_t t_acc = tmem_base + static_cast<uint32_t>(wg * 256);
        const uint32_t t_act = t_acc + static_cast<uint32_t>(kPW);      // hi pairs (80 columns)
        const uint32_t t_lo = t_act + static_cast<uint32_t>(kPW / 2);   // lo pairs (X = 3)
        const uint32_t lane_off = static_cast<uint32_t>(wq * 32) << 16;
        const int my_row = wq * 32 + lane;
        // the MMA warp of the group: lane 0 issues while lanes 1..31 wait at
        // the warp's reconvergence point (not on the mbarriers: a diverged
        // warp spinning there would slow the issuing lane down)
        const bool mma_warp = wt < 32, leader = wt == 0;
        const uint32_t id_h = idesc_bf16(128, kPW), id_o = idesc_bf16(128, 16);
        uint8_t *term = term0 + wg * kTermImg;
        const uint64_t d_sel = plain_desc(smem_u32(sel), 128u, 0u);
        const uint64_t d_term = plain_desc(smem_u32(term), 0u, 128u);
        // the term of layer l (vec[q][l], or the output bias when l == nh)
        // for row wt of the image: loaded ahead, written as BF16 hi + lo in K
        // columns 0 and 1 once the MMAs reading the image have completed
        auto load_term = [&](int q, int l) {
            float v = 0.f;
            if (wt < kPW) {
                if (l < a.nh)
                    v = __ldg(a.vec + (static_cast<size_t>(q) * (kPaperMaxLayers - 1) + l) * kPW + wt);
                else if (wt < WRF_OUT)
                    v = __ldg(a.bout + wt);
            }
            return v;
        };
        auto write_term = [&](float v) {
            if (wt < kPW) {
                const uint32_t hi = pack_bf16(v, 0.f) & 0xFFFFu;
                const uint32_t lo = pack_bf16(__fsub_rn(v, __uint_as_float(hi << 16)), 0.f) & 0xFFFFu;
                *reinterpret_cast<uint4 *>(term + wt * 16) = make_uint4(hi | (lo << 16), 0u, 0u, 0u);
            }
        };
        // MMAs of one weight panel (hi, and lo when X = 3) at K offsets
        // 0 .. nk-1 of 16: A from tensor memory (activation pairs from
        // column a_col) or from the gamma(mean) panel in shared memory
        // (descriptors advanced from their bases by one add per MMA)
        const uint64_t d_g = sw128_desc(g_addr);
        auto panel_mmas = [&](uint32_t bh, uint32_t bl, bool gamma, int a_col, int nk) {
            const uint64_t dbh0 = sw128_desc(bh), dbl0 = sw128_desc(bl);
            for (int kk = 0; kk < nk; ++kk) {
                const uint32_t ko = static_cast<uint32_t>(kk) * 32u;
                const uint64_t dbh = desc_adv(dbh0, ko);
                if (gamma) {
                    const uint64_t dg = desc_adv(d_g, ko);
                    mma_bf16(t_acc, dg, dbh, id_h, 1u);
                    if (X == 3) {
                        mma_bf16(t_acc, dg, desc_adv(dbl0, ko), id_h, 1u);
                        mma_bf16(t_acc, desc_adv(d_g, kGPanel + ko), dbh, id_h, 1u);
                    }
                } else {
                    const uint32_t col = static_cast<uint32_t>((a_col + kk) * 8);
                    mma_bf16_ts(t_acc, t_act + col, dbh, id_h, 1u);
                    if (X == 3) {
                        mma_bf16_ts(t_acc, t_act + col, desc_adv(dbl0, ko), id_h, 1u);
                        mma_bf16_ts(t_acc, t_lo + col, dbh, id_h, 1u);
                    }
                }
            }
        };
        uint32_t phase = 0, g = 0;
        wait_or_abort(wbar, 0, abort_flag, a.status);
        for (int p = blockIdx.x; p < rounds_total; p += gridDim.x) {
            if (wg_bar_any(1 + wg, *abort_flag != 0, kGroup)) break;
            const int tile = kWGs * p + wg;
            const bool tv = tile < a.ntiles;
            const int q = tv ? tile / a.tpq : 0;
            const int n = tv ? (tile % a.tpq) * kTile + my_row : a.N;
            const bool rv = n < a.N;
            // gamma(mean_n) -> this tile's panel(s), 16-byte chunks 4 half .. 4 half + 3
            for (int t = 0; t < kTerms; ++t) {
                const uint4 *src = reinterpret_cast<const uint4 *>(
                    a.G + (static_cast<size_t>(t) * a.N + (rv ? n : 0)) * kGammaCols);
#pragma unroll
                for (int c = 4 * half; c < 4 * half + 4; ++c) {
                    const uint4 v = rv ? __ldg(src + c) : make_uint4(0u, 0u, 0u, 0u);
                    *reinterpret_cast<uint4 *>(G + t * kGPanel + my_row * 128 +
                                               ((c ^ (my_row & 7)) << 4)) = v;
                }
            }
            write_term(load_term(q, 0));
            fence_async_smem();
            named_bar(1 + wg, kGroup);
            for (int l = 0; l < a.nh; ++l) {
                if (leader) {
                    tc_fence_after();
                    // D = vec[q][l] (hi + lo), then += W_l x
                    mma_bf16(t_acc, d_sel, d_term, id_h, 0u);
                    const int np = panels_of(l);
                    for (int i = 0; i < np; ++i) {
                        const int pid = (l == 0 || i == 3) ? kGammaPanel : i;
                        uint32_t b_addr[2];
                        int slots[2];
                        for (int t = 0; t < kTerms; ++t, ++g) {
                            slots[t] = static_cast<int>(g % kRing);
                            wait_or_abort(&full[slots[t]], (g / kRing) & 1u, abort_flag, a.status);
                            b_addr[t] = ring_addr + static_cast<uint32_t>(slots[t]) * kBPanel;
                        }
                        tc_fence_after();
                        if (pid == kGammaPanel) {
                            panel_mmas(b_addr[0], b_addr[kTerms - 1], true, 0, 4);
                        } else {
                            // activations K 64 pid .. (K 128..159 for pid 2)
                            panel_mmas(b_addr[0], b_addr[kTerms - 1], false, 4 * pid,
                                       pid == 2 ? 2 : 4);
                        }
                        for (int t = 0; t < kTerms; ++t) mma_commit(&empty[slots[t]]);
                    }
                    mma_commit(&accb[wg]);
                }
                if (mma_warp) __syncwarp();
                const float tnext = load_term(q, l + 1);  // in flight during the MMAs
                wait_or_abort(&accb[wg], phase, abort_flag, a.status);
                phase ^= 1u;
                tc_fence_after();
                write_term(tnext);  // the layer-l MMAs that read the image are complete
                // this warp's 80 accumulator columns -> 40 activation columns
                // (and, X = 3, 40 columns of the BF16 remainders)
                if (X == 3) {
                    // five chunks of 16 columns; the next chunk's load is in flight
                    // while this one is converted and stored
                    uint32_t ra[16], rb[16];
                    auto convert = [&](const uint32_t (&r)[16], int c) {
                        const int col = 80 * half + 16 * c;
                        uint32_t pk[8], pl[8];
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const float v0 = __uint_as_float(r[2 * j]), v1 = __uint_as_float(r[2 * j + 1]);
                            pk[j] = pack_bf16_relu(v0, v1);
                            if (X == 3) {
                                const float r0 = fmaxf(v0, 0.f), r1 = fmaxf(v1, 0.f);
                                pl[j] = pack_bf16(__fsub_rn(r0, __uint_as_float(pk[j] << 16)),
                                                  __fsub_rn(r1, __uint_as_float(pk[j] & 0xFFFF0000u)));
                            }
                        }
                        tmem_st8(t_act + lane_off + col / 2, pk);
                        if (X == 3) tmem_st8(t_lo + lane_off + col / 2, pl);
                    };
                    const uint32_t c0 = t_acc + lane_off + 80 * half;
                    tmem_ld16_issue(c0, ra);
                    tmem_ld16_wait(ra);
                    tmem_ld16_issue(c0 + 16, rb);
                    convert(ra, 0);
                    tmem_ld16_wait(rb);
                    tmem_ld16_issue(c0 + 32, ra);
                    convert(rb, 1);
                    tmem_ld16_wait(ra);
                    tmem_ld16_issue(c0 + 48, rb);
                    convert(ra, 2);
                    tmem_ld16_wait(rb);
                    tmem_ld16_issue(c0 + 64, ra);
                    convert(rb, 3);
                    tmem_ld16_wait(ra);
                    convert(ra, 4);
                } else {
                    // (BF16 alone: one chunk at a time; the overlapped form
                    // spills registers in this instance)
#pragma unroll 1
                    for (int c = 0; c < 3; ++c) {
                        const int col = 80 * half + 32 * c;
                        const int nv = c < 2 ? 32 : 16;
                        float v[32];
                        uint32_t pk[16], pl[16];
                        if (c < 2)
                            tmem_ld32(t_acc + lane_off + col, v);
                        else
                            tmem_ld16(t_acc + lane_off + col, v);
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            if (2 * j >= nv) break;
                            pk[j] = pack_bf16_relu(v[2 * j], v[2 * j + 1]);
                            if (X == 3) {
                                const float r0 = fmaxf(v[2 * j], 0.f), r1 = fmaxf(v[2 * j + 1], 0.f);
                                pl[j] = pack_bf16(__fsub_rn(r0, __uint_as_float(pk[j] << 16)),
                                                  __fsub_rn(r1, __uint_as_float(pk[j] & 0xFFFF0000u)));
                            }
                        }
                        if (c < 2) {
                            tmem_st16(t_act + lane_off + col / 2, pk);
                            if (X == 3) tmem_st16(t_lo + lane_off + col / 2, pl);
                        } else {
                            tmem_st8(t_act + lane_off + col / 2, pk);
                            if (X == 3) tmem_st8(t_lo + lane_off + col / 2, pl);
                        }
                    }
                }
                tmem_wait_st();
                tc_fence_before();
                fence_async_smem();
                named_bar(1 + wg, kGroup);
            }
            // output layer: N = 16 (5 used), K 0..159, resident weights
            if (leader) {
                tc_fence_after();
                mma_bf16(t_acc, d_sel, d_term, id_o, 0u);  // D = output bias (hi + lo)
                const uint64_t d_o = sw128_desc(o_addr);
#pragma unroll
                for (int kk = 0; kk < kPW / 16; ++kk) {
                    const uint32_t oo = static_cast<uint32_t>(kk >> 2) * kOutPanel +
                                        static_cast<uint32_t>(kk & 3) * 32u;
                    const uint64_t dob = desc_adv(d_o, oo);
                    mma_bf16_ts(t_acc, t_act + static_cast<uint32_t>(kk * 8), dob, id_o, 1u);
                    if (X == 3) {
                        mma_bf16_ts(t_acc, t_act + static_cast<uint32_t>(kk * 8),
                                    desc_adv(d_o, oo + kOutImg), id_o, 1u);
                        mma_bf16_ts(t_acc, t_lo + static_cast<uint32_t>(kk * 8), dob, id_o, 1u);
                    }
                }
                mma_commit(&accb[wg]);
            }
            if (mma_warp) __syncwarp();
            wait_or_abort(&accb[wg], phase, abort_flag, a.status);
            phase ^= 1u;
            tc_fence_after();
            float o[16];
            tmem_ld16(t_acc + lane_off, o);
            tc_fence_before();
            if (half == 0 && tv && rv && !*abort_flag) {
                float d[5];
#pragma unroll
                for (int i = 0; i < WRF_OUT; ++i) d[i] = o[i];
                paper_project(a.s, n, q, d, a.g, a.rec, a.rec_im);
            }
            named_bar(1 + wg, kGroup);  // TMEM columns and the gamma panel are free again
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
    // room for the hi and lo images (three-product precision)
    return 2 * (static_cast<size_t>(seq_len(n_hidden)) * kBPanel + kOutImg);
}

namespace {

template <int X>
cudaError_t launch_paper_tc_x(const PaperSceneView &sv, const PaperMlpView &mv, const GridView &g,
                              const float *tx, int Q, const PaperWs &ws, float4 *rec, int *status,
                              cudaStream_t st) {
    using Cfg = TcCfg<X>;
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
    uint16_t *oimg = ws.img + static_cast<size_t>(Cfg::Terms * nseq) * kBPanel / 2;
    {
        const int nb_vec = Q * (kPaperMaxLayers - 1);
        const int nb_gamma = (sv.n + kPW - 1) / kPW;
        const int nb_w = 148 * 4;  // 592 x 160 threads, about the 296 x 256 of a separate launch
        paper_tc_prep_kernel<<<nb_vec + nb_gamma + nb_w, kPW, 0, st>>>(
            m, nseq, wimg, oimg, s, ws.G, tx, ws.vec, nb_vec, nb_gamma, Cfg::Terms);
    }
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
    a.rec = rec;
    a.rec_im = reinterpret_cast<float *>(rec + 2 * rows);
    a.status = status;
    const size_t smem = Cfg::smem;
    cudaError_t e = cudaFuncSetAttribute(paper_tc_kernel<X>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int rounds = (a.ntiles + Cfg::WGs - 1) / Cfg::WGs;
    const int grid = rounds < sms ? rounds : sms;
    paper_tc_kernel<X><<<grid, Cfg::Threads, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_paper_tc(const PaperSceneView &sv, const PaperMlpView &mv, const GridView &g,
                            const float *tx, int Q, const PaperWs &ws, float4 *rec, int *status,
                            int precision, cudaStream_t st) {
    return precision == WRF_BF16X3
               ? launch_paper_tc_x<3>(sv, mv, g, tx, Q, ws, rec, status, st)
               : launch_paper_tc_x<1>(sv, mv, g, tx, Q, ws, rec, status, st);
}

}  // namespace wrf
