// Tile rasteriser for the order-free Gaussian sum (Sec. 4.1 Eq. 8-9,
// Sec. 4.2 Eq. 13) and its backward.
//
// Forward: one CTA per (tile, query), one thread per two pixels (or four, a
// launch knob); warp w owns an 8 x 8 pixel block of the tile and lane l the
// pixels (l % 8, l / 8) and (l % 8, l / 8 + 4) of it (with four pixels a
// 16 x 8 block, also the columns + 8).  The tile's Gaussian list (ascending
// id) is streamed through shared memory in batches of one record per thread
// (or two, a launch knob) into two landing buffers that alternate, so the
// batch after next is in flight while the current one is evaluated, by one
// of two staging paths (a launch knob): every thread copies its own records
// with two 16-byte cp.async each into its own slots and waits for its own
// copies only (cp.async.wait_group; the thread that copies a record is the
// one that sets it up), or TMA gathers (cp.async.bulk.tensor tile::gather4,
// four records per copy) completing on one mbarrier per buffer.  Once per
// (tile, Gaussian) a thread turns the record into the polynomial
//   -q'(lx, ly) = c0 + c1 lx + c2 ly + c3 lx^2 + c4 lx ly + c5 ly^2
// in the pixel's offset (lx, ly) from the tile centre (q' = q log2(e)/2), and
// a bitmask of the warp blocks its footprint rectangle touches.  Each warp
// then compacts (ballot + popc) the batch into its own list, ascending, and
// evaluates only those.  Set-up stores, per tile row y, alpha(y) and beta(y)
// with
//   -q'(lx, y) = alpha(y) + beta(y) lx + c3 lx^2,
// the rows y and y + 4 of a thread side by side in one 16-byte entry
// (alpha(y), alpha(y+4), beta(y), beta(y+4)), so a pixel costs two FMAs (one
// two-lane fma.rn.f32x2 each for both pixels), one compare, one ex2 and one
// FMA, and one list entry, one (alpha, beta) load and one (c3, w) load serve
// both pixels of a thread.
// Every pixel adds its contributions in ascending Gaussian id, so a query's
// spectrum does not depend on the other queries in the launch.  The finished
// tile goes through shared memory (the row-pair area, dead by then) to
// float4 stores.
//
// Backward: one CTA per (tile, query); the tile's dL/dA is staged in shared
// memory, a warp cuts 32 keys of the list into (key, box row) items shared
// out evenly over its lanes, recomputes exp(-q/2) over each row's in-cutoff
// span and accumulates dL/d(mx, my, A, B, C, w) per key, then adds them to
// the per-(query, Gaussian) gradient with atomics (a Gaussian spans several
// tiles).
#include <cuda.h>

#include <cstring>
#include <mutex>

#include "kernels.h"

namespace wrf {

namespace {

// d = a * b + c on two FP32 lanes in one instruction (fma.rn.f32x2); each
// lane rounds exactly like fmaf.
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\t"
        "mov.b64 rb, {%4, %5};\n\t"
        "mov.b64 rc, {%6, %7};\n\t"
        "fma.rn.f32x2 rd, ra, rb, rc;\n\t"
        "mov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}

// TMA gather of four 32-byte records (rows r0..r3 of the record tensor map,
// 8 FP32 columns from column 0) into 128 contiguous bytes of shared memory,
// completion counted in bytes on `bar`.  dst 128-byte aligned.
__device__ __forceinline__ void tma_gather4(void *dst, const CUtensorMap *map, int r0, int r1,
                                            int r2, int r3, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile::gather4.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(r0), "r"(r1), "r"(r2), "r"(r3),
        "r"(smem_u32(bar))
        : "memory");
}

// Shared-memory carve-up of the forward kernel for a tile with NT threads
// and TH rows: a batch holds B = BF x NT records, BF per thread.  WIM: the
// staged imaginary weights (two channels with TMA staging; the cp.async path
// keeps them in registers).  The finished tile is staged in the row-pair
// area, which is dead once the last batch is evaluated.  Kept small enough
// for eight CTAs per SM at 32 x 16 tiles with four pixels per thread.
template <int NT, int TH, int BF, bool WIM>
struct FwdSmem {
    static constexpr int B = NT * BF, NW = NT / 32, RS = B + 1;  // RS: bank spread
    static constexpr size_t raw = 0;                           // [2][B][2] float4, TMA landing
    static constexpr size_t rowc = raw + 2 * B * 32;           // [TH/2][RS] float4, row pairs
    static constexpr size_t gc = rowc + (TH / 2) * RS * 16;    // [B] float4 (c3, c3, w, 0)
    static constexpr size_t mask = gc + B * 16;                // [B] u8, warp blocks touched
    static constexpr size_t lists = mask + B;                  // [NW][B] u16, per-warp compaction
    static constexpr size_t wim = lists + NW * B * 2;          // [2][B] f32, imaginary weights
    static constexpr size_t bytes = wim + (WIM ? 2 * B * 4 : 0);
};

// CH = 1: one channel, out [Q][H][W].  CH = 2: real and imaginary channels
// (weights w from the records, w_im from rec_im [Q][N]) summed with one ex2
// per pixel and Gaussian, out [Q][2][H][W] = magnitude, phase (Sec. 6.1).
// PX: pixels per thread, 2 (rows y, y + 4 of an 8 x 8 warp block) or 4 (also
// columns x + 8: a 16 x 8 warp block; one row-pair entry serves both
// columns).  BF: records per thread in a staged batch (the batch holds
// BF x threads Gaussians).
// TMA: record staging by TMA gathers (one cp.async.bulk.tensor tile::gather4
// of four records per issuing thread, completion counted in bytes on one
// mbarrier per landing buffer, bounded waits) or, with TMA = false, by
// per-thread cp.async (each thread copies the records it sets up itself,
// completion by cp.async.wait_group).  Both stage the same bytes in the same
// slots; the rest of the kernel is shared.
template <int TW, int TH, int CH, bool WRAP, int PX, int BF, bool TMA>
__global__ void __launch_bounds__(TW *TH / PX, 1024 * PX / (TW * TH)) render_kernel(
    const float4 *__restrict__ rec, const uint32_t *__restrict__ gids,
    const uint32_t *__restrict__ offs, const long long *__restrict__ n_keys, long long cap, int n,
    GridView g, float ncut, float *__restrict__ out, int *status, const float *__restrict__ rec_im,
    const long long *__restrict__ qbase, const __grid_constant__ CUtensorMap rmap) {
    constexpr int NT = TW * TH / PX, B = NT * BF, NW = NT / 32;
    constexpr int NG = B / 4;  // four-record gathers per full batch
    static_assert(NG <= NT, "one gather per thread at most");
    constexpr int BW = 4 * PX;   // warp block width: 8 or 16 columns
    constexpr int NSX = TW / BW;  // warp blocks of BW x 8 pixels: NSX across, TH/8 down
    static_assert(NW == NSX * (TH / 8), "one warp block per warp");
    using L = FwdSmem<NT, TH, BF, CH == 2 && TMA>;
    static_assert(NW <= 8, "warp-block masks are 8 bits");
    static_assert(L::gc - L::rowc >= static_cast<size_t>(CH) * TH * TW * 4,
                  "the output tile fits in the row-pair area");
    extern __shared__ __align__(128) unsigned char smem[];
    float4 *raw = reinterpret_cast<float4 *>(smem + L::raw);
    float4 *rowc = reinterpret_cast<float4 *>(smem + L::rowc);
    float4 *gcoef = reinterpret_cast<float4 *>(smem + L::gc);
    uint8_t *mask = smem + L::mask;
    uint16_t *lists = reinterpret_cast<uint16_t *>(smem + L::lists);
    float *wim_s = reinterpret_cast<float *>(smem + L::wim);  // two channels: [2][B]
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ int abort_flag;
    // the finished tile (and its phase plane), written after the last batch
    float(*stile)[TW] = reinterpret_cast<float(*)[TW]>(smem + L::rowc);
    float(*stile_im)[TW] = stile + TH;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int t = blockIdx.y, q = blockIdx.x;  // tile-major launch order
    const int x0 = (t % g.ntx) * TW, y0 = (t / g.ntx) * TH;
    // this thread's pixels (tile-local): column pxl (and pxl + 8 when PX = 4),
    // rows pyl and pyl + 4; lx = the column's offset from the tile centre
    const int pxl = (warp % NSX) * BW + (lane & 7);
    const int pyl = (warp / NSX) * 8 + (lane >> 3);
    const float lx = static_cast<float>(pxl - TW / 2);
    const float xcen = static_cast<float>(x0 + TW / 2), ycen = static_cast<float>(y0 + TH / 2);

    // the offsets array always has Q x T + 1 entries, so both loads are
    // issued together with the key count; an overflowed binning renders zero
    uint32_t s0 = offs[static_cast<size_t>(q) * g.T + t];
    uint32_t s1 = offs[static_cast<size_t>(q) * g.T + t + 1];
    if (*n_keys > cap) s0 = s1 = 0;
    const int total = static_cast<int>(s1 - s0);
    const int nb = (total + B - 1) / B;
    // records of this query (multi-scene batches: at qbase[q]): rows from rb
    const long long rb = qbase ? qbase[q] : static_cast<long long>(q) * n;
    const float4 *qrec = rec + static_cast<size_t>(rb) * 2;
    const float *qim = CH == 2 ? rec_im + static_cast<size_t>(q) * n : nullptr;

    // Thread g < NG gathers records 4g .. 4g+3 of a batch; gq holds their
    // Gaussian ids, loaded one batch before the gather is issued (a group
    // past the batch's end repeats its first id: the bytes land in unused
    // slots).
    uint32_t gq[4] = {0u, 0u, 0u, 0u};
    auto load_group = [&](int bb) {
        const int cnt = min(B, total - bb * B), i0 = 4 * tid;
        if (tid < NG && i0 < cnt) {
            const uint32_t *src = gids + s0 + bb * B + i0;
            gq[0] = src[0];
#pragma unroll
            for (int j = 1; j < 4; ++j) gq[j] = i0 + j < cnt ? src[j] : gq[0];
        }
    };
    auto gather = [&](int bb) {
        const int buf = bb & 1, cnt = min(B, total - bb * B);
        if (4 * tid < cnt) {
            tma_gather4(raw + (buf * B + 4 * tid) * 2, &rmap, static_cast<int>(rb + gq[0]),
                        static_cast<int>(rb + gq[1]), static_cast<int>(rb + gq[2]),
                        static_cast<int>(rb + gq[3]), &bar[buf]);
            if (CH == 2) {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (4 * tid + j < cnt) wim_s[buf * B + 4 * tid + j] = qim[gq[j]];
            }
        }
    };
    auto batch_bytes = [&](int bb) {
        return static_cast<uint32_t>((min(B, total - bb * B) + 3) / 4) * 128u;
    };
    // cp.async staging: this thread's records of batch bb (their ids in
    // gnext, loaded one batch early), one commit group per batch slot, empty
    // or not, so "all but the newest group done" always means "this batch
    // landed"
    uint32_t gnext[BF];
    // two channels: the imaginary weights of this thread's records, per
    // landing buffer (registers; the TMA path keeps them in shared memory)
    float wim_r[2][BF];
#pragma unroll
    for (int k = 0; k < BF; ++k) wim_r[0][k] = wim_r[1][k] = 0.f;
    auto load_own = [&](int bb) {
#pragma unroll
        for (int k = 0; k < BF; ++k) {
            const int i = tid + k * NT;
            gnext[k] = i < total - bb * B ? gids[s0 + bb * B + i] : 0u;
        }
    };
    auto copy_own = [&](int bb) {
        const int buf = bb & 1;
#pragma unroll
        for (int k = 0; k < BF; ++k) {
            const int i = tid + k * NT;
            if (i < total - bb * B) {
                const float4 *src = qrec + 2 * static_cast<size_t>(gnext[k]);
                cp_async16(raw + (buf * B + i) * 2, src);
                cp_async16(raw + (buf * B + i) * 2 + 1, src + 1);
                if (CH == 2) {
                    if (buf) wim_r[1][k] = qim[gnext[k]];
                    else wim_r[0][k] = qim[gnext[k]];
                }
            }
        }
        cp_async_commit();
    };

    if (TMA) {
        if (tid == 0) {
            mbar_init(&bar[0], 1);
            mbar_init(&bar[1], 1);
            fence_mbar_init();
            for (int bb = 0; bb < 2 && bb < nb; ++bb)
                mbar_arrive_expect_tx(&bar[bb], batch_bytes(bb));
        }
        load_group(0);
        __syncthreads();
        if (nb > 0) gather(0);
        load_group(1);
        if (nb > 1) gather(1);
        load_group(2);  // ids of batch 2, gathered after batch 0 is set up
        if (CH == 2) __syncthreads();  // the imaginary weights of batches 0 and 1
    } else {
        load_own(0);
        copy_own(0);
        load_own(1);
        copy_own(1);
        load_own(2);
    }
    if (TMA) {
        // (the cp.async path has no bounded wait and so no abort)
        if (tid == 0) abort_flag = 0;
        __syncthreads();
    }

    float acc0 = 0.f, acc1 = 0.f, acc0i = 0.f, acc1i = 0.f;
    // PX = 4: column pxl + 8, rows pyl and pyl + 4
    float acc2 = 0.f, acc3 = 0.f, acc2i = 0.f, acc3i = 0.f;
    uint16_t *mylist = lists + warp * B;
    int b = 0;
    for (; b < nb; ++b) {
        const int buf = b & 1;
        const int cnt = min(B, total - b * B);
        if (TMA) {
            if (!mbar_wait(&bar[buf], (b >> 1) & 1, status)) abort_flag = 1;
            if (tid == 0 && b + 2 < nb) mbar_arrive_expect_tx(&bar[buf], batch_bytes(b + 2));
        } else {
            cp_async_wait_pending<1>();  // this thread's records of batch b
        }
        // ---- per-record set-up, once per (tile, Gaussian):
        // -q'(p) for p = tile centre + (lx, ly) as a polynomial in lx, ly:
        //   dx = lx - ux, dy = ly - uy, u = centre - tile centre,
        //   -q' = c0 + c1 lx + c2 ly + c3 lx^2 + c4 lx ly + c5 ly^2
        // and the mask of 8x8 warp blocks its footprint rectangle touches.
#pragma unroll
        for (int k = 0; k < BF; ++k) {
            const int ri = tid + k * NT;  // the record this thread sets up
            if (ri >= cnt) break;
            const float4 r0 = raw[(buf * B + ri) * 2], r1 = raw[(buf * B + ri) * 2 + 1];
            // with azimuth wrap, the image of the Gaussian nearest to this tile
            const float mx = WRAP ? nearest_image_x(r0.x, xcen, g) : r0.x;
            const float ux = mx - xcen, uy = r0.y - ycen;
            const float h1 = fmaf(r0.z, ux, r0.w * uy), h2 = fmaf(r0.w, ux, r1.x * uy);
            const float c0 = -fmaf(ux, h1, uy * h2);
            const float c1 = 2.f * h1, c2 = 2.f * h2, c4 = -2.f * r0.w, c5 = -r1.x;
            // per tile row: -q'(lx) = alpha + beta lx + c3 lx^2; entry p of
            // the record holds rows y(p) and y(p) + 4, y(p) = 8 (p / 4) + p % 4
            // both rows of an entry at once: two-lane FMAs, each lane rounded
            // like fmaf (alpha = (c5 ly + c2) ly + c0, beta = c4 ly + c1)
            const float2 c5v = make_float2(c5, c5), c2v = make_float2(c2, c2);
            const float2 c0v = make_float2(c0, c0), c4v = make_float2(c4, c4);
            const float2 c1v = make_float2(c1, c1);
#pragma unroll
            for (int pr = 0; pr < TH / 2; ++pr) {
                const float ly0 = static_cast<float>((pr >> 2) * 8 + (pr & 3) - TH / 2);
                const float2 ly = make_float2(ly0, ly0 + 4.f);
                const float2 al = fma2(fma2(c5v, ly, c2v), ly, c0v);
                const float2 be = fma2(c4v, ly, c1v);
                rowc[pr * L::RS + ri] = make_float4(al.x, al.y, be.x, be.y);
            }
            const float wi = CH == 2 ? (TMA ? wim_s[buf * B + ri] : (buf ? wim_r[1][k] : wim_r[0][k]))
                                     : 0.f;
            gcoef[ri] = make_float4(-r0.z, -r0.z, r1.y, wi);
            uint32_t mk = 0;
            const float xlo = ceilf(__fsub_rn(mx, r1.z)) - static_cast<float>(x0);
            const float xhi = floorf(__fadd_rn(mx, r1.z)) - static_cast<float>(x0);
            const float ylo = ceilf(__fsub_rn(r0.y, r1.w)) - static_cast<float>(y0);
            const float yhi = floorf(__fadd_rn(r0.y, r1.w)) - static_cast<float>(y0);
            if (xhi >= 0.f && xlo <= TW - 1.f && yhi >= 0.f && ylo <= TH - 1.f) {
                const int bx0 = static_cast<int>(fmaxf(xlo, 0.f)) / BW;
                const int bx1 = static_cast<int>(fminf(xhi, TW - 1.f)) / BW;
                const int by0 = static_cast<int>(fmaxf(ylo, 0.f)) >> 3;
                const int by1 = static_cast<int>(fminf(yhi, TH - 1.f)) >> 3;
                const uint32_t row = (2u << bx1) - (1u << bx0);
                for (int by = by0; by <= by1; ++by) mk |= row << (by * NSX);
            }
            mask[ri] = static_cast<uint8_t>(mk);
        }
        __syncthreads();
        // raw[buf] is consumed: the copies of batch b+2 can land there now
        if (TMA) {
            if (b + 2 < nb) {
                gather(b + 2);
                load_group(b + 3);
            }
        } else {
            copy_own(b + 2);  // (commits an empty group past the last batch)
            load_own(b + 3);
        }
        // ---- this warp's list: records touching its block, ascending index
        // (the mask loads of all rounds are independent: unrolled, they
        // overlap)
        int m = 0;
#pragma unroll
        for (int base = 0; base < B; base += 32) {
            if (base >= cnt) break;
            const int i = base + lane;
            const bool hit = i < cnt && ((mask[i] >> warp) & 1u);
            const uint32_t bal = __ballot_sync(0xffffffffu, hit);
            // entries are byte offsets i * 16 into the (c3, c3, w, 0) array
            if (hit) mylist[m + __popc(bal & ((1u << lane) - 1u))] = static_cast<uint16_t>(i * 16);
            m += __popc(bal);
        }
        __syncwarp();
        // ---- accumulate: w * 2^(-q') where q <= q_cut (Eq. 8-9)
        const char *mypair = reinterpret_cast<const char *>(
            rowc + ((pyl >> 3) * 4 + (pyl & 3)) * L::RS);
        const char *gcb = reinterpret_cast<const char *>(gcoef);
        const float2 lx2 = make_float2(lx, lx);
        const float2 lxb = make_float2(lx + 8.f, lx + 8.f);  // PX = 4: the second column
        // unrolled 8 deep with four pixels per thread and one channel (1.3 %
        // faster than 4 at 32 x 16) and at 32 x 8 tiles with two (0.5 %), 4
        // elsewhere (8 spills a register at 16 x 16 with two)
        constexpr int kUnroll = ((PX == 4 && CH == 1) || (TW == 32 && TH == 8)) ? 8 : 4;
#pragma unroll kUnroll
        for (int j = 0; j < m; ++j) {
            const int o = mylist[j];  // = record index * 16
            const float4 ab = *reinterpret_cast<const float4 *>(mypair + o);  // alpha x 2, beta x 2
            const float4 cw = *reinterpret_cast<const float4 *>(gcb + o);    // c3, c3, w, 0
            const float2 t = fma2(make_float2(cw.x, cw.y), lx2, make_float2(ab.z, ab.w));
            const float2 nq = fma2(t, lx2, make_float2(ab.x, ab.y));
            if (CH == 1) {
                if (nq.x >= ncut) acc0 = fmaf(cw.z, ex2_approx(nq.x), acc0);
                if (nq.y >= ncut) acc1 = fmaf(cw.z, ex2_approx(nq.y), acc1);
                if (PX == 4) {
                    const float2 tb = fma2(make_float2(cw.x, cw.y), lxb, make_float2(ab.z, ab.w));
                    const float2 nqb = fma2(tb, lxb, make_float2(ab.x, ab.y));
                    if (nqb.x >= ncut) acc2 = fmaf(cw.z, ex2_approx(nqb.x), acc2);
                    if (nqb.y >= ncut) acc3 = fmaf(cw.z, ex2_approx(nqb.y), acc3);
                }
            } else {
                if (nq.x >= ncut) {
                    const float e = ex2_approx(nq.x);
                    acc0 = fmaf(cw.z, e, acc0);
                    acc0i = fmaf(cw.w, e, acc0i);
                }
                if (nq.y >= ncut) {
                    const float e = ex2_approx(nq.y);
                    acc1 = fmaf(cw.z, e, acc1);
                    acc1i = fmaf(cw.w, e, acc1i);
                }
                if (PX == 4) {
                    const float2 tb = fma2(make_float2(cw.x, cw.y), lxb, make_float2(ab.z, ab.w));
                    const float2 nqb = fma2(tb, lxb, make_float2(ab.x, ab.y));
                    if (nqb.x >= ncut) {
                        const float e = ex2_approx(nqb.x);
                        acc2 = fmaf(cw.z, e, acc2);
                        acc2i = fmaf(cw.w, e, acc2i);
                    }
                    if (nqb.y >= ncut) {
                        const float e = ex2_approx(nqb.y);
                        acc3 = fmaf(cw.z, e, acc3);
                        acc3i = fmaf(cw.w, e, acc3i);
                    }
                }
            }
        }
        __syncthreads();  // coef / mask / lists are rewritten by the next batch
        if (TMA && abort_flag) break;
    }
    if (!TMA) cp_async_wait_all();  // nothing may be in flight when the CTA exits
    if (TMA && abort_flag) {
        // drain gathers still in flight (bounded waits) before the CTA exits
        for (int bb = b; bb < nb && bb <= b + 2; ++bb)
            mbar_wait(&bar[bb & 1], (bb >> 1) & 1, status);
        return;
    }
    if (CH == 1) {
        stile[pyl][pxl] = acc0;
        stile[pyl + 4][pxl] = acc1;
        if (PX == 4) {
            stile[pyl][pxl + 8] = acc2;
            stile[pyl + 4][pxl + 8] = acc3;
        }
    } else {
        // magnitude and phase of re + i im (arg 0 = 0)
        stile[pyl][pxl] = sqrtf(fmaf(acc0, acc0, acc0i * acc0i));
        stile[pyl + 4][pxl] = sqrtf(fmaf(acc1, acc1, acc1i * acc1i));
        stile_im[pyl][pxl] = atan2f(acc0i, acc0);
        stile_im[pyl + 4][pxl] = atan2f(acc1i, acc1);
        if (PX == 4) {
            stile[pyl][pxl + 8] = sqrtf(fmaf(acc2, acc2, acc2i * acc2i));
            stile[pyl + 4][pxl + 8] = sqrtf(fmaf(acc3, acc3, acc3i * acc3i));
            stile_im[pyl][pxl + 8] = atan2f(acc2i, acc2);
            stile_im[pyl + 4][pxl + 8] = atan2f(acc3i, acc3);
        }
    }
    __syncthreads();
    const size_t plane = static_cast<size_t>(g.H) * g.W;
    const bool vec = (g.W & 3) == 0;
    for (int c = 0; c < CH; ++c) {
        float *oq = out + (static_cast<size_t>(q) * CH + c) * plane;
        float(*st)[TW] = c == 0 ? stile : stile_im;
        for (int i = tid; i < TH * TW / 4; i += NT) {
            const int r = i / (TW / 4), c4 = (i % (TW / 4)) * 4;
            const int y = y0 + r, x = x0 + c4;
            if (y >= g.H || x >= g.W) continue;
            const float4 v = *reinterpret_cast<const float4 *>(&st[r][c4]);
            float *dst = oq + static_cast<size_t>(y) * g.W + x;
            if (vec) {
                *reinterpret_cast<float4 *>(dst) = v;
            } else {
                const float vv[4] = {v.x, v.y, v.z, v.w};
                for (int k = 0; k < 4 && x + k < g.W; ++k) dst[k] = vv[k];
            }
        }
    }
}

// Backward of the order-free sum (Eq. 9) for one (tile, query): per key
// (record n of the tile's list) the sums over its in-cutoff pixels of
//   ge = dL/dA(p) e(p),  e = exp(-q/2):
//   S0 = sum ge, S1 = sum ge dx, S2 = sum ge dy,
//   S3 = sum ge dx^2, S4 = sum ge dx dy, S5 = sum ge dy^2,
// from which dL/dw = S0, dL/dmean = w (Sigma^-1 (S1, S2)) and
// dL/d(A, B, C) = -w (S3 / 2, S4, S5 / 2) (the conic in record units).
//
// Work split: a warp takes 32 keys at a time and cuts them into items of one
// row of a key's box (within the tile).  Each lane gets a contiguous range of
// the items (all ranges equal to within one), so the lanes of a warp run
// equally long instead of as long as the warp's largest box; within a row
// only the x-interval where the quadratic form can be under the cutoff is
// visited (solved per row with a margin; the per-pixel test decides).  A
// lane keeps the sums of its current key in registers (the row terms of S2,
// S4, S5 folded at each row end) and adds them into the warp's per-key sums
// in shared memory when it moves to the next key; one lane per key then
// adds the six gradients to d_rec.
template <int TW, int TH>
__global__ void __launch_bounds__(128) render_bwd_kernel(
    const float4 *__restrict__ rec, const uint32_t *__restrict__ gids,
    const uint32_t *__restrict__ offs, const long long *__restrict__ n_keys, long long cap, int n,
    GridView g, float cut_s, const float *__restrict__ dA, float *__restrict__ d_rec) {
    __shared__ float sg[TH][TW];
    __shared__ float4 kpar[4][32][3];  // per warp and key: mx, my, A, B | C, 1/A, xa, xb | ya
    __shared__ int kpre[4][33];        // per warp: item (row) prefix over its 32 keys
    __shared__ float kacc[4][32][6];   // per warp and key: S0 .. S5
    const int t = blockIdx.y, q = blockIdx.x;  // tile-major, as the forward
    const int x0 = (t % g.ntx) * TW, y0 = (t / g.ntx) * TH;
    for (int i = threadIdx.x; i < TH * TW; i += blockDim.x) {
        int y = y0 + i / TW, x = x0 + i % TW;
        sg[i / TW][i % TW] =
            (y < g.H && x < g.W) ? dA[(static_cast<size_t>(q) * g.H + y) * g.W + x] : 0.f;
    }
    __syncthreads();
    if (*n_keys > cap) return;
    const uint32_t s0 = offs[static_cast<size_t>(q) * g.T + t];
    const uint32_t s1 = offs[static_cast<size_t>(q) * g.T + t + 1];
    const float inv = 1.f / kHalfLog2e;
    const int xe = min(x0 + TW, g.W) - 1, ye = min(y0 + TH, g.H) - 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float4(*par)[3] = kpar[warp];
    int *pre = kpre[warp];
    float(*acc)[6] = kacc[warp];
    for (uint32_t base = s0 + 32u * warp; base < s1; base += 128u) {
        // ---- this lane's key: its box within the tile and its row count
        const uint32_t i = base + lane;
        size_t r = 0;
        float w = 0.f, A = 0.f, Bc = 0.f, Cc = 0.f;
        int rows = 0;
        if (i < s1) {
            r = static_cast<size_t>(q) * n + gids[i];
            float4 r0 = rec[2 * r];
            const float4 r1 = rec[2 * r + 1];
            // with azimuth wrap, the image of the Gaussian nearest to this tile
            r0.x = nearest_image_x(r0.x, static_cast<float>(x0) + 0.5f * TW, g);
            const int xa = max(x0, static_cast<int>(ceilf(fmaxf(r0.x - r1.z, static_cast<float>(x0)))));
            const int xb = min(xe, static_cast<int>(floorf(fminf(r0.x + r1.z, static_cast<float>(xe)))));
            const int ya = max(y0, static_cast<int>(ceilf(fmaxf(r0.y - r1.w, static_cast<float>(y0)))));
            const int yb = min(ye, static_cast<int>(floorf(fminf(r0.y + r1.w, static_cast<float>(ye)))));
            rows = (xa <= xb && ya <= yb) ? yb - ya + 1 : 0;
            A = r0.z * inv;
            Bc = r0.w * inv;
            Cc = r1.x * inv;
            w = r1.y;
            par[lane][0] = r0;
            par[lane][1] = make_float4(r1.x, 1.f / r0.z, static_cast<float>(xa),
                                       static_cast<float>(xb));
            par[lane][2] = make_float4(static_cast<float>(ya), 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int j = 0; j < 6; ++j) acc[lane][j] = 0.f;
        int incl = rows;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        pre[lane + 1] = incl;
        if (lane == 0) pre[0] = 0;
        __syncwarp();
        // ---- this lane's items [it0, it1): rows of consecutive keys
        const int it0 = static_cast<int>(static_cast<long long>(total) * lane / 32);
        const int it1 = static_cast<int>(static_cast<long long>(total) * (lane + 1) / 32);
        if (it0 < it1) {
            int k = 0;  // the last key whose items start at or before it0
            for (int step = 16; step > 0; step >>= 1)
                if (k + step <= 32 && pre[k + step] <= it0) k += step;
            int row = it0 - pre[k], nrow = pre[k + 1] - pre[k];
            float4 p0 = par[k][0], p1 = par[k][1];
            float yk = par[k][2].x;
            float S0 = 0.f, S1 = 0.f, S2 = 0.f, S3 = 0.f, S4 = 0.f, S5 = 0.f;
            for (int it = it0; it < it1; ++it) {
                if (row == nrow) {
                    // next key with rows: hand this key's sums to the warp
                    atomicAdd(&acc[k][0], S0);
                    atomicAdd(&acc[k][1], S1);
                    atomicAdd(&acc[k][2], S2);
                    atomicAdd(&acc[k][3], S3);
                    atomicAdd(&acc[k][4], S4);
                    atomicAdd(&acc[k][5], S5);
                    S0 = S1 = S2 = S3 = S4 = S5 = 0.f;
                    do {
                        ++k;
                    } while (pre[k + 1] == pre[k]);
                    row = 0;
                    nrow = pre[k + 1] - pre[k];
                    p0 = par[k][0];
                    p1 = par[k][1];
                    yk = par[k][2].x;
                }
                const int y = static_cast<int>(yk) + row;
                ++row;
                const float dy = static_cast<float>(y) - p0.y;
                // x-interval of this row where the form r0.z dx^2 + 2 r0.w dx dy +
                // r1.x dy^2 can be <= cut_s (margin 1/64 px; the test below decides)
                const float bq = p0.w * dy;
                const float disc = fmaf(bq, bq, -p0.z * fmaf(p1.x * dy, dy, -cut_s));
                if (!(disc >= 0.f)) continue;
                const float sq = sqrtf(disc);
                const float xlo = fmaxf(ceilf(p0.x + (-bq - sq) * p1.y - 0.015625f), p1.z);
                const float xhi = fminf(floorf(p0.x + (-bq + sq) * p1.y + 0.015625f), p1.w);
                if (!(xlo <= xhi)) continue;
                const int xl = static_cast<int>(xlo), xh = static_cast<int>(xhi);
                const float b2 = 2.f * p0.w * dy, c0 = p1.x * dy * dy;
                const float *grow = &sg[y - y0][0];
                float R0 = 0.f, R1 = 0.f;  // this row's sums of ge and ge dx
                float dx = static_cast<float>(xl) - p0.x;
                for (int x = xl; x <= xh; ++x, dx += 1.f) {
                    const float nq = -(dx * fmaf(p0.z, dx, b2) + c0);
                    if (nq >= -cut_s) {
                        const float ge = grow[x - x0] * ex2_approx(nq);
                        const float tx = ge * dx;
                        R0 += ge;
                        R1 += tx;
                        S3 = fmaf(tx, dx, S3);
                    }
                }
                S0 += R0;
                S1 += R1;
                S2 = fmaf(R0, dy, S2);
                S4 = fmaf(R1, dy, S4);
                S5 = fmaf(R0 * dy, dy, S5);
            }
            atomicAdd(&acc[k][0], S0);
            atomicAdd(&acc[k][1], S1);
            atomicAdd(&acc[k][2], S2);
            atomicAdd(&acc[k][3], S3);
            atomicAdd(&acc[k][4], S4);
            atomicAdd(&acc[k][5], S5);
        }
        __syncwarp();
        // ---- one lane per key: the six gradients of its record
        if (rows > 0) {
            const float S0 = acc[lane][0], S1 = acc[lane][1], S2 = acc[lane][2];
            const float S3 = acc[lane][3], S4 = acc[lane][4], S5 = acc[lane][5];
            float *o = d_rec + r * 6;
            atomicAdd(o + 0, w * fmaf(A, S1, Bc * S2));
            atomicAdd(o + 1, w * fmaf(Bc, S1, Cc * S2));
            atomicAdd(o + 2, -0.5f * w * S3);
            atomicAdd(o + 3, -w * S4);
            atomicAdd(o + 4, -0.5f * w * S5);
            atomicAdd(o + 5, S0);
        }
        __syncwarp();  // par / pre / acc are rewritten for the next 32 keys
    }
}

// The record tensor map: rows of 8 FP32 (32 bytes), a box of one row (the
// gather's shape).
cudaError_t record_map(const float4 *rec, unsigned long long rows, CUtensorMap *m) {
    std::memset(m, 0, sizeof(*m));
    if (!rec || rows == 0) return cudaSuccess;  // no records: the map is never used
    EncodeTiledFn f = encode_tiled();
    if (!f) return cudaErrorSymbolNotFound;
    const cuuint64_t dims[2] = {8, rows};
    const cuuint64_t strides[1] = {32};
    const cuuint32_t box[2] = {8, 1};
    const cuuint32_t elem[2] = {1, 1};
    const CUresult r = f(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float4 *>(rec), dims,
                         strides, box, elem, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int TW, int TH, int CH, int PX, int BF>
cudaError_t launch_fwd_x(const float4 *rec, const uint32_t *gids, const uint32_t *offs,
                         const long long *n_keys, long long cap, int n, int Q, const GridView &g,
                         float *out, int *status, cudaStream_t st, const long long *qbase) {
    const size_t smem = g.tma && CH == 2 ? FwdSmem<TW * TH / PX, TH, BF, true>::bytes
                                         : FwdSmem<TW * TH / PX, TH, BF, false>::bytes;
    auto kern = g.tma ? (g.wrap ? render_kernel<TW, TH, CH, true, PX, BF, true>
                                : render_kernel<TW, TH, CH, false, PX, BF, true>)
                      : (g.wrap ? render_kernel<TW, TH, CH, true, PX, BF, false>
                                : render_kernel<TW, TH, CH, false, PX, BF, false>);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    // record rows the gathers may address: Q x n, or (multi-scene batches,
    // rows from the device-side query bases) up to the int32 row limit
    const unsigned long long rows =
        qbase ? 0x7fffffffull : static_cast<unsigned long long>(Q) * static_cast<unsigned>(n);
    if (rows > 0x7fffffffull) return cudaErrorInvalidValue;
    CUtensorMap rmap;  // used by the TMA staging only
    if ((e = record_map(g.tma ? rec : nullptr, rows, &rmap)) != cudaSuccess) return e;
    // CTAs in tile-major order: the grid is Q x T, query fastest, so one tile
    // position runs for all queries, then the next (0.914 -> 0.880 ms on 20k
    // Gaussians x 256 TX, 360 x 90, 32 x 16 tiles); T <= 3000 (grid check)
    const dim3 grid(Q, g.T);
    // two channels: the imaginary weights follow the Q x N records
    const float *rec_im =
        CH == 2 ? reinterpret_cast<const float *>(rec + 2 * static_cast<size_t>(Q) * n) : nullptr;
    kern<<<grid, TW * TH / PX, smem, st>>>(rec, gids, offs, n_keys, cap, n, g,
                                           -g.q_cut * kHalfLog2e, out, status, rec_im, qbase,
                                           rmap);
    return cudaGetLastError();
}

// The rasteriser's knobs (pixels per thread, records per thread per batch):
// every combination (PX = 4 needs tiles at least 16 wide).
template <int TW, int TH, int CH>
cudaError_t launch_fwd(const float4 *rec, const uint32_t *gids, const uint32_t *offs,
                       const long long *n_keys, long long cap, int n, int Q, const GridView &g,
                       float *out, int *status, cudaStream_t st, const long long *qbase) {
    if (g.px == 2 && g.bpt == 1)
        return launch_fwd_x<TW, TH, CH, 2, 1>(rec, gids, offs, n_keys, cap, n, Q, g, out, status, st, qbase);
    if (g.px == 2 && g.bpt == 2)
        return launch_fwd_x<TW, TH, CH, 2, 2>(rec, gids, offs, n_keys, cap, n, Q, g, out, status, st, qbase);
    if constexpr (TW >= 16) {
        if (g.px == 4 && g.bpt == 1)
            return launch_fwd_x<TW, TH, CH, 4, 1>(rec, gids, offs, n_keys, cap, n, Q, g, out, status, st, qbase);
        if (g.px == 4 && g.bpt == 2)
            return launch_fwd_x<TW, TH, CH, 4, 2>(rec, gids, offs, n_keys, cap, n, Q, g, out, status, st, qbase);
    }
    return cudaErrorInvalidValue;
}

template <int CH>
cudaError_t launch_any(const float4 *rec, const uint32_t *gids, const uint32_t *offsets,
                       const long long *n_keys, long long cap, int n, int Q, const GridView &g,
                       float *out, int *status, cudaStream_t st, const long long *qb) {
    if (Q == 0) return cudaSuccess;
    if (g.tw == 8 && g.th == 8) return launch_fwd<8, 8, CH>(rec, gids, offsets, n_keys, cap, n, Q, g, out, status, st, qb);
    if (g.tw == 16 && g.th == 8) return launch_fwd<16, 8, CH>(rec, gids, offsets, n_keys, cap, n, Q, g, out, status, st, qb);
    if (g.tw == 16 && g.th == 16) return launch_fwd<16, 16, CH>(rec, gids, offsets, n_keys, cap, n, Q, g, out, status, st, qb);
    if (g.tw == 32 && g.th == 8) return launch_fwd<32, 8, CH>(rec, gids, offsets, n_keys, cap, n, Q, g, out, status, st, qb);
    if (g.tw == 32 && g.th == 16) return launch_fwd<32, 16, CH>(rec, gids, offsets, n_keys, cap, n, Q, g, out, status, st, qb);
    return cudaErrorInvalidValue;
}

template <int TW, int TH>
cudaError_t launch_bwd(const float4 *rec, const uint32_t *gids, const uint32_t *offs,
                       const long long *n_keys, long long cap, int n, int Q, const GridView &g,
                       const float *dA, float *d_rec, cudaStream_t st) {
    const dim3 grid(Q, g.T);  // tile-major, as the forward
    render_bwd_kernel<TW, TH><<<grid, 128, 0, st>>>(rec, gids, offs, n_keys, cap, n, g,
                                                    g.q_cut * kHalfLog2e, dA, d_rec);
    return cudaGetLastError();
}

}  // namespace

// cuTensorMapEncodeTiled, fetched from the driver at the first use (the
// library does not link libcuda).
EncodeTiledFn encode_tiled() {
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult r;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                             &r) == cudaSuccess &&
            r == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(f);
    });
    return fn;
}

bool render_config_supported(int tw, int th) {
    return (tw == 8 && th == 8) || (tw == 16 && th == 8) || (tw == 16 && th == 16) ||
           (tw == 32 && th == 8) || (tw == 32 && th == 16);
}

cudaError_t launch_render(const float4 *rec, const uint32_t *gids, const uint32_t *offsets,
                          const long long *n_keys, long long cap, int n, int Q,
                          const GridView &g, float *out, int *status, cudaStream_t st,
                          const long long *qbase) {
    return launch_any<1>(rec, gids, offsets, n_keys, cap, n, Q, g, out, status, st, qbase);
}

cudaError_t launch_render_complex(const float4 *rec, const uint32_t *gids,
                                  const uint32_t *offsets, const long long *n_keys, long long cap,
                                  int n, int Q, const GridView &g, float *out, int *status,
                                  cudaStream_t st) {
    return launch_any<2>(rec, gids, offsets, n_keys, cap, n, Q, g, out, status, st, nullptr);
}

cudaError_t launch_render_bwd(const float4 *rec, const uint32_t *gids, const uint32_t *offsets,
                              const long long *n_keys, long long cap, int n, int Q,
                              const GridView &g, const float *dA, float *d_rec, int *status,
                              cudaStream_t st) {
    (void)status;
    if (Q == 0) return cudaSuccess;
    if (g.tw == 8 && g.th == 8) return launch_bwd<8, 8>(rec, gids, offsets, n_keys, cap, n, Q, g, dA, d_rec, st);
    if (g.tw == 16 && g.th == 8) return launch_bwd<16, 8>(rec, gids, offsets, n_keys, cap, n, Q, g, dA, d_rec, st);
    if (g.tw == 16 && g.th == 16) return launch_bwd<16, 16>(rec, gids, offsets, n_keys, cap, n, Q, g, dA, d_rec, st);
    if (g.tw == 32 && g.th == 8) return launch_bwd<32, 8>(rec, gids, offsets, n_keys, cap, n, Q, g, dA, d_rec, st);
    if (g.tw == 32 && g.th == 16) return launch_bwd<32, 16>(rec, gids, offsets, n_keys, cap, n, Q, g, dA, d_rec, st);
    return cudaErrorInvalidValue;
}

}  // namespace wrf
