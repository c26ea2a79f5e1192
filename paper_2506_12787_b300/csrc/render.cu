// Tile rasteriser for the order-free Gaussian sum (Sec. 4.1 Eq. 8-9,
// Sec. 4.2 Eq. 13) and its backward.
//
// Forward: one CTA per (tile, query).  The tile's Gaussian list (ascending
// id) is streamed through shared memory in batches of NT records: every
// thread issues one 32-byte cp.async.bulk (TMA bulk copy) for one record,
// completion is counted in bytes on an mbarrier, and two buffers alternate so
// the next batch lands while the current one is evaluated.  Each thread owns
// a column of PPT consecutive pixels and walks them with an incremental
// quadratic form (two adds per pixel); a warp skips a Gaussian whose bounding
// box misses the warp's pixel block, and a pixel adds w * 2^(-q') only when
// q <= q_cut.  The finished tile goes through shared memory to float4 stores.
//
// Backward: one CTA per (tile, query); the tile's dL/dA is staged in shared
// memory and each thread takes one Gaussian of the list, walks the pixels of
// its bounding box inside the tile, recomputes exp(-q/2) and accumulates
// dL/d(mx, my, A, B, C, w), then adds them to the per-(query, Gaussian)
// gradient with atomics (a Gaussian spans several tiles).
#include "kernels.h"

namespace wrf {

namespace {

template <int TW, int TH, int PPT>
__global__ void __launch_bounds__(TW *TH / PPT) render_kernel(
    const float4 *__restrict__ rec, const uint32_t *__restrict__ gids,
    const uint32_t *__restrict__ offs, const long long *__restrict__ n_keys, long long cap, int n,
    GridView g, float cut_s, float *__restrict__ out, int *status) {
    constexpr int NT = TW * TH / PPT;
    constexpr int B = NT;
    __shared__ __align__(128) float4 srec[2][B][2];
    __shared__ __align__(16) float stile[TH][TW];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ int abort_flag;

    const int t = blockIdx.x, q = blockIdx.y;
    const int x0 = (t % g.ntx) * TW, y0 = (t / g.ntx) * TH;
    const int lx = threadIdx.x % TW, ly = (threadIdx.x / TW) * PPT;
    const float px = static_cast<float>(x0 + lx), py = static_cast<float>(y0 + ly);
    // pixel block of this warp (used to skip Gaussians that cannot reach it)
    const int tid0 = threadIdx.x & ~31, tid1 = tid0 + 31;
    float wx0, wx1;
    if (TW >= 32) {
        wx0 = static_cast<float>(x0 + tid0 % TW);
        wx1 = wx0 + 31.f;
    } else {
        wx0 = static_cast<float>(x0);
        wx1 = static_cast<float>(x0 + TW - 1);
    }
    const float wy0 = static_cast<float>(y0 + (tid0 / TW) * PPT);
    const float wy1 = static_cast<float>(y0 + (tid1 / TW) * PPT + PPT - 1);

    uint32_t s0 = 0, s1 = 0;
    if (*n_keys <= cap) {
        s0 = offs[static_cast<size_t>(q) * g.T + t];
        s1 = offs[static_cast<size_t>(q) * g.T + t + 1];
    }
    const int total = static_cast<int>(s1 - s0);
    const int nb = (total + B - 1) / B;
    const float4 *qrec = rec + static_cast<size_t>(q) * n * 2;

    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
        abort_flag = 0;
        for (int b = 0; b < 2 && b < nb; ++b)
            mbar_arrive_expect_tx(&bar[b], static_cast<uint32_t>(min(B, total - b * B)) * 32u);
    }
    __syncthreads();
    for (int b = 0; b < 2 && b < nb; ++b) {
        int i = threadIdx.x;
        if (i < total - b * B) {
            uint32_t gid = gids[s0 + b * B + i];
            bulk_g2s(&srec[b][i][0], qrec + 2 * static_cast<size_t>(gid), 32, &bar[b]);
        }
    }

    float acc[PPT];
#pragma unroll
    for (int j = 0; j < PPT; ++j) acc[j] = 0.f;
    const float ncut = -cut_s;
    int b = 0;
    for (; b < nb; ++b) {
        const int buf = b & 1;
        if (!mbar_wait(&bar[buf], (b >> 1) & 1, status)) abort_flag = 1;
        const int cnt = min(B, total - b * B);
        for (int i = 0; i < cnt; ++i) {
            const float4 r0 = srec[buf][i][0];
            const float4 r1 = srec[buf][i][1];
            if (r0.x + r1.z < wx0 || r0.x - r1.z > wx1 || r0.y + r1.w < wy0 ||
                r0.y - r1.w > wy1)
                continue;
            const float dx = px - r0.x, dy = py - r0.y;
            float nq = -(dx * fmaf(r0.z, dx, 2.f * r0.w * dy) + r1.x * dy * dy);
            float step = -(2.f * fmaf(r0.w, dx, r1.x * dy) + r1.x);
            const float step2 = -2.f * r1.x;
#pragma unroll
            for (int j = 0; j < PPT; ++j) {
                if (nq >= ncut) acc[j] = fmaf(r1.y, ex2_approx(nq), acc[j]);
                nq += step;
                step += step2;
            }
        }
        if (threadIdx.x == 0 && b + 2 < nb)
            mbar_arrive_expect_tx(&bar[buf], static_cast<uint32_t>(min(B, total - (b + 2) * B)) * 32u);
        __syncthreads();
        if (abort_flag) break;
        if (b + 2 < nb) {
            int i = threadIdx.x;
            if (i < total - (b + 2) * B) {
                uint32_t gid = gids[s0 + (b + 2) * B + i];
                bulk_g2s(&srec[buf][i][0], qrec + 2 * static_cast<size_t>(gid), 32, &bar[buf]);
            }
        }
    }
    if (abort_flag) {
        // drain copies still in flight (batches b and b+1; bounded) before the CTA exits
        for (int bb = b; bb < nb && bb <= b + 1; ++bb) mbar_wait(&bar[bb & 1], (bb >> 1) & 1, status);
        return;
    }
#pragma unroll
    for (int j = 0; j < PPT; ++j) stile[ly + j][lx] = acc[j];
    __syncthreads();
    float *oq = out + static_cast<size_t>(q) * g.H * g.W;
    const bool vec = (g.W & 3) == 0;
    for (int i = threadIdx.x; i < TH * TW / 4; i += NT) {
        const int r = i / (TW / 4), c4 = (i % (TW / 4)) * 4;
        const int y = y0 + r, x = x0 + c4;
        if (y >= g.H || x >= g.W) continue;
        const float4 v = *reinterpret_cast<const float4 *>(&stile[r][c4]);
        float *dst = oq + static_cast<size_t>(y) * g.W + x;
        if (vec) {
            *reinterpret_cast<float4 *>(dst) = v;
        } else {
            const float vv[4] = {v.x, v.y, v.z, v.w};
            for (int k = 0; k < 4 && x + k < g.W; ++k) dst[k] = vv[k];
        }
    }
}

template <int TW, int TH>
__global__ void __launch_bounds__(128) render_bwd_kernel(
    const float4 *__restrict__ rec, const uint32_t *__restrict__ gids,
    const uint32_t *__restrict__ offs, const long long *__restrict__ n_keys, long long cap, int n,
    GridView g, float cut_s, const float *__restrict__ dA, float *__restrict__ d_rec) {
    __shared__ float sg[TH][TW];
    const int t = blockIdx.x, q = blockIdx.y;
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
    for (uint32_t i = s0 + threadIdx.x; i < s1; i += blockDim.x) {
        const uint32_t gid = gids[i];
        const size_t r = static_cast<size_t>(q) * n + gid;
        const float4 r0 = rec[2 * r], r1 = rec[2 * r + 1];
        int xa = max(x0, static_cast<int>(ceilf(fmaxf(r0.x - r1.z, static_cast<float>(x0)))));
        int xb = min(xe, static_cast<int>(floorf(fminf(r0.x + r1.z, static_cast<float>(xe)))));
        int ya = max(y0, static_cast<int>(ceilf(fmaxf(r0.y - r1.w, static_cast<float>(y0)))));
        int yb = min(ye, static_cast<int>(floorf(fminf(r0.y + r1.w, static_cast<float>(ye)))));
        const float A = r0.z * inv, Bc = r0.w * inv, Cc = r1.x * inv, w = r1.y;
        float gmx = 0.f, gmy = 0.f, gA = 0.f, gB = 0.f, gC = 0.f, gw = 0.f;
        for (int y = ya; y <= yb; ++y) {
            const float dy = static_cast<float>(y) - r0.y;
            for (int x = xa; x <= xb; ++x) {
                const float dx = static_cast<float>(x) - r0.x;
                const float nq = -(dx * fmaf(r0.z, dx, 2.f * r0.w * dy) + r1.x * dy * dy);
                if (!(nq >= -cut_s)) continue;
                const float e = ex2_approx(nq);
                const float gp = sg[y - y0][x - x0];
                const float ge = gp * e, gwe = ge * w;
                gw += ge;
                gmx = fmaf(gwe, fmaf(A, dx, Bc * dy), gmx);
                gmy = fmaf(gwe, fmaf(Bc, dx, Cc * dy), gmy);
                gA = fmaf(-0.5f * gwe, dx * dx, gA);
                gB = fmaf(-gwe, dx * dy, gB);
                gC = fmaf(-0.5f * gwe, dy * dy, gC);
            }
        }
        float *o = d_rec + r * 6;
        atomicAdd(o + 0, gmx);
        atomicAdd(o + 1, gmy);
        atomicAdd(o + 2, gA);
        atomicAdd(o + 3, gB);
        atomicAdd(o + 4, gC);
        atomicAdd(o + 5, gw);
    }
}

template <int TW, int TH, int PPT>
cudaError_t launch_fwd(const float4 *rec, const uint32_t *gids, const uint32_t *offs,
                       const long long *n_keys, long long cap, int n, int Q, const GridView &g,
                       float *out, int *status, cudaStream_t st) {
    dim3 grid(g.T, Q);
    render_kernel<TW, TH, PPT><<<grid, TW * TH / PPT, 0, st>>>(rec, gids, offs, n_keys, cap, n, g,
                                                               g.q_cut * kHalfLog2e, out, status);
    return cudaGetLastError();
}

template <int TW, int TH>
cudaError_t launch_bwd(const float4 *rec, const uint32_t *gids, const uint32_t *offs,
                       const long long *n_keys, long long cap, int n, int Q, const GridView &g,
                       const float *dA, float *d_rec, cudaStream_t st) {
    dim3 grid(g.T, Q);
    render_bwd_kernel<TW, TH><<<grid, 128, 0, st>>>(rec, gids, offs, n_keys, cap, n, g,
                                                    g.q_cut * kHalfLog2e, dA, d_rec);
    return cudaGetLastError();
}

}  // namespace

bool render_config_supported(int tw, int th) {
    return (tw == 8 && th == 8) || (tw == 16 && th == 8) || (tw == 16 && th == 16) ||
           (tw == 32 && th == 8) || (tw == 32 && th == 16);
}

cudaError_t launch_render(const float4 *rec, const uint32_t *gids, const uint32_t *offsets,
                          const long long *n_keys, long long cap, int n, int Q,
                          const GridView &g, float *out, int *status, cudaStream_t st) {
    if (Q == 0) return cudaSuccess;
    if (g.tw == 8 && g.th == 8) return launch_fwd<8, 8, 2>(rec, gids, offsets, n_keys, cap, n, Q, g, out, status, st);
    if (g.tw == 16 && g.th == 8) return launch_fwd<16, 8, 2>(rec, gids, offsets, n_keys, cap, n, Q, g, out, status, st);
    if (g.tw == 16 && g.th == 16) return launch_fwd<16, 16, 4>(rec, gids, offsets, n_keys, cap, n, Q, g, out, status, st);
    if (g.tw == 32 && g.th == 8) return launch_fwd<32, 8, 2>(rec, gids, offsets, n_keys, cap, n, Q, g, out, status, st);
    if (g.tw == 32 && g.th == 16) return launch_fwd<32, 16, 4>(rec, gids, offsets, n_keys, cap, n, Q, g, out, status, st);
    return cudaErrorInvalidValue;
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
