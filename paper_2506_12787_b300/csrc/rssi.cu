// RSSI head (Sec. 7.2): the spectrum map of a query, rendered from a small
// scene (the paper uses 50 Gaussians on a 16 x 16 map), reduced by a global
// average pool to one value; RSSI is the spectrum magnitude averaged over
// azimuth and elevation (Sec. 6.6).
//
// In this tiny-N regime the whole path is latency-bound, so one CTA per query
// runs every step in one launch, with nothing in HBM between them:
//   1. layer 1 from the factorised terms U[n] + V[q] (prep.cu, FP32), ReLU;
//   2. hidden layers in FP32 on the CUDA cores as a register-tiled product:
//      the scene's rows are padded to 64, activations are kept transposed
//      ([input k][row]) in shared memory, and thread t owns the 4 x 8 output
//      tile rows 4 (t % 16) .. +3, columns 8 (t / 16) .. +7, so each input k
//      costs one 16-byte activation load and two 16-byte weight loads for 32
//      independent FMAs; the layer's transposed FP32 weights are staged into
//      shared memory 64 inputs (32 KB) at a time with coalesced 16-byte loads.
//      Each output still sums bias + w_k h_k in ascending k;
//   3. the output layer and the deform + project step (Eq. 12-13) per
//      Gaussian, records kept in shared memory;
//   4. every pixel against every Gaussian in ascending id with the q <= q_cut
//      footprint test (Eq. 9/13), one thread per pixel;
//   5. the magnitudes summed in a fixed order (per-thread pixel order, then a
//      shared-memory tree), divided by H W.
// The pooled value does not depend on the other queries of the launch.
#include "kernels.h"

namespace wrf {

namespace {

constexpr int kThreads = 256;
constexpr int kKChunk = 64;  // weight rows (inputs) staged per pass: 32 KB
constexpr int kRows = kRssiMaxN;       // rows padded to 64
constexpr int kPitch = kRows + 4;      // floats per input of the transposed activations

struct RssiArgs {
    SceneView s;
    MlpView m;
    GridView g;
    const float *U;   // [N][128] W0[:, :dm] gamma(mean_n)
    const float *V;   // [Q][128] W0[:, dm:] gamma(tx_q) + b0
    const float *wt;  // hidden layers transposed [l][k][j]
    const float *wo;  // output layer transposed [k][8]
    int nh;
    float *rssi;      // [Q]
    float *map;       // [Q][H][W] or null
};

__global__ void __launch_bounds__(kThreads) rssi_kernel(RssiArgs a) {
    // [kKChunk][128] staged weights, then two [128][kPitch] transposed activations
    extern __shared__ __align__(16) float smem[];
    float *wbuf = smem;
    float *hin = smem + kKChunk * WRF_HIDDEN, *hout = hin + WRF_HIDDEN * kPitch;
    __shared__ float4 recs[kRssiMaxN][2];
    __shared__ float wims[kRssiMaxN];  // imaginary weights (two channels)
    __shared__ float dout[kRssiMaxN][8];
    __shared__ float red[kThreads];
    const int q = blockIdx.x, tid = threadIdx.x, N = a.s.n;

    // 1. layer 1: h[r][j] = relu(U[r][j] + V[q][j]), stored as hin[j][r]
    //    (rows >= N are zero; loads unrolled so they are in flight together)
    const float *vq = a.V + static_cast<size_t>(q) * WRF_HIDDEN;
    const float vj = vq[tid & (WRF_HIDDEN - 1)];
#pragma unroll
    for (int c = 0; c < kRows * WRF_HIDDEN / kThreads; ++c) {
        const int e = tid + c * kThreads, r = e >> 7, j = e & (WRF_HIDDEN - 1);
        hin[j * kPitch + r] = r < N ? fmaxf(__ldg(a.U + e) + vj, 0.f) : 0.f;
    }
    // 2. hidden layers: thread tile rows 4 rg .. 4 rg + 3, columns 8 cg .. 8 cg + 7;
    //    the next 32 KB weight chunk is loaded into registers while the
    //    current one is used
    const int rg = tid & 15, cg = tid >> 4;
    constexpr int kPer = kKChunk * WRF_HIDDEN / 4 / kThreads;  // float4 per thread per chunk
    float4 pre[kPer];
    auto load_chunk = [&](int l, int k0) {
        const float4 *src = reinterpret_cast<const float4 *>(
            a.wt + static_cast<size_t>(l) * WRF_HIDDEN * WRF_HIDDEN) + k0 * (WRF_HIDDEN / 4);
#pragma unroll
        for (int c = 0; c < kPer; ++c) pre[c] = __ldg(src + tid + c * kThreads);
    };
    if (a.nh > 0) load_chunk(0, 0);
    for (int l = 0; l < a.nh; ++l) {
        float acc[4][8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const float b = a.m.bh[l][8 * cg + c];
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[r][c] = b;
        }
        for (int k0 = 0; k0 < WRF_HIDDEN; k0 += kKChunk) {
            __syncthreads();  // the previous chunk (or layer's outputs) is done with
#pragma unroll
            for (int c = 0; c < kPer; ++c)
                reinterpret_cast<float4 *>(wbuf)[tid + c * kThreads] = pre[c];
            __syncthreads();
            if (k0 + kKChunk < WRF_HIDDEN)
                load_chunk(l, k0 + kKChunk);
            else if (l + 1 < a.nh)
                load_chunk(l + 1, 0);
#pragma unroll 4
            for (int k = 0; k < kKChunk; ++k) {
                const float4 hv = *reinterpret_cast<const float4 *>(hin + (k0 + k) * kPitch + 4 * rg);
                const float4 wa = *reinterpret_cast<const float4 *>(wbuf + k * WRF_HIDDEN + 8 * cg);
                const float4 wb = *reinterpret_cast<const float4 *>(wbuf + k * WRF_HIDDEN + 8 * cg + 4);
                const float h[4] = {hv.x, hv.y, hv.z, hv.w};
                const float w[8] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w};
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int c = 0; c < 8; ++c) acc[r][c] = fmaf(w[c], h[r], acc[r][c]);
            }
        }
#pragma unroll
        for (int c = 0; c < 8; ++c)
            *reinterpret_cast<float4 *>(hout + (8 * cg + c) * kPitch + 4 * rg) =
                make_float4(fmaxf(acc[0][c], 0.f), fmaxf(acc[1][c], 0.f), fmaxf(acc[2][c], 0.f),
                            fmaxf(acc[3][c], 0.f));
        float *t = hin;
        hin = hout;
        hout = t;
    }
    __syncthreads();
    // 3. output layer (5 residuals per Gaussian; its 4 KB transposed weights
    //    staged in shared memory first), then deform + project
    for (int i = tid; i < WRF_HIDDEN * 8 / 4; i += kThreads)
        reinterpret_cast<float4 *>(wbuf)[i] = __ldg(reinterpret_cast<const float4 *>(a.wo) + i);
    __syncthreads();
    for (int e = tid; e < N * 8; e += kThreads) {
        const int r = e >> 3, o = e & 7;
        if (o < WRF_OUT) {
            float acc = a.m.bo[o];
            for (int k = 0; k < WRF_HIDDEN; ++k) acc = fmaf(wbuf[k * 8 + o], hin[k * kPitch + r], acc);
            dout[r][o] = acc;
        }
    }
    __syncthreads();
    if (tid < N) {
        float4 r0, r1;
        const GaussParams p = load_params(a.s, tid);
        project_geom(p, dout[tid][0], dout[tid][1], dout[tid][2], dout[tid][3], dout[tid][4], a.g,
                     r0, r1);
        recs[tid][0] = r0;
        recs[tid][1] = r1;
        wims[tid] = weight_im(p);
    }
    __syncthreads();
    // 4. every pixel against every Gaussian (ascending id), footprint test
    //    -q' >= -q_cut log2(e)/2 with q' = q log2(e)/2 from the pre-scaled conic
    const int HW = a.g.H * a.g.W;
    const float ncut = -a.g.q_cut * kHalfLog2e;
    float part = 0.f;
    for (int p = tid; p < HW; p += kThreads) {
        const float x = static_cast<float>(p % a.g.W), y = static_cast<float>(p / a.g.W);
        float acc = 0.f, acc_im = 0.f;
        for (int n = 0; n < N; ++n) {
            const float4 r0 = recs[n][0], r1 = recs[n][1];
            float dx = x - r0.x;
            const float dy = y - r0.y;
            if (a.g.wrap) dx -= static_cast<float>(a.g.W) * rintf(dx / static_cast<float>(a.g.W));
            const float t = fmaf(r0.z, dx, 2.f * r0.w * dy);
            const float nq = -fmaf(dx, t, r1.x * dy * dy);
            if (nq >= ncut) {
                const float e = ex2_approx(nq);
                acc = fmaf(r1.y, e, acc);
                acc_im = fmaf(wims[n], e, acc_im);
            }
        }
        // magnitude of the (one- or two-channel) value
        const float mag = a.s.channels == 2 ? sqrtf(fmaf(acc, acc, acc_im * acc_im)) : fabsf(acc);
        if (a.map) a.map[static_cast<size_t>(q) * HW + p] = a.s.channels == 2 ? mag : acc;
        part += mag;
    }
    // 5. fixed-order reduction
    red[tid] = part;
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
        if (tid < s) red[tid] += red[tid + s];
        __syncthreads();
    }
    if (tid == 0) a.rssi[q] = red[0] / static_cast<float>(HW);
}

}  // namespace

cudaError_t launch_rssi(const SceneView &s, const MlpView &m, const GridView &g, int Q,
                        const DeformWs &ws, float *rssi, float *map, cudaStream_t st) {
    if (Q == 0) return cudaSuccess;
    if (s.n > kRssiMaxN || m.n_layers < 2) return cudaErrorInvalidValue;
    RssiArgs a{};
    a.s = s;
    a.m = m;
    a.g = g;
    a.U = ws.U;
    a.V = ws.V;
    a.wt = ws.wt_f32;
    a.wo = ws.wo_f32;
    a.nh = m.n_layers - 2;
    a.rssi = rssi;
    a.map = map;
    const size_t smem = (static_cast<size_t>(kKChunk) * WRF_HIDDEN + 2 * WRF_HIDDEN * kPitch) * 4;
    cudaError_t e = cudaFuncSetAttribute(rssi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    rssi_kernel<<<Q, kThreads, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace wrf
