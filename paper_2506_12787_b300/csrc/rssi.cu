// RSSI head (Sec. 7.2): the spectrum map of a query, rendered from a small
// scene (the paper uses 50 Gaussians on a 16 x 16 map), reduced by a global
// average pool to one value; RSSI is the spectrum magnitude averaged over
// azimuth and elevation (Sec. 6.6).
//
// In this tiny-N regime the whole path is latency-bound, so one CTA per query
// runs every step in one launch, with nothing in HBM between them:
//   1. layer 1 from the factorised terms U[n] + V[q] (prep.cu, FP32), ReLU;
//   2. hidden layers in FP32 on the CUDA cores: thread (j, half) owns output
//      column j of the rows n = half, half + 2, ...; weights stream from the
//      transposed FP32 image (coalesced over j, L1/L2 resident), activations
//      are read from shared memory as broadcasts;
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
    extern __shared__ float hbuf[];  // [2][N][128] activations
    __shared__ float4 recs[kRssiMaxN][2];
    __shared__ float dout[kRssiMaxN][8];
    __shared__ float red[kThreads];
    const int q = blockIdx.x, tid = threadIdx.x, N = a.s.n;
    float *hin = hbuf, *hout = hbuf + N * WRF_HIDDEN;

    // 1. layer 1: relu(U[n] + V[q])
    const float *vq = a.V + static_cast<size_t>(q) * WRF_HIDDEN;
    for (int e = tid; e < N * WRF_HIDDEN; e += kThreads)
        hin[e] = fmaxf(a.U[e] + vq[e & (WRF_HIDDEN - 1)], 0.f);
    // 2. hidden layers
    const int j = tid & (WRF_HIDDEN - 1), half = tid >> 7;
    for (int l = 0; l < a.nh; ++l) {
        __syncthreads();
        const float bj = a.m.bh[l][j];
        float acc[kRssiMaxN / 2];
#pragma unroll
        for (int i = 0; i < kRssiMaxN / 2; ++i) acc[i] = bj;
        const float *w = a.wt + static_cast<size_t>(l) * WRF_HIDDEN * WRF_HIDDEN + j;
#pragma unroll 2
        for (int k = 0; k < WRF_HIDDEN; ++k) {
            const float wk = __ldg(w + k * WRF_HIDDEN);
#pragma unroll
            for (int i = 0; i < kRssiMaxN / 2; ++i) {
                const int r = 2 * i + half;
                if (r < N) acc[i] = fmaf(wk, hin[r * WRF_HIDDEN + k], acc[i]);
            }
        }
#pragma unroll
        for (int i = 0; i < kRssiMaxN / 2; ++i) {
            const int r = 2 * i + half;
            if (r < N) hout[r * WRF_HIDDEN + j] = fmaxf(acc[i], 0.f);
        }
        float *t = hin;
        hin = hout;
        hout = t;
    }
    __syncthreads();
    // 3. output layer (5 residuals per Gaussian), then deform + project
    for (int e = tid; e < N * 8; e += kThreads) {
        const int r = e >> 3, o = e & 7;
        if (o < WRF_OUT) {
            float acc = a.m.bo[o];
            const float *h = hin + r * WRF_HIDDEN;
            for (int k = 0; k < WRF_HIDDEN; ++k) acc = fmaf(__ldg(a.wo + k * 8 + o), h[k], acc);
            dout[r][o] = acc;
        }
    }
    __syncthreads();
    if (tid < N) {
        float4 r0, r1;
        project_params(load_params(a.s, tid), dout[tid][0], dout[tid][1], dout[tid][2],
                       dout[tid][3], dout[tid][4], a.g, r0, r1);
        recs[tid][0] = r0;
        recs[tid][1] = r1;
    }
    __syncthreads();
    // 4. every pixel against every Gaussian (ascending id), footprint test
    //    -q' >= -q_cut log2(e)/2 with q' = q log2(e)/2 from the pre-scaled conic
    const int HW = a.g.H * a.g.W;
    const float ncut = -a.g.q_cut * kHalfLog2e;
    float part = 0.f;
    for (int p = tid; p < HW; p += kThreads) {
        const float x = static_cast<float>(p % a.g.W), y = static_cast<float>(p / a.g.W);
        float acc = 0.f;
        for (int n = 0; n < N; ++n) {
            const float4 r0 = recs[n][0], r1 = recs[n][1];
            const float dx = x - r0.x, dy = y - r0.y;
            const float t = fmaf(r0.z, dx, 2.f * r0.w * dy);
            const float nq = -fmaf(dx, t, r1.x * dy * dy);
            if (nq >= ncut) acc = fmaf(r1.y, ex2_approx(nq), acc);
        }
        if (a.map) a.map[static_cast<size_t>(q) * HW + p] = acc;
        part += fabsf(acc);
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
    const size_t smem = static_cast<size_t>(2) * (s.n > 0 ? s.n : 1) * WRF_HIDDEN * 4;
    cudaError_t e = cudaFuncSetAttribute(rssi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    rssi_kernel<<<Q, kThreads, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace wrf
