// Deformation MLP on the CUDA cores in FP32 (Sec. 4.2, Eq. 14).
//
// A CTA takes ROWS consecutive (query, Gaussian) rows (64, or 32 for small
// problems so that more SMs take part).  Activations live in shared memory
// transposed ([unit][row], padded pitch), and thread t computes a 4-row x
// 8-unit register tile of every hidden layer: rows 4 (t % (ROWS/4)) .., units
// 8 (t / (ROWS/4)) ..; per input k it reads one float4 of activations and two
// float4 of weights for 32 FMAs.  The transposed weights ([k][unit]) stream
// through two shared buffers of 16 inputs each with cp.async, one chunk
// ahead of the products.  Every output sums its bias, then w_k h_k in
// ascending k.  Layer 1 starts from ReLU(U[n] + V[q]) (see prep.cu).  The
// epilogue evaluates the output layer and either stores the residual row or
// deforms and projects the Gaussian.  On request (training) every hidden
// activation is also stored, acts [layer][row][128] FP32, for the backward.
#include "kernels.h"

namespace wrf {

namespace {

constexpr int kH = WRF_HIDDEN;  // 128
constexpr int kKC = 16;         // inputs per staged weight chunk


template <int ROWS>
struct F32Cfg {
    static constexpr int RG = ROWS / 4;          // row groups
    static constexpr int THREADS = RG * (kH / 8);  // x 16 unit groups
    static constexpr int PITCH = ROWS + 4;       // floats per unit of the activations
    static constexpr size_t smem = (static_cast<size_t>(2 * kKC) * kH + 2 * kH * PITCH + kH * 8) * 4;
};

template <int ROWS>
__global__ void __launch_bounds__(F32Cfg<ROWS>::THREADS) mlp_f32_kernel(
    SceneView s, MlpView m, GridView g, int Q, DeformWs ws, int mode, float *resid, float4 *rec,
    uint32_t *count, float *rec_im, float *acts) {
    using C = F32Cfg<ROWS>;
    constexpr int T = C::THREADS, P = C::PITCH;
    extern __shared__ __align__(16) float smem[];
    float *wbuf = smem;                       // [2][kKC][kH]
    float *hin = wbuf + 2 * kKC * kH;         // [kH][P]
    float *hout = hin + kH * P;               // [kH][P]
    float *wo = hout + kH * P;                // [kH][8]
    __shared__ float dout[ROWS][8];
    const int tid = threadIdx.x;
    const int rg = tid % C::RG, cg = tid / C::RG;
    const long long rows = static_cast<long long>(Q) * s.n;
    const long long r0 = static_cast<long long>(blockIdx.x) * ROWS;
    const int nh = m.n_layers - 2;
    const int nchunk = nh * (kH / kKC);
    auto stage = [&](int c) {
        const int l = c / (kH / kKC), k0 = (c % (kH / kKC)) * kKC;
        const float4 *src = reinterpret_cast<const float4 *>(
            ws.wt_f32 + (static_cast<size_t>(l) * kH + k0) * kH);
        float4 *dst = reinterpret_cast<float4 *>(wbuf + (c & 1) * kKC * kH);
        for (int i = tid; i < kKC * kH / 4; i += T) cp_async16(dst + i, src + i);
        cp_async_commit();
    };
    if (nchunk > 0) stage(0);
    for (int i = tid; i < kH * 8 / 4; i += T)
        reinterpret_cast<float4 *>(wo)[i] = reinterpret_cast<const float4 *>(ws.wo_f32)[i];
    // layer 1: h = ReLU(U[n] + V[q]); lanes take consecutive rows (conflict-
    // free transposed stores), each loading 4 units
    for (int e = tid; e < ROWS * kH / 4; e += T) {
        const int r = e % ROWS, j4 = 4 * (e / ROWS);
        const long long row = r0 + r;
        float4 h = make_float4(0.f, 0.f, 0.f, 0.f);
        if (row < rows) {
            const int q = static_cast<int>(row / s.n), n = static_cast<int>(row % s.n);
            const float4 u = __ldg(reinterpret_cast<const float4 *>(ws.U + static_cast<size_t>(n) * kH + j4));
            const float4 v = __ldg(reinterpret_cast<const float4 *>(ws.V + static_cast<size_t>(q) * kH + j4));
            h = make_float4(fmaxf(u.x + v.x, 0.f), fmaxf(u.y + v.y, 0.f), fmaxf(u.z + v.z, 0.f),
                            fmaxf(u.w + v.w, 0.f));
        }
        if (acts && row < rows)
            *reinterpret_cast<float4 *>(acts + static_cast<size_t>(row) * kH + j4) = h;
        hin[(j4 + 0) * P + r] = h.x;
        hin[(j4 + 1) * P + r] = h.y;
        hin[(j4 + 2) * P + r] = h.z;
        hin[(j4 + 3) * P + r] = h.w;
    }
    float acc[4][8];
    for (int c = 0; c < nchunk; ++c) {
        const int l = c / (kH / kKC), kc = c % (kH / kKC);
        if (kc == 0) {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const float bv = __ldg(m.bh[l] + 8 * cg + j);
#pragma unroll
                for (int r = 0; r < 4; ++r) acc[r][j] = bv;
            }
        }
        // chunk c has landed for every thread, every thread is done with the
        // buffer the next chunk overwrites and with the previous layer
        cp_async_wait_all();
        __syncthreads();
        if (c + 1 < nchunk) stage(c + 1);
        const float *wb = wbuf + (c & 1) * kKC * kH;
        const float *hk = hin + kc * kKC * P;
#pragma unroll 8
        for (int k = 0; k < kKC; ++k) {
            const float4 hv = *reinterpret_cast<const float4 *>(hk + k * P + 4 * rg);
            const float4 wa = *reinterpret_cast<const float4 *>(wb + k * kH + 8 * cg);
            const float4 wc = *reinterpret_cast<const float4 *>(wb + k * kH + 8 * cg + 4);
            const float h[4] = {hv.x, hv.y, hv.z, hv.w};
            const float w[8] = {wa.x, wa.y, wa.z, wa.w, wc.x, wc.y, wc.z, wc.w};
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[r][j] = fmaf(w[j], h[r], acc[r][j]);
        }
        if (kc == kH / kKC - 1) {
#pragma unroll
            for (int j = 0; j < 8; ++j)
                *reinterpret_cast<float4 *>(hout + (8 * cg + j) * P + 4 * rg) =
                    make_float4(fmaxf(acc[0][j], 0.f), fmaxf(acc[1][j], 0.f),
                                fmaxf(acc[2][j], 0.f), fmaxf(acc[3][j], 0.f));
            if (acts) {
                float *al = acts + static_cast<size_t>(l + 1) * rows * kH;
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const long long row = r0 + 4 * rg + r;
                    if (row >= rows) continue;
                    float4 *dst = reinterpret_cast<float4 *>(al + static_cast<size_t>(row) * kH + 8 * cg);
                    dst[0] = make_float4(fmaxf(acc[r][0], 0.f), fmaxf(acc[r][1], 0.f),
                                         fmaxf(acc[r][2], 0.f), fmaxf(acc[r][3], 0.f));
                    dst[1] = make_float4(fmaxf(acc[r][4], 0.f), fmaxf(acc[r][5], 0.f),
                                         fmaxf(acc[r][6], 0.f), fmaxf(acc[r][7], 0.f));
                }
            }
            float *t = hin;
            hin = hout;
            hout = t;
        }
    }
    __syncthreads();
    // output layer: (row, output) pairs over the threads
    for (int i = tid; i < ROWS * WRF_OUT; i += T) {
        const int r = i / WRF_OUT, o = i % WRF_OUT;
        float a = __ldg(m.bo + o);
        for (int k = 0; k < kH; ++k) a = fmaf(wo[k * 8 + o], hin[k * P + r], a);
        dout[r][o] = a;
    }
    __syncthreads();
    if (tid >= ROWS) return;
    const long long row = r0 + tid;
    if (row >= rows) return;
    const float *o = dout[tid];
    if (mode == 0) {
        float *dst = resid + row * WRF_OUT;
#pragma unroll
        for (int j = 0; j < WRF_OUT; ++j) dst[j] = o[j];
    } else {
        const int n = static_cast<int>(row % s.n);
        float4 a, b;
        const GaussParams p = load_params(s, n);
        project_geom(p, o[0], o[1], o[2], o[3], o[4], g, a, b);
        rec[2 * row] = a;
        rec[2 * row + 1] = b;
        if (rec_im) rec_im[row] = weight_im(p);
        if (count) count[row] = record_tiles(a, b, g);
    }
}

template <int ROWS>
cudaError_t launch_rows(const SceneView &s, const MlpView &m, const GridView &g, int Q,
                        const DeformWs &ws, int mode, float *resid, float4 *rec, uint32_t *count,
                        float *rec_im, float *acts, long long rows, cudaStream_t st) {
    using C = F32Cfg<ROWS>;
    cudaError_t e = cudaFuncSetAttribute(mlp_f32_kernel<ROWS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(C::smem));
    if (e != cudaSuccess) return e;
    const long long blocks = (rows + ROWS - 1) / ROWS;
    mlp_f32_kernel<ROWS><<<static_cast<unsigned>(blocks), C::THREADS, C::smem, st>>>(
        s, m, g, Q, ws, mode, resid, rec, count, rec_im, acts);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_mlp_f32(const SceneView &s, const MlpView &m, const GridView &g, int Q,
                           const DeformWs &ws, int mode, float *resid, float4 *rec,
                           uint32_t *count, float *acts, cudaStream_t st) {
    const long long rows = static_cast<long long>(Q) * s.n;
    if (rows == 0) return cudaSuccess;
    // two channels: the imaginary weights follow the Q x N records
    float *rec_im = (mode == 1 && s.channels == 2) ? reinterpret_cast<float *>(rec + 2 * rows)
                                                   : nullptr;
    // small problems: 32-row CTAs so that more SMs take part
    if (rows < 148LL * 64 * 4)
        return launch_rows<32>(s, m, g, Q, ws, mode, resid, rec, count, rec_im, acts, rows, st);
    return launch_rows<64>(s, m, g, Q, ws, mode, resid, rec, count, rec_im, acts, rows, st);
}

}  // namespace wrf
