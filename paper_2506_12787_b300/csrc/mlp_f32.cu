// Deformation MLP on the CUDA cores in FP32 (Sec. 4.2, Eq. 14).
//
// One CTA takes 32 (query, Gaussian) rows.  Activations live in shared
// memory column-major ([unit][row]) so that lane = row reads them without
// bank conflicts; warp w produces hidden units 32w..32w+31 for all 32 rows,
// reading the transposed weights as warp-uniform float4 broadcasts.
// Layer 1 starts from ReLU(U[n] + V[q]) (see prep.cu).  The epilogue either
// stores the residual row or deforms and projects the Gaussian in place.
#include "kernels.h"

namespace wrf {

namespace {

constexpr int kRows = 32;

__global__ void __launch_bounds__(128) mlp_f32_kernel(SceneView s, MlpView m, GridView g, int Q,
                                                      DeformWs ws, int mode, float *resid,
                                                      float4 *rec, uint32_t *count,
                                                      float *rec_im) {
    extern __shared__ __align__(16) float smem[];
    float *act0 = smem;                                   // [128][32]
    float *act1 = act0 + WRF_HIDDEN * kRows;              // [128][32]
    float *wt = act1 + WRF_HIDDEN * kRows;                // [128][128]
    float *wo = wt + WRF_HIDDEN * WRF_HIDDEN;             // [128][8]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long rows = static_cast<long long>(Q) * s.n;
    const long long r0 = static_cast<long long>(blockIdx.x) * kRows;

    // Layer 1: h1 = ReLU(U[n] + V[q]).  Lane = row; warp w fills units
    // 32w..32w+31 (each lane walks its own row of U, so the 128-byte line is
    // reused from L1 across the 32 iterations).
    {
        const long long row = r0 + lane;
        const bool ok = row < rows;
        const int q = ok ? static_cast<int>(row / s.n) : 0;
        const int n = ok ? static_cast<int>(row % s.n) : 0;
        const float *u = ws.U + static_cast<size_t>(n) * WRF_HIDDEN + warp * 32;
        const float *v = ws.V + static_cast<size_t>(q) * WRF_HIDDEN + warp * 32;
        for (int jj = 0; jj < 32; ++jj)
            act0[(warp * 32 + jj) * kRows + lane] = ok ? fmaxf(u[jj] + v[jj], 0.f) : 0.f;
    }
    for (int i = threadIdx.x; i < WRF_HIDDEN * 8 / 4; i += blockDim.x)
        reinterpret_cast<float4 *>(wo)[i] = reinterpret_cast<const float4 *>(ws.wo_f32)[i];

    float *in = act0, *out = act1;
    for (int l = 0; l < m.n_layers - 2; ++l) {
        __syncthreads();  // previous layer's activations and weight reads done
        const float4 *src = reinterpret_cast<const float4 *>(ws.wt_f32 +
                                                             static_cast<size_t>(l) * WRF_HIDDEN *
                                                                 WRF_HIDDEN);
        for (int i = threadIdx.x; i < WRF_HIDDEN * WRF_HIDDEN / 4; i += blockDim.x)
            reinterpret_cast<float4 *>(wt)[i] = src[i];
        __syncthreads();
        float acc[32];
        const float *bl = m.bh[l] + warp * 32;
#pragma unroll
        for (int jj = 0; jj < 32; ++jj) acc[jj] = bl[jj];
#pragma unroll 2
        for (int k = 0; k < WRF_HIDDEN; ++k) {
            float h = in[k * kRows + lane];
            const float4 *wk = reinterpret_cast<const float4 *>(wt + k * WRF_HIDDEN + warp * 32);
#pragma unroll
            for (int v4 = 0; v4 < 8; ++v4) {
                float4 w = wk[v4];
                acc[4 * v4 + 0] = fmaf(w.x, h, acc[4 * v4 + 0]);
                acc[4 * v4 + 1] = fmaf(w.y, h, acc[4 * v4 + 1]);
                acc[4 * v4 + 2] = fmaf(w.z, h, acc[4 * v4 + 2]);
                acc[4 * v4 + 3] = fmaf(w.w, h, acc[4 * v4 + 3]);
            }
        }
#pragma unroll
        for (int jj = 0; jj < 32; ++jj) out[(warp * 32 + jj) * kRows + lane] = fmaxf(acc[jj], 0.f);
        float *t = in;
        in = out;
        out = t;
    }
    __syncthreads();
    if (warp != 0) return;
    const long long row = r0 + lane;
    if (row >= rows) return;
    float o[WRF_OUT];
#pragma unroll
    for (int j = 0; j < WRF_OUT; ++j) o[j] = m.bo[j];
    for (int k = 0; k < WRF_HIDDEN; ++k) {
        float h = in[k * kRows + lane];
        float4 w0 = reinterpret_cast<const float4 *>(wo + k * 8)[0];
        float w4 = wo[k * 8 + 4];
        o[0] = fmaf(w0.x, h, o[0]);
        o[1] = fmaf(w0.y, h, o[1]);
        o[2] = fmaf(w0.z, h, o[2]);
        o[3] = fmaf(w0.w, h, o[3]);
        o[4] = fmaf(w4, h, o[4]);
    }
    if (mode == 0) {
        float *dst = resid + row * WRF_OUT;
#pragma unroll
        for (int j = 0; j < WRF_OUT; ++j) dst[j] = o[j];
    } else {
        int n = static_cast<int>(row % s.n);
        float4 a, b;
        const GaussParams p = load_params(s, n);
        project_geom(p, o[0], o[1], o[2], o[3], o[4], g, a, b);
        rec[2 * row] = a;
        rec[2 * row + 1] = b;
        if (rec_im) rec_im[row] = weight_im(p);
        if (count) count[row] = record_tiles(a, b, g);
    }
}

}  // namespace

cudaError_t launch_mlp_f32(const SceneView &s, const MlpView &m, const GridView &g, int Q,
                           const DeformWs &ws, int mode, float *resid, float4 *rec,
                           uint32_t *count, cudaStream_t st) {
    long long rows = static_cast<long long>(Q) * s.n;
    if (rows == 0) return cudaSuccess;
    size_t smem = (2 * WRF_HIDDEN * kRows + WRF_HIDDEN * WRF_HIDDEN + WRF_HIDDEN * 8) * 4;
    cudaError_t e = cudaFuncSetAttribute(mlp_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    long long blocks = (rows + kRows - 1) / kRows;
    // two channels: the imaginary weights follow the Q x N records
    float *rec_im = (mode == 1 && s.channels == 2) ? reinterpret_cast<float *>(rec + 2 * rows)
                                                   : nullptr;
    mlp_f32_kernel<<<static_cast<unsigned>(blocks), 128, smem, st>>>(s, m, g, Q, ws, mode, resid,
                                                                     rec, count, rec_im);
    return cudaGetLastError();
}

}  // namespace wrf
