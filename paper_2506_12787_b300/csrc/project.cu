// Deformation + projection of every (query, Gaussian) row (Sec. 4.2
// Eq. 12-13) and its backward.
#include "kernels.h"

namespace wrf {

namespace {

__global__ void project_kernel(SceneView s, const float *resid, int Q, GridView g, float4 *rec,
                               uint32_t *count, float *rec_im) {
    const long long rows = static_cast<long long>(Q) * s.n;
    for (long long r = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; r < rows;
         r += static_cast<long long>(gridDim.x) * blockDim.x) {
        int n = static_cast<int>(r % s.n);
        float d[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
        if (resid) {
#pragma unroll
            for (int j = 0; j < 5; ++j) d[j] = resid[r * 5 + j];
        }
        float4 a, b;
        const GaussParams p = load_params(s, n);
        project_geom(p, d[0], d[1], d[2], d[3], d[4], g, a, b);
        rec[2 * r] = a;
        rec[2 * r + 1] = b;
        if (rec_im) rec_im[r] = weight_im(p);
        if (count) count[r] = record_tiles(a, b, g);
    }
}

// Chain rule of project_geom for one row: from dL/d(mx, my, A, B, C, w) to
// dL/d(dx, dy, drot, dls1, dls2) and dL/d(opacity_logit, amp).
//   A = c^2 i1 + s^2 i2, B = cs (i1 - i2), C = s^2 i1 + c^2 i2, i_k = e^{-2 l_k}
//   dA/dth = -2cs(i1-i2), dB/dth = (c^2-s^2)(i1-i2), dC/dth = 2cs(i1-i2)
//   d/dl1 = -2 i1 (c^2, cs, s^2),  d/dl2 = -2 i2 (s^2, -cs, c^2)
__device__ __forceinline__ void project_grad_row(const SceneView &s, int n, const float *d,
                                                 const float *gr, float *out, float &g_op,
                                                 float &g_amp) {
    float th = s.rot[n] + (d ? d[2] : 0.f);
    float l1 = s.log_scale[2 * n] + (d ? d[3] : 0.f);
    float l2 = s.log_scale[2 * n + 1] + (d ? d[4] : 0.f);
    float sn, cs;
    sincosf(th, &sn, &cs);
    float i1 = expf(-2.f * l1), i2 = expf(-2.f * l2);
    float cc = cs * cs, ss = sn * sn, csn = cs * sn, di = i1 - i2;
    out[0] = gr[0];
    out[1] = gr[1];
    out[2] = gr[2] * (-2.f * csn * di) + gr[3] * ((cc - ss) * di) + gr[4] * (2.f * csn * di);
    out[3] = -2.f * i1 * (gr[2] * cc + gr[3] * csn + gr[4] * ss);
    out[4] = -2.f * i2 * (gr[2] * ss - gr[3] * csn + gr[4] * cc);
    float sg = 1.f / (1.f + expf(-s.opacity_logit[n]));
    g_op = gr[5] * s.amp[n] * sg * (1.f - sg);
    g_amp = gr[5] * sg;
}

// One thread per Gaussian, looping over queries: per-Gaussian sums are
// accumulated in registers in query order (deterministic), and d_resid rows
// are written as they are produced.
__global__ void project_bwd_kernel(SceneView s, const float *resid, int Q, const float *d_rec,
                                   float *d_resid, float *d_mean, float *d_ls, float *d_rot,
                                   float *d_op, float *d_amp) {
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= s.n) return;
    float acc[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int q = 0; q < Q; ++q) {
        long long r = static_cast<long long>(q) * s.n + n;
        float gr[6];
#pragma unroll
        for (int j = 0; j < 6; ++j) gr[j] = d_rec[r * 6 + j];
        float o[5], gop, gamp;
        project_grad_row(s, n, resid ? resid + r * 5 : nullptr, gr, o, gop, gamp);
        if (d_resid) {
#pragma unroll
            for (int j = 0; j < 5; ++j) d_resid[r * 5 + j] = o[j];
        }
#pragma unroll
        for (int j = 0; j < 5; ++j) acc[j] += o[j];
        acc[5] += gop;
        acc[6] += gamp;
    }
    d_mean[2 * n] = acc[0];
    d_mean[2 * n + 1] = acc[1];
    d_rot[n] = acc[2];
    d_ls[2 * n] = acc[3];
    d_ls[2 * n + 1] = acc[4];
    d_op[n] = acc[5];
    d_amp[n] = acc[6];
}

}  // namespace

cudaError_t launch_project(const SceneView &s, const float *resid, int Q, const GridView &g,
                           float4 *rec, uint32_t *count, cudaStream_t st) {
    long long rows = static_cast<long long>(Q) * s.n;
    if (rows == 0) return cudaSuccess;
    long long blocks = (rows + 255) / 256;
    if (blocks > 148 * 64) blocks = 148 * 64;
    // two channels: the imaginary weights follow the Q x N records
    float *rec_im = s.channels == 2 ? reinterpret_cast<float *>(rec + 2 * rows) : nullptr;
    project_kernel<<<static_cast<unsigned>(blocks), 256, 0, st>>>(s, resid, Q, g, rec, count,
                                                                  rec_im);
    return cudaGetLastError();
}

cudaError_t launch_project_bwd(const SceneView &s, const float *resid, int Q, const float *d_rec,
                               float *d_resid, float *d_mean, float *d_ls, float *d_rot,
                               float *d_op, float *d_amp, cudaStream_t st) {
    if (s.n == 0) return cudaSuccess;
    project_bwd_kernel<<<(s.n + 127) / 128, 128, 0, st>>>(s, resid, Q, d_rec, d_resid, d_mean,
                                                          d_ls, d_rot, d_op, d_amp);
    return cudaGetLastError();
}

}  // namespace wrf
