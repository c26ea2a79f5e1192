// Back-propagation through the deformation MLP (Sec. 4.2 Eq. 14-15; the
// paper fits all parameters by gradient descent, Sec. 4.4), FP32 on the
// CUDA cores.
//
// Given dL/d(resid) for every (query, Gaussian) row, produces dL/dW and
// dL/db of every layer and, unless positions are stop-gradded (the paper's
// fine stage, Sec. 4.4), the derivative through gamma(mean) added into
// d_mean.  Rows are processed in chunks of kChunk:
//   rows kernel  - 32 rows per CTA: recompute the forward activations
//                  (layer 1 from the exact split U[n] + V[q], see prep.cu),
//                  then walk the layers backwards, delta_l = (W_{l+1}^T
//                  delta_{l+1}) * [z_l > 0]; store every layer's input row
//                  H_l and pre-activation gradient G_l = delta_l in the chunk
//                  buffers; add W0m^T delta_1 through the derivative of the
//                  positional encoding into d_mean (atomics).
//   dW kernel    - dW_l += G_l^T H_{l-1} over the chunk's rows: 32 x 32
//                  output tiles, a slice of rows per CTA, shared-memory
//                  tiles of 32 rows, one atomic add per output per slice;
//                  the bias gradient is the same sum with H = 1.
#include "kernels.h"

namespace wrf {

namespace {

constexpr int kRows = 32;
constexpr int kChunk = 8192;

inline size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

// Chunk buffers, row-major [kChunk][width].
struct ChunkBufs {
    float *H0;        // [kChunk][din]   first-layer input [gamma(mean), gamma(tx)]
    float *Hh[7];     // [kChunk][128]   input of layer l (= activation h_l), l = 1..n_layers-1
    float *G[8];      // [kChunk][dout]  pre-activation gradient of layer l (G[L-1] width 5)
    float *gam_m;     // [N][dm]         gamma(mean_n)
    float *gam_t;     // [Q][dt]         gamma(tx_q)
};

// gamma tables (Eq. 15), same feature order and phase reduction as prep.cu.
__device__ void encode_row(const PeArg *x, int d, int L, float *out) {
    for (int i = 0; i < d; ++i) out[i] = pe_value(x[i]);
    for (int k = 0; k < L; ++k)
        for (int i = 0; i < d; ++i) {
            float s, c;
            pe_band(x[i], k, s, c);
            out[d + k * d + i] = s;
            out[d + L * d + k * d + i] = c;
        }
}

__global__ void gamma_tables_kernel(SceneView s, MlpView m, GridView g, const float *tx, int Q,
                                    float *gam_m, float *gam_t) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < s.n) {
        const float2 mu = reinterpret_cast<const float2 *>(s.mean)[i];
        const PeArg x[2] = {pe_arg(mu.x, 0.f, static_cast<float>(g.W)),
                            pe_arg(mu.y, 0.f, static_cast<float>(g.H))};
        encode_row(x, 2, m.L_mean, gam_m + static_cast<size_t>(i) * m.dm);
    } else if (i < s.n + Q) {
        const int q = i - s.n;
        PeArg x[3];
        for (int c = 0; c < 3; ++c) x[c] = pe_arg(tx[3 * q + c], m.room_min[c], m.room_size[c]);
        encode_row(x, 3, m.L_tx, gam_t + static_cast<size_t>(q) * m.dt);
    }
}

struct RowsArgs {
    SceneView s;
    MlpView m;
    GridView g;
    DeformWs fw;
    ChunkBufs cb;
    const float *d_resid;
    long long row0, nrows;  // rows of this chunk
    float *d_mean;          // null: stop-grad through gamma(mean)
};

// act layout in shared memory: [unit][row] (lane = row).
__global__ void __launch_bounds__(128) mlp_bwd_rows_kernel(RowsArgs a) {
    extern __shared__ __align__(16) float sm[];
    const int L = a.m.n_layers, nh = L - 2;
    float *h = sm;                               // [L-1][128][32] activations h_1..h_{L-1}
    float *dl = h + (L - 1) * WRF_HIDDEN * kRows;  // [2][128][32] deltas (ping-pong)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long lr = static_cast<long long>(blockIdx.x) * kRows + lane;  // row in chunk
    const long long row = a.row0 + lr;
    const bool ok = lr < a.nrows;
    const int q = ok ? static_cast<int>(row / a.s.n) : 0;
    const int n = ok ? static_cast<int>(row % a.s.n) : 0;

    // ---- forward recompute
    {
        const float *u = a.fw.U + static_cast<size_t>(n) * WRF_HIDDEN + warp * 32;
        const float *v = a.fw.V + static_cast<size_t>(q) * WRF_HIDDEN + warp * 32;
        for (int jj = 0; jj < 32; ++jj)
            h[(warp * 32 + jj) * kRows + lane] = ok ? fmaxf(u[jj] + v[jj], 0.f) : 0.f;
    }
    for (int l = 0; l < nh; ++l) {
        __syncthreads();
        const float *in = h + l * WRF_HIDDEN * kRows;
        float *out = h + (l + 1) * WRF_HIDDEN * kRows;
        const float *Wt = a.fw.wt_f32 + static_cast<size_t>(l) * WRF_HIDDEN * WRF_HIDDEN;  // [k][j]
        float acc[32];
#pragma unroll
        for (int jj = 0; jj < 32; ++jj) acc[jj] = a.m.bh[l][warp * 32 + jj];
        for (int k = 0; k < WRF_HIDDEN; ++k) {
            const float x = in[k * kRows + lane];
            const float4 *wk = reinterpret_cast<const float4 *>(Wt + k * WRF_HIDDEN + warp * 32);
#pragma unroll
            for (int v4 = 0; v4 < 8; ++v4) {
                const float4 w = wk[v4];
                acc[4 * v4 + 0] = fmaf(w.x, x, acc[4 * v4 + 0]);
                acc[4 * v4 + 1] = fmaf(w.y, x, acc[4 * v4 + 1]);
                acc[4 * v4 + 2] = fmaf(w.z, x, acc[4 * v4 + 2]);
                acc[4 * v4 + 3] = fmaf(w.w, x, acc[4 * v4 + 3]);
            }
        }
#pragma unroll
        for (int jj = 0; jj < 32; ++jj) out[(warp * 32 + jj) * kRows + lane] = fmaxf(acc[jj], 0.f);
    }
    __syncthreads();

    // ---- output layer: delta_out = d_resid row
    float g5[WRF_OUT];
#pragma unroll
    for (int j = 0; j < WRF_OUT; ++j) g5[j] = ok ? a.d_resid[row * WRF_OUT + j] : 0.f;
    if (warp == 0 && ok) {
#pragma unroll
        for (int j = 0; j < WRF_OUT; ++j) a.cb.G[L - 1][lr * WRF_OUT + j] = g5[j];
    }
    // delta of the last hidden pre-activation: (Wo^T g5) * [h_{L-1} > 0]
    float *dcur = dl;
    {
        const float *hl = h + nh * WRF_HIDDEN * kRows;
        for (int jj = 0; jj < 32; ++jj) {
            const int k = warp * 32 + jj;
            float sacc = 0.f;
#pragma unroll
            for (int j = 0; j < WRF_OUT; ++j) sacc = fmaf(a.m.Wo[j * WRF_HIDDEN + k], g5[j], sacc);
            dcur[k * kRows + lane] = hl[k * kRows + lane] > 0.f ? sacc : 0.f;
        }
    }
    // hidden layers backwards: layer l maps h_{l+1} -> z_{l+2}
    for (int l = nh - 1; l >= -1; --l) {
        __syncthreads();
        // store G of the layer whose pre-activation dcur is, and its input H
        const int layer = l + 1;  // 0 = first layer
        if (ok) {
            float *G = a.cb.G[layer] + lr * WRF_HIDDEN;
            for (int jj = 0; jj < 32; ++jj) G[warp * 32 + jj] = dcur[(warp * 32 + jj) * kRows + lane];
        }
        if (l < 0) break;
        // delta_{prev} = (W_l^T dcur) * [h_{l+1} > 0], W_l = Wh[l] [j][k]
        float *dnext = dcur == dl ? dl + WRF_HIDDEN * kRows : dl;
        const float *hin = h + l * WRF_HIDDEN * kRows;
        const float *Wl = a.m.Wh[l];
        float acc[32];
#pragma unroll
        for (int kk = 0; kk < 32; ++kk) acc[kk] = 0.f;
        for (int j = 0; j < WRF_HIDDEN; ++j) {
            const float d = dcur[j * kRows + lane];
            const float4 *wj = reinterpret_cast<const float4 *>(Wl + j * WRF_HIDDEN + warp * 32);
#pragma unroll
            for (int v4 = 0; v4 < 8; ++v4) {
                const float4 w = wj[v4];
                acc[4 * v4 + 0] = fmaf(w.x, d, acc[4 * v4 + 0]);
                acc[4 * v4 + 1] = fmaf(w.y, d, acc[4 * v4 + 1]);
                acc[4 * v4 + 2] = fmaf(w.z, d, acc[4 * v4 + 2]);
                acc[4 * v4 + 3] = fmaf(w.w, d, acc[4 * v4 + 3]);
            }
        }
#pragma unroll
        for (int kk = 0; kk < 32; ++kk) {
            const int k = warp * 32 + kk;
            dnext[k * kRows + lane] = hin[k * kRows + lane] > 0.f ? acc[kk] : 0.f;
        }
        dcur = dnext;
    }
    // ---- layer inputs H: activations h_1..h_{L-1} and the first-layer features
    if (ok) {
        for (int l = 0; l < L - 1; ++l) {
            float *Hr = a.cb.Hh[l] + lr * WRF_HIDDEN;
            for (int jj = 0; jj < 32; ++jj)
                Hr[warp * 32 + jj] = h[(l * WRF_HIDDEN + warp * 32 + jj) * kRows + lane];
        }
        const int din = a.m.dm + a.m.dt;
        float *H0 = a.cb.H0 + lr * din;
        for (int k = warp; k < din; k += 4)
            H0[k] = k < a.m.dm ? a.cb.gam_m[static_cast<size_t>(n) * a.m.dm + k]
                               : a.cb.gam_t[static_cast<size_t>(q) * a.m.dt + (k - a.m.dm)];
    }
    // ---- d_mean through gamma(mean): d gamma / d x for x = mean / (W, H)
    if (a.d_mean && ok && warp == 0) {
        const int din = a.m.dm + a.m.dt, Lm = a.m.L_mean;
        const float2 mu = reinterpret_cast<const float2 *>(a.s.mean)[n];
        const PeArg x[2] = {pe_arg(mu.x, 0.f, static_cast<float>(a.g.W)),
                            pe_arg(mu.y, 0.f, static_cast<float>(a.g.H))};
        float gx[2] = {0.f, 0.f};
        for (int f = 0; f < a.m.dm; ++f) {
            // dL/dgamma_f = sum_j W0[j][f] delta1[j]
            float s = 0.f;
            for (int j = 0; j < WRF_HIDDEN; ++j) s = fmaf(a.m.W0[j * din + f], dcur[j * kRows + lane], s);
            const int i = f % 2, grp = f / 2;
            float dg = 1.f;
            if (grp >= 1) {
                const int k = (grp - 1) % Lm;
                float sn, cs;
                pe_band(x[i], k, sn, cs);
                const float w = ldexpf(3.14159265358979f, k);
                dg = grp <= Lm ? w * cs : -w * sn;
            }
            gx[i] = fmaf(s, dg, gx[i]);
        }
        atomicAdd(a.d_mean + 2 * n, gx[0] / static_cast<float>(a.g.W));
        atomicAdd(a.d_mean + 2 * n + 1, gx[1] / static_cast<float>(a.g.H));
    }
}

// dW[j][k] += sum_r G[r][j] H[r][k] (and db[j] += sum_r G[r][j] when k-tile 0
// carries the bias column) over rows [r0, r1) of the chunk.
struct DwJob {
    const float *G;  // [R][dout]
    const float *H;  // [R][din]
    float *dW;       // [dout][din]
    float *db;       // [dout]
    int dout, din;
};
struct DwArgs {
    DwJob job[8];
    int njobs;
    long long nrows;
    int slice;  // rows per CTA
};

__global__ void __launch_bounds__(256) dw_kernel(DwArgs a) {
    __shared__ float sG[32][33];
    __shared__ float sH[32][33];
    const DwJob jb = a.job[blockIdx.z];
    const int j0 = blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
    // output tile: rows j0..j0+31 of dW, columns k0..k0+31 (blockIdx.x encodes k-tile and slice)
    const int nkt = (jb.din + 31) / 32 + 1;  // +1: the bias column tile
    const int kt = blockIdx.x % nkt;
    const int sl = blockIdx.x / nkt;
    if (j0 >= jb.dout) return;
    const long long r0 = static_cast<long long>(sl) * a.slice;
    if (r0 >= a.nrows) return;
    const long long r1 = min(a.nrows, r0 + a.slice);
    const bool bias = kt == nkt - 1;
    const int k0 = kt * 32;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};  // rows j = j0 + ty + 8i, column k = k0 + tx
    for (long long rb = r0; rb < r1; rb += 32) {
        // load 32 rows of G (columns j0..j0+31) and H (columns k0..k0+31)
        for (int i = ty; i < 32; i += 8) {
            const long long r = rb + i;
            const bool rok = r < r1;
            const int j = j0 + tx, k = k0 + tx;
            sG[i][tx] = (rok && j < jb.dout) ? jb.G[r * jb.dout + j] : 0.f;
            sH[i][tx] = bias ? (rok ? 1.f : 0.f) : ((rok && k < jb.din) ? jb.H[r * jb.din + k] : 0.f);
        }
        __syncthreads();
#pragma unroll 8
        for (int i = 0; i < 32; ++i) {
            const float hv = sH[i][tx];
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[u] = fmaf(sG[i][ty + 8 * u], hv, acc[u]);
        }
        __syncthreads();
    }
    for (int u = 0; u < 4; ++u) {
        const int j = j0 + ty + 8 * u, k = k0 + tx;
        if (j >= jb.dout) continue;
        if (bias) {
            if (tx == 0) atomicAdd(jb.db + j, acc[u]);
        } else if (k < jb.din) {
            atomicAdd(jb.dW + static_cast<size_t>(j) * jb.din + k, acc[u]);
        }
    }
}

}  // namespace

size_t deform_bwd_ws_layout(int n, int Q, const MlpView &m, DeformWs *fw, DeformBwdWs *bw,
                            char *base) {
    size_t off = align256(deform_ws_layout(n, Q, m.n_layers, fw, base));
    auto take = [&](size_t bytes) {
        char *p = base ? base + off : nullptr;
        off = align256(off + bytes);
        return reinterpret_cast<float *>(p);
    };
    DeformBwdWs w{};
    const int din = m.dm + m.dt;
    const int L = m.n_layers;
    w.cb_H0 = take(static_cast<size_t>(kChunk) * din * 4);
    for (int l = 0; l < L - 1; ++l) w.cb_Hh[l] = take(static_cast<size_t>(kChunk) * WRF_HIDDEN * 4);
    for (int l = 0; l < L; ++l)
        w.cb_G[l] = take(static_cast<size_t>(kChunk) * (l == L - 1 ? WRF_OUT : WRF_HIDDEN) * 4);
    w.gam_m = take(static_cast<size_t>(n) * m.dm * 4);
    w.gam_t = take(static_cast<size_t>(Q) * m.dt * 4);
    if (bw) *bw = w;
    return off;
}

cudaError_t launch_mlp_bwd(const SceneView &s, const MlpView &m, const GridView &g,
                           const float *tx, int Q, const DeformWs &fw, const DeformBwdWs &bw,
                           const float *d_resid, float *const *dW, float *const *db,
                           float *d_mean, int stop_grad_mean, cudaStream_t st) {
    const int L = m.n_layers;
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
    gamma_tables_kernel<<<static_cast<int>((s.n + Q + 127) / 128), 128, 0, st>>>(
        s, m, g, tx, Q, bw.gam_m, bw.gam_t);
    const size_t smem = static_cast<size_t>((L - 1) + 2) * WRF_HIDDEN * kRows * 4;
    cudaError_t e = cudaFuncSetAttribute(mlp_bwd_rows_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    RowsArgs ra{};
    ra.s = s;
    ra.m = m;
    ra.g = g;
    ra.fw = fw;
    ra.cb.H0 = bw.cb_H0;
    for (int l = 0; l < L - 1; ++l) ra.cb.Hh[l] = bw.cb_Hh[l];
    for (int l = 0; l < L; ++l) ra.cb.G[l] = bw.cb_G[l];
    ra.cb.gam_m = bw.gam_m;
    ra.cb.gam_t = bw.gam_t;
    ra.d_resid = d_resid;
    ra.d_mean = stop_grad_mean ? nullptr : d_mean;
    DwArgs da{};
    da.njobs = L;
    for (int l = 0; l < L; ++l) {
        DwJob &j = da.job[l];
        j.G = bw.cb_G[l];
        j.H = l == 0 ? bw.cb_H0 : bw.cb_Hh[l - 1];
        j.dW = dW[l];
        j.db = db[l];
        j.dout = l == L - 1 ? WRF_OUT : WRF_HIDDEN;
        j.din = l == 0 ? din : WRF_HIDDEN;
    }
    da.slice = 1024;
    int max_kt = 0;
    for (int l = 0; l < L; ++l) max_kt = max(max_kt, (da.job[l].din + 31) / 32 + 1);
    for (long long r0 = 0; r0 < rows; r0 += kChunk) {
        const long long nr = min(static_cast<long long>(kChunk), rows - r0);
        ra.row0 = r0;
        ra.nrows = nr;
        mlp_bwd_rows_kernel<<<static_cast<int>((nr + kRows - 1) / kRows), 128, smem, st>>>(ra);
        da.nrows = nr;
        const int nslices = static_cast<int>((nr + da.slice - 1) / da.slice);
        dim3 grid(max_kt * nslices, WRF_HIDDEN / 32, L);
        dw_kernel<<<grid, 256, 0, st>>>(da);
    }
    return cudaGetLastError();
}

}  // namespace wrf
