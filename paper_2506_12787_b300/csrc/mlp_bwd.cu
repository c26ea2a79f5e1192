// Back-propagation through the deformation MLP (Sec. 4.2 Eq. 14-15; the
// paper fits all parameters by gradient descent, Sec. 4.4).
//
// Given dL/d(resid) for every (query, Gaussian) row, produces dL/dW and
// dL/db of every layer and, unless positions are stop-gradded (the paper's
// fine stage, Sec. 4.4), the derivative through gamma(mean) added into
// d_mean.  Every step over rows is a dense product, so rows are processed in
// chunks of up to kChunk as plain GEMMs (cuBLAS, FP32 inputs and outputs computed
// on the tensor cores with the three-term BF16 split of FP32,
// CUBLAS_COMPUTE_32F_EMULATED_16BFX9) between small hand-written kernels:
//   features   H0 = [gamma(mean_n), gamma(tx_q)], H1 = ReLU(U[n] + V[q])
//   forward    Z_l = H_{l-1} W_{l-1}^T; H_l = ReLU(Z_l + b)       (hidden layers)
//              -- both skipped for H1.. when the forward saved its hidden
//              activations (acts), which are then read in place
//   deltas     D_last = (G_out W_out) * [H_last > 0]; D_{l-1} = (D_l W_l) * [H_{l-1} > 0]
//   gradients  dW_l += D_l^T H_{l-1} (GEMM over rows, accumulated across
//              chunks), db_l += column sums of D_l,
//              dgamma(mean) = D_1 W0m -> d_mean through d gamma / d mean.
// All matrices are row-major [rows][width]; cuBLAS sees them column-major
// transposed.  The GEMM workspace comes from the caller's workspace; one
// cuBLAS handle per device is created on the first call.
#include <cublas_v2.h>

#include <mutex>

#include "kernels.h"

namespace wrf {

namespace {

// Rows per chunk: large chunks keep the launch count low and the weight-
// gradient GEMMs (a reduction over the chunk's rows) long; the buffers take
// ~8.2 KB per row of the chunk (1M rows: 8.6 GB of workspace).
constexpr long long kChunk = 1 << 20;

// Rows per chunk for a problem of Q x n rows.
inline long long chunk_rows(int n, int Q) {
    const long long rows = static_cast<long long>(Q) * n;
    return rows < kChunk ? (rows > 0 ? rows : 1) : kChunk;
}
constexpr size_t kCublasWs = size_t(32) << 20;

inline size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }


__global__ void gamma_tables_kernel(SceneView s, MlpView m, GridView g, const float *tx, int Q,
                                    float *gam_m, float *gam_t) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < s.n) {
        const float2 mu = reinterpret_cast<const float2 *>(s.mean)[i];
        const PeArg x[2] = {pe_arg(mu.x, 0.f, static_cast<float>(g.W)),
                            pe_arg(mu.y, 0.f, static_cast<float>(g.H))};
        pe_encode(x, 2, m.L_mean, gam_m + static_cast<size_t>(i) * m.dm);
    } else if (i < s.n + Q) {
        const int q = i - s.n;
        PeArg x[3];
        for (int c = 0; c < 3; ++c) x[c] = pe_arg(tx[3 * q + c], m.room_min[c], m.room_size[c]);
        pe_encode(x, 3, m.L_tx, gam_t + static_cast<size_t>(q) * m.dt);
    }
}

// H0[r] = [gamma(mean_n), gamma(tx_q)], H1[r] = ReLU(U[n] + V[q]) for the
// chunk's rows (row = row0 + r, q = row / N, n = row % N).
__global__ void features_kernel(int N, long long row0, int nrows, int dm, int dt,
                                const float *gam_m, const float *gam_t, const float *U,
                                const float *V, float *H0, float *H1) {
    const int din = dm + dt;
    const int ncol = din + (H1 ? WRF_HIDDEN : 0);  // H1 is NULL when saved by the forward
    const long long total = static_cast<long long>(nrows) * ncol;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long r = e / ncol;
        const int c = static_cast<int>(e % ncol);
        const long long row = row0 + r;
        const int q = static_cast<int>(row / N), n = static_cast<int>(row % N);
        if (c < din) {
            H0[r * din + c] = c < dm ? gam_m[static_cast<size_t>(n) * dm + c]
                                     : gam_t[static_cast<size_t>(q) * dt + (c - dm)];
        } else {
            const int j = c - din;
            H1[r * WRF_HIDDEN + j] = fmaxf(U[static_cast<size_t>(n) * WRF_HIDDEN + j] +
                                               V[static_cast<size_t>(q) * WRF_HIDDEN + j],
                                           0.f);
        }
    }
}

// Z = ReLU(Z + b) in place, Z [nrows][128].
__global__ void bias_relu_kernel(float *Z, const float *b, long long n) {
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < n;
         e += static_cast<long long>(gridDim.x) * blockDim.x)
        Z[e] = fmaxf(Z[e] + b[e & (WRF_HIDDEN - 1)], 0.f);
}

// D = D * [H > 0] in place.
__global__ void relu_mask_kernel(float *D, const float *H, long long n) {
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < n;
         e += static_cast<long long>(gridDim.x) * blockDim.x)
        if (!(H[e] > 0.f)) D[e] = 0.f;
}

// db[j] += sum_r D[r][j] for D [nrows][width]: each block sums a slice of
// rows per column, one atomic add per (block, column).
__global__ void colsum_kernel(const float *D, int nrows, int width, float *db) {
    const int j = threadIdx.x;
    if (j >= width) return;
    const int rows_per = (nrows + gridDim.x - 1) / gridDim.x;
    const int r0 = blockIdx.x * rows_per, r1 = min(nrows, r0 + rows_per);
    float s = 0.f;
    for (int r = r0; r < r1; ++r) s += D[static_cast<size_t>(r) * width + j];
    if (r1 > r0) atomicAdd(db + j, s);
}

// d_mean[n] += dgamma(mean_n) . d gamma / d (mean / (W, H)) / (W, H).
__global__ void dmean_kernel(SceneView s, MlpView m, GridView g, int N, long long row0, int nrows,
                             const float *dgm, float *d_mean) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrows) return;
    const long long row = row0 + r;
    const int n = static_cast<int>(row % N);
    const float2 mu = reinterpret_cast<const float2 *>(s.mean)[n];
    const PeArg x[2] = {pe_arg(mu.x, 0.f, static_cast<float>(g.W)),
                        pe_arg(mu.y, 0.f, static_cast<float>(g.H))};
    const int Lm = m.L_mean;
    float gx[2] = {0.f, 0.f};
    for (int f = 0; f < m.dm; ++f) {
        const int i = f % 2, grp = f / 2;
        float dg = 1.f;
        if (grp >= 1) {
            const int k = (grp - 1) % Lm;
            float sn, cs;
            pe_band(x[i], k, sn, cs);
            const float w = ldexpf(3.14159265358979f, k);
            dg = grp <= Lm ? w * cs : -w * sn;
        }
        gx[i] = fmaf(dgm[static_cast<size_t>(r) * m.dm + f], dg, gx[i]);
    }
    atomicAdd(d_mean + 2 * n, gx[0] / static_cast<float>(g.W));
    atomicAdd(d_mean + 2 * n + 1, gx[1] / static_cast<float>(g.H));
}

int grid_for(long long n) {
    long long b = (n + 255) / 256;
    return static_cast<int>(b > 148 * 16 ? 148 * 16 : (b < 1 ? 1 : b));
}

// One cuBLAS handle per device, created on first use.
cublasHandle_t handle_for_device() {
    static cublasHandle_t handles[64] = {nullptr};
    static std::mutex mu;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (!handles[dev]) {
        cublasHandle_t h = nullptr;
        if (cublasCreate(&h) != CUBLAS_STATUS_SUCCESS) return nullptr;
        handles[dev] = h;
    }
    return handles[dev];
}

// C^T (m x n) = opA(A) (m x k) * opB(B) (k x n) in cuBLAS column-major terms
// (a row-major [rows][width] matrix is a column-major [width][rows] one).
cublasStatus_t gemm(cublasHandle_t h, cublasOperation_t ta, cublasOperation_t tb, int m, int n,
                    int k, const float *A, int lda, const float *B, int ldb, float beta, float *C,
                    int ldc) {
    const float alpha = 1.f;
    return cublasGemmEx(h, ta, tb, m, n, k, &alpha, A, CUDA_R_32F, lda, B, CUDA_R_32F, ldb, &beta, C,
                        CUDA_R_32F, ldc, CUBLAS_COMPUTE_32F_EMULATED_16BFX9, CUBLAS_GEMM_DEFAULT);
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
    const size_t C = static_cast<size_t>(chunk_rows(n, Q));
    w.cb_H0 = take(C * din * 4);
    for (int l = 0; l < L - 1; ++l) w.cb_Hh[l] = take(C * WRF_HIDDEN * 4);
    for (int l = 0; l < L - 1; ++l) w.cb_G[l] = take(C * WRF_HIDDEN * 4);
    w.cb_G[L - 1] = nullptr;  // the output layer's delta is d_resid itself
    w.dgm = take(C * m.dm * 4);
    w.gam_m = take(static_cast<size_t>(n) * m.dm * 4);
    w.gam_t = take(static_cast<size_t>(Q) * m.dt * 4);
    w.cublas_ws = reinterpret_cast<char *>(take(kCublasWs));
    w.cublas_ws_bytes = kCublasWs;
    if (bw) *bw = w;
    return off;
}

cudaError_t launch_mlp_bwd(const SceneView &s, const MlpView &m, const GridView &g,
                           const float *tx, int Q, const DeformWs &fw, const DeformBwdWs &bw,
                           const float *d_resid, const float *acts, float *const *dW,
                           float *const *db, float *d_mean, int stop_grad_mean, cudaStream_t st) {
    const int L = m.n_layers, nh = L - 2;
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
    cublasHandle_t h = handle_for_device();
    if (!h) return cudaErrorUnknown;
    if (cublasSetStream(h, st) != CUBLAS_STATUS_SUCCESS ||
        cublasSetWorkspace(h, bw.cublas_ws, bw.cublas_ws_bytes) != CUBLAS_STATUS_SUCCESS)
        return cudaErrorUnknown;
    gamma_tables_kernel<<<static_cast<int>((s.n + Q + 127) / 128), 128, 0, st>>>(
        s, m, g, tx, Q, bw.gam_m, bw.gam_t);
    const cublasOperation_t N_ = CUBLAS_OP_N, T_ = CUBLAS_OP_T;
    const long long CH = chunk_rows(s.n, Q);
    for (long long r0 = 0; r0 < rows; r0 += CH) {
        const int R = static_cast<int>(rows - r0 < CH ? rows - r0 : CH);
        const long long nH = static_cast<long long>(R) * WRF_HIDDEN;
        // hidden activations of this chunk: saved by the forward, or recomputed
        const float *Hh[8];
        for (int l = 0; l <= nh; ++l)
            Hh[l] = acts ? acts + (static_cast<size_t>(l) * rows + r0) * WRF_HIDDEN : bw.cb_Hh[l];
        features_kernel<<<grid_for(static_cast<long long>(R) * (din + (acts ? 0 : WRF_HIDDEN))),
                          256, 0, st>>>(s.n, r0, R, m.dm, m.dt, bw.gam_m, bw.gam_t, fw.U, fw.V,
                                        bw.cb_H0, acts ? nullptr : bw.cb_Hh[0]);
        // forward recompute of the hidden layers: H_{l+1} = ReLU(H_l Wh[l]^T + bh[l])
        for (int l = 0; l < nh && !acts; ++l) {
            if (gemm(h, T_, N_, WRF_HIDDEN, R, WRF_HIDDEN, m.Wh[l], WRF_HIDDEN, bw.cb_Hh[l],
                     WRF_HIDDEN, 0.f, bw.cb_Hh[l + 1], WRF_HIDDEN) != CUBLAS_STATUS_SUCCESS)
                return cudaErrorUnknown;
            bias_relu_kernel<<<grid_for(nH), 256, 0, st>>>(bw.cb_Hh[l + 1], m.bh[l], nH);
        }
        const float *Gout = d_resid + r0 * WRF_OUT;
        // delta of the last hidden layer: (G_out W_out) * [H_last > 0]
        float *Dl = bw.cb_G[nh];
        if (gemm(h, N_, N_, WRF_HIDDEN, R, WRF_OUT, m.Wo, WRF_HIDDEN, Gout, WRF_OUT, 0.f, Dl,
                 WRF_HIDDEN) != CUBLAS_STATUS_SUCCESS)
            return cudaErrorUnknown;
        relu_mask_kernel<<<grid_for(nH), 256, 0, st>>>(Dl, Hh[nh], nH);
        // output layer gradients: dWo += G_out^T H_last, dbo += colsum(G_out)
        if (gemm(h, N_, T_, WRF_HIDDEN, WRF_OUT, R, Hh[nh], WRF_HIDDEN, Gout, WRF_OUT, 1.f,
                 dW[L - 1], WRF_HIDDEN) != CUBLAS_STATUS_SUCCESS)
            return cudaErrorUnknown;
        colsum_kernel<<<296, 32, 0, st>>>(Gout, R, WRF_OUT, db[L - 1]);
        // hidden layers backwards: layer l+1 (Wh[l]) maps H_l -> Z_{l+1}
        for (int l = nh - 1; l >= 0; --l) {
            float *D = bw.cb_G[l + 1];  // delta of Z_{l+1}
            if (gemm(h, N_, T_, WRF_HIDDEN, WRF_HIDDEN, R, Hh[l], WRF_HIDDEN, D, WRF_HIDDEN,
                     1.f, dW[l + 1], WRF_HIDDEN) != CUBLAS_STATUS_SUCCESS)
                return cudaErrorUnknown;
            colsum_kernel<<<296, 128, 0, st>>>(D, R, WRF_HIDDEN, db[l + 1]);
            float *Dp = bw.cb_G[l];  // delta of Z_l = (D Wh[l]) * [H_l > 0]
            if (gemm(h, N_, N_, WRF_HIDDEN, R, WRF_HIDDEN, m.Wh[l], WRF_HIDDEN, D, WRF_HIDDEN, 0.f,
                     Dp, WRF_HIDDEN) != CUBLAS_STATUS_SUCCESS)
                return cudaErrorUnknown;
            relu_mask_kernel<<<grid_for(nH), 256, 0, st>>>(Dp, Hh[l], nH);
        }
        // first layer: dW0 += D_0^T H0, db0 += colsum(D_0)
        if (gemm(h, N_, T_, din, WRF_HIDDEN, R, bw.cb_H0, din, bw.cb_G[0], WRF_HIDDEN, 1.f, dW[0],
                 din) != CUBLAS_STATUS_SUCCESS)
            return cudaErrorUnknown;
        colsum_kernel<<<296, 128, 0, st>>>(bw.cb_G[0], R, WRF_HIDDEN, db[0]);
        if (!stop_grad_mean) {
            // dgamma(mean) [R][dm] = D_0 W0[:, :dm]
            if (gemm(h, N_, N_, m.dm, R, WRF_HIDDEN, m.W0, din, bw.cb_G[0], WRF_HIDDEN, 0.f,
                     bw.dgm, m.dm) != CUBLAS_STATUS_SUCCESS)
                return cudaErrorUnknown;
            dmean_kernel<<<(R + 127) / 128, 128, 0, st>>>(s, m, g, s.n, r0, R, bw.dgm, d_mean);
        }
    }
    return cudaGetLastError();
}

}  // namespace wrf
