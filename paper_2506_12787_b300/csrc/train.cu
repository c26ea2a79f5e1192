// Training-protocol kernels (Sec. 4.4).
//
// Loss of Eq. 16 over a batch of Q maps:
//   L = lambda_1 mean|A_hat - A| + (1 - lambda_1) (1 - mean_q SSIM(A_hat_q, A_q)),
// with SSIM in its standard form: local means, variances and covariance under
// an 11 x 11 Gaussian window (sigma 1.5, weights summing to 1, zero outside the
// map), C1 = (0.01 L)^2, C2 = (0.03 L)^2 with L = 1, averaged over the map.
// Two tiled passes (32 x 32 output pixels per CTA, the separable window as an
// 11-tap row pass and an 11-tap column pass over a shared-memory halo):
//   1. ssim_stats_kernel: the five window sums, the per-pixel index s, and the
//      three coefficient maps of its derivative
//        c1 = ds/dmx - 2 mx ds/dsxx - my ds/dsxy,  c2 = ds/dsxx,  c3 = ds/dsxy,
//      plus per-tile partial sums of s and |A_hat - A|;
//   2. ssim_grad_kernel: dSSIM/dA_hat = (G*c1 + 2 A_hat G*c2 + A G*c3) / (H W)
//      (the window's adjoint is the same zero-padded window sum), fused with
//      the L1 term into dL/dA_hat;
//   3. loss_reduce_kernel: the partials summed in a fixed order -> L and the
//      per-map SSIM.
// Adam (the paper trains with PyTorch's Adam, learning rates in Table I):
// one launch updates up to kAdamGroups parameter tensors.
// Anneal smoothing (Eq. 17-18): the fine stage's noisy TX positions, gathered
// from the training set in the same launch.
#include "kernels.h"

namespace wrf {

namespace {

constexpr int kTile = 32;                 // output pixels per CTA side
constexpr int kHalo = 5;                  // window radius
constexpr int kIn = kTile + 2 * kHalo;    // 42
constexpr int kSsimThreads = 256;
constexpr float kC1 = 0.01f * 0.01f, kC2 = 0.03f * 0.03f;

// 11-tap Gaussian, sigma 1.5, normalised: every CTA computes the weights
// into shared memory (the sum in a fixed order).
__device__ __forceinline__ void make_window(float *w) {
    if (threadIdx.x < 2 * kHalo + 1) {
        const float r = static_cast<float>(static_cast<int>(threadIdx.x) - kHalo);
        w[threadIdx.x] = expf(-r * r / (2.f * 1.5f * 1.5f));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int t = 0; t < 2 * kHalo + 1; ++t) s += w[t];
        for (int t = 0; t < 2 * kHalo + 1; ++t) w[t] /= s;
    }
    __syncthreads();
}

struct LossView {
    const float *x, *y;   // prediction A_hat, target A: [Q][H][W]
    int Q, H, W, tx, ty;  // tiles across / down
    float lam;
    float *coef;          // [3][Q][H][W]
    float *part;          // [Q][tx*ty][2]: sum s, sum |x - y|
    float *dx;            // [Q][H][W] or null
    float *out;           // [1 + Q]: L, SSIM_q
};

__global__ void __launch_bounds__(kSsimThreads) ssim_stats_kernel(LossView v) {
    __shared__ float sx[kIn][kIn + 1], sy[kIn][kIn + 1];
    __shared__ float hs[5][kIn][kTile];
    __shared__ float red[2][kSsimThreads / 32];
    __shared__ float c_win[2 * kHalo + 1];
    make_window(c_win);
    const int q = blockIdx.z, tid = threadIdx.x;
    const int x0 = blockIdx.x * kTile, y0 = blockIdx.y * kTile;
    const size_t base = static_cast<size_t>(q) * v.H * v.W;
    for (int i = tid; i < kIn * kIn; i += kSsimThreads) {
        const int r = i / kIn, c = i % kIn, gy = y0 - kHalo + r, gx = x0 - kHalo + c;
        const bool in = gy >= 0 && gy < v.H && gx >= 0 && gx < v.W;
        sx[r][c] = in ? v.x[base + static_cast<size_t>(gy) * v.W + gx] : 0.f;
        sy[r][c] = in ? v.y[base + static_cast<size_t>(gy) * v.W + gx] : 0.f;
    }
    __syncthreads();
    // row pass: 42 rows x 32 output columns, five products
    for (int i = tid; i < kIn * kTile; i += kSsimThreads) {
        const int r = i / kTile, c = i % kTile;
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f, a4 = 0.f;
#pragma unroll
        for (int t = 0; t < 2 * kHalo + 1; ++t) {
            const float g = c_win[t], xv = sx[r][c + t], yv = sy[r][c + t];
            a0 = fmaf(g, xv, a0);
            a1 = fmaf(g, yv, a1);
            a2 = fmaf(g, xv * xv, a2);
            a3 = fmaf(g, yv * yv, a3);
            a4 = fmaf(g, xv * yv, a4);
        }
        hs[0][r][c] = a0;
        hs[1][r][c] = a1;
        hs[2][r][c] = a2;
        hs[3][r][c] = a3;
        hs[4][r][c] = a4;
    }
    __syncthreads();
    // column pass and the per-pixel index
    const int c = tid & 31;
    float ps = 0.f, pl1 = 0.f;
    for (int r = tid >> 5; r < kTile; r += kSsimThreads / 32) {
        float m[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int t = 0; t < 2 * kHalo + 1; ++t) {
            const float g = c_win[t];
#pragma unroll
            for (int k = 0; k < 5; ++k) m[k] = fmaf(g, hs[k][r + t][c], m[k]);
        }
        const int gy = y0 + r, gx = x0 + c;
        if (gy >= v.H || gx >= v.W) continue;
        const float mx = m[0], my = m[1];
        const float sxx = m[2] - mx * mx, syy = m[3] - my * my, sxy = m[4] - mx * my;
        const float A = 2.f * mx * my + kC1, B = 2.f * sxy + kC2;
        const float Cc = mx * mx + my * my + kC1, D = sxx + syy + kC2;
        const float inv = 1.f / (Cc * D);
        const float s = A * B * inv;
        const float d_mx = 2.f * my * B * inv - s * 2.f * mx / Cc;
        const float d_sxx = -s / D;
        const float d_sxy = 2.f * A * inv;
        const size_t p = base + static_cast<size_t>(gy) * v.W + gx;
        const size_t plane = static_cast<size_t>(v.Q) * v.H * v.W;
        v.coef[p] = d_mx - 2.f * mx * d_sxx - my * d_sxy;
        v.coef[plane + p] = d_sxx;
        v.coef[2 * plane + p] = d_sxy;
        ps += s;
        pl1 += fabsf(sx[r + kHalo][c + kHalo] - sy[r + kHalo][c + kHalo]);
    }
    // fixed-order block sums
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ps += __shfl_down_sync(0xffffffffu, ps, o);
        pl1 += __shfl_down_sync(0xffffffffu, pl1, o);
    }
    if ((tid & 31) == 0) {
        red[0][tid >> 5] = ps;
        red[1][tid >> 5] = pl1;
    }
    __syncthreads();
    if (tid == 0) {
        float a = 0.f, b = 0.f;
        for (int w = 0; w < kSsimThreads / 32; ++w) {
            a += red[0][w];
            b += red[1][w];
        }
        float *pp = v.part + (static_cast<size_t>(q) * v.tx * v.ty + blockIdx.y * v.tx + blockIdx.x) * 2;
        pp[0] = a;
        pp[1] = b;
    }
}

__global__ void __launch_bounds__(kSsimThreads) ssim_grad_kernel(LossView v) {
    __shared__ float sc[3][kIn][kIn + 1];
    __shared__ float hs[3][kIn][kTile];
    __shared__ float c_win[2 * kHalo + 1];
    make_window(c_win);
    const int q = blockIdx.z, tid = threadIdx.x;
    const int x0 = blockIdx.x * kTile, y0 = blockIdx.y * kTile;
    const size_t base = static_cast<size_t>(q) * v.H * v.W;
    const size_t plane = static_cast<size_t>(v.Q) * v.H * v.W;
    for (int i = tid; i < kIn * kIn; i += kSsimThreads) {
        const int r = i / kIn, c = i % kIn, gy = y0 - kHalo + r, gx = x0 - kHalo + c;
        const bool in = gy >= 0 && gy < v.H && gx >= 0 && gx < v.W;
        const size_t p = base + static_cast<size_t>(gy) * v.W + gx;
        sc[0][r][c] = in ? v.coef[p] : 0.f;
        sc[1][r][c] = in ? v.coef[plane + p] : 0.f;
        sc[2][r][c] = in ? v.coef[2 * plane + p] : 0.f;
    }
    __syncthreads();
    for (int i = tid; i < kIn * kTile; i += kSsimThreads) {
        const int r = i / kTile, c = i % kTile;
        float a0 = 0.f, a1 = 0.f, a2 = 0.f;
#pragma unroll
        for (int t = 0; t < 2 * kHalo + 1; ++t) {
            const float g = c_win[t];
            a0 = fmaf(g, sc[0][r][c + t], a0);
            a1 = fmaf(g, sc[1][r][c + t], a1);
            a2 = fmaf(g, sc[2][r][c + t], a2);
        }
        hs[0][r][c] = a0;
        hs[1][r][c] = a1;
        hs[2][r][c] = a2;
    }
    __syncthreads();
    const int c = tid & 31;
    const float P = static_cast<float>(v.H) * static_cast<float>(v.W);
    const float w_ssim = (1.f - v.lam) / (static_cast<float>(v.Q) * P);
    const float w_l1 = v.lam / (static_cast<float>(v.Q) * P);
    for (int r = tid >> 5; r < kTile; r += kSsimThreads / 32) {
        const int gy = y0 + r, gx = x0 + c;
        if (gy >= v.H || gx >= v.W) continue;
        float g0 = 0.f, g1 = 0.f, g2 = 0.f;
#pragma unroll
        for (int t = 0; t < 2 * kHalo + 1; ++t) {
            const float g = c_win[t];
            g0 = fmaf(g, hs[0][r + t][c], g0);
            g1 = fmaf(g, hs[1][r + t][c], g1);
            g2 = fmaf(g, hs[2][r + t][c], g2);
        }
        const size_t p = base + static_cast<size_t>(gy) * v.W + gx;
        const float xv = v.x[p], yv = v.y[p];
        const float dssim = g0 + 2.f * xv * g1 + yv * g2;
        const float sgn = xv > yv ? 1.f : (xv < yv ? -1.f : 0.f);
        v.dx[p] = w_l1 * sgn - w_ssim * dssim;
    }
}

// One block: per-map SSIM and the loss, partials summed in a fixed order.
__global__ void __launch_bounds__(256) loss_reduce_kernel(LossView v) {
    __shared__ float red[2][256];
    const int T = v.tx * v.ty;
    const float P = static_cast<float>(v.H) * static_cast<float>(v.W);
    float ssum = 0.f, l1 = 0.f;
    for (int q = threadIdx.x; q < v.Q; q += blockDim.x) {
        float a = 0.f, b = 0.f;
        for (int t = 0; t < T; ++t) {
            a += v.part[(static_cast<size_t>(q) * T + t) * 2];
            b += v.part[(static_cast<size_t>(q) * T + t) * 2 + 1];
        }
        v.out[1 + q] = a / P;
        ssum += a / P;
        l1 += b;
    }
    red[0][threadIdx.x] = ssum;
    red[1][threadIdx.x] = l1;
    __syncthreads();
    if (threadIdx.x == 0) {
        float a = 0.f, b = 0.f;
        for (int i = 0; i < blockDim.x; ++i) {
            a += red[0][i];
            b += red[1][i];
        }
        const float Q = static_cast<float>(v.Q);
        v.out[0] = v.lam * b / (Q * P) + (1.f - v.lam) * (1.f - a / Q);
    }
}

struct AdamArgs {
    AdamGroup g[kAdamGroups];
    long long start[kAdamGroups + 1];  // prefix sums of the group sizes
    int n;
    float beta1, beta2, eps, bc1, bc2;
};

__global__ void adam_kernel(AdamArgs a) {
    const long long total = a.start[a.n];
    int grp = 0;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        while (i >= a.start[grp + 1]) ++grp;
        const AdamGroup &G = a.g[grp];
        const long long k = i - a.start[grp];
        const float g = G.grad[k];
        const float m = fmaf(a.beta1, G.m[k], (1.f - a.beta1) * g);
        const float v = fmaf(a.beta2, G.v[k], (1.f - a.beta2) * g * g);
        G.m[k] = m;
        G.v[k] = v;
        const float denom = sqrtf(v / a.bc2) + a.eps;
        G.param[k] -= G.lr * (m / a.bc1) / denom;
    }
}

// Eq. 17-18 anneal smoothing of the MLP's TX input: for row q,
// out[q] = tx[idx[q]] + room_size * normals[q] * gamma (2 / cbrt(N_s)) (1 - i / tau)
// while i < tau, else tx[idx[q]] (idx NULL: row q itself).
__global__ void anneal_kernel(const float *tx, const int *idx, const float *normals, int Q,
                              int iter, int n_pos, float gamma, int tau, float rx, float ry,
                              float rz, float *out) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= Q) return;
    const int src = idx ? idx[q] : q;
    const float scale = iter < tau ? gamma * (2.f / cbrtf(static_cast<float>(n_pos))) *
                                         (1.f - static_cast<float>(iter) / static_cast<float>(tau))
                                   : 0.f;
    const float room[3] = {rx, ry, rz};
    for (int c = 0; c < 3; ++c)
        out[3 * q + c] = fmaf(room[c] * normals[3 * q + c], scale, tx[3 * src + c]);
}

}  // namespace

cudaError_t launch_anneal(const float *tx, const int *idx, const float *normals, int Q, int iter,
                          int n_pos, float gamma, int tau, const float *room_size, float *out,
                          cudaStream_t st) {
    if (Q == 0) return cudaSuccess;
    anneal_kernel<<<(Q + 127) / 128, 128, 0, st>>>(tx, idx, normals, Q, iter, n_pos, gamma, tau,
                                                   room_size[0], room_size[1], room_size[2], out);
    return cudaGetLastError();
}

size_t loss_ws_layout(int Q, int H, int W, float **coef, float **part) {
    const int tx = (W + kTile - 1) / kTile, ty = (H + kTile - 1) / kTile;
    const size_t c = (static_cast<size_t>(3) * Q * H * W * 4 + 255) & ~static_cast<size_t>(255);
    const size_t p = static_cast<size_t>(Q) * tx * ty * 2 * 4;
    if (coef) *coef = nullptr;
    if (part) *part = nullptr;
    return c + p;
}

cudaError_t launch_loss(const float *pred, const float *target, int Q, int H, int W, float lam,
                        float *out, float *d_pred, char *ws, cudaStream_t st) {
    if (Q == 0) return cudaSuccess;
    LossView v{};
    v.x = pred;
    v.y = target;
    v.Q = Q;
    v.H = H;
    v.W = W;
    v.tx = (W + kTile - 1) / kTile;
    v.ty = (H + kTile - 1) / kTile;
    v.lam = lam;
    const size_t c = (static_cast<size_t>(3) * Q * H * W * 4 + 255) & ~static_cast<size_t>(255);
    v.coef = reinterpret_cast<float *>(ws);
    v.part = reinterpret_cast<float *>(ws + c);
    v.dx = d_pred;
    v.out = out;
    dim3 grid(v.tx, v.ty, Q);
    ssim_stats_kernel<<<grid, kSsimThreads, 0, st>>>(v);
    if (d_pred) ssim_grad_kernel<<<grid, kSsimThreads, 0, st>>>(v);
    loss_reduce_kernel<<<1, 256, 0, st>>>(v);
    return cudaGetLastError();
}

cudaError_t launch_adam(const AdamGroup *groups, int n, int step, float beta1, float beta2,
                        float eps, cudaStream_t st) {
    if (n < 1 || n > kAdamGroups || step < 1) return cudaErrorInvalidValue;
    AdamArgs a{};
    a.n = n;
    a.start[0] = 0;
    for (int i = 0; i < n; ++i) {
        a.g[i] = groups[i];
        a.start[i + 1] = a.start[i] + groups[i].n;
    }
    a.beta1 = beta1;
    a.beta2 = beta2;
    a.eps = eps;
    a.bc1 = static_cast<float>(1.0 - std::pow(static_cast<double>(beta1), step));
    a.bc2 = static_cast<float>(1.0 - std::pow(static_cast<double>(beta2), step));
    const long long total = a.start[n];
    if (total == 0) return cudaSuccess;
    long long blocks = (total + 255) / 256;
    if (blocks > 148 * 8) blocks = 148 * 8;
    adam_kernel<<<static_cast<int>(blocks), 256, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace wrf
