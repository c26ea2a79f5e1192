// The paper's own primitive and deformation head (Sec. 4.1-4.2, Sec. 6.1).
//
// Primitive n: raw angular centre (u, v) normalised by the hyperbolic map
// (x = W (tanh u + 1) / 2 on the [0, 2 pi] azimuth axis, y = H (tanh v + 1) / 2
// on the [0, pi/2] elevation axis), covariance Sigma = L L^T from its Cholesky
// entries L = [[l1, 0], [l2, l3]] (Sec. 3.2), attenuation delta = sigmoid(a),
// complex response psi = (re, im).  The deformation network F (Eq. 14) maps
// [gamma(x/W, y/H), gamma(s)] to residuals (dmu_x, dmu_y, dpsi_re, dpsi_im,
// ddelta); the frame at s is (mu + dmu, Sigma, psi + dpsi, delta + ddelta)
// (Eq. 12, no covariance residual), rendered per channel with the weight
// (delta + ddelta) (psi_c + dpsi_c) (Eq. 13) by the two-channel rasteriser.
//
// Network: n_hidden Linear+ReLU layers of width <= 160 (the paper: 8 x 156),
// the encoded input concatenated to the activations entering hidden layers 2,
// 4 and 6 (0-based: a skip every two layers), a Linear output of width 5.  A
// layer whose input holds the encoding splits exactly into
//   W [h; gamma(mu_n); gamma(s_q)] + b = W_h h + U[n] + V[q],
// U[n] = W_mu gamma(mu_n) once per Gaussian, V[q] = W_s gamma(s_q) + b once per
// query (prep kernels), so a row pays only the hidden-to-hidden products.
// Those run as a register-tiled FP32 product: a CTA holds 64 rows of one
// query, activations transposed ([input][row]) in shared memory, thread t the
// 4 x 8 output tile rows 4 (t % 16) .., columns 8 (t / 16) .. (320 threads over
// 64 x 160), weights streamed 16 inputs (10 KB) at a time through two cp.async
// buffers (two CTAs per SM); each output sums its
// add-term then w_k h_k in ascending k.  The epilogue evaluates the output
// layer and the projection and writes the records (w = real weight) and the
// imaginary weights after them.
#include "kernels.h"
#include "paper.cuh"

namespace wrf {

namespace {

constexpr int kPW = kPaperMaxWidth;   // padded width (160)
constexpr int kRows = 64;             // rows per CTA
constexpr int kThreads = 320;         // 16 row groups x 20 column groups
constexpr int kPitch = kRows + 4;     // floats per input of the transposed activations
constexpr int kKC = 16;               // weight rows (inputs) per staged chunk (two buffers)
constexpr int kEnc = 4;               // layers with the encoding in their input: 0, 2, 4, 6


struct PaperNet {
    int n_hidden, width, dm, dt, L_mean, L_tx;
    float room_min[3], room_size[3];
    const float *W[kPaperMaxLayers], *b[kPaperMaxLayers];
};

// Column offset of the mean-encoding block in layer l's input.
__device__ __forceinline__ int mu_off(const PaperNet &m, int l) { return l == 0 ? 0 : m.width; }
__device__ __forceinline__ int in_dim(const PaperNet &m, int l) {
    return (l == 0 ? 0 : m.width) + (l == 0 || is_skip(l) ? m.dm + m.dt : 0);
}

// U[e][n][j] for the encoding layers, 32 Gaussians per block, thread = j.
__global__ void __launch_bounds__(kPW) paper_mean_kernel(PaperView s, PaperNet m, GridView g,
                                                         float *U) {
    __shared__ float gam[32][2 * (2 * 15 + 1)];
    const int n0 = blockIdx.x * 32;
    if (threadIdx.x < 32 && n0 + threadIdx.x < s.n) {
        const float2 mu = reinterpret_cast<const float2 *>(s.mu)[n0 + threadIdx.x];
        const PeArg a[2] = {unit_centre(mu.x), unit_centre(mu.y)};
        pe_encode(a, 2, m.L_mean, gam[threadIdx.x]);
    }
    __syncthreads();
    const int j = threadIdx.x;
    for (int l = 0; l < m.n_hidden; ++l) {
        if (l != 0 && !is_skip(l)) continue;
        float acc[32];
#pragma unroll
        for (int r = 0; r < 32; ++r) acc[r] = 0.f;
        if (j < m.width) {
            const float *wr = m.W[l] + static_cast<size_t>(j) * in_dim(m, l) + mu_off(m, l);
            for (int k = 0; k < m.dm; ++k) {
                const float w = __ldg(wr + k);
#pragma unroll
                for (int r = 0; r < 32; ++r) acc[r] = fmaf(w, gam[r][k], acc[r]);
            }
        }
        float *Ue = U + static_cast<size_t>(enc_index(l)) * s.n * kPW;
        for (int r = 0; r < 32 && n0 + r < s.n; ++r) Ue[static_cast<size_t>(n0 + r) * kPW + j] = acc[r];
    }
}

// V[e][q][j] = W_s gamma(s_q) + b for the encoding layers, one query per block.
__global__ void __launch_bounds__(kPW) paper_tx_kernel(PaperNet m, const float *tx, int Q, float *V) {
    __shared__ float gam[3 * (2 * 15 + 1)];
    const int q = blockIdx.x;
    if (threadIdx.x == 0) {
        PeArg a[3];
        for (int c = 0; c < 3; ++c) a[c] = pe_arg(tx[3 * q + c], m.room_min[c], m.room_size[c]);
        pe_encode(a, 3, m.L_tx, gam);
    }
    __syncthreads();
    const int j = threadIdx.x;
    for (int l = 0; l < m.n_hidden; ++l) {
        if (l != 0 && !is_skip(l)) continue;
        float acc = 0.f;
        if (j < m.width) {
            const float *wr = m.W[l] + static_cast<size_t>(j) * in_dim(m, l) + mu_off(m, l) + m.dm;
            for (int k = 0; k < m.dt; ++k) acc = fmaf(__ldg(wr + k), gam[k], acc);
            acc += m.b[l][j];
        }
        V[(static_cast<size_t>(enc_index(l)) * Q + q) * kPW + j] = acc;
    }
}

// Transposed, zero-padded hidden-to-hidden weights Wt[l][k][j] (l = 1 ..
// n_hidden-1), biases of the layers without the encoding, output layer
// Wo[k][8].
__global__ void paper_weights_kernel(PaperNet m, float *Wt, float *bh, float *Wo) {
    const long long per = static_cast<long long>(kPW) * kPW;
    const long long total = (kPaperMaxLayers - 1) * per + kPaperMaxLayers * kPW + kPW * 8;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        if (i < (kPaperMaxLayers - 1) * per) {
            const int l = 1 + static_cast<int>(i / per);
            const int k = static_cast<int>((i % per) / kPW), j = static_cast<int>(i % kPW);
            float v = 0.f;
            if (l < m.n_hidden && k < m.width && j < m.width)
                v = m.W[l][static_cast<size_t>(j) * in_dim(m, l) + k];
            Wt[i] = v;
        } else if (i < (kPaperMaxLayers - 1) * per + kPaperMaxLayers * kPW) {
            const long long e = i - (kPaperMaxLayers - 1) * per;
            const int l = static_cast<int>(e / kPW), j = static_cast<int>(e % kPW);
            bh[e] = (l > 0 && l < m.n_hidden && !is_skip(l) && j < m.width) ? m.b[l][j] : 0.f;
        } else {
            const long long e = i - (kPaperMaxLayers - 1) * per - kPaperMaxLayers * kPW;
            const int k = static_cast<int>(e / 8), o = static_cast<int>(e % 8);
            Wo[e] = (k < m.width && o < WRF_OUT) ? m.W[m.n_hidden][static_cast<size_t>(o) * m.width + k]
                                                 : 0.f;
        }
    }
}

struct PaperArgs {
    PaperView s;
    PaperNet m;
    GridView g;
    int Q, tpq;
    const float *U, *V, *Wt, *bh, *Wo;
    int deform;  // 0: no network (residuals 0)
    float4 *rec;
    float *rec_im;
};

__global__ void __launch_bounds__(kThreads, 2) paper_mlp_kernel(PaperArgs a) {
    extern __shared__ __align__(16) float smem[];
    float *wbuf = smem;                                  // [kKC][kPW]
    float *hin = smem + 2 * kKC * kPW, *hout = hin + kPW * kPitch;
    __shared__ float dout[kRows][8];
    const int tid = threadIdx.x, q = blockIdx.y;
    const int n0 = blockIdx.x * kRows;
    const int N = a.s.n;
    const int rg = tid % 16, cg = tid / 16;
    const PaperNet &m = a.m;
    if (a.deform) {
        // weight chunks (kKC inputs x 160 outputs) stream through two buffers
        // with cp.async, one chunk ahead of the products
        const int nchunk = (m.n_hidden - 1) * (kPW / kKC);
        auto stage = [&](int s) {
            const int l = 1 + s / (kPW / kKC), k0 = (s % (kPW / kKC)) * kKC;
            const float4 *src = reinterpret_cast<const float4 *>(
                a.Wt + (static_cast<size_t>(l - 1) * kPW + k0) * kPW);
            float4 *dst = reinterpret_cast<float4 *>(wbuf + (s & 1) * kKC * kPW);
            for (int i = tid; i < kKC * kPW / 4; i += kThreads) cp_async16(dst + i, src + i);
            cp_async_commit();
        };
        if (nchunk > 0) stage(0);
        // layer 0: h = relu(U0[n] + V0[q]); lanes take consecutive rows so the
        // transposed stores are conflict-free, each loading 4 columns
        const float *U0 = a.U, *V0 = a.V + static_cast<size_t>(q) * kPW;
        for (int e = tid; e < kRows * kPW / 4; e += kThreads) {
            const int r = e % kRows, j4 = 4 * (e / kRows), n = n0 + r;
            float4 u = make_float4(0.f, 0.f, 0.f, 0.f);
            if (n < N) u = __ldg(reinterpret_cast<const float4 *>(U0 + static_cast<size_t>(n) * kPW + j4));
            const float4 v = __ldg(reinterpret_cast<const float4 *>(V0 + j4));
            const bool ok = n < N;
            hin[(j4 + 0) * kPitch + r] = ok ? fmaxf(u.x + v.x, 0.f) : 0.f;
            hin[(j4 + 1) * kPitch + r] = ok ? fmaxf(u.y + v.y, 0.f) : 0.f;
            hin[(j4 + 2) * kPitch + r] = ok ? fmaxf(u.z + v.z, 0.f) : 0.f;
            hin[(j4 + 3) * kPitch + r] = ok ? fmaxf(u.w + v.w, 0.f) : 0.f;
        }
        float acc[4][8];
        for (int s = 0; s < nchunk; ++s) {
            const int l = 1 + s / (kPW / kKC), kc = s % (kPW / kKC);
            if (kc == 0) {
                if (is_skip(l)) {
                    const float *Ul = a.U + static_cast<size_t>(enc_index(l)) * N * kPW;
                    const float *Vl = a.V + (static_cast<size_t>(enc_index(l)) * a.Q + q) * kPW;
                    const float4 va = __ldg(reinterpret_cast<const float4 *>(Vl + 8 * cg));
                    const float4 vb = __ldg(reinterpret_cast<const float4 *>(Vl + 8 * cg + 4));
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        const int n = min(n0 + 4 * rg + r, N - 1);
                        const float *ur = Ul + static_cast<size_t>(n) * kPW + 8 * cg;
                        const float4 ua = __ldg(reinterpret_cast<const float4 *>(ur));
                        const float4 ub = __ldg(reinterpret_cast<const float4 *>(ur + 4));
                        acc[r][0] = ua.x + va.x;
                        acc[r][1] = ua.y + va.y;
                        acc[r][2] = ua.z + va.z;
                        acc[r][3] = ua.w + va.w;
                        acc[r][4] = ub.x + vb.x;
                        acc[r][5] = ub.y + vb.y;
                        acc[r][6] = ub.z + vb.z;
                        acc[r][7] = ub.w + vb.w;
                    }
                } else {
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        const float bv = a.bh[l * kPW + 8 * cg + c];
#pragma unroll
                        for (int r = 0; r < 4; ++r) acc[r][c] = bv;
                    }
                }
            }
            // chunk s has landed for every thread, and every thread is done
            // with the buffer the next chunk overwrites (and with the layer
            // outputs written before this point)
            cp_async_wait_all();
            __syncthreads();
            if (s + 1 < nchunk) stage(s + 1);
            const float *wb = wbuf + (s & 1) * kKC * kPW;
            const float *hk = hin + kc * kKC * kPitch;
#pragma unroll 8
            for (int k = 0; k < kKC; ++k) {
                const float4 hv = *reinterpret_cast<const float4 *>(hk + k * kPitch + 4 * rg);
                const float4 wa = *reinterpret_cast<const float4 *>(wb + k * kPW + 8 * cg);
                const float4 wc = *reinterpret_cast<const float4 *>(wb + k * kPW + 8 * cg + 4);
                const float h[4] = {hv.x, hv.y, hv.z, hv.w};
                const float w[8] = {wa.x, wa.y, wa.z, wa.w, wc.x, wc.y, wc.z, wc.w};
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int c = 0; c < 8; ++c) acc[r][c] = fmaf(w[c], h[r], acc[r][c]);
            }
            if (kc == kPW / kKC - 1) {
#pragma unroll
                for (int c = 0; c < 8; ++c)
                    *reinterpret_cast<float4 *>(hout + (8 * cg + c) * kPitch + 4 * rg) =
                        make_float4(fmaxf(acc[0][c], 0.f), fmaxf(acc[1][c], 0.f),
                                    fmaxf(acc[2][c], 0.f), fmaxf(acc[3][c], 0.f));
                float *t = hin;
                hin = hout;
                hout = t;
            }
        }
        __syncthreads();
        // output layer: thread (row, output) = (tid / 5, tid % 5)
        for (int i = tid; i < kPW * 8; i += kThreads) wbuf[i] = a.Wo[i];  // 2 x 16 x 160 >= 1280
        __syncthreads();
        {
            const int r = tid / WRF_OUT, o = tid % WRF_OUT;
            float acc = m.b[m.n_hidden][o];
            for (int k = 0; k < kPW; ++k) acc = fmaf(wbuf[k * 8 + o], hin[k * kPitch + r], acc);
            dout[r][o] = acc;
        }
    } else if (tid < kRows * WRF_OUT) {
        dout[tid / WRF_OUT][tid % WRF_OUT] = 0.f;
    }
    __syncthreads();
    // projection (Eq. 12-13 with the paper's primitive), one thread per row
    if (tid < kRows && n0 + tid < N)
        paper_project(a.s, n0 + tid, q, dout[tid], a.g, a.rec, a.rec_im);
}

inline size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

}  // namespace

size_t paper_ws_layout(int n, int Q, PaperWs *ws, char *base) {
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char *p = base ? base + off : nullptr;
        off = align256(off + bytes);
        return reinterpret_cast<float *>(p);
    };
    PaperWs w{};
    w.U = take(static_cast<size_t>(kEnc) * (n > 0 ? n : 1) * kPW * 4);
    w.V = take(static_cast<size_t>(kEnc) * (Q > 0 ? Q : 1) * kPW * 4);
    w.Wt = take(static_cast<size_t>(kPaperMaxLayers - 1) * kPW * kPW * 4);
    w.bh = take(static_cast<size_t>(kPaperMaxLayers) * kPW * 4);
    w.Wo = take(static_cast<size_t>(kPW) * 8 * 4);
    // BF16 gamma(mean) rows [N][64], then (three-product precision) their remainders
    w.G = reinterpret_cast<uint16_t *>(take(static_cast<size_t>(n > 0 ? n : 1) * 64 * 2 * 2));
    w.vec = take(static_cast<size_t>(Q > 0 ? Q : 1) * (kPaperMaxLayers - 1) * kPW * 4);
    w.img = reinterpret_cast<uint16_t *>(take(paper_tc_image_bytes(kPaperMaxLayers - 1)));
    if (ws) *ws = w;
    return off;
}

cudaError_t launch_paper(const PaperSceneView &sv, const PaperMlpView *mv, const GridView &g,
                         const float *tx, int Q, const PaperWs &ws, float4 *rec, cudaStream_t st) {
    const long long rows = static_cast<long long>(Q) * sv.n;
    if (rows == 0) return cudaSuccess;
    PaperArgs a{};
    a.s = PaperView{sv.n, sv.mu, sv.chol, sv.attn_logit, sv.psi};
    a.g = g;
    a.Q = Q;
    a.tpq = (sv.n + kRows - 1) / kRows;
    a.rec = rec;
    a.rec_im = reinterpret_cast<float *>(rec + 2 * rows);
    a.deform = mv != nullptr;
    if (mv) {
        PaperNet &m = a.m;
        m.n_hidden = mv->n_hidden;
        m.width = mv->width;
        m.L_mean = mv->L_mean;
        m.L_tx = mv->L_tx;
        m.dm = 2 * (2 * mv->L_mean + 1);
        m.dt = 3 * (2 * mv->L_tx + 1);
        for (int i = 0; i < 3; ++i) {
            m.room_min[i] = mv->room_min[i];
            m.room_size[i] = mv->room_size[i];
        }
        for (int l = 0; l <= mv->n_hidden; ++l) {
            m.W[l] = mv->W[l];
            m.b[l] = mv->b[l];
        }
        a.U = ws.U;
        a.V = ws.V;
        a.Wt = ws.Wt;
        a.bh = ws.bh;
        a.Wo = ws.Wo;
        paper_mean_kernel<<<(sv.n + 31) / 32, kPW, 0, st>>>(a.s, m, g, ws.U);
        paper_tx_kernel<<<Q, kPW, 0, st>>>(m, tx, Q, ws.V);
        paper_weights_kernel<<<148 * 4, 256, 0, st>>>(m, ws.Wt, ws.bh, ws.Wo);
    }
    const size_t smem = (static_cast<size_t>(2 * kKC) * kPW + 2 * kPW * kPitch) * 4;
    cudaError_t e = cudaFuncSetAttribute(paper_mlp_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    dim3 grid(a.tpq, Q);
    paper_mlp_kernel<<<grid, kThreads, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace wrf
