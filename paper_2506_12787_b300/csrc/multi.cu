// Multi-scene batches: one launch sequence over queries of several resident
// scenes (Sec. 4.2: every scene is its own set of Gaussians G^0 with its own
// deformation network; a query is a TX position in one of them).
//
// A prepared scene set holds, per scene, what does not depend on the queries:
// the BF16 gamma(mean) rows and the BF16 tensor-core weight images (built by
// the single-scene preparation kernel), plus a device table of the scenes.
// Per batch the setup kernel turns the per-query scene indices into record
// offsets (qbase: query q's records are rows qbase[q] .. qbase[q+1]-1) and
// 128-row MLP tile ranges (tstart), and the per-query layer-1 term V[q] is
// formed with the query's own scene's first layer; then the tensor-core MLP
// (multi-scene variant), binning and the rasteriser run once over the whole
// batch.  A query's records and spectrum are computed exactly as in a
// single-scene launch, so they do not depend on the rest of the batch.
#include "kernels.h"

namespace wrf {

namespace {

inline size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

struct TableArgs {
    SceneEntry e[kMaxScenes];
    int S;
};

__global__ void multi_table_kernel(TableArgs t, SceneEntry *table) {
    const int i = threadIdx.x;
    if (i < t.S) table[i] = t.e[i];
}

// One block: qbase (records) and tstart (128-row tiles) as exclusive prefix
// sums over the queries; a query whose scene index is out of range has no
// Gaussians.  If the records exceed the capacity, every query is emptied and
// WRF_ENOSPC recorded.
constexpr int kSetupThreads = 1024;
__global__ void __launch_bounds__(kSetupThreads) multi_setup_kernel(
    const SceneEntry *table, int S, const int *scene_of, int Q, long long rec_capacity,
    long long *qbase, int *tstart, int *status) {
    __shared__ long long wr[32];
    __shared__ int wt[32];
    __shared__ long long carry_r;
    __shared__ int carry_t;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        carry_r = 0;
        carry_t = 0;
    }
    __syncthreads();
    for (int q0 = 0; q0 < Q; q0 += kSetupThreads) {
        const int q = q0 + threadIdx.x;
        int n = 0;
        if (q < Q) {
            const int sc = scene_of[q];
            n = (sc >= 0 && sc < S) ? table[sc].s.n : 0;
        }
        long long r = n;
        int t = (n + 127) / 128;
        // inclusive warp scans, then over warps
        for (int o = 1; o < 32; o <<= 1) {
            const long long yr = __shfl_up_sync(0xffffffffu, r, o);
            const int yt = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) {
                r += yr;
                t += yt;
            }
        }
        if (lane == 31) {
            wr[w] = r;
            wt[w] = t;
        }
        __syncthreads();
        if (w == 0) {
            long long a = wr[lane];
            int b = wt[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const long long ya = __shfl_up_sync(0xffffffffu, a, o);
                const int yb = __shfl_up_sync(0xffffffffu, b, o);
                if (lane >= o) {
                    a += ya;
                    b += yb;
                }
            }
            wr[lane] = a;
            wt[lane] = b;
        }
        __syncthreads();
        const long long br = carry_r + (w > 0 ? wr[w - 1] : 0);
        const int bt = carry_t + (w > 0 ? wt[w - 1] : 0);
        if (q < Q) {
            qbase[q] = br + r - n;
            tstart[q] = bt + t - (n + 127) / 128;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            carry_r += wr[31];
            carry_t += wt[31];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        qbase[Q] = carry_r;
        tstart[Q] = carry_t;
    }
    __syncthreads();
    if (carry_r > rec_capacity) {
        for (int q = threadIdx.x; q <= Q; q += kSetupThreads) {
            qbase[q] = 0;
            tstart[q] = 0;
        }
        if (threadIdx.x == 0) record_status(status, WRF_ENOSPC);
    }
}

// V[q][j] = W0(s_q)[j, dm:] gamma(tx_q) + b0(s_q)[j], four queries per block,
// thread j: the same features and summation order as the single-scene
// preparation, so a query's V is bit-identical to it.
constexpr int kVq = 4;
constexpr int kMaxPe = 3 * (2 * 15 + 1);
__global__ void __launch_bounds__(128) multi_v_kernel(const SceneEntry *table, int S,
                                                      const int *scene_of, MlpView m,
                                                      const float *tx, int Q, float *V) {
    __shared__ float gam[kVq][kMaxPe];
    const int q0 = blockIdx.x * kVq;
    const int din = m.dm + m.dt;
    const int L = m.L_tx;
    for (int e = threadIdx.x; e < kVq * m.dt; e += blockDim.x) {
        const int r = e / m.dt, f = e % m.dt, q = q0 + r;
        if (q >= Q) continue;
        const int i = f % 3, grp = f / 3;
        const PeArg x = pe_arg(tx[3 * q + i], m.room_min[i], m.room_size[i]);
        float val = pe_value(x);
        if (grp >= 1) {
            float sn, cs;
            pe_band(x, (grp - 1) % L, sn, cs);
            val = grp <= L ? sn : cs;
        }
        gam[r][f] = val;
    }
    __syncthreads();
    const int j = threadIdx.x;
    for (int r = 0; r < kVq; ++r) {
        const int q = q0 + r;
        if (q >= Q) break;
        const int sc = scene_of[q];
        if (sc < 0 || sc >= S) continue;
        const float *wrow = table[sc].W0 + static_cast<size_t>(j) * din + m.dm;
        float acc = 0.f;
#pragma unroll 16
        for (int k = 0; k < m.dt; ++k) acc = fmaf(wrow[k], gam[r][k], acc);
        V[static_cast<size_t>(q) * WRF_HIDDEN + j] = acc + table[sc].b0[j];
    }
}

// Bytes of one scene's BF16 weight images (as the single-scene preparation
// lays them out: W1m, hidden layers, output layer, bias image, selectors).
size_t image_bytes(int n_layers) {
    const int nh = n_layers - 2;
    return static_cast<size_t>(WRF_HIDDEN) * 128 + static_cast<size_t>(nh) * WRF_HIDDEN *
                                                        WRF_HIDDEN * 2 +
           16 * WRF_HIDDEN * 2 + kBiasImageBytes + kSelImageBytes;
}

}  // namespace

size_t multi_set_layout(const SceneView *s, int S, int n_layers, int k1, MultiSet *ms,
                        char *base) {
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char *p = base ? base + off : nullptr;
        off = align256(off + bytes);
        return p;
    };
    MultiSet m{};
    m.table = reinterpret_cast<SceneEntry *>(take(kMaxScenes * sizeof(SceneEntry)));
    m.wt_scratch = reinterpret_cast<float *>(take(static_cast<size_t>(6) * WRF_HIDDEN * WRF_HIDDEN * 4));
    m.wo_scratch = reinterpret_cast<float *>(take(WRF_HIDDEN * 8 * 4));
    for (int i = 0; i < S; ++i) {
        m.G[i] = reinterpret_cast<uint16_t *>(take(static_cast<size_t>(s[i].n > 0 ? s[i].n : 1) * k1 * 2));
        m.img[i] = reinterpret_cast<uint16_t *>(take(image_bytes(n_layers)));
    }
    if (ms) *ms = m;
    return off;
}

cudaError_t launch_multi_prepare(const SceneView *s, const MlpView *m, int S, const GridView &g,
                                 const MultiSet &ms, cudaStream_t st) {
    TableArgs t{};
    t.S = S;
    for (int i = 0; i < S; ++i) {
        DeformWs w{};
        w.G = ms.G[i];
        w.w_bf16 = ms.img[i];
        w.wt_f32 = ms.wt_scratch;  // the FP32 images are not used here
        w.wo_f32 = ms.wo_scratch;
        cudaError_t e = launch_prep(s[i], m[i], g, nullptr, 0, w, WRF_BF16, st);
        if (e != cudaSuccess) return e;
        t.e[i] = SceneEntry{s[i], ms.G[i], ms.img[i], m[i].W0, m[i].b0};
    }
    multi_table_kernel<<<1, 32, 0, st>>>(t, ms.table);
    return cudaGetLastError();
}

size_t multi_ws_layout(int Q, MultiWs *mw, char *base) {
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char *p = base ? base + off : nullptr;
        off = align256(off + bytes);
        return p;
    };
    MultiWs w{};
    w.tstart = reinterpret_cast<int *>(take(static_cast<size_t>(Q + 1) * 4));
    w.V = reinterpret_cast<float *>(take(static_cast<size_t>(Q > 0 ? Q : 1) * WRF_HIDDEN * 4));
    if (mw) *mw = w;
    return off;
}

cudaError_t launch_deform_project_multi(const MultiSet &ms, int S, const MlpView &m,
                                        const GridView &g, const int *scene_of, const float *tx,
                                        int Q, float4 *rec, long long rec_capacity,
                                        long long *qbase, const MultiWs &w, int *status,
                                        cudaStream_t st) {
    if (Q == 0) return cudaSuccess;
    multi_setup_kernel<<<1, kSetupThreads, 0, st>>>(ms.table, S, scene_of, Q, rec_capacity, qbase,
                                                    w.tstart, status);
    multi_v_kernel<<<(Q + kVq - 1) / kVq, WRF_HIDDEN, 0, st>>>(ms.table, S, scene_of, m, tx, Q,
                                                               w.V);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_mlp_tc_multi(ms.table, m, g, Q, scene_of, qbase, w.tstart, w.V, rec, status, st);
}

}  // namespace wrf
