// C ABI entry points (include/wrf.h): argument checks, workspace carve-up and
// kernel launches.  No entry point allocates device memory or synchronises,
// except wrf_status_read which is documented to synchronise its stream.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <cuda.h>

#include <mutex>

#include "kernels.h"

namespace {

thread_local char g_err[512] = "";

__device__ int g_status;  // first device-side error since the last read

wrf_status fail(wrf_status s, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return s;
}

wrf_status cuda_fail(cudaError_t e, const char *where) {
    return fail(WRF_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

// Device address of a __device__ symbol in the current device's context,
// cached per device together with the context it was looked up in: after a
// device reset (a new primary context, where the module and its symbols may
// sit elsewhere) the address is looked up again.  The first lookup in a
// context should happen outside stream capture.  Returns the CUDA error.
struct SymbolCache {
    void *ptr[64] = {nullptr};
    unsigned long long ctx_id[64] = {0};  // unique id of the context (never reused)
    std::mutex mu;
};

cudaError_t symbol_ptr(SymbolCache &c, const void *symbol, void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    // make the device's primary context current (initialises it if needed)
    e = cudaSetDevice(dev);
    if (e != cudaSuccess) return e;
    // the driver calls are fetched through the runtime, so the library has
    // no link-time dependency on the driver library
    using GetCurrentFn = CUresult (*)(CUcontext *);
    using GetIdFn = CUresult (*)(CUcontext, unsigned long long *);
    static GetCurrentFn get_current = nullptr;
    static GetIdFn get_id = nullptr;
    {
        std::lock_guard<std::mutex> lock(c.mu);
        if (!get_current || !get_id) {
            void *f0 = nullptr, *f1 = nullptr;
            cudaDriverEntryPointQueryResult r0, r1;
            if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f0, 12000, cudaEnableDefault,
                                                 &r0) != cudaSuccess ||
                cudaGetDriverEntryPointByVersion("cuCtxGetId", &f1, 12000, cudaEnableDefault,
                                                 &r1) != cudaSuccess ||
                r0 != cudaDriverEntryPointSuccess || r1 != cudaDriverEntryPointSuccess)
                return cudaErrorSymbolNotFound;
            get_current = reinterpret_cast<GetCurrentFn>(f0);
            get_id = reinterpret_cast<GetIdFn>(f1);
        }
    }
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
        return cudaErrorDeviceUninitialized;
    std::lock_guard<std::mutex> lock(c.mu);
    if (!c.ptr[dev] || c.ctx_id[dev] != id) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, symbol);
        if (e != cudaSuccess) return e;
        c.ptr[dev] = p;
        c.ctx_id[dev] = id;
    }
    *out = c.ptr[dev];
    return cudaSuccess;
}

// Device address of g_status for the current device, or NULL.
int *status_ptr() {
    static SymbolCache cache;
    void *p = nullptr;
    if (symbol_ptr(cache, reinterpret_cast<const void *>(&g_status), &p) != cudaSuccess)
        return nullptr;
    return static_cast<int *>(p);
}

// Scratch for wrf_bin_noalloc: a fixed array in device memory that exists on
// every device that loads this library, for the life of the process.  Host
// code may not use the symbol as an address; bin_scratch_ptr() asks the
// runtime for its device address.
constexpr size_t kBinScratchBytes = size_t(4) << 20;  // 4 MiB
__device__ __align__(256) unsigned char g_bin_scratch[kBinScratchBytes];

// Device address of g_bin_scratch on the current device (see symbol_ptr: the
// first wrf_bin_noalloc call in a context should come before any stream
// capture).  Returns the CUDA error.
cudaError_t bin_scratch_ptr(void **out) {
    static SymbolCache cache;
    return symbol_ptr(cache, reinterpret_cast<const void *>(g_bin_scratch), out);
}

bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

wrf_status check_scene(const wrf_scene *s) {
    if (!s) return fail(WRF_EINVAL, "scene is NULL");
    if (s->n < 0) return fail(WRF_EINVAL, "scene.n < 0");
    if (s->channels != 1 && s->channels != 2)
        return fail(WRF_EUNSUPPORTED, "channels must be 1 or 2");
    if (s->n > 0 && (!s->mean || !s->log_scale || !s->rot || !s->opacity_logit || !s->amp))
        return fail(WRF_EINVAL, "scene array is NULL");
    if (s->n > 0 && (!aligned(s->mean, 8) || !aligned(s->log_scale, 8)))
        return fail(WRF_EINVAL, "scene.mean / log_scale must be 8-byte aligned");
    return WRF_OK;
}

wrf_status check_grid(const wrf_grid *g, wrf::GridView *v) {
    if (!g) return fail(WRF_EINVAL, "grid is NULL");
    if (g->H < 1 || g->W < 1 || g->H > 65536 || g->W > 65536)
        return fail(WRF_EINVAL, "grid H/W out of range");
    // every supported shape is a power of two on both axes: the device code
    // takes tile indices by shift (tile_of)
    if (!wrf::render_config_supported(g->tile_w, g->tile_h))
        return fail(WRF_EUNSUPPORTED, "tile %dx%d not supported", g->tile_w, g->tile_h);
    if (!(g->q_cut > 0.f)) return fail(WRF_EINVAL, "q_cut must be > 0 (or +inf)");
    v->H = g->H;
    v->W = g->W;
    v->tw = g->tile_w;
    v->th = g->tile_h;
    v->ntx = (g->W + g->tile_w - 1) / g->tile_w;
    v->nty = (g->H + g->tile_h - 1) / g->tile_h;
    v->T = v->ntx * v->nty;
    v->q_cut = g->q_cut;
    if (g->wrap_x != 0 && g->wrap_x != 1) return fail(WRF_EINVAL, "wrap_x must be 0 or 1");
    if (g->wrap_x && !(g->q_cut < INFINITY)) return fail(WRF_EINVAL, "wrap_x needs a finite q_cut");
    v->wrap = g->wrap_x;
    if (v->T > 3000) return fail(WRF_EUNSUPPORTED, "more than 3000 tiles");
    v->px = g->px_per_thread ? g->px_per_thread : 2;
    v->bpt = g->batch_factor ? g->batch_factor : 1;
    if (v->px != 2 && v->px != 4) return fail(WRF_EUNSUPPORTED, "px_per_thread must be 2 or 4");
    if (v->bpt != 1 && v->bpt != 2) return fail(WRF_EUNSUPPORTED, "batch_factor must be 1 or 2");
    if (v->px == 4 && g->tile_w < 16)
        return fail(WRF_EUNSUPPORTED, "px_per_thread 4 needs tile_w >= 16");
    if (g->tma_staging != 0 && g->tma_staging != 1)
        return fail(WRF_EINVAL, "tma_staging must be 0 or 1");
    v->tma = g->tma_staging;
    return WRF_OK;
}

wrf_status check_mlp(const wrf_mlp *m, wrf::MlpView *v) {
    if (!m) return fail(WRF_EINVAL, "mlp is NULL");
    if (m->n_layers < 2 || m->n_layers > WRF_MAX_LAYERS)
        return fail(WRF_EUNSUPPORTED, "n_layers must be in [2, 8]");
    if (m->L_mean < 0 || m->L_mean > 15 || m->L_tx < 0 || m->L_tx > 15)
        return fail(WRF_EUNSUPPORTED, "frequency bands must be in [0, 15]");
    const int dm = 2 * (2 * m->L_mean + 1), dt = 3 * (2 * m->L_tx + 1);
    if (m->dims[0] != dm + dt) return fail(WRF_EINVAL, "dims[0] != 2(2L_mean+1)+3(2L_tx+1)");
    for (int l = 1; l < m->n_layers; ++l)
        if (m->dims[l] != WRF_HIDDEN) return fail(WRF_EUNSUPPORTED, "hidden widths must be 128");
    if (m->dims[m->n_layers] != WRF_OUT) return fail(WRF_EUNSUPPORTED, "output width must be 5");
    for (int l = 0; l < m->n_layers; ++l)
        if (!m->W[l] || !m->b[l]) return fail(WRF_EINVAL, "weight %d is NULL", l);
    for (int i = 0; i < 3; ++i)
        if (!(m->room_size[i] > 0.f)) return fail(WRF_EINVAL, "room_size must be > 0");
    if (m->precision != WRF_FP32 && m->precision != WRF_BF16 && m->precision != WRF_BF16X3)
        return fail(WRF_EINVAL, "unknown precision");
    if (m->precision != WRF_FP32 && m->n_layers > 5)
        return fail(WRF_EUNSUPPORTED, "tensor-core path keeps <= 3 hidden layers resident");
    v->n_layers = m->n_layers;
    v->dm = dm;
    v->dt = dt;
    v->L_mean = m->L_mean;
    v->L_tx = m->L_tx;
    for (int i = 0; i < 3; ++i) {
        v->room_min[i] = m->room_min[i];
        v->room_size[i] = m->room_size[i];
    }
    v->W0 = m->W[0];
    v->b0 = m->b[0];
    for (int l = 0; l < 8; ++l) {
        v->Wh[l] = (l + 1 < m->n_layers - 1) ? m->W[l + 1] : nullptr;
        v->bh[l] = (l + 1 < m->n_layers - 1) ? m->b[l + 1] : nullptr;
    }
    v->Wo = m->W[m->n_layers - 1];
    v->bo = m->b[m->n_layers - 1];
    return WRF_OK;
}

wrf::SceneView view(const wrf_scene *s) {
    return wrf::SceneView{s->n, s->mean, s->log_scale, s->rot, s->opacity_logit, s->amp,
                          s->channels};
}

bool rows_ok(int n, int Q) { return static_cast<long long>(n) * Q < (1ll << 31); }

// One thread waits, with the library's bounded wait, on an mbarrier phase
// that never completes (arrival count 2, one arrival): the wait gives up
// after limit_ns and records WRF_ETIMEOUT.  Nothing faults or hangs.
__global__ void selftest_wait_kernel(unsigned long long limit_ns, int *status, int *waited) {
    __shared__ __align__(8) uint64_t bar;
    wrf::mbar_init(&bar, 2);
    wrf::fence_mbar_init();
    wrf::mbar_arrive(&bar);
    const bool ok = wrf::mbar_wait(&bar, 0, status, limit_ns);
    *waited = ok ? 1 : 0;
}

}  // namespace

extern "C" {

int32_t wrf_version(void) { return 1; }

wrf_status wrf_selftest_wait(int64_t limit_ns, int32_t *completed, void *stream) {
    if (limit_ns <= 0 || limit_ns > 2000000000ll)
        return fail(WRF_EINVAL, "limit_ns must be in (0, 2e9]");
    if (!completed) return fail(WRF_EINVAL, "completed is NULL");
    int *st = status_ptr();
    if (!st) return fail(WRF_ECUDA, "status word unavailable");
    selftest_wait_kernel<<<1, 1, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<unsigned long long>(limit_ns), st, completed);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "wrf_selftest_wait");
    return WRF_OK;
}

const char *wrf_last_error(void) { return g_err; }

wrf_status wrf_status_read(void *stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int *p = status_ptr();
    if (!p) return fail(WRF_ECUDA, "status word unavailable");
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, p, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "wrf_status_read");
    if (h != 0) {
        int z = 0;
        e = cudaMemcpyAsync(p, &z, sizeof(int), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "wrf_status_read");
        return fail(static_cast<wrf_status>(h), "device status %d", h);
    }
    return WRF_OK;
}

size_t wrf_deform_workspace_size(int32_t n, int32_t Q, const wrf_mlp *mlp) {
    int nl = mlp ? mlp->n_layers : 5;
    return wrf::deform_ws_layout(n < 0 ? 0 : n, Q < 0 ? 0 : Q, nl, nullptr, nullptr);
}

static wrf_status deform_common(const wrf_scene *scene, const wrf_mlp *mlp, const wrf_grid *grid,
                                const float *tx, int32_t Q, int mode, float *resid, float *rec,
                                uint32_t *tile_count, float *acts, void *ws, size_t ws_bytes,
                                void *stream) {
    wrf_status s;
    wrf::GridView g{};
    wrf::MlpView m{};
    if ((s = check_scene(scene)) != WRF_OK) return s;
    if ((s = check_mlp(mlp, &m)) != WRF_OK) return s;
    if ((s = check_grid(grid, &g)) != WRF_OK) return s;
    if (Q < 0) return fail(WRF_EINVAL, "Q < 0");
    if (!rows_ok(scene->n, Q)) return fail(WRF_EUNSUPPORTED, "Q*N must be < 2^31");
    if (Q > 0 && !tx) return fail(WRF_EINVAL, "tx is NULL");
    if (mode == 0 && Q > 0 && scene->n > 0 && !resid) return fail(WRF_EINVAL, "resid is NULL");
    if (acts && mlp->precision == WRF_BF16)
        return fail(WRF_EUNSUPPORTED, "saved activations need the FP32 or BF16X3 MLP");
    if (acts && !aligned(acts, 16)) return fail(WRF_EINVAL, "acts must be 16-byte aligned");
    if (mode == 1 && Q > 0 && scene->n > 0 && (!rec || !aligned(rec, 16)))
        return fail(WRF_EINVAL, "rec must be non-NULL and 16-byte aligned");
    size_t need = wrf::deform_ws_layout(scene->n, Q, mlp->n_layers, nullptr, nullptr);
    if (ws_bytes < need || !ws || !aligned(ws, 256))
        return fail(WRF_EINVAL, "workspace: need %zu bytes, 256-byte aligned", need);
    if (Q == 0 || scene->n == 0) return WRF_OK;
    wrf::DeformWs w{};
    wrf::deform_ws_layout(scene->n, Q, mlp->n_layers, &w, static_cast<char *>(ws));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    wrf::SceneView sv = view(scene);
    int *status = status_ptr();
    cudaError_t e = wrf::launch_prep(sv, m, g, tx, Q, w, mlp->precision, st);
    if (e != cudaSuccess) return cuda_fail(e, "prep");
    if (mlp->precision == WRF_BF16)
        e = wrf::launch_mlp_tc(sv, m, g, Q, w, mode, resid, reinterpret_cast<float4 *>(rec),
                               tile_count, status, st);
    else if (mlp->precision == WRF_BF16X3)
        e = wrf::launch_mlp_x3(sv, m, g, Q, w, mode, resid, reinterpret_cast<float4 *>(rec),
                               tile_count, acts, status, st);
    else
        e = wrf::launch_mlp_f32(sv, m, g, Q, w, mode, resid, reinterpret_cast<float4 *>(rec),
                                tile_count, acts, st);
    if (e != cudaSuccess) return cuda_fail(e, "mlp");
    return WRF_OK;
}

wrf_status wrf_deform(const wrf_scene *scene, const wrf_mlp *mlp, const wrf_grid *grid,
                      const float *tx, int32_t Q, float *resid, void *ws, size_t ws_bytes,
                      void *stream) {
    return deform_common(scene, mlp, grid, tx, Q, 0, resid, nullptr, nullptr, nullptr, ws,
                         ws_bytes, stream);
}

wrf_status wrf_deform_acts(const wrf_scene *scene, const wrf_mlp *mlp, const wrf_grid *grid,
                           const float *tx, int32_t Q, float *resid, float *acts, void *ws,
                           size_t ws_bytes, void *stream) {
    if (Q > 0 && scene && scene->n > 0 && !acts) return fail(WRF_EINVAL, "acts is NULL");
    return deform_common(scene, mlp, grid, tx, Q, 0, resid, nullptr, nullptr, acts, ws, ws_bytes,
                         stream);
}

wrf_status wrf_deform_project(const wrf_scene *scene, const wrf_mlp *mlp, const wrf_grid *grid,
                              const float *tx, int32_t Q, float *rec, uint32_t *tile_count,
                              void *ws, size_t ws_bytes, void *stream) {
    return deform_common(scene, mlp, grid, tx, Q, 1, nullptr, rec, tile_count, nullptr, ws,
                         ws_bytes, stream);
}

size_t wrf_loss_workspace_size(int32_t Q, int32_t H, int32_t W) {
    if (Q < 0 || H < 1 || W < 1) return 0;
    return wrf::loss_ws_layout(Q, H, W, nullptr, nullptr);
}

wrf_status wrf_loss(const float *pred, const float *target, int32_t Q, int32_t H, int32_t W,
                    float lambda1, float *out, float *d_pred, void *ws, size_t ws_bytes,
                    void *stream) {
    if (Q < 0 || H < 1 || W < 1) return fail(WRF_EINVAL, "loss: Q >= 0, H >= 1, W >= 1");
    if (static_cast<long long>(Q) * H * W >= (1ll << 31))
        return fail(WRF_EUNSUPPORTED, "loss: Q*H*W must be < 2^31");
    if (!(lambda1 >= 0.f && lambda1 <= 1.f)) return fail(WRF_EINVAL, "lambda1 must be in [0, 1]");
    if (Q == 0) return WRF_OK;
    if (!pred || !target || !out) return fail(WRF_EINVAL, "pred / target / out is NULL");
    const size_t need = wrf::loss_ws_layout(Q, H, W, nullptr, nullptr);
    if (ws_bytes < need || !ws || !aligned(ws, 256))
        return fail(WRF_EINVAL, "workspace: need %zu bytes, 256-byte aligned", need);
    cudaError_t e = wrf::launch_loss(pred, target, Q, H, W, lambda1, out, d_pred,
                                     static_cast<char *>(ws), static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "loss");
    return WRF_OK;
}

wrf_status wrf_adam(const wrf_adam_group *groups, int32_t n_groups, int32_t step, float beta1,
                    float beta2, float eps, void *stream) {
    if (n_groups < 1 || n_groups > wrf::kAdamGroups || !groups)
        return fail(WRF_EINVAL, "adam: 1..%d groups", wrf::kAdamGroups);
    if (step < 1) return fail(WRF_EINVAL, "adam: step >= 1");
    if (!(beta1 >= 0.f && beta1 < 1.f && beta2 >= 0.f && beta2 < 1.f && eps > 0.f))
        return fail(WRF_EINVAL, "adam: betas in [0, 1), eps > 0");
    wrf::AdamGroup g[wrf::kAdamGroups];
    for (int i = 0; i < n_groups; ++i) {
        const wrf_adam_group &a = groups[i];
        if (a.n < 0) return fail(WRF_EINVAL, "adam: group %d has n < 0", i);
        if (a.n > 0 && (!a.param || !a.grad || !a.m || !a.v))
            return fail(WRF_EINVAL, "adam: group %d has a NULL array", i);
        g[i] = wrf::AdamGroup{a.param, a.grad, a.m, a.v, static_cast<long long>(a.n), a.lr};
    }
    cudaError_t e = wrf::launch_adam(g, n_groups, step, beta1, beta2, eps,
                                     static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "adam");
    return WRF_OK;
}

wrf_status wrf_anneal_tx(const float *tx, const int32_t *idx, int32_t n_positions,
                         const float *normals, int32_t Q, int32_t iter, float gamma, int32_t tau,
                         const float room_size[3], float *tx_out, void *stream) {
    if (Q < 0 || n_positions < 1 || tau < 1 || iter < 0)
        return fail(WRF_EINVAL, "anneal: Q >= 0, n_positions >= 1, tau >= 1, iter >= 0");
    if (!room_size || !(room_size[0] > 0.f && room_size[1] > 0.f && room_size[2] > 0.f))
        return fail(WRF_EINVAL, "anneal: room_size must be > 0");
    if (!(gamma >= 0.f)) return fail(WRF_EINVAL, "anneal: gamma >= 0");
    if (Q == 0) return WRF_OK;
    if (!tx || !normals || !tx_out) return fail(WRF_EINVAL, "anneal: NULL pointer");
    cudaError_t e = wrf::launch_anneal(tx, idx, normals, Q, iter, n_positions, gamma, tau,
                                       room_size, tx_out, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "anneal");
    return WRF_OK;
}

wrf_status wrf_rssi(const wrf_scene *scene, const wrf_mlp *mlp, const wrf_grid *grid,
                    const float *tx, int32_t Q, float *rssi, float *map, void *ws,
                    size_t ws_bytes, void *stream) {
    wrf_status s;
    wrf::MlpView m{};
    if ((s = check_scene(scene)) != WRF_OK) return s;
    if ((s = check_mlp(mlp, &m)) != WRF_OK) return s;
    if (!grid) return fail(WRF_EINVAL, "grid is NULL");
    if (grid->H < 1 || grid->W < 1 ||
        static_cast<long long>(grid->H) * grid->W > wrf::kRssiMaxPixels)
        return fail(WRF_EUNSUPPORTED, "RSSI head: H*W must be in [1, %d]", wrf::kRssiMaxPixels);
    if (!(grid->q_cut > 0.f)) return fail(WRF_EINVAL, "q_cut must be > 0 (or +inf)");
    if (scene->n > wrf::kRssiMaxN)
        return fail(WRF_EUNSUPPORTED, "RSSI head: at most %d Gaussians", wrf::kRssiMaxN);
    if (Q < 0) return fail(WRF_EINVAL, "Q < 0");
    if (Q > 0 && (!tx || !rssi)) return fail(WRF_EINVAL, "tx / rssi is NULL");
    size_t need = wrf::deform_ws_layout(scene->n, Q, mlp->n_layers, nullptr, nullptr);
    if (ws_bytes < need || !ws || !aligned(ws, 256))
        return fail(WRF_EINVAL, "workspace: need %zu bytes, 256-byte aligned", need);
    if (Q == 0) return WRF_OK;
    wrf::GridView g{};
    g.H = grid->H;
    g.W = grid->W;
    g.tw = g.th = 16;
    g.ntx = (g.W + 15) / 16;
    g.nty = (g.H + 15) / 16;
    g.T = g.ntx * g.nty;
    g.q_cut = grid->q_cut;
    if (grid->wrap_x != 0 && grid->wrap_x != 1) return fail(WRF_EINVAL, "wrap_x must be 0 or 1");
    if (grid->wrap_x && !(grid->q_cut < INFINITY))
        return fail(WRF_EINVAL, "wrap_x needs a finite q_cut");
    g.wrap = grid->wrap_x;
    wrf::DeformWs w{};
    wrf::deform_ws_layout(scene->n, Q, mlp->n_layers, &w, static_cast<char *>(ws));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    wrf::SceneView sv = view(scene);
    cudaError_t e = wrf::launch_prep(sv, m, g, tx, Q, w, WRF_FP32, st);
    if (e != cudaSuccess) return cuda_fail(e, "prep");
    e = wrf::launch_rssi(sv, m, g, Q, w, rssi, map, st);
    if (e != cudaSuccess) return cuda_fail(e, "rssi");
    return WRF_OK;
}

wrf_status wrf_measure_alu_peaks(double *fma_flops, double *fma2_flops, double *ex2_per_s,
                                 void *stream) {
    if (!fma_flops || !fma2_flops || !ex2_per_s) return fail(WRF_EINVAL, "output is NULL");
    double r[3] = {0, 0, 0};
    cudaError_t e = wrf::measure_alu_peaks(r, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "peak probes");
    *fma_flops = r[0];
    *fma2_flops = r[1];
    *ex2_per_s = r[2];
    return WRF_OK;
}

size_t wrf_paper_workspace_size(int32_t n, int32_t Q) {
    return wrf::paper_ws_layout(n < 0 ? 0 : n, Q < 0 ? 0 : Q, nullptr, nullptr);
}

wrf_status wrf_paper_deform_project(const wrf_paper_scene *scene, const wrf_paper_mlp *mlp,
                                    const wrf_grid *grid, const float *tx, int32_t Q, float *rec,
                                    void *ws, size_t ws_bytes, void *stream) {
    static_assert(WRF_PAPER_MAX_LAYERS == wrf::kPaperMaxLayers, "layer bound");
    static_assert(WRF_PAPER_MAX_WIDTH == wrf::kPaperMaxWidth, "width bound");
    wrf_status s;
    wrf::GridView g{};
    if (!scene) return fail(WRF_EINVAL, "scene is NULL");
    if (scene->n < 0) return fail(WRF_EINVAL, "scene.n < 0");
    if (scene->n > 0 && (!scene->mu || !scene->chol || !scene->attn_logit || !scene->psi))
        return fail(WRF_EINVAL, "scene array is NULL");
    if (scene->n > 0 && (!aligned(scene->mu, 8) || !aligned(scene->psi, 8)))
        return fail(WRF_EINVAL, "scene.mu / psi must be 8-byte aligned");
    if ((s = check_grid(grid, &g)) != WRF_OK) return s;
    if (Q < 0) return fail(WRF_EINVAL, "Q < 0");
    if (Q > 65535) return fail(WRF_EUNSUPPORTED, "Q must be <= 65535");
    if (!rows_ok(scene->n, Q)) return fail(WRF_EUNSUPPORTED, "Q*N must be < 2^31");
    wrf::PaperMlpView mv{};
    if (mlp) {
        if (mlp->n_hidden < 1 || mlp->n_hidden > 8)
            return fail(WRF_EUNSUPPORTED, "n_hidden must be in [1, 8]");
        if (mlp->width < 1 || mlp->width > WRF_PAPER_MAX_WIDTH)
            return fail(WRF_EUNSUPPORTED, "width must be in [1, 160]");
        if (mlp->L_mean < 0 || mlp->L_mean > 15 || mlp->L_tx < 0 || mlp->L_tx > 15)
            return fail(WRF_EUNSUPPORTED, "frequency bands must be in [0, 15]");
        for (int l = 0; l <= mlp->n_hidden; ++l)
            if (!mlp->W[l] || !mlp->b[l]) return fail(WRF_EINVAL, "weight %d is NULL", l);
        for (int i = 0; i < 3; ++i)
            if (!(mlp->room_size[i] > 0.f)) return fail(WRF_EINVAL, "room_size must be > 0");
        if (Q > 0 && !tx) return fail(WRF_EINVAL, "tx is NULL");
        if (mlp->precision != WRF_FP32 && mlp->precision != WRF_BF16 &&
            mlp->precision != WRF_BF16X3)
            return fail(WRF_EINVAL, "unknown precision");
        const bool tc = mlp->precision == WRF_BF16 || mlp->precision == WRF_BF16X3;
        if (tc && 2 * (2 * mlp->L_mean + 1) > 64)
            return fail(WRF_EUNSUPPORTED, "BF16 path: 2(2 L_mean + 1) must be <= 64");
        if (tc && Q > 0 && scene->n > 0 &&
            (static_cast<long long>(Q) * ((scene->n + 127) / 128) >= (1ll << 30)))
            return fail(WRF_EUNSUPPORTED, "too many tiles");
        mv.n_hidden = mlp->n_hidden;
        mv.width = mlp->width;
        mv.L_mean = mlp->L_mean;
        mv.L_tx = mlp->L_tx;
        for (int i = 0; i < 3; ++i) {
            mv.room_min[i] = mlp->room_min[i];
            mv.room_size[i] = mlp->room_size[i];
        }
        for (int l = 0; l <= mlp->n_hidden; ++l) {
            mv.W[l] = mlp->W[l];
            mv.b[l] = mlp->b[l];
        }
    }
    if (Q == 0 || scene->n == 0) return WRF_OK;
    if (!rec || !aligned(rec, 16)) return fail(WRF_EINVAL, "rec must be 16-byte aligned");
    size_t need = wrf::paper_ws_layout(scene->n, Q, nullptr, nullptr);
    if (mlp && (ws_bytes < need || !ws || !aligned(ws, 256)))
        return fail(WRF_EINVAL, "workspace: need %zu bytes, 256-byte aligned", need);
    wrf::PaperWs w{};
    if (mlp) wrf::paper_ws_layout(scene->n, Q, &w, static_cast<char *>(ws));
    wrf::PaperSceneView sv{scene->n, scene->mu, scene->chol, scene->attn_logit, scene->psi};
    cudaError_t e;
    if (mlp && (mlp->precision == WRF_BF16 || mlp->precision == WRF_BF16X3))
        e = wrf::launch_paper_tc(sv, mv, g, tx, Q, w, reinterpret_cast<float4 *>(rec), status_ptr(),
                                 mlp->precision, static_cast<cudaStream_t>(stream));
    else
        e = wrf::launch_paper(sv, mlp ? &mv : nullptr, g, tx, Q, w,
                              reinterpret_cast<float4 *>(rec), static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "paper head");
    return WRF_OK;
}

wrf_status wrf_project(const wrf_scene *scene, const float *resid, int32_t Q,
                       const wrf_grid *grid, float *rec, uint32_t *tile_count, void *stream) {
    wrf_status s;
    wrf::GridView g{};
    if ((s = check_scene(scene)) != WRF_OK) return s;
    if ((s = check_grid(grid, &g)) != WRF_OK) return s;
    if (Q < 0) return fail(WRF_EINVAL, "Q < 0");
    if (!rows_ok(scene->n, Q)) return fail(WRF_EUNSUPPORTED, "Q*N must be < 2^31");
    if (Q == 0 || scene->n == 0) return WRF_OK;
    if (!rec || !aligned(rec, 16)) return fail(WRF_EINVAL, "rec must be 16-byte aligned");
    cudaError_t e = wrf::launch_project(view(scene), resid, Q, g, reinterpret_cast<float4 *>(rec),
                                        tile_count, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "project");
    return WRF_OK;
}

size_t wrf_bin_workspace_size(int32_t n, int32_t Q, const wrf_grid *grid) {
    wrf::GridView g{};
    if (!grid || check_grid(grid, &g) != WRF_OK) return 0;
    return wrf::bin_ws_layout(n < 0 ? 0 : n, Q < 0 ? 0 : Q, g, nullptr, nullptr);
}

wrf_status wrf_bin(const float *rec, int32_t n, int32_t Q, const wrf_grid *grid, uint32_t *gids,
                   int64_t key_capacity, int64_t *n_keys_out, uint32_t *tile_offsets, void *ws,
                   size_t ws_bytes, void *stream) {
    wrf_status s;
    wrf::GridView g{};
    if ((s = check_grid(grid, &g)) != WRF_OK) return s;
    if (n < 0 || Q < 0 || key_capacity < 0) return fail(WRF_EINVAL, "negative size");
    if (Q > 65535) return fail(WRF_EUNSUPPORTED, "Q > 65535 per call");
    if (!rows_ok(n, Q)) return fail(WRF_EUNSUPPORTED, "Q*N must be < 2^31");
    if (!n_keys_out || !tile_offsets) return fail(WRF_EINVAL, "n_keys_out / tile_offsets NULL");
    if (n > 0 && Q > 0 && (!rec || !aligned(rec, 16))) return fail(WRF_EINVAL, "rec alignment");
    if (key_capacity > 0 && !gids) return fail(WRF_EINVAL, "gids is NULL");
    size_t need = wrf::bin_ws_layout(n, Q, g, nullptr, nullptr);
    if (ws_bytes < need || !ws || !aligned(ws, 256))
        return fail(WRF_EINVAL, "workspace: need %zu bytes, 256-byte aligned", need);
    if (Q == 0) {  // no keys: the count and the one CSR entry are still written
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        cudaError_t e = cudaMemsetAsync(n_keys_out, 0, sizeof(int64_t), st);
        if (e == cudaSuccess) e = cudaMemsetAsync(tile_offsets, 0, sizeof(uint32_t), st);
        if (e != cudaSuccess) return cuda_fail(e, "bin (Q = 0)");
        return WRF_OK;
    }
    wrf::BinWs w{};
    wrf::bin_ws_layout(n, Q, g, &w, static_cast<char *>(ws));
    cudaError_t e = wrf::launch_bin(reinterpret_cast<const float4 *>(rec), n, Q, g, gids,
                                    key_capacity, reinterpret_cast<long long *>(n_keys_out),
                                    tile_offsets, w, status_ptr(), static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "bin");
    return WRF_OK;
}

wrf_status wrf_bin_noalloc(const float *rec, int32_t n, int32_t Q, const wrf_grid *grid,
                           uint32_t *gids, int64_t key_capacity, int64_t *n_keys_out,
                           uint32_t *tile_offsets, void *stream) {
    wrf::GridView g{};
    wrf_status s;
    if ((s = check_grid(grid, &g)) != WRF_OK) return s;
    if (n < 0 || Q < 0 || key_capacity < 0) return fail(WRF_EINVAL, "negative size");
    const size_t need = wrf::bin_ws_layout(n, Q, g, nullptr, nullptr);
    if (need > kBinScratchBytes)
        return fail(WRF_EINVAL,
                    "wrf_bin_noalloc: this size needs %zu bytes of scratch, the built-in "
                    "scratch holds %zu; use wrf_bin with a caller workspace",
                    need, kBinScratchBytes);
    void *ws = nullptr;
    cudaError_t e = bin_scratch_ptr(&ws);
    if (e != cudaSuccess) return cuda_fail(e, "wrf_bin_noalloc: scratch address");
    // The scratch needs no clearing: binning writes every count and block
    // sum it later reads.
    return wrf_bin(rec, n, Q, grid, gids, key_capacity, n_keys_out, tile_offsets, ws,
                   kBinScratchBytes, stream);
}

// ------------------------------------------------------ multi-scene batches
static wrf_status check_multi(const wrf_scene *scenes, const wrf_mlp *mlps, int32_t S,
                              wrf::SceneView *sv, wrf::MlpView *mv) {
    if (!scenes || !mlps) return fail(WRF_EINVAL, "scenes / mlps is NULL");
    if (S < 1 || S > wrf::kMaxScenes)
        return fail(WRF_EUNSUPPORTED, "multi-scene: 1 <= S <= %d scenes", wrf::kMaxScenes);
    wrf_status s;
    for (int i = 0; i < S; ++i) {
        if ((s = check_scene(&scenes[i])) != WRF_OK) return s;
        if (scenes[i].channels != 1)
            return fail(WRF_EUNSUPPORTED, "multi-scene: one channel per scene");
        if ((s = check_mlp(&mlps[i], &mv[i])) != WRF_OK) return s;
        if (mlps[i].precision != WRF_BF16)
            return fail(WRF_EUNSUPPORTED, "multi-scene: BF16 tensor-core MLPs");
        const wrf_mlp &a = mlps[0], &b = mlps[i];
        bool same = a.n_layers == b.n_layers && a.L_mean == b.L_mean && a.L_tx == b.L_tx;
        for (int k = 0; k < 3; ++k)
            same = same && a.room_min[k] == b.room_min[k] && a.room_size[k] == b.room_size[k];
        if (!same)
            return fail(WRF_EUNSUPPORTED,
                        "multi-scene: every scene's MLP has the same layers, bands and room");
        sv[i] = view(&scenes[i]);
    }
    return WRF_OK;
}

size_t wrf_multi_set_size(const wrf_scene *scenes, const wrf_mlp *mlps, int32_t S) {
    wrf::SceneView sv[wrf::kMaxScenes];
    wrf::MlpView mv[wrf::kMaxScenes];
    if (check_multi(scenes, mlps, S, sv, mv) != WRF_OK) return 0;
    return wrf::multi_set_layout(sv, S, mlps[0].n_layers, wrf::mlp_k1(mv[0].dm), nullptr,
                                 nullptr);
}

wrf_status wrf_multi_set_prepare(const wrf_scene *scenes, const wrf_mlp *mlps, int32_t S,
                                 const wrf_grid *grid, void *set, size_t set_bytes,
                                 void *stream) {
    wrf::SceneView sv[wrf::kMaxScenes];
    wrf::MlpView mv[wrf::kMaxScenes];
    wrf::GridView g{};
    wrf_status s;
    if ((s = check_multi(scenes, mlps, S, sv, mv)) != WRF_OK) return s;
    if ((s = check_grid(grid, &g)) != WRF_OK) return s;
    const size_t need = wrf::multi_set_layout(sv, S, mlps[0].n_layers, wrf::mlp_k1(mv[0].dm),
                                              nullptr, nullptr);
    if (!set || set_bytes < need || !aligned(set, 256))
        return fail(WRF_EINVAL, "scene set: need %zu bytes, 256-byte aligned", need);
    wrf::MultiSet ms{};
    wrf::multi_set_layout(sv, S, mlps[0].n_layers, wrf::mlp_k1(mv[0].dm), &ms,
                          static_cast<char *>(set));
    cudaError_t e = wrf::launch_multi_prepare(sv, mv, S, g, ms, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "multi-scene prepare");
    return WRF_OK;
}

size_t wrf_multi_workspace_size(int32_t Q) {
    return wrf::multi_ws_layout(Q < 0 ? 0 : Q, nullptr, nullptr);
}

wrf_status wrf_deform_project_multi(const wrf_scene *scenes, const wrf_mlp *mlps, int32_t S,
                                    const void *set, const int32_t *scene_of, const float *tx,
                                    int32_t Q, const wrf_grid *grid, float *rec,
                                    int64_t rec_capacity, int64_t *query_base, void *ws,
                                    size_t ws_bytes, void *stream) {
    wrf::SceneView sv[wrf::kMaxScenes];
    wrf::MlpView mv[wrf::kMaxScenes];
    wrf::GridView g{};
    wrf_status s;
    if ((s = check_multi(scenes, mlps, S, sv, mv)) != WRF_OK) return s;
    if ((s = check_grid(grid, &g)) != WRF_OK) return s;
    if (Q < 0 || Q > 65535) return fail(WRF_EUNSUPPORTED, "multi-scene: 0 <= Q <= 65535");
    if (rec_capacity < 0) return fail(WRF_EINVAL, "rec_capacity < 0");
    // the rasteriser addresses record rows with 32-bit coordinates
    if (rec_capacity > 0x7fffffffll) return fail(WRF_EUNSUPPORTED, "rec_capacity >= 2^31");
    if (!query_base) return fail(WRF_EINVAL, "query_base is NULL");
    if (Q == 0) {
        cudaError_t e = cudaMemsetAsync(query_base, 0, sizeof(int64_t),
                                        static_cast<cudaStream_t>(stream));
        if (e != cudaSuccess) return cuda_fail(e, "multi-scene (Q = 0)");
        return WRF_OK;
    }
    if (!set || !aligned(set, 256) || !scene_of || !tx)
        return fail(WRF_EINVAL, "set / scene_of / tx is NULL (or set not 256-byte aligned)");
    if (rec_capacity > 0 && (!rec || !aligned(rec, 16)))
        return fail(WRF_EINVAL, "rec must be non-NULL and 16-byte aligned");
    const size_t need = wrf::multi_ws_layout(Q, nullptr, nullptr);
    if (!ws || ws_bytes < need || !aligned(ws, 256))
        return fail(WRF_EINVAL, "workspace: need %zu bytes, 256-byte aligned", need);
    wrf::MultiSet ms{};
    wrf::multi_set_layout(sv, S, mlps[0].n_layers, wrf::mlp_k1(mv[0].dm), &ms,
                          static_cast<char *>(const_cast<void *>(set)));
    wrf::MultiWs w{};
    wrf::multi_ws_layout(Q, &w, static_cast<char *>(ws));
    cudaError_t e = wrf::launch_deform_project_multi(
        ms, S, mv[0], g, scene_of, tx, Q, reinterpret_cast<float4 *>(rec), rec_capacity,
        reinterpret_cast<long long *>(query_base), w, status_ptr(),
        static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "deform_project_multi");
    return WRF_OK;
}

wrf_status wrf_bin_multi(const float *rec, const int64_t *query_base, int32_t n_max, int32_t Q,
                         const wrf_grid *grid, uint32_t *gids, int64_t key_capacity,
                         int64_t *n_keys_out, uint32_t *tile_offsets, void *ws, size_t ws_bytes,
                         void *stream) {
    wrf_status s;
    wrf::GridView g{};
    if ((s = check_grid(grid, &g)) != WRF_OK) return s;
    if (n_max < 0 || Q < 0 || key_capacity < 0) return fail(WRF_EINVAL, "negative size");
    if (Q > 65535) return fail(WRF_EUNSUPPORTED, "Q > 65535 per call");
    if (!rows_ok(n_max, Q)) return fail(WRF_EUNSUPPORTED, "Q*n_max must be < 2^31");
    if (!n_keys_out || !tile_offsets) return fail(WRF_EINVAL, "n_keys_out / tile_offsets NULL");
    if (Q > 0 && !query_base) return fail(WRF_EINVAL, "query_base is NULL");
    if (n_max > 0 && Q > 0 && (!rec || !aligned(rec, 16))) return fail(WRF_EINVAL, "rec alignment");
    if (key_capacity > 0 && !gids) return fail(WRF_EINVAL, "gids is NULL");
    size_t need = wrf::bin_ws_layout(n_max, Q, g, nullptr, nullptr);
    if (ws_bytes < need || !ws || !aligned(ws, 256))
        return fail(WRF_EINVAL, "workspace: need %zu bytes, 256-byte aligned", need);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (Q == 0) {
        cudaError_t e = cudaMemsetAsync(n_keys_out, 0, sizeof(int64_t), st);
        if (e == cudaSuccess) e = cudaMemsetAsync(tile_offsets, 0, sizeof(uint32_t), st);
        if (e != cudaSuccess) return cuda_fail(e, "bin_multi (Q = 0)");
        return WRF_OK;
    }
    wrf::BinWs w{};
    wrf::bin_ws_layout(n_max, Q, g, &w, static_cast<char *>(ws));
    cudaError_t e = wrf::launch_bin(reinterpret_cast<const float4 *>(rec), n_max, Q, g, gids,
                                    key_capacity, reinterpret_cast<long long *>(n_keys_out),
                                    tile_offsets, w, status_ptr(), st,
                                    reinterpret_cast<const long long *>(query_base));
    if (e != cudaSuccess) return cuda_fail(e, "bin_multi");
    return WRF_OK;
}

wrf_status wrf_render_multi(const float *rec, const int64_t *query_base, const uint32_t *gids,
                            const uint32_t *tile_offsets, const int64_t *n_keys,
                            int64_t key_capacity, int32_t Q, const wrf_grid *grid, float *spectra,
                            void *stream) {
    wrf_status s;
    wrf::GridView g{};
    if ((s = check_grid(grid, &g)) != WRF_OK) return s;
    if (Q < 0) return fail(WRF_EINVAL, "negative size");
    if (Q > 65535) return fail(WRF_EUNSUPPORTED, "Q > 65535 per call");
    if (Q == 0) return WRF_OK;
    if (!query_base || !tile_offsets || !n_keys || !spectra)
        return fail(WRF_EINVAL, "NULL pointer");
    if (!aligned(spectra, 16) || (rec && !aligned(rec, 16)))
        return fail(WRF_EINVAL, "spectra / rec must be 16-byte aligned");
    cudaError_t e = wrf::launch_render(reinterpret_cast<const float4 *>(rec), gids, tile_offsets,
                                       reinterpret_cast<const long long *>(n_keys), key_capacity,
                                       0, Q, g, spectra, status_ptr(),
                                       static_cast<cudaStream_t>(stream),
                                       reinterpret_cast<const long long *>(query_base));
    if (e != cudaSuccess) return cuda_fail(e, "render_multi");
    return WRF_OK;
}

wrf_status wrf_render(const float *rec, const uint32_t *gids, const uint32_t *tile_offsets,
                      const int64_t *n_keys, int64_t key_capacity, int32_t n, int32_t Q,
                      const wrf_grid *grid, float *spectra, void *stream) {
    wrf_status s;
    wrf::GridView g{};
    if ((s = check_grid(grid, &g)) != WRF_OK) return s;
    if (n < 0 || Q < 0) return fail(WRF_EINVAL, "negative size");
    if (Q > 65535) return fail(WRF_EUNSUPPORTED, "Q > 65535 per call");
    if (Q == 0) return WRF_OK;
    if (!tile_offsets || !n_keys || !spectra) return fail(WRF_EINVAL, "NULL pointer");
    if (!aligned(spectra, 16) || (n > 0 && !aligned(rec, 16)))
        return fail(WRF_EINVAL, "spectra / rec must be 16-byte aligned");
    cudaError_t e = wrf::launch_render(reinterpret_cast<const float4 *>(rec), gids, tile_offsets,
                                       reinterpret_cast<const long long *>(n_keys), key_capacity,
                                       n, Q, g, spectra, status_ptr(),
                                       static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "render");
    return WRF_OK;
}

wrf_status wrf_render_complex(const float *rec, const uint32_t *gids,
                              const uint32_t *tile_offsets, const int64_t *n_keys,
                              int64_t key_capacity, int32_t n, int32_t Q, const wrf_grid *grid,
                              float *out, void *stream) {
    wrf_status s;
    wrf::GridView g{};
    if ((s = check_grid(grid, &g)) != WRF_OK) return s;
    if (n < 0 || Q < 0) return fail(WRF_EINVAL, "negative size");
    if (Q > 65535) return fail(WRF_EUNSUPPORTED, "Q > 65535 per call");
    if (Q == 0) return WRF_OK;
    if (!tile_offsets || !n_keys || !out) return fail(WRF_EINVAL, "NULL pointer");
    if (!aligned(out, 16) || (n > 0 && !aligned(rec, 16)))
        return fail(WRF_EINVAL, "out / rec must be 16-byte aligned");
    cudaError_t e = wrf::launch_render_complex(
        reinterpret_cast<const float4 *>(rec), gids, tile_offsets,
        reinterpret_cast<const long long *>(n_keys), key_capacity, n, Q, g, out, status_ptr(),
        static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "render_complex");
    return WRF_OK;
}

wrf_status wrf_render_backward(const float *rec, const uint32_t *gids,
                               const uint32_t *tile_offsets, const int64_t *n_keys,
                               int64_t key_capacity, int32_t n, int32_t Q, const wrf_grid *grid,
                               const float *dL_dspectra, float *d_rec, void *stream) {
    wrf_status s;
    wrf::GridView g{};
    if ((s = check_grid(grid, &g)) != WRF_OK) return s;
    if (n < 0 || Q < 0) return fail(WRF_EINVAL, "negative size");
    if (Q > 65535) return fail(WRF_EUNSUPPORTED, "Q > 65535 per call");
    if (Q == 0 || n == 0) return WRF_OK;
    if (!rec || !tile_offsets || !n_keys || !dL_dspectra || !d_rec)
        return fail(WRF_EINVAL, "NULL pointer");
    cudaError_t e = wrf::launch_render_bwd(reinterpret_cast<const float4 *>(rec), gids,
                                           tile_offsets,
                                           reinterpret_cast<const long long *>(n_keys),
                                           key_capacity, n, Q, g, dL_dspectra, d_rec,
                                           status_ptr(), static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "render_backward");
    return WRF_OK;
}

wrf_status wrf_project_backward(const wrf_scene *scene, const float *resid, int32_t Q,
                                const float *d_rec, float *d_resid, float *d_mean,
                                float *d_log_scale, float *d_rot, float *d_opacity, float *d_amp,
                                void *stream) {
    wrf_status s;
    if ((s = check_scene(scene)) != WRF_OK) return s;
    if (scene->channels != 1)
        return fail(WRF_EUNSUPPORTED, "the backward takes one channel");
    if (Q < 0) return fail(WRF_EINVAL, "Q < 0");
    if (!rows_ok(scene->n, Q)) return fail(WRF_EUNSUPPORTED, "Q*N must be < 2^31");
    if (scene->n == 0) return WRF_OK;
    if ((Q > 0 && !d_rec) || !d_mean || !d_log_scale || !d_rot || !d_opacity || !d_amp)
        return fail(WRF_EINVAL, "NULL pointer");
    cudaError_t e = wrf::launch_project_bwd(view(scene), resid, Q, d_rec, d_resid, d_mean,
                                            d_log_scale, d_rot, d_opacity, d_amp,
                                            static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "project_backward");
    return WRF_OK;
}

size_t wrf_deform_backward_workspace_size(int32_t n, int32_t Q, const wrf_mlp *mlp) {
    wrf::MlpView m{};
    if (!mlp || check_mlp(mlp, &m) != WRF_OK) return 0;
    return wrf::deform_bwd_ws_layout(n < 0 ? 0 : n, Q < 0 ? 0 : Q, m, nullptr, nullptr, nullptr);
}

wrf_status wrf_deform_backward(const wrf_scene *scene, const wrf_mlp *mlp, const wrf_grid *grid,
                               const float *tx, int32_t Q, const float *d_resid,
                               const float *acts, float *const *dW, float *const *db,
                               float *d_mean, int32_t stop_grad_mean, void *ws, size_t ws_bytes,
                               void *stream) {
    wrf_status s;
    wrf::GridView g{};
    wrf::MlpView m{};
    if ((s = check_scene(scene)) != WRF_OK) return s;
    if (scene->channels != 1)
        return fail(WRF_EUNSUPPORTED, "the backward takes one channel");
    if ((s = check_mlp(mlp, &m)) != WRF_OK) return s;
    if ((s = check_grid(grid, &g)) != WRF_OK) return s;
    if (Q < 0) return fail(WRF_EINVAL, "Q < 0");
    if (!rows_ok(scene->n, Q)) return fail(WRF_EUNSUPPORTED, "Q*N must be < 2^31");
    if (!dW || !db) return fail(WRF_EINVAL, "dW / db NULL");
    for (int l = 0; l < mlp->n_layers; ++l)
        if (!dW[l] || !db[l]) return fail(WRF_EINVAL, "dW[%d] / db[%d] NULL", l, l);
    if (!stop_grad_mean && scene->n > 0 && !d_mean) return fail(WRF_EINVAL, "d_mean NULL");
    if (Q > 0 && (!tx || !d_resid)) return fail(WRF_EINVAL, "tx / d_resid NULL");
    size_t need = wrf::deform_bwd_ws_layout(scene->n, Q, m, nullptr, nullptr, nullptr);
    if (ws_bytes < need || !ws || !aligned(ws, 256))
        return fail(WRF_EINVAL, "workspace: need %zu bytes, 256-byte aligned", need);
    wrf::DeformWs fw{};
    wrf::DeformBwdWs bw{};
    wrf::deform_bwd_ws_layout(scene->n, Q, m, &fw, &bw, static_cast<char *>(ws));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    wrf::SceneView sv = view(scene);
    cudaError_t e = cudaSuccess;
    if (Q > 0 && scene->n > 0) {
        e = wrf::launch_prep(sv, m, g, tx, Q, fw, WRF_FP32, st);
        if (e != cudaSuccess) return cuda_fail(e, "prep");
    }
    e = wrf::launch_mlp_bwd(sv, m, g, tx, Q, fw, bw, d_resid, acts, dW, db, d_mean,
                            stop_grad_mean, status_ptr(), st);
    if (e != cudaSuccess) return cuda_fail(e, "mlp_backward");
    return WRF_OK;
}

}  // extern "C"

namespace wrf {

wrf_status check_forward(const wrf_scene *scene, const wrf_mlp *mlp, const wrf_grid *grid, int Q) {
    wrf_status s;
    GridView g{};
    MlpView m{};
    if ((s = check_scene(scene)) != WRF_OK) return s;
    if ((s = check_mlp(mlp, &m)) != WRF_OK) return s;
    if ((s = check_grid(grid, &g)) != WRF_OK) return s;
    if (Q < 1 || Q > 65535) return fail(WRF_EINVAL, "Q must be in [1, 65535]");
    if (!rows_ok(scene->n, Q)) return fail(WRF_EUNSUPPORTED, "Q*N must be < 2^31");
    return WRF_OK;
}

wrf_status set_error(wrf_status s, const char *where, cudaError_t e) {
    if (e != cudaSuccess) return fail(s, "%s: %s", where, cudaGetErrorString(e));
    return fail(s, "%s", where);
}

}  // namespace wrf
