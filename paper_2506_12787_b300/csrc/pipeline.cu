// Host-to-host forward pipeline (wrf_pipeline_*, include/wrf.h): TX positions
// in host memory go in, spectra in host memory come out (the problem as Sec.
// 4.1-4.2 state it), with the device work of a step -- wrf_deform_project,
// wrf_bin and wrf_render (wrf_render_complex for two channels) -- replayed
// from a CUDA graph.
//
// Two slots, each with its own device TX and spectrum buffers, key count and
// graph; the records, workspaces and tile lists are shared, since the compute
// stream runs one step after the other.  Step i uses slot i % 2: its TX goes
// through the slot's pinned staging to the device, the graph runs on the
// compute stream, and the spectra and the key count are read back on the
// copy stream, so that step i's read-back overlaps step i + 1's compute.
// Before a slot is reused the host waits for its previous step's read-back
// and checks that step's key count against the capacity its graph ran with;
// a step that did not fit is recomputed (capacity grown, graphs captured
// again) into the same host buffer.
#include <cstring>

#include "kernels.h"

struct wrf_pipeline {
    int dev = 0;
    wrf_scene scene{};
    wrf_mlp mlp{};
    wrf_grid grid{};
    int Q = 0, n = 0;
    float margin = 1.25f;
    size_t out_bytes = 0;  // one step's spectra
    cudaStream_t compute = nullptr, copy = nullptr;
    float *rec = nullptr;
    void *dws = nullptr, *bws = nullptr;
    size_t dws_bytes = 0, bws_bytes = 0;
    uint32_t *gids = nullptr;
    int64_t cap = 0;
    uint32_t *offs = nullptr;
    int64_t *nkeys = nullptr;    // device [2]: each slot's key count
    int64_t *nk_host = nullptr;  // pinned [2]: the same, read back
    float *tx_dev[2] = {nullptr, nullptr};
    float *out_dev[2] = {nullptr, nullptr};
    float *tx_pin[2] = {nullptr, nullptr};  // pinned staging of each slot's TX
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    cudaEvent_t done[2] = {nullptr, nullptr}, freed[2] = {nullptr, nullptr};
    float *dst[2] = {nullptr, nullptr};  // the host buffer of each slot's pending step
    int64_t cap_used[2] = {0, 0};        // the capacity that step's graph ran with
    bool pending[2] = {false, false};
    long long steps = 0;
};

namespace {

// The pipeline's device is current for the duration of a call; the caller's
// device is restored on return.
struct DeviceScope {
    int prev = -1;
    explicit DeviceScope(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceScope() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

wrf_status cuda_err(cudaError_t e, const char *where) {
    return wrf::set_error(WRF_ECUDA, where, e);
}

// One forward of slot k on stream st: records, tile lists, spectra.
wrf_status enqueue_forward(wrf_pipeline *p, int k, cudaStream_t st) {
    wrf_status s = wrf_deform_project(&p->scene, &p->mlp, &p->grid, p->tx_dev[k], p->Q, p->rec,
                                      nullptr, p->dws, p->dws_bytes, st);
    if (s != WRF_OK) return s;
    s = wrf_bin(p->rec, p->n, p->Q, &p->grid, p->gids, p->cap, p->nkeys + k, p->offs, p->bws,
                p->bws_bytes, st);
    if (s != WRF_OK) return s;
    if (p->scene.channels == 2)
        return wrf_render_complex(p->rec, p->gids, p->offs, p->nkeys + k, p->cap, p->n, p->Q,
                                  &p->grid, p->out_dev[k], st);
    return wrf_render(p->rec, p->gids, p->offs, p->nkeys + k, p->cap, p->n, p->Q, &p->grid,
                      p->out_dev[k], st);
}

// Both slots' graphs, captured on the compute stream (the key capacity and
// the tile-list buffer are baked into them).
wrf_status capture(wrf_pipeline *p) {
    for (int k = 0; k < 2; ++k) {
        if (p->exec[k]) {
            cudaGraphExecDestroy(p->exec[k]);
            p->exec[k] = nullptr;
        }
        cudaError_t e = cudaStreamBeginCapture(p->compute, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_err(e, "pipeline capture");
        const wrf_status s = enqueue_forward(p, k, p->compute);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(p->compute, &g);
        if (s != WRF_OK) {
            if (g) cudaGraphDestroy(g);
            return s;
        }
        if (e != cudaSuccess) return cuda_err(e, "pipeline capture");
        e = cudaGraphInstantiate(&p->exec[k], g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_err(e, "pipeline graph instantiate");
    }
    return WRF_OK;
}

wrf_status alloc_keys(wrf_pipeline *p, int64_t cap) {
    if (cap <= p->cap) return WRF_OK;
    if (p->gids) cudaFree(p->gids);
    p->gids = nullptr;
    p->cap = 0;
    cudaError_t e = cudaMalloc(&p->gids, static_cast<size_t>(cap) * sizeof(uint32_t));
    if (e != cudaSuccess) return cuda_err(e, "pipeline key buffer");
    p->cap = cap;
    return WRF_OK;
}

int64_t grown(const wrf_pipeline *p, int64_t need) {
    return static_cast<int64_t>(static_cast<double>(need) * p->margin) + 1024;
}

// Slot k's step again, without the graph, synchronously: TX from the slot's
// staging, spectra into the slot's device buffer, key count into nk_host[k].
wrf_status run_slot_sync(wrf_pipeline *p, int k) {
    const size_t txb = static_cast<size_t>(p->Q) * 3 * sizeof(float);
    cudaError_t e = cudaMemcpyAsync(p->tx_dev[k], p->tx_pin[k], txb, cudaMemcpyHostToDevice,
                                    p->compute);
    if (e != cudaSuccess) return cuda_err(e, "pipeline upload");
    const wrf_status s = enqueue_forward(p, k, p->compute);
    if (s != WRF_OK) return s;
    e = cudaMemcpyAsync(p->nk_host + k, p->nkeys + k, sizeof(int64_t), cudaMemcpyDeviceToHost,
                        p->compute);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->compute);
    return e == cudaSuccess ? WRF_OK : cuda_err(e, "pipeline step");
}

// The status word after a step whose keys did not fit: WRF_ENOSPC is that
// step's own record; anything else is an error to report.
wrf_status clear_overflow(wrf_pipeline *p) {
    const wrf_status st = wrf_status_read(p->compute);
    return (st == WRF_OK || st == WRF_ENOSPC) ? WRF_OK : st;
}

// Waits for slot k's pending step (its read-back) and, if its keys did not
// fit the capacity its graph ran with, recomputes it into its host buffer.
wrf_status finish_slot(wrf_pipeline *p, int k) {
    if (!p->pending[k]) return WRF_OK;
    p->pending[k] = false;
    cudaError_t e = cudaEventSynchronize(p->freed[k]);
    if (e != cudaSuccess) return cuda_err(e, "pipeline wait");
    if (p->nk_host[k] <= p->cap_used[k]) return WRF_OK;
    // nothing of the pipeline may run while buffers and graphs change
    e = cudaStreamSynchronize(p->compute);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->copy);
    if (e != cudaSuccess) return cuda_err(e, "pipeline wait");
    wrf_status s = clear_overflow(p);
    if (s != WRF_OK) return s;
    if (p->nk_host[k] > p->cap) {
        if ((s = alloc_keys(p, grown(p, p->nk_host[k]))) != WRF_OK) return s;
        if ((s = capture(p)) != WRF_OK) return s;
    }
    if ((s = run_slot_sync(p, k)) != WRF_OK) return s;
    if (p->nk_host[k] > p->cap) return wrf::set_error(WRF_ENOSPC, "pipeline: key count grew");
    e = cudaMemcpy(p->dst[k], p->out_dev[k], p->out_bytes, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? WRF_OK : cuda_err(e, "pipeline read-back");
}

// The first step's sizing: an eager run of its TX positions, the capacity
// from its key count, then both graphs.
wrf_status size_and_capture(wrf_pipeline *p) {
    wrf_status s = run_slot_sync(p, 0);
    if (s != WRF_OK) return s;
    if (p->nk_host[0] > p->cap) {
        if ((s = clear_overflow(p)) != WRF_OK) return s;
    }
    if ((s = alloc_keys(p, grown(p, p->nk_host[0]))) != WRF_OK) return s;
    return capture(p);
}

void release(wrf_pipeline *p) {
    for (int k = 0; k < 2; ++k) {
        if (p->exec[k]) cudaGraphExecDestroy(p->exec[k]);
        if (p->done[k]) cudaEventDestroy(p->done[k]);
        if (p->freed[k]) cudaEventDestroy(p->freed[k]);
        cudaFree(p->tx_dev[k]);
        cudaFree(p->out_dev[k]);
        cudaFreeHost(p->tx_pin[k]);
    }
    cudaFree(p->rec);
    cudaFree(p->dws);
    cudaFree(p->bws);
    cudaFree(p->gids);
    cudaFree(p->offs);
    cudaFree(p->nkeys);
    cudaFreeHost(p->nk_host);
    if (p->compute) cudaStreamDestroy(p->compute);
    if (p->copy) cudaStreamDestroy(p->copy);
    delete p;
}

}  // namespace

extern "C" {

wrf_status wrf_pipeline_create(const wrf_scene *scene, const wrf_mlp *mlp, const wrf_grid *grid,
                               int32_t Q, float key_margin, wrf_pipeline **out) {
    if (!out) return wrf::set_error(WRF_EINVAL, "pipeline: out is NULL");
    *out = nullptr;
    wrf_status s = wrf::check_forward(scene, mlp, grid, Q);
    if (s != WRF_OK) return s;
    if (!(key_margin == 0.f || (key_margin >= 1.f && key_margin <= 1e6f)))
        return wrf::set_error(WRF_EINVAL, "pipeline: key_margin must be 0 or in [1, 1e6]");
    wrf_pipeline *p = new wrf_pipeline();
    cudaError_t e = cudaGetDevice(&p->dev);
    if (e != cudaSuccess) {
        delete p;
        return cuda_err(e, "pipeline device");
    }
    p->scene = *scene;
    p->mlp = *mlp;
    p->grid = *grid;
    p->Q = Q;
    p->n = scene->n;
    if (key_margin != 0.f) p->margin = key_margin;
    const size_t rows = static_cast<size_t>(Q) * static_cast<size_t>(scene->n);
    const size_t ch = static_cast<size_t>(scene->channels);
    const int T = ((grid->W + grid->tile_w - 1) / grid->tile_w) *
                  ((grid->H + grid->tile_h - 1) / grid->tile_h);
    p->out_bytes = static_cast<size_t>(Q) * grid->H * grid->W * ch * sizeof(float);
    p->dws_bytes = wrf_deform_workspace_size(scene->n, Q, mlp);
    p->bws_bytes = wrf_bin_workspace_size(scene->n, Q, grid);
    const size_t txb = static_cast<size_t>(Q) * 3 * sizeof(float);
    auto dev_alloc = [&](void **ptr, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(ptr, bytes < 256 ? 256 : bytes);
    };
    dev_alloc(reinterpret_cast<void **>(&p->rec), rows * 32 + (ch == 2 ? rows * 4 : 0));
    dev_alloc(&p->dws, p->dws_bytes);
    dev_alloc(&p->bws, p->bws_bytes);
    dev_alloc(reinterpret_cast<void **>(&p->offs), (static_cast<size_t>(Q) * T + 1) * 4);
    dev_alloc(reinterpret_cast<void **>(&p->nkeys), 2 * sizeof(int64_t));
    for (int k = 0; k < 2; ++k) {
        dev_alloc(reinterpret_cast<void **>(&p->tx_dev[k]), txb);
        dev_alloc(reinterpret_cast<void **>(&p->out_dev[k]), p->out_bytes);
        if (e == cudaSuccess) e = cudaHostAlloc(&p->tx_pin[k], txb, cudaHostAllocDefault);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->done[k], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->freed[k], cudaEventDisableTiming);
    }
    if (e == cudaSuccess)
        e = cudaHostAlloc(reinterpret_cast<void **>(&p->nk_host), 2 * sizeof(int64_t),
                          cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->compute, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->copy, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        release(p);
        return cuda_err(e, "pipeline allocation");
    }
    if ((s = alloc_keys(p, 1024)) != WRF_OK) {
        release(p);
        return s;
    }
    *out = p;
    return WRF_OK;
}

wrf_status wrf_pipeline_step(wrf_pipeline *p, const float *tx_host, float *spectra_host) {
    if (!p || !tx_host || !spectra_host)
        return wrf::set_error(WRF_EINVAL, "pipeline / tx_host / spectra_host is NULL");
    DeviceScope scope(p->dev);
    const size_t txb = static_cast<size_t>(p->Q) * 3 * sizeof(float);
    wrf_status s;
    if (p->steps == 0) {
        std::memcpy(p->tx_pin[0], tx_host, txb);
        if ((s = size_and_capture(p)) != WRF_OK) return s;
    }
    const int k = static_cast<int>(p->steps & 1);
    if ((s = finish_slot(p, k)) != WRF_OK) return s;  // the step two before, same slot
    std::memcpy(p->tx_pin[k], tx_host, txb);
    cudaError_t e = cudaMemcpyAsync(p->tx_dev[k], p->tx_pin[k], txb, cudaMemcpyHostToDevice,
                                    p->compute);
    if (e == cudaSuccess) e = cudaGraphLaunch(p->exec[k], p->compute);
    if (e == cudaSuccess) e = cudaEventRecord(p->done[k], p->compute);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p->copy, p->done[k], 0);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(spectra_host, p->out_dev[k], p->out_bytes, cudaMemcpyDeviceToHost,
                            p->copy);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p->nk_host + k, p->nkeys + k, sizeof(int64_t),
                            cudaMemcpyDeviceToHost, p->copy);
    if (e == cudaSuccess) e = cudaEventRecord(p->freed[k], p->copy);
    if (e != cudaSuccess) return cuda_err(e, "pipeline step");
    p->dst[k] = spectra_host;
    p->cap_used[k] = p->cap;
    p->pending[k] = true;
    ++p->steps;
    return WRF_OK;
}

wrf_status wrf_pipeline_wait(wrf_pipeline *p) {
    if (!p) return wrf::set_error(WRF_EINVAL, "pipeline is NULL");
    DeviceScope scope(p->dev);
    const int older = static_cast<int>(p->steps & 1);  // slot of the earlier pending step
    wrf_status s = finish_slot(p, older);
    if (s != WRF_OK) return s;
    if ((s = finish_slot(p, older ^ 1)) != WRF_OK) return s;
    return p->steps > 0 ? clear_overflow(p) : WRF_OK;
}

wrf_status wrf_pipeline_destroy(wrf_pipeline *p) {
    if (!p) return WRF_OK;
    DeviceScope scope(p->dev);
    cudaStreamSynchronize(p->compute);
    cudaStreamSynchronize(p->copy);
    release(p);
    return WRF_OK;
}

}  // extern "C"
