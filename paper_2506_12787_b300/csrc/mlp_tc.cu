// Deformation MLP on the 5th-generation tensor cores (tcgen05), BF16
// operands with FP32 accumulation in tensor memory (Sec. 4.2, Eq. 14).
//
// Rows are the (query, Gaussian) pairs, flattened as row = q*N + n and cut
// into tiles of 128 rows (one tcgen05 M=128 tile; TMEM lane = row).  A CTA
// has two warpgroups that each own a tile at a time and run independently,
// so one warpgroup's epilogue on the CUDA cores overlaps the other's MMAs on
// the tensor core.  Per tile and warpgroup:
//   1. layer 1 activation h1 = ReLU(U[n] + V[q]) (FP32, see prep.cu) is
//      rounded to BF16 into a 128x128 K-major, 128-byte-swizzled smem tile;
//   2. for every hidden layer: one elected thread issues 8 MMAs
//      (128x128x16, kind::f16) reading the activation tile and the layer's
//      resident weight image, and commits them to an mbarrier; the 128
//      threads then read their row from TMEM (tcgen05.ld 32x32b), add the
//      bias, apply ReLU, round to BF16 and write the next activation tile;
//   3. the output layer is one 128x16x128 MMA chain (5 useful columns);
//      its epilogue adds the bias and either stores the residual row or
//      deforms and projects the Gaussian (fused Eq. 12-13) into its record.
// All weights (<= 3 hidden layers + output, <= 100 KB of BF16) are copied
// into shared memory once per CTA with bulk (TMA) copies.
#include "kernels.h"

namespace wrf {

namespace {

constexpr int kTileRows = 128;
constexpr int kThreads = 256;             // two warpgroups
constexpr uint32_t kLayerBytes = 128 * 128 * 2;
constexpr uint32_t kOutBytes = 16 * 128 * 2;
constexpr uint32_t kActBytes = 128 * 128 * 2;
constexpr uint32_t kTmemCols = 512;       // 2 x (128 hidden + 16 output), rounded to a power of 2

// ------------------------------------------------------------ tcgen05 PTX
__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void named_bar(int id, int count) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
// Barrier over the 128 threads of one warpgroup that also ORs `pred` across
// them, so every thread of the warpgroup takes the same branch afterwards.
__device__ __forceinline__ bool wg_bar_any(int id, bool pred) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, %2, 128, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"(static_cast<uint32_t>(pred)), "r"(id)
        : "memory");
    return r != 0;
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle,
// 8-row core-matrix groups 1024 bytes apart (stride byte offset), start
// address in 16-byte units, descriptor version 1 (bit 46).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);
    d |= static_cast<uint64_t>(1) << 16;                 // leading byte offset (unused here)
    d |= static_cast<uint64_t>(1024 >> 4) << 32;         // stride byte offset
    d |= static_cast<uint64_t>(1) << 46;                 // version
    d |= static_cast<uint64_t>(2) << 61;                 // SWIZZLE_128B
    return d;
}

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
           (static_cast<uint32_t>(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float *v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(b), "f"(a));  // a -> low half
    return r;
}

// Wait on an mbarrier phase; gives up (returning false) when another thread
// has flagged an abort or after kWaitLimitNs, flagging it.  Threads never
// leave a tile early on an abort: they finish it (on garbage) so that every
// named barrier of the tile is reached by all 128 threads, and the tile loop
// ends at the next uniform check.
__device__ __forceinline__ bool wait_or_abort(uint64_t *bar, uint32_t parity,
                                              volatile int *abort_flag, int *status) {
    if (mbar_try_wait(bar, parity)) return true;
    unsigned long long t0 = globaltimer_ns();
    for (;;) {
        for (int i = 0; i < 32; ++i)
            if (mbar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
        if (globaltimer_ns() - t0 > kWaitLimitNs) {
            *abort_flag = 1;
            record_status(status, WRF_ETIMEOUT);
            return false;
        }
    }
}

struct TcArgs {
    SceneView s;
    GridView g;
    const float *U, *V;
    const uint16_t *w_img;   // BF16 images: hidden layers then output layer
    const float *bh[3];
    const float *bo;
    int nh;                  // hidden 128x128 layers (0..3)
    int Q;
    long long rows;
    int ntiles;
    int mode;
    float *resid;
    float4 *rec;
    uint32_t *count;
    int *status;
};

__global__ void __launch_bounds__(kThreads, 1) mlp_tc_kernel(TcArgs a) {
    extern __shared__ uint8_t smem_raw[];
    // 1024-byte aligned base (128-byte swizzle atoms must be 1024-aligned)
    const uint32_t raw = smem_u32(smem_raw);
    uint8_t *base = smem_raw + (((raw + 1023u) & ~1023u) - raw);
    const uint32_t w_bytes = a.nh * kLayerBytes + kOutBytes;
    uint8_t *wsm = base;
    uint8_t *act[2] = {base + w_bytes, base + w_bytes + kActBytes};
    float *bias = reinterpret_cast<float *>(base + w_bytes + 2 * kActBytes);  // [nh*128 + 16]
    uint64_t *bars = reinterpret_cast<uint64_t *>(bias + a.nh * 128 + 16);    // wbar, mbar[2]
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 3);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int wg = warp >> 2, wq = warp & 3;  // warpgroup, warp within warpgroup

    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        mbar_init(&bars[2], 1);
        fence_mbar_init();
        *abort_flag = 0;
    }
    for (int i = tid; i < a.nh * 128; i += kThreads) bias[i] = a.bh[i >> 7][i & 127];
    if (tid < 16) bias[a.nh * 128 + tid] = tid < WRF_OUT ? a.bo[tid] : 0.f;
    if (warp == 0) tmem_alloc(tmem_slot, kTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    if (tid == 0) {
        mbar_arrive_expect_tx(&bars[0], w_bytes);
        const uint8_t *src = reinterpret_cast<const uint8_t *>(a.w_img);
        for (uint32_t off = 0; off < w_bytes; off += 16384u) {
            uint32_t len = w_bytes - off < 16384u ? w_bytes - off : 16384u;
            bulk_g2s(wsm + off, src + off, len, &bars[0]);
        }
    }
    bool ok = wait_or_abort(&bars[0], 0, abort_flag, a.status);
    (void)ok;
    __syncthreads();

    uint64_t *mbar = &bars[1 + wg];
    uint32_t phase = 0;
    uint8_t *A = act[wg];
    const uint32_t a_addr = smem_u32(A);
    const uint32_t w_addr = smem_u32(wsm);
    const uint32_t t_hid = tmem_base + static_cast<uint32_t>(wg * 256);
    const uint32_t t_out = t_hid + 128u;
    const uint32_t lane_off = static_cast<uint32_t>(wq * 32) << 16;  // TMEM lane field
    const int my_row = wq * 32 + lane;                               // row within the tile
    const bool leader = (tid & 127) == 0;
    const float4 *U4 = reinterpret_cast<const float4 *>(a.U);
    const float4 *V4 = reinterpret_cast<const float4 *>(a.V);
    const uint32_t id128 = idesc_bf16(128, 128), id16 = idesc_bf16(128, 16);

    for (int tile = blockIdx.x * 2 + wg; tile < a.ntiles; tile += gridDim.x * 2) {
        // uniform per warpgroup: a timed-out wait anywhere ends the loop for
        // all 128 threads together (no thread is left at a named barrier)
        if (wg_bar_any(1 + wg, *abort_flag != 0)) break;
        const long long row0 = static_cast<long long>(tile) * kTileRows;
        // ---- layer 1: h1 = ReLU(U[n] + V[q]) -> BF16 swizzled tile.
        // Warp wq fills rows 32wq..32wq+31; lane covers K columns 4*lane..4*lane+3.
        {
            const int half = lane >> 4, chunk = (lane & 15) >> 1, sub = (lane & 1) * 8;
            for (int rr = 0; rr < 32; ++rr) {
                const int r = wq * 32 + rr;
                const long long row = row0 + r;
                uint2 packed = make_uint2(0u, 0u);
                if (row < a.rows) {
                    const int q = static_cast<int>(row / a.s.n);
                    const int n = static_cast<int>(row - static_cast<long long>(q) * a.s.n);
                    const float4 u = U4[static_cast<size_t>(n) * 32 + lane];
                    const float4 v = V4[static_cast<size_t>(q) * 32 + lane];
                    packed.x = pack_bf16(fmaxf(u.x + v.x, 0.f), fmaxf(u.y + v.y, 0.f));
                    packed.y = pack_bf16(fmaxf(u.z + v.z, 0.f), fmaxf(u.w + v.w, 0.f));
                }
                *reinterpret_cast<uint2 *>(A + half * 16384 + r * 128 +
                                           ((chunk ^ (r & 7)) << 4) + sub) = packed;
            }
        }
        fence_async_smem();
        named_bar(1 + wg, 128);

        // ---- hidden layers
        for (int l = 0; l < a.nh; ++l) {
            if (leader) {
                tc_fence_after();
                const uint32_t wl = w_addr + l * kLayerBytes;
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const uint32_t koff = (k >> 2) * 16384u + (k & 3) * 32u;
                    mma_bf16(t_hid, sw128_desc(a_addr + koff), sw128_desc(wl + koff), id128,
                             k > 0 ? 1u : 0u);
                }
                mma_commit(mbar);
            }
            wait_or_abort(mbar, phase, abort_flag, a.status);
            phase ^= 1u;
            tc_fence_after();
            const float *bl = bias + l * 128;
#pragma unroll 1
            for (int c = 0; c < 4; ++c) {
                float v[32];
                tmem_ld32(t_hid + lane_off + c * 32, v);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    uint4 p;
                    const float *b = bl + c * 32 + j * 8;
                    p.x = pack_bf16(fmaxf(v[j * 8 + 0] + b[0], 0.f), fmaxf(v[j * 8 + 1] + b[1], 0.f));
                    p.y = pack_bf16(fmaxf(v[j * 8 + 2] + b[2], 0.f), fmaxf(v[j * 8 + 3] + b[3], 0.f));
                    p.z = pack_bf16(fmaxf(v[j * 8 + 4] + b[4], 0.f), fmaxf(v[j * 8 + 5] + b[5], 0.f));
                    p.w = pack_bf16(fmaxf(v[j * 8 + 6] + b[6], 0.f), fmaxf(v[j * 8 + 7] + b[7], 0.f));
                    const int kc = c * 4 + j;  // 16-byte chunk 0..15 along K
                    *reinterpret_cast<uint4 *>(A + (kc >> 3) * 16384 + my_row * 128 +
                                               (((kc & 7) ^ (my_row & 7)) << 4)) = p;
                }
            }
            tc_fence_before();
            fence_async_smem();
            named_bar(1 + wg, 128);
        }

        // ---- output layer (N = 16, columns 0..4 used)
        if (leader) {
            tc_fence_after();
            const uint32_t wo = w_addr + a.nh * kLayerBytes;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const uint32_t ka = (k >> 2) * 16384u + (k & 3) * 32u;
                const uint32_t kb = (k >> 2) * 2048u + (k & 3) * 32u;
                mma_bf16(t_out, sw128_desc(a_addr + ka), sw128_desc(wo + kb), id16,
                         k > 0 ? 1u : 0u);
            }
            mma_commit(mbar);
        }
        wait_or_abort(mbar, phase, abort_flag, a.status);
        phase ^= 1u;
        tc_fence_after();
        float o[16];
        tmem_ld16(t_out + lane_off, o);
        tc_fence_before();
        const long long row = row0 + my_row;
        if (row < a.rows && !*abort_flag) {
            const float *bo = bias + a.nh * 128;
            const float d0 = o[0] + bo[0], d1 = o[1] + bo[1], d2 = o[2] + bo[2],
                        d3 = o[3] + bo[3], d4 = o[4] + bo[4];
            if (a.mode == 0) {
                float *dst = a.resid + row * WRF_OUT;
                dst[0] = d0;
                dst[1] = d1;
                dst[2] = d2;
                dst[3] = d3;
                dst[4] = d4;
            } else {
                const int n = static_cast<int>(row % a.s.n);
                float4 r0, r1;
                uint32_t c = project_one(a.s, n, d0, d1, d2, d3, d4, a.g, r0, r1);
                a.rec[2 * row] = r0;
                a.rec[2 * row + 1] = r1;
                if (a.count) a.count[row] = c;
            }
        }
        named_bar(1 + wg, 128);  // TMEM output columns and the tile are free again
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem_base, kTmemCols);
    }
}

}  // namespace

cudaError_t launch_mlp_tc(const SceneView &s, const MlpView &m, const GridView &g, int Q,
                          const DeformWs &ws, int mode, float *resid, float4 *rec,
                          uint32_t *count, int *status, cudaStream_t st) {
    const long long rows = static_cast<long long>(Q) * s.n;
    if (rows == 0) return cudaSuccess;
    const int nh = m.n_layers - 2;
    if (nh < 0 || nh > 3) return cudaErrorInvalidValue;
    TcArgs a{};
    a.s = s;
    a.g = g;
    a.U = ws.U;
    a.V = ws.V;
    a.w_img = ws.w_bf16;
    for (int l = 0; l < 3; ++l) a.bh[l] = l < nh ? m.bh[l] : nullptr;
    a.bo = m.bo;
    a.nh = nh;
    a.Q = Q;
    a.rows = rows;
    a.ntiles = static_cast<int>((rows + kTileRows - 1) / kTileRows);
    a.mode = mode;
    a.resid = resid;
    a.rec = rec;
    a.count = count;
    a.status = status;
    const size_t smem = 1024 + nh * kLayerBytes + kOutBytes + 2 * kActBytes +
                        (nh * 128 + 16) * 4 + 3 * 8 + 8 + 64;
    cudaError_t e = cudaFuncSetAttribute(mlp_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int grid = (a.ntiles + 1) / 2;
    if (grid > sms) grid = sms;
    mlp_tc_kernel<<<grid, kThreads, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace wrf
