// Shared device helpers for the spectrum-synthesis kernels (sm_103a).
//
// Contents: status codes, bounded waits, PTX wrappers for mbarriers and bulk
// (TMA) copies, the per-Gaussian projection (Sec. 4.2 Eq. 12-13 with the
// residual head dx, dy, drot, dls1, dls2) and the footprint tile rectangle.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/wrf.h"

namespace wrf {

// log2(e)/2: exp(-q/2) == exp2(-q * kHalfLog2e).
constexpr float kHalfLog2e = 0.72134752044448170368f;

// Bounded waits give up after this many nanoseconds of %globaltimer.
constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // 2 s

struct GridView {
    int H, W, tw, th, ntx, nty, T;
    float q_cut;
    int wrap;  // azimuth wrap: columns 0 and W are the same direction
    int px;    // rasteriser: pixels per thread (2 or 4)
    int bpt;   // rasteriser: Gaussian records per thread in a staged batch (1 or 2)
    int tma;   // rasteriser: records staged by TMA gathers (1) or per-thread cp.async (0)
};

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void record_status(int *status, int code) {
    if (status) atomicCAS(status, 0, code);
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// ---------------------------------------------------------------- mbarrier
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Wait for phase `parity` of `bar` to complete; gives up after limit_ns of
// %globaltimer, records WRF_ETIMEOUT and returns false.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int *status,
                                          unsigned long long limit_ns = kWaitLimitNs) {
    if (mbar_try_wait(bar, parity)) return true;
    unsigned long long t0 = globaltimer_ns();
    for (;;) {
        for (int i = 0; i < 64; ++i)
            if (mbar_try_wait(bar, parity)) return true;
        if (globaltimer_ns() - t0 > limit_ns) {
            record_status(status, WRF_ETIMEOUT);
            return false;
        }
    }
}

// ------------------------------------------------------------ bulk copies
// Non-tensor bulk copy global -> shared, completion counted in bytes on
// `bar`.  Both addresses 16-byte aligned, size a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// ------------------------------------------------------- footprint rectangle
// Tiles covered by a record's footprint: pixels ceil(my-ry)..floor(my+ry)
// clipped to the grid, divided by the tile height; columns ceil(mx-rx)..
// floor(mx+rx) clipped to the grid, or, with azimuth wrap (0 and W the same
// direction), taken modulo W, divided by the tile width.  The columns come as
// up to two tile intervals [tx0, tx1] and [tx2, tx3] (the second empty,
// tx2 > tx3, unless a wrapped footprint crosses the seam).  Every step is an
// exactly rounded FP32 operation so the result is a fixed integer function of
// the stored record.
// WRAP: whether g.wrap is set, as a compile-time flag for the binning
// kernels (the general form below reads it at run time).
template <bool WRAP>
__device__ __forceinline__ bool tile_rect_t(float mx, float my, float rx, float ry,
                                            const GridView &g, int &tx0, int &tx1, int &tx2,
                                            int &tx3, int &ty0, int &ty1);

__device__ __forceinline__ bool tile_rect(float mx, float my, float rx, float ry,
                                          const GridView &g, int &tx0, int &tx1, int &tx2,
                                          int &tx3, int &ty0, int &ty1) {
    return g.wrap ? tile_rect_t<true>(mx, my, rx, ry, g, tx0, tx1, tx2, tx3, ty0, ty1)
                  : tile_rect_t<false>(mx, my, rx, ry, g, tx0, tx1, tx2, tx3, ty0, ty1);
}

// a / t for a >= 0 and a tile size t that is a power of two (every
// supported tile shape is: 8, 16 or 32 wide, 8 or 16 high).
__device__ __forceinline__ int tile_of(int a, int t) { return a >> (__ffs(t) - 1); }

template <bool WRAP>
__device__ __forceinline__ bool tile_rect_t(float mx, float my, float rx, float ry,
                                            const GridView &g, int &tx0, int &tx1, int &tx2,
                                            int &tx3, int &ty0, int &ty1) {
    tx2 = 1;
    tx3 = 0;
    const float ylo = __fsub_rn(my, ry), yhi = __fadd_rn(my, ry);
    const float hm = static_cast<float>(g.H - 1);
    if (!(yhi >= 0.f) || !(ylo <= hm)) return false;
    const float ay = ceilf(fmaxf(ylo, 0.f)), by = floorf(fminf(yhi, hm));
    if (ay > by) return false;
    ty0 = tile_of(static_cast<int>(ay), g.th);
    ty1 = tile_of(static_cast<int>(by), g.th);
    const float xlo = __fsub_rn(mx, rx), xhi = __fadd_rn(mx, rx);
    if (!WRAP) {
        const float wm = static_cast<float>(g.W - 1);
        if (!(xhi >= 0.f) || !(xlo <= wm)) return false;
        const float ax = ceilf(fmaxf(xlo, 0.f)), bx = floorf(fminf(xhi, wm));
        if (ax > bx) return false;
        tx0 = tile_of(static_cast<int>(ax), g.tw);
        tx1 = tile_of(static_cast<int>(bx), g.tw);
        return true;
    }
    const float lo = ceilf(xlo), hi = floorf(xhi);
    if (!(lo <= hi)) return false;
    if (__fadd_rn(__fsub_rn(hi, lo), 1.f) >= static_cast<float>(g.W)) {
        tx0 = 0;
        tx1 = g.ntx - 1;
        return true;
    }
    // columns modulo W (|column| < 2^24 for any footprint the rasteriser can
    // use, so 32-bit integers are exact)
    const int c0 = static_cast<int>(lo), c1 = static_cast<int>(hi);
    int a = c0 % g.W, b = c1 % g.W;
    if (a < 0) a += g.W;
    if (b < 0) b += g.W;
    if (a <= b) {
        tx0 = tile_of(a, g.tw);
        tx1 = tile_of(b, g.tw);
        return true;
    }
    const int ta = tile_of(a, g.tw), tb = tile_of(b, g.tw);
    tx0 = 0;
    if (ta <= tb) {  // both pieces of the wrapped footprint meet in one tile
        tx1 = g.ntx - 1;
        return true;
    }
    tx1 = tb;
    tx2 = ta;
    tx3 = g.ntx - 1;
    return true;
}

// Column tiles covered (both intervals of tile_rect).
__device__ __forceinline__ int tile_cols(int tx0, int tx1, int tx2, int tx3) {
    return (tx1 - tx0 + 1) + (tx3 >= tx2 ? tx3 - tx2 + 1 : 0);
}

// Centre x of the image of a Gaussian nearest to column position xc (azimuth
// wrap: the images are mx + k W); mx itself without wrap.
__device__ __forceinline__ float nearest_image_x(float mx, float xc, const GridView &g) {
    if (!g.wrap) return mx;
    const float W = static_cast<float>(g.W);
    return __fsub_rn(mx, W * rintf(__fdiv_rn(__fsub_rn(mx, xc), W)));
}

// ------------------------------------------------------------- projection
struct SceneView {
    int n;
    const float *mean, *log_scale, *rot, *opacity_logit, *amp;  // amp [n][channels]
    int channels;  // 1, or 2 (real and imaginary amplitude)
};

// Reference-frame parameters of one Gaussian (amp_im = 0 with one channel).
struct GaussParams {
    float mx, my, rot, ls1, ls2, op, amp, amp_im;
};
__device__ __forceinline__ GaussParams load_params(const SceneView &s, int n) {
    const float2 m = reinterpret_cast<const float2 *>(s.mean)[n];
    const float2 ls = reinterpret_cast<const float2 *>(s.log_scale)[n];
    const float *a = s.amp + static_cast<size_t>(n) * s.channels;
    return GaussParams{m.x, m.y, s.rot[n], ls.x, ls.y, s.opacity_logit[n], a[0],
                       s.channels == 2 ? a[1] : 0.f};
}

// Weight of the second (imaginary) channel: sigmoid(a) * amp_im, stored by
// the record writers in the tail after the Q x N records ([Q][N] floats).
__device__ __forceinline__ float weight_im(const GaussParams &p) {
    return p.amp_im / (1.f + expf(-p.op));
}

// Number of tiles a record's footprint rectangle covers.
__device__ __forceinline__ uint32_t record_tiles(const float4 &r0, const float4 &r1,
                                                 const GridView &g) {
    int a, b, a2, b2, c, d;
    if (!tile_rect(r0.x, r0.y, r1.z, r1.w, g, a, b, a2, b2, c, d)) return 0u;
    return static_cast<uint32_t>(tile_cols(a, b, a2, b2) * (d - c + 1));
}

// Deform a Gaussian by its residual (Eq. 12) and project it to a record:
// centre, log2(e)/2-scaled inverse covariance of R(th) diag(s1^2, s2^2) R^T,
// weight sigmoid(a) * amp (Sec. 4.1) and footprint half-widths.
__device__ __forceinline__ void project_geom(const GaussParams &p, float d0, float d1, float d2,
                                             float d3, float d4, const GridView &g, float4 &r0,
                                             float4 &r1) {
    float mx = p.mx + d0, my = p.my + d1;
    float th = p.rot + d2;
    float l1 = p.ls1 + d3, l2 = p.ls2 + d4;
    float sn, cs;
    sincosf(th, &sn, &cs);
    float v1 = expf(2.f * l1), v2 = expf(2.f * l2);
    float i1 = expf(-2.f * l1), i2 = expf(-2.f * l2);
    float cc = cs * cs, ss = sn * sn, csn = cs * sn;
    float sxx = cc * v1 + ss * v2, syy = ss * v1 + cc * v2;
    float A = cc * i1 + ss * i2, B = csn * (i1 - i2), C = ss * i1 + cc * i2;
    float w = p.amp / (1.f + expf(-p.op));
    float rx = sqrtf(g.q_cut * sxx), ry = sqrtf(g.q_cut * syy);
    r0 = make_float4(mx, my, A * kHalfLog2e, B * kHalfLog2e);
    r1 = make_float4(C * kHalfLog2e, w, rx, ry);
}

// project_geom, returning the number of tiles the footprint covers.
__device__ __forceinline__ uint32_t project_params(const GaussParams &p, float d0, float d1,
                                                   float d2, float d3, float d4,
                                                   const GridView &g, float4 &r0, float4 &r1) {
    project_geom(p, d0, d1, d2, d3, d4, g, r0, r1);
    return record_tiles(r0, r1, g);
}


// ------------------------------------------------------ positional encoding
// Eq. 15 applies sin and cos to 2^k pi x for k up to L-1 (2^9 pi at L = 10):
// a rounding of x by one FP32 ulp would move the phase of the top band by
// ~1e-4.  x = (a - b) / d is therefore carried as an unevaluated sum
// hi + lo of two FP32 numbers (TwoSum for a - b, the exact FMA remainder for
// the division), and the phase 2^k (hi + lo) is reduced modulo 2 exactly
// before sincospif, so every band keeps FP32 accuracy.
struct PeArg {
    float hi, lo;
};
__device__ __forceinline__ PeArg pe_arg(float a, float b, float d) {
    const float t = __fsub_rn(a, b);
    const float nb = -b;
    const float bb = __fsub_rn(t, a);  // TwoSum: a + nb = t + e exactly
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(t, bb)), __fsub_rn(nb, bb));
    const float hi = __fdiv_rn(t, d);
    const float r = fmaf(-hi, d, t);  // t - hi d, exact
    return PeArg{hi, __fdiv_rn(__fadd_rn(r, e), d)};
}
__device__ __forceinline__ float pe_value(PeArg x) { return __fadd_rn(x.hi, x.lo); }
// sin(2^k pi x), cos(2^k pi x): 2^k hi is exact, and so is its reduction by
// the nearest even integer (Sterbenz), leaving |phase| <= 1 plus 2^k lo.
__device__ __forceinline__ void pe_band(PeArg x, int k, float &s, float &c) {
    const float h = ldexpf(x.hi, k);
    const float n2 = 2.f * rintf(0.5f * h);
    const float red = __fadd_rn(__fsub_rn(h, n2), ldexpf(x.lo, k));
    sincospif(red, &s, &c);
}

// gamma(x) of Eq. 15 for a d-vector, written to out[d(2L+1)] in the order
// [x, sin band 0 (all d), ..., sin band L-1, cos band 0, ..., cos band L-1].
__device__ inline void pe_encode(const PeArg *x, int d, int L, float *out) {
    for (int i = 0; i < d; ++i) out[i] = pe_value(x[i]);
    for (int k = 0; k < L; ++k)
        for (int i = 0; i < d; ++i) {
            float s, c;
            pe_band(x[i], k, s, c);
            out[d + k * d + i] = s;
            out[d + L * d + k * d + i] = c;
        }
}

// ------------------------------------------------------------ cp.async
// 16-byte global -> shared copy (L2 only), its commit and a wait for all.
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
// Wait until at most N of this thread's committed groups are still pending.
template <int N>
__device__ __forceinline__ void cp_async_wait_pending() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

}  // namespace wrf
