// Pieces of the paper's primitive and head (Sec. 4.1-4.2) shared by the FP32
// and the tensor-core network kernels: the skip layout, the tanh centre map
// and the projection to two-channel records (the encoding of Eq. 15 is
// pe_encode in common.cuh).
#pragma once
#include "common.cuh"

namespace wrf {

// hidden layers whose input also holds the encoding (a skip every two layers)
__host__ __device__ inline bool is_skip(int l) { return l == 2 || l == 4 || l == 6; }
// index of an encoding layer among {0, 2, 4, 6}
__host__ __device__ inline int enc_index(int l) { return l / 2; }

struct PaperView {
    int n;
    const float *mu, *chol, *attn, *psi;
};

// (tanh u + 1) / 2 as an unevaluated sum hi + lo (Fast2Sum of 1 + tanh u,
// |tanh u| <= 1; halving is exact), the encoding's input on the unit square.
__device__ __forceinline__ PeArg unit_centre(float u) {
    const float t = tanhf(u);
    const float s = __fadd_rn(1.f, t);
    const float e = __fadd_rn(__fsub_rn(1.f, s), t);
    return PeArg{0.5f * s, 0.5f * e};
}

// Reference centre in pixels: x = W (tanh u + 1) / 2, y = H (tanh v + 1) / 2.
__device__ __forceinline__ void centre(const PaperView &s, int n, const GridView &g, float &x,
                                       float &y) {
    const float2 m = reinterpret_cast<const float2 *>(s.mu)[n];
    x = static_cast<float>(g.W) * pe_value(unit_centre(m.x));
    y = static_cast<float>(g.H) * pe_value(unit_centre(m.y));
}


// Record of Gaussian n for query q (Eq. 12-13 with the paper's primitive):
// centre x0 + dmu, inverse of Sigma = L L^T (scaled by log2(e)/2), real
// weight (delta + ddelta)(psi_re + dpsi_re) in the record, imaginary weight
// (delta + ddelta)(psi_im + dpsi_im) after the records.  d = (dmu_x, dmu_y,
// dpsi_re, dpsi_im, ddelta).
__device__ __forceinline__ void paper_project(const PaperView &s, int n, int q, const float *d,
                                              const GridView &g, float4 *rec, float *rec_im) {
    float x, y;
    centre(s, n, g, x, y);
    const float mx = x + d[0], my = y + d[1];
    const float *L = s.chol + static_cast<size_t>(n) * 3;
    const float l1 = L[0], l2 = L[1], l3 = L[2];
    const float sxx = l1 * l1, sxy = l1 * l2, syy = fmaf(l2, l2, l3 * l3);
    const float det = (l1 * l3) * (l1 * l3);
    const float inv = 1.f / det;
    const float A = syy * inv, B = -sxy * inv, C = sxx * inv;
    const float delta = 1.f / (1.f + expf(-s.attn[n])) + d[4];
    const float2 ps = reinterpret_cast<const float2 *>(s.psi)[n];
    const float rx = sqrtf(g.q_cut * sxx), ry = sqrtf(g.q_cut * syy);
    const size_t row = static_cast<size_t>(q) * s.n + n;
    rec[2 * row] = make_float4(mx, my, A * kHalfLog2e, B * kHalfLog2e);
    rec[2 * row + 1] = make_float4(C * kHalfLog2e, delta * (ps.x + d[2]), rx, ry);
    rec_im[row] = delta * (ps.y + d[3]);
}

}  // namespace wrf
