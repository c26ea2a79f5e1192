/*
 * FP64 CPU oracle for SwiftWRF spectrum synthesis (arXiv 2506.12787).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or
 * calls this file; only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg do.  It shares no code, header or constant table with the
 * CUDA library.
 *
 * Each function restates one definition of the paper in plain double
 * precision, with no blocking, fusion or reordering beyond what the
 * definition states:
 *   or_pe          positional encoding gamma(x), Sec. 4.2 Eq. 15
 *   or_mlp_row     the deformation MLP F_theta, Sec. 4.2 Eq. 14 (unfactorised)
 *   or_deform      residuals for every (query, Gaussian) pair, Eqs. 12 and 14
 *   or_project     deformed centre, inverse covariance and weight, Eqs. 8, 12
 *   or_render      the order-free truncated Gaussian sum, Eqs. 9 and 13
 *   or_bin_f32     tile lists: an integer function of FP32 records (Sec. 4.1,
 *                  "the spectrum domain partitioned into parallel tiles")
 *   or_*_grad      analytic derivatives of the above (Sec. 4.1, 4.4: the
 *                  parameters are fitted by back-propagation)
 *
 * Readings where the paper is silent (stated once here, used throughout):
 *   - pixel (j,k) of an H x W spectrum sits at x = j (azimuth column),
 *     y = k (elevation row), integer units, Sec. 3.1 Eq. 5 layout;
 *   - a Gaussian contributes to a pixel only where q = d^T Sigma^-1 d <= q_cut;
 *     q_cut = +inf means no cutoff;
 *   - Sigma = R(theta) diag(sigma1^2, sigma2^2) R(theta)^T with
 *     sigma_i = exp(log_scale_i); the MLP outputs (dx, dy, drot, dls1, dls2);
 *   - weight w = sigmoid(opacity_logit) * amp (Sec. 4.1, delta = sigma(a));
 *   - PE inputs: mean normalised to (x/W, y/H), TX to (s - room_min)/room_size.
 *
 * Parity pins: every function here is checked in tests/test_oracle.py
 * against closed forms, invariants or an independent brute force.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_EINVAL (-1)
#define OR_ENOSPC (-2)
#define OR_MAX_LAYERS 8
#define OR_MAX_WIDTH 512

/* ---------------------------------------------------------------- PE ---- */
/* Eq. 15: gamma(s) = [s, sin(2^k pi s)_{k<L}, cos(2^k pi s)_{k<L}], each term
 * applied to every component; output length d(2L+1), ordered
 * [s_0..s_{d-1}, sin k=0 (all d), ..., sin k=L-1, cos k=0, ..., cos k=L-1]. */
void or_pe(const double *x, int d, int L, double *out)
{
    for (int i = 0; i < d; ++i) out[i] = x[i];
    for (int k = 0; k < L; ++k) {
        double f = ldexp(M_PI, k); /* 2^k * pi */
        for (int i = 0; i < d; ++i) {
            out[d + k * d + i] = sin(f * x[i]);
            out[d + L * d + k * d + i] = cos(f * x[i]);
        }
    }
}

/* -------------------------------------------------------------- MLP ---- */
/* params: for each layer l, W_l [dims[l+1]][dims[l]] row-major then b_l. */
static size_t param_count(int n_layers, const int *dims)
{
    size_t c = 0;
    for (int l = 0; l < n_layers; ++l) c += (size_t)dims[l + 1] * dims[l] + dims[l + 1];
    return c;
}

/* One row through F_theta: hidden layers Linear+ReLU, last layer Linear.
 * If `pre` is non-NULL the pre-activations of every layer are stored there
 * ([n_layers][OR_MAX_WIDTH]) for the backward pass. */
void or_mlp_row(const double *in, int n_layers, const int *dims, const double *params,
                double *out, double *pre)
{
    double a[OR_MAX_WIDTH], z[OR_MAX_WIDTH];
    memcpy(a, in, sizeof(double) * dims[0]);
    const double *p = params;
    for (int l = 0; l < n_layers; ++l) {
        int din = dims[l], dout = dims[l + 1];
        const double *Wl = p, *bl = p + (size_t)dout * din;
        for (int j = 0; j < dout; ++j) {
            double s = bl[j];
            for (int k = 0; k < din; ++k) s += Wl[(size_t)j * din + k] * a[k];
            z[j] = s;
        }
        if (pre) memcpy(pre + (size_t)l * OR_MAX_WIDTH, z, sizeof(double) * dout);
        if (l + 1 < n_layers)
            for (int j = 0; j < dout; ++j) a[j] = z[j] > 0.0 ? z[j] : 0.0;
        else
            memcpy(out, z, sizeof(double) * dout);
        p += (size_t)dout * din + dout;
    }
}

/* The MLP input for (Gaussian n, query s): [gamma(mean_n normalised),
 * gamma(tx normalised)], Eq. 14. */
static void mlp_input(const double *mean_n, int H, int W, const double *tx, int L_mean,
                      int L_tx, const double *room_min, const double *room_size, double *in)
{
    double mu[2] = {mean_n[0] / W, mean_n[1] / H};
    double s[3];
    for (int i = 0; i < 3; ++i) s[i] = (tx[i] - room_min[i]) / room_size[i];
    or_pe(mu, 2, L_mean, in);
    or_pe(s, 3, L_tx, in + 2 * (2 * L_mean + 1));
}

/* Residuals [Q][N][out] for every (query, Gaussian) row: Eq. 14 evaluated
 * row by row, no factorisation. */
int or_deform(int N, const double *mean, int H, int W, int Q, const double *tx, int L_mean,
              int L_tx, const double *room_min, const double *room_size, int n_layers,
              const int *dims, const double *params, double *resid)
{
    if (n_layers < 1 || n_layers > OR_MAX_LAYERS) return OR_EINVAL;
    if (dims[0] != 2 * (2 * L_mean + 1) + 3 * (2 * L_tx + 1)) return OR_EINVAL;
    for (int l = 0; l <= n_layers; ++l)
        if (dims[l] < 1 || dims[l] > OR_MAX_WIDTH) return OR_EINVAL;
    int dout = dims[n_layers];
    long long rows = (long long)N * Q;
#pragma omp parallel for schedule(static)
    for (long long r = 0; r < rows; ++r) {
        int q = (int)(r / N), n = (int)(r % N);
        double in[OR_MAX_WIDTH];
        mlp_input(mean + 2 * (size_t)n, H, W, tx + 3 * (size_t)q, L_mean, L_tx, room_min,
                  room_size, in);
        or_mlp_row(in, n_layers, dims, params, resid + (size_t)r * dout, NULL);
    }
    return OR_OK;
}

/* ---------------------------------------------------------- project ---- */
/* Deformed Gaussian for (q, n), Eq. 12/13 with the residual head
 * (dx, dy, drot, dls1, dls2).  proj row = [mx, my, A, B, C, w, rx, ry] where
 * [[A,B],[B,C]] = Sigma^-1 and rx, ry = sqrt(q_cut * Sigma_xx),
 * sqrt(q_cut * Sigma_yy) are the axis extents of the q <= q_cut ellipse. */
void or_project(int N, const double *mean, const double *log_scale, const double *rot,
                const double *opacity_logit, const double *amp, int Q, const double *resid,
                double q_cut, double *proj)
{
    long long rows = (long long)N * Q;
#pragma omp parallel for schedule(static)
    for (long long r = 0; r < rows; ++r) {
        int n = (int)(r % N);
        const double *d = resid ? resid + (size_t)r * 5 : NULL;
        double mx = mean[2 * n] + (d ? d[0] : 0.0);
        double my = mean[2 * n + 1] + (d ? d[1] : 0.0);
        double th = rot[n] + (d ? d[2] : 0.0);
        double l1 = log_scale[2 * n] + (d ? d[3] : 0.0);
        double l2 = log_scale[2 * n + 1] + (d ? d[4] : 0.0);
        double c = cos(th), s = sin(th);
        double v1 = exp(2.0 * l1), v2 = exp(2.0 * l2); /* sigma_i^2 */
        double sxx = c * c * v1 + s * s * v2;
        double syy = s * s * v1 + c * c * v2;
        double i1 = 1.0 / v1, i2 = 1.0 / v2;
        double A = c * c * i1 + s * s * i2;
        double B = c * s * (i1 - i2);
        double C = s * s * i1 + c * c * i2;
        double w = amp[n] / (1.0 + exp(-opacity_logit[n]));
        double *o = proj + (size_t)r * 8;
        o[0] = mx; o[1] = my; o[2] = A; o[3] = B; o[4] = C; o[5] = w;
        o[6] = sqrt(q_cut * sxx);
        o[7] = sqrt(q_cut * syy);
    }
}

/* ----------------------------------------------------------- render ---- */
/* Integer pixel range [lo, hi] of the extent centre +- r on an axis of
 * `size` pixels; returns 0 when empty.  Infinite r covers the whole axis. */
static int pixel_range(double centre, double r, int size, int *lo, int *hi)
{
    if (isnan(centre) || isnan(r)) return 0;
    if (isinf(r)) { *lo = 0; *hi = size - 1; return size > 0; }
    double a = ceil(centre - r), b = floor(centre + r);
    if (a < 0) a = 0;
    if (b > size - 1) b = size - 1;
    if (a > b) return 0;
    *lo = (int)a; *hi = (int)b;
    return 1;
}

/* Eq. 9 / 13: A(y, x) = sum_n [q_n <= q_cut] w_n exp(-q_n / 2), summed per
 * pixel in ascending n.  `slack` (optional) receives, per pixel, the sum of
 * |w| exp(-q/2) over the Gaussians whose q lies within band*q_cut of q_cut,
 * where an FP32 evaluation may legitimately fall on the other side: a bound
 * on the magnitude of what either decision adds, whatever the sign of w. */
/* Images of a Gaussian along the azimuth axis: with wrap (0 and W columns
 * the same direction) the sum runs over the centres mx + m W whose extent
 * +- r meets [0, W-1]; without wrap only m = 0.  r must be finite with wrap. */
static void image_range(double mx, double r, int W, int wrap, int *m_lo, int *m_hi)
{
    if (!wrap) { *m_lo = 0; *m_hi = 0; return; }
    *m_lo = (int)ceil((-r - mx) / W);
    *m_hi = (int)floor((W - 1 + r - mx) / W);
}

int or_render_w(int Q, int N, const double *proj, int H, int W, double q_cut, double band,
                int wrap, double *out, double *slack);

int or_render(int Q, int N, const double *proj, int H, int W, double q_cut, double band,
              double *out, double *slack)
{
    return or_render_w(Q, N, proj, H, W, q_cut, band, 0, out, slack);
}

int or_render_w(int Q, int N, const double *proj, int H, int W, double q_cut, double band,
                int wrap, double *out, double *slack)
{
    if (H < 1 || W < 1) return OR_EINVAL;
    if (wrap && isinf(q_cut)) return OR_EINVAL;
    double widen = sqrt(1.0 + band);
#pragma omp parallel for schedule(dynamic, 1)
    for (int q = 0; q < Q; ++q) {
        double *A = out + (size_t)q * H * W;
        double *S = slack ? slack + (size_t)q * H * W : NULL;
        memset(A, 0, sizeof(double) * H * W);
        if (S) memset(S, 0, sizeof(double) * H * W);
        for (int n = 0; n < N; ++n) {
            const double *p = proj + ((size_t)q * N + n) * 8;
            int m_lo, m_hi, y0, y1;
            if (!pixel_range(p[1], p[7] * widen, H, &y0, &y1)) continue;
            image_range(p[0], p[6] * widen, W, wrap, &m_lo, &m_hi);
            for (int m = m_lo; m <= m_hi; ++m) {
                double cx = p[0] + (double)m * W;
                int x0, x1;
                if (!pixel_range(cx, p[6] * widen, W, &x0, &x1)) continue;
                for (int y = y0; y <= y1; ++y)
                    for (int x = x0; x <= x1; ++x) {
                        double dx = x - cx, dy = y - p[1];
                        double qq = p[2] * dx * dx + 2.0 * p[3] * dx * dy + p[4] * dy * dy;
                        double e = p[5] * exp(-0.5 * qq);
                        if (qq <= q_cut) A[(size_t)y * W + x] += e;
                        if (S && fabs(qq - q_cut) <= band * q_cut) S[(size_t)y * W + x] += fabs(e);
                    }
            }
        }
    }
    return OR_OK;
}

/* -------------------------------------------------------------- bin ---- */
/* Tile rectangle of an FP32 record, decided in FP32 (the precision the
 * records are stored in): pixels ceil(mx-rx)..floor(mx+rx) clipped to the
 * grid, then divided by the tile size.  Returns 0 for an empty footprint. */
static int rect_f32(const float *r, int H, int W, int tw, int th, int *tx0, int *tx1,
                    int *ty0, int *ty1)
{
    float mx = r[0], my = r[1], rx = r[6], ry = r[7];
    float xlo = mx - rx, xhi = mx + rx, ylo = my - ry, yhi = my + ry;
    float wm = (float)(W - 1), hm = (float)(H - 1);
    if (!(xhi >= 0.0f) || !(xlo <= wm) || !(yhi >= 0.0f) || !(ylo <= hm)) return 0;
    float ax = ceilf(fmaxf(xlo, 0.0f)), bx = floorf(fminf(xhi, wm));
    float ay = ceilf(fmaxf(ylo, 0.0f)), by = floorf(fminf(yhi, hm));
    if (ax > bx || ay > by) return 0;
    *tx0 = (int)ax / tw; *tx1 = (int)bx / tw;
    *ty0 = (int)ay / th; *ty1 = (int)by / th;
    return 1;
}

/* Tile lists: for each query q and tile t (row-major over tiles), the ids n
 * of the Gaussians whose rectangle covers t, in ascending n.  offsets has
 * Q*T+1 entries (CSR); counts[q*N+n] = number of tiles of (q, n).  When the
 * total exceeds `cap`, no ids are written and OR_ENOSPC is returned with
 * *n_keys set to the required total. */
/* With azimuth wrap: the column pixels ceil(mx-rx)..floor(mx+rx) (FP32)
 * taken modulo W, as the tile intervals [a0, a1] and [b0, b1] (the second
 * empty, b0 > b1, unless the footprint crosses the 0 / W seam); rows as
 * without wrap.  Returns 0 for an empty footprint. */
static int rect_f32_wrap(const float *r, int H, int W, int tw, int th, int *a0, int *a1, int *b0,
                         int *b1, int *ty0, int *ty1)
{
    float mx = r[0], my = r[1], rx = r[6], ry = r[7];
    float ylo = my - ry, yhi = my + ry, hm = (float)(H - 1);
    if (!(yhi >= 0.0f) || !(ylo <= hm)) return 0;
    float ay = ceilf(fmaxf(ylo, 0.0f)), by = floorf(fminf(yhi, hm));
    if (ay > by) return 0;
    float lo = ceilf(mx - rx), hi = floorf(mx + rx);
    if (!(lo <= hi)) return 0;
    int ntx = (W + tw - 1) / tw;
    *ty0 = (int)ay / th; *ty1 = (int)by / th;
    *b0 = 1; *b1 = 0;
    if (hi - lo + 1.0f >= (float)W) { *a0 = 0; *a1 = ntx - 1; return 1; }
    long c0 = (long)lo, c1 = (long)hi;
    long a = ((c0 % W) + W) % W, b = ((c1 % W) + W) % W;
    if (a <= b) { *a0 = (int)(a / tw); *a1 = (int)(b / tw); return 1; }
    int ta = (int)(a / tw), tb = (int)(b / tw);
    if (ta <= tb) { *a0 = 0; *a1 = ntx - 1; return 1; }  /* both pieces in one tile */
    *a0 = 0; *a1 = tb; *b0 = ta; *b1 = ntx - 1;
    return 1;
}

/* Column tile intervals of a record: [a0,a1] and [b0,b1] (b empty unless
 * wrapped); returns 0 when the footprint is empty. */
static int rect_any(const float *r, int H, int W, int tw, int th, int wrap, int *a0, int *a1,
                    int *b0, int *b1, int *ty0, int *ty1)
{
    if (wrap) return rect_f32_wrap(r, H, W, tw, th, a0, a1, b0, b1, ty0, ty1);
    *b0 = 1; *b1 = 0;
    return rect_f32(r, H, W, tw, th, a0, a1, ty0, ty1);
}

int or_bin_f32_w(int Q, int N, const float *rec, int H, int W, int tw, int th, int wrap,
                 uint32_t *counts, uint32_t *gids, int64_t cap, int64_t *n_keys,
                 uint32_t *offsets);

int or_bin_f32(int Q, int N, const float *rec, int H, int W, int tw, int th, uint32_t *counts,
               uint32_t *gids, int64_t cap, int64_t *n_keys, uint32_t *offsets)
{
    return or_bin_f32_w(Q, N, rec, H, W, tw, th, 0, counts, gids, cap, n_keys, offsets);
}

int or_bin_f32_w(int Q, int N, const float *rec, int H, int W, int tw, int th, int wrap,
                 uint32_t *counts, uint32_t *gids, int64_t cap, int64_t *n_keys,
                 uint32_t *offsets)
{
    if (tw < 1 || th < 1 || H < 1 || W < 1) return OR_EINVAL;
    int ntx = (W + tw - 1) / tw, nty = (H + th - 1) / th, T = ntx * nty;
    uint64_t *cnt = calloc((size_t)Q * T, sizeof(uint64_t));
    if (!cnt) return OR_EINVAL;
    for (int q = 0; q < Q; ++q)
        for (int n = 0; n < N; ++n) {
            int a, b, a2, b2, c, d, k = 0;
            if (rect_any(rec + ((size_t)q * N + n) * 8, H, W, tw, th, wrap, &a, &b, &a2, &b2, &c,
                         &d)) {
                for (int ty = c; ty <= d; ++ty) {
                    for (int tx = a; tx <= b; ++tx) { cnt[(size_t)q * T + ty * ntx + tx]++; ++k; }
                    for (int tx = a2; tx <= b2; ++tx) { cnt[(size_t)q * T + ty * ntx + tx]++; ++k; }
                }
            }
            if (counts) counts[(size_t)q * N + n] = (uint32_t)k;
        }
    uint64_t run = 0;
    for (size_t i = 0; i < (size_t)Q * T; ++i) {
        uint64_t c = cnt[i];
        offsets[i] = (uint32_t)run;
        cnt[i] = run; /* becomes the fill cursor */
        run += c;
    }
    offsets[(size_t)Q * T] = (uint32_t)run;
    *n_keys = (int64_t)run;
    if ((int64_t)run > cap || run > 0xffffffffull) { free(cnt); return OR_ENOSPC; }
    for (int q = 0; q < Q; ++q)
        for (int n = 0; n < N; ++n) {
            int a, b, a2, b2, c, d;
            if (!rect_any(rec + ((size_t)q * N + n) * 8, H, W, tw, th, wrap, &a, &b, &a2, &b2, &c,
                          &d))
                continue;
            for (int ty = c; ty <= d; ++ty) {
                for (int tx = a; tx <= b; ++tx) gids[cnt[(size_t)q * T + ty * ntx + tx]++] = n;
                for (int tx = a2; tx <= b2; ++tx) gids[cnt[(size_t)q * T + ty * ntx + tx]++] = n;
            }
        }
    free(cnt);
    return OR_OK;
}

/* -------------------------------------------------------- gradients ---- */
/* d/d(proj) of L given dL/dA: dproj row = [dmx, dmy, dA, dB, dC, dw].  The
 * cutoff indicator is piecewise constant and contributes no derivative. */
int or_render_grad_w(int Q, int N, const double *proj, int H, int W, double q_cut, int wrap,
                     const double *dA, double *dproj);

int or_render_grad(int Q, int N, const double *proj, int H, int W, double q_cut,
                   const double *dA, double *dproj)
{
    return or_render_grad_w(Q, N, proj, H, W, q_cut, 0, dA, dproj);
}

int or_render_grad_w(int Q, int N, const double *proj, int H, int W, double q_cut, int wrap,
                     const double *dA, double *dproj)
{
    if (wrap && isinf(q_cut)) return OR_EINVAL;
#pragma omp parallel for schedule(dynamic, 1)
    for (int q = 0; q < Q; ++q) {
        const double *G = dA + (size_t)q * H * W;
        for (int n = 0; n < N; ++n) {
            const double *p = proj + ((size_t)q * N + n) * 8;
            double *g = dproj + ((size_t)q * N + n) * 6;
            for (int i = 0; i < 6; ++i) g[i] = 0.0;
            int m_lo, m_hi, y0, y1;
            if (!pixel_range(p[1], p[7], H, &y0, &y1)) continue;
            image_range(p[0], p[6], W, wrap, &m_lo, &m_hi);
            for (int m = m_lo; m <= m_hi; ++m) {
                double cx = p[0] + (double)m * W;
                int x0, x1;
                if (!pixel_range(cx, p[6], W, &x0, &x1)) continue;
                for (int y = y0; y <= y1; ++y)
                    for (int x = x0; x <= x1; ++x) {
                        double dx = x - cx, dy = y - p[1];
                        double qq = p[2] * dx * dx + 2.0 * p[3] * dx * dy + p[4] * dy * dy;
                        if (!(qq <= q_cut)) continue;
                        double e = exp(-0.5 * qq), gp = G[(size_t)y * W + x];
                        double gw = gp * p[5] * e;
                        g[0] += gw * (p[2] * dx + p[3] * dy);
                        g[1] += gw * (p[3] * dx + p[4] * dy);
                        g[2] += -0.5 * gw * dx * dx;
                        g[3] += -gw * dx * dy;
                        g[4] += -0.5 * gw * dy * dy;
                        g[5] += gp * e;
                    }
            }
        }
    }
    return OR_OK;
}

/* Chain rule through or_project: from dproj [Q,N,6] to dresid [Q,N,5]
 * (d of dx, dy, drot, dls1, dls2) and the reference-frame parameters summed
 * over queries (d_mean [N,2], d_log_scale [N,2], d_rot, d_opacity, d_amp). */
void or_project_grad(int N, const double *log_scale, const double *rot,
                     const double *opacity_logit, const double *amp, int Q,
                     const double *resid, const double *dproj, double *dresid, double *d_mean,
                     double *d_log_scale, double *d_rot, double *d_opacity, double *d_amp)
{
    memset(d_mean, 0, sizeof(double) * 2 * N);
    memset(d_log_scale, 0, sizeof(double) * 2 * N);
    memset(d_rot, 0, sizeof(double) * N);
    memset(d_opacity, 0, sizeof(double) * N);
    memset(d_amp, 0, sizeof(double) * N);
#pragma omp parallel for schedule(static)
    for (int n = 0; n < N; ++n) {
        for (int q = 0; q < Q; ++q) {
            size_t r = (size_t)q * N + n;
            const double *d = resid ? resid + r * 5 : NULL;
            const double *g = dproj + r * 6;
            double th = rot[n] + (d ? d[2] : 0.0);
            double l1 = log_scale[2 * n] + (d ? d[3] : 0.0);
            double l2 = log_scale[2 * n + 1] + (d ? d[4] : 0.0);
            double c = cos(th), s = sin(th);
            double i1 = exp(-2.0 * l1), i2 = exp(-2.0 * l2);
            /* dA/dth, dB/dth, dC/dth */
            double dAt = -2.0 * c * s * (i1 - i2), dBt = (c * c - s * s) * (i1 - i2),
                   dCt = 2.0 * c * s * (i1 - i2);
            double gth = g[2] * dAt + g[3] * dBt + g[4] * dCt;
            double gl1 = -2.0 * i1 * (g[2] * c * c + g[3] * c * s + g[4] * s * s);
            double gl2 = -2.0 * i2 * (g[2] * s * s - g[3] * c * s + g[4] * c * c);
            double sg = 1.0 / (1.0 + exp(-opacity_logit[n]));
            if (dresid) {
                double *dr = dresid + r * 5;
                dr[0] = g[0]; dr[1] = g[1]; dr[2] = gth; dr[3] = gl1; dr[4] = gl2;
            }
            d_mean[2 * n] += g[0];
            d_mean[2 * n + 1] += g[1];
            d_rot[n] += gth;
            d_log_scale[2 * n] += gl1;
            d_log_scale[2 * n + 1] += gl2;
            d_opacity[n] += g[5] * amp[n] * sg * (1.0 - sg);
            d_amp[n] += g[5] * sg;
        }
    }
}

/* Back-propagation of one row through F_theta (Sec. 4.4: every parameter is
 * fitted by gradient descent).  `pre` holds the row's pre-activations from
 * or_mlp_row.  The ReLU decision of hidden unit j of layer l is z > 0, except
 * for the one unit (flip_l, flip_j), if flip_l >= 0, whose decision is taken
 * the other way round (its activation then counts as 0: it lies within
 * rounding of zero).  Adds the row's parameter gradient into gp (params
 * layout) and, unless stop_grad_mean is set, the derivative through
 * gamma(mean) into gm[2]. */
static void row_backward(const double *in, const double *pre, int n_layers, const int *dims,
                         const double *params, const size_t *off, const double *dres,
                         int flip_l, int flip_j, int stop_grad_mean, const double *mu, int H,
                         int W, int L_mean, double *gp, double *gm)
{
    double delta[OR_MAX_WIDTH], prev[OR_MAX_WIDTH], act[OR_MAX_WIDTH];
    int dl = dims[n_layers];
    memcpy(delta, dres, sizeof(double) * dl);
    for (int l = n_layers - 1; l >= 0; --l) {
        int din = dims[l], dout = dims[l + 1];
        const double *Wl = params + off[l];
        double *gW = gp + off[l], *gb = gW + (size_t)dout * din;
        /* input activation of layer l: ReLU of layer l-1's pre-activation */
        if (l == 0) memcpy(act, in, sizeof(double) * din);
        else
            for (int k = 0; k < din; ++k) {
                double z = pre[(size_t)(l - 1) * OR_MAX_WIDTH + k];
                int on = z > 0.0;
                if (l - 1 == flip_l && k == flip_j) { on = !on; z = 0.0; }
                act[k] = on ? z : 0.0;
            }
        for (int j = 0; j < dout; ++j) {
            gb[j] += delta[j];
            for (int k = 0; k < din; ++k) gW[(size_t)j * din + k] += delta[j] * act[k];
        }
        for (int k = 0; k < din; ++k) {
            double sum = 0.0;
            for (int j = 0; j < dout; ++j) sum += Wl[(size_t)j * din + k] * delta[j];
            prev[k] = sum;
        }
        if (l > 0)
            for (int k = 0; k < din; ++k) {
                int on = pre[(size_t)(l - 1) * OR_MAX_WIDTH + k] > 0.0;
                if (l - 1 == flip_l && k == flip_j) on = !on;
                delta[k] = on ? prev[k] : 0.0;
            }
        else
            memcpy(delta, prev, sizeof(double) * din);
    }
    if (!stop_grad_mean) {
        /* delta now holds dL/d(input features); the first dm belong to gamma(mean). */
        for (int i = 0; i < 2; ++i) {
            double g = delta[i];
            for (int k = 0; k < L_mean; ++k) {
                double f = ldexp(M_PI, k);
                g += delta[2 + k * 2 + i] * f * cos(f * mu[i]);
                g -= delta[2 + L_mean * 2 + k * 2 + i] * f * sin(f * mu[i]);
            }
            gm[i] += g / (i == 0 ? W : H);
        }
    }
}

/* Back-propagation through F_theta for every row: accumulates d_params
 * (same layout as params) and, unless stop_grad_mean is set, adds the
 * derivative through gamma(mean) to d_mean [N,2] (the paper freezes position
 * gradients in its fine stage, Sec. 4.4; the flag reproduces that).
 *
 * Ambiguous ReLU decisions: a hidden pre-activation z with
 * |z| <= band * (|b_j| + sum_k |W_jk a_k|) lies within the rounding error of
 * an FP32 evaluation of the same row, so an FP32 forward may take its ReLU
 * decision either way and both gradients are correct.  If slack is non-NULL
 * (params layout, and dmean_slack [N,2]) it receives, summed over every such
 * decision of every row, the absolute change of each gradient element when
 * that one decision is taken the other way (band = 0: no ambiguous
 * decision, zero slack). */
int or_mlp_grad_slack(int N, const double *mean, int H, int W, int Q, const double *tx,
                      int L_mean, int L_tx, const double *room_min, const double *room_size,
                      int n_layers, const int *dims, const double *params, const double *dresid,
                      int stop_grad_mean, double band, double *d_params, double *d_mean,
                      double *slack, double *dmean_slack)
{
    if (n_layers < 1 || n_layers > OR_MAX_LAYERS) return OR_EINVAL;
    size_t P = param_count(n_layers, dims);
    int nthreads = 1;
#ifdef _OPENMP
    nthreads = omp_get_max_threads();
#endif
    double *part = calloc((size_t)nthreads * P, sizeof(double));
    double *dmp = calloc((size_t)nthreads * 2 * N, sizeof(double));
    double *spart = slack ? calloc((size_t)nthreads * P, sizeof(double)) : NULL;
    double *smp = slack ? calloc((size_t)nthreads * 2 * N, sizeof(double)) : NULL;
    if (!part || !dmp || (slack && (!spart || !smp))) {
        free(part); free(dmp); free(spart); free(smp);
        return OR_EINVAL;
    }
#pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *gp = part + (size_t)tid * P;
        double *gm = dmp + (size_t)tid * 2 * N;
        double *pre = malloc(sizeof(double) * OR_MAX_LAYERS * OR_MAX_WIDTH);
        double *rowA = slack ? malloc(sizeof(double) * P) : NULL;
        double *rowB = slack ? malloc(sizeof(double) * P) : NULL;
        double in[OR_MAX_WIDTH], outv[OR_MAX_WIDTH], a[OR_MAX_WIDTH];
        size_t off[OR_MAX_LAYERS + 1];
        off[0] = 0;
        for (int l = 0; l < n_layers; ++l)
            off[l + 1] = off[l] + (size_t)dims[l + 1] * dims[l] + dims[l + 1];
#pragma omp for schedule(static)
        for (long long r = 0; r < (long long)N * Q; ++r) {
            int q = (int)(r / N), n = (int)(r % N);
            double mu[2] = {mean[2 * n] / W, mean[2 * n + 1] / H};
            mlp_input(mean + 2 * (size_t)n, H, W, tx + 3 * (size_t)q, L_mean, L_tx, room_min,
                      room_size, in);
            or_mlp_row(in, n_layers, dims, params, outv, pre);
            const double *dres = dresid + (size_t)r * dims[n_layers];
            /* ambiguous ReLU decisions of this row */
            int nflip = 0;
            if (slack && band > 0.0) {
                memcpy(a, in, sizeof(double) * dims[0]);
                for (int l = 0; l + 1 < n_layers; ++l) {
                    int din = dims[l], dout = dims[l + 1];
                    const double *Wl = params + off[l], *bl = Wl + (size_t)dout * din;
                    for (int j = 0; j < dout; ++j) {
                        double mag = fabs(bl[j]);
                        for (int k = 0; k < din; ++k) mag += fabs(Wl[(size_t)j * din + k] * a[k]);
                        if (fabs(pre[(size_t)l * OR_MAX_WIDTH + j]) <= band * mag) ++nflip;
                    }
                    for (int j = 0; j < dout; ++j) {
                        double z = pre[(size_t)l * OR_MAX_WIDTH + j];
                        a[j] = z > 0.0 ? z : 0.0;
                    }
                }
            }
            if (nflip == 0) {
                row_backward(in, pre, n_layers, dims, params, off, dres, -1, -1, stop_grad_mean,
                             mu, H, W, L_mean, gp, gm + 2 * n);
                continue;
            }
            double gmA[2] = {0.0, 0.0}, gmB[2];
            memset(rowA, 0, sizeof(double) * P);
            row_backward(in, pre, n_layers, dims, params, off, dres, -1, -1, stop_grad_mean, mu,
                         H, W, L_mean, rowA, gmA);
            double *sp = spart + (size_t)tid * P, *sm = smp + (size_t)tid * 2 * N;
            memcpy(a, in, sizeof(double) * dims[0]);
            for (int l = 0; l + 1 < n_layers; ++l) {
                int din = dims[l], dout = dims[l + 1];
                const double *Wl = params + off[l], *bl = Wl + (size_t)dout * din;
                for (int j = 0; j < dout; ++j) {
                    double mag = fabs(bl[j]);
                    for (int k = 0; k < din; ++k) mag += fabs(Wl[(size_t)j * din + k] * a[k]);
                    if (!(fabs(pre[(size_t)l * OR_MAX_WIDTH + j]) <= band * mag)) continue;
                    memset(rowB, 0, sizeof(double) * P);
                    gmB[0] = gmB[1] = 0.0;
                    row_backward(in, pre, n_layers, dims, params, off, dres, l, j,
                                 stop_grad_mean, mu, H, W, L_mean, rowB, gmB);
                    for (size_t i = 0; i < P; ++i) sp[i] += fabs(rowB[i] - rowA[i]);
                    sm[2 * n] += fabs(gmB[0] - gmA[0]);
                    sm[2 * n + 1] += fabs(gmB[1] - gmA[1]);
                }
                for (int j = 0; j < dout; ++j) {
                    double z = pre[(size_t)l * OR_MAX_WIDTH + j];
                    a[j] = z > 0.0 ? z : 0.0;
                }
            }
            for (size_t i = 0; i < P; ++i) gp[i] += rowA[i];
            gm[2 * n] += gmA[0];
            gm[2 * n + 1] += gmA[1];
        }
        free(pre);
        free(rowA);
        free(rowB);
    }
    memset(d_params, 0, sizeof(double) * P);
    for (int t = 0; t < nthreads; ++t)
        for (size_t i = 0; i < P; ++i) d_params[i] += part[(size_t)t * P + i];
    for (int t = 0; t < nthreads; ++t)
        for (int i = 0; i < 2 * N; ++i) d_mean[i] += dmp[(size_t)t * 2 * N + i];
    if (slack) {
        memset(slack, 0, sizeof(double) * P);
        for (int t = 0; t < nthreads; ++t)
            for (size_t i = 0; i < P; ++i) slack[i] += spart[(size_t)t * P + i];
        if (dmean_slack)
            for (int t = 0; t < nthreads; ++t)
                for (int i = 0; i < 2 * N; ++i) dmean_slack[i] += smp[(size_t)t * 2 * N + i];
    }
    free(part);
    free(dmp);
    free(spart);
    free(smp);
    return OR_OK;
}

int or_mlp_grad(int N, const double *mean, int H, int W, int Q, const double *tx, int L_mean,
                int L_tx, const double *room_min, const double *room_size, int n_layers,
                const int *dims, const double *params, const double *dresid, int stop_grad_mean,
                double *d_params, double *d_mean)
{
    return or_mlp_grad_slack(N, mean, H, W, Q, tx, L_mean, L_tx, room_min, room_size, n_layers,
                             dims, params, dresid, stop_grad_mean, 0.0, d_params, d_mean, NULL,
                             NULL);
}

/* Number of OpenMP threads the oracle runs with (reported by benchmarks). */
int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
