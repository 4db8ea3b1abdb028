/*
 * FP64 CPU oracle for Dense Inverse Search (DIS) optical flow
 * (Kroeger, Timofte, Dai, Van Gool, "Fast Optical Flow using Dense Inverse Search").
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this file.  It shares no code, header, table or
 * helper with the CUDA path: everything below is written out from the paper in plain
 * loops, double precision, single thread, with no blocking, fusion or reordering beyond
 * what each formula states.
 *
 * Layouts: images are dense row-major H x W doubles; colour images are C such planes
 * back to back.  Flow fields are H x W x 2 interleaved (u along x / columns, v along y / rows).
 * A flow U maps pixel x of frame t to x + U(x) in frame t+1, i.e. I_{t+1}(x + U(x)) ~ I_t(x)
 * (Sec. 2.1, Eq. 1).
 *
 * Readings of passages that are silent or ambiguous are marked [Rn] and listed together
 * with the rest of the design notes of the repository.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Robust penalizer Psi(a^2) = sqrt(a^2 + eps^2) with eps = 0.001 (Sec. 2.3). */
#define OR_EPS 0.001
/* Normalisation beta = (|grad_2 .|^2 + 0.01)^-1 (Sec. 2.3, after Zimmer et al.). */
#define OR_BETA_REG 0.01
/* [R7] A patch whose template Hessian has det <= 1e-6 (tr/2)^2 is treated as flat. */
#define OR_DEGENERATE_REL 1e-6

typedef struct or_params {
    int patch_size;        /* theta_ps */
    double overlap;        /* theta_ov in [0,1) */
    int stride_override;   /* > 0: use this patch stride instead of the one derived from theta_ov */
    int grad_iters;        /* theta_it */
    int coarsest_scale;    /* theta_ss, < 0: automatic (Sec. 3.1) */
    int finest_scale;      /* theta_sf */
    int refine;            /* variational refinement on/off (Sec. 2.3) */
    int var_outer;         /* theta_vo, < 0: s + 1 (Sec. 3.1) */
    int var_inner;         /* theta_vi */
    double delta, gamma, alpha; /* data / gradient / smoothness weights (Sec. 3.1: 5, 10, 10) */
    double sor_omega;      /* [R14] over-relaxation factor */
    double intensity_scale;/* [R1] inputs in [0,1] are multiplied by this (255) */
    int channels;          /* 1 or 3 */
    int dof;               /* 2: optical flow; 1: horizontal displacement only (supp. depth from stereo) [R20] */
    int norm;              /* search error norm (supp. robust error norms): 0 L2, 1 L1, 2 Huber [R21] */
    double huber_b;        /* Huber threshold b on the intensity scale [R21] */
    int fb;                /* 1: forward-backward consistency (supp. Sec. B (ii)) [R22] */
    double term_eps;       /* > 0: a patch stops once its update step is at most this long (supp. Sec. C) [R23] */
    int polish;            /* > 0 with frozen increments: each patch restarts at u_init + frozen and runs the
                            * update to convergence (at most this many steps): the converged search whose
                            * implicit-function gradient the differentiable form offers [R24] */
} or_params;

enum { OR_NORM_L2 = 0, OR_NORM_L1 = 1, OR_NORM_HUBER = 2 };

/* [R21] Robust error norms (supplementary, robust error norms): before the update, the error of
 * every pixel is transformed so that squaring it gives the L1 or the Huber penalty:
 *   L1:    e <- sign(e) sqrt(|e|)
 *   Huber: e <- e if |e| < b, else sign(e) sqrt(2 b |e| - b^2)
 * (the printed condition "e < b" is read as |e| < b; b is a parameter). */
double or_robust_error(double e, int norm, double b)
{
    if (norm == OR_NORM_L1) return (e < 0 ? -1.0 : 1.0) * sqrt(fabs(e));
    if (norm == OR_NORM_HUBER) {
        if (fabs(e) < b) return e;
        return (e < 0 ? -1.0 : 1.0) * sqrt(2.0 * b * fabs(e) - b * b);
    }
    return e;
}

enum { OR_OK = 0, OR_ERR_INVALID = 1, OR_ERR_TOO_SMALL = 4 };
enum { OR_PATCH_OK = 0, OR_PATCH_RESET = 1, OR_PATCH_FLAT = 2 };

/* ---- decision trace --------------------------------------------------------------
 * Optional FNV-1a hash over every discrete decision taken (bilinear cell, clamping,
 * max(1,|d|) branch, reset).  Two evaluations with equal hashes took the same
 * branches everywhere, so a finite difference between them is free of kinks. */
static _Thread_local uint64_t* t_hash = NULL;
static void note(int64_t v)
{
    if (t_hash) {
        *t_hash ^= (uint64_t)v;
        *t_hash *= 1099511628211ULL;
    }
}

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* ---- bilinear interpolation -------------------------------------------------------
 * Sub-pixel extraction used by the search (Sec. 2.1), the densification weights (Eq. 3)
 * and the refinement warp.  [R9] Coordinates are clamped to the image before
 * interpolating (pixel centres at integer coordinates). */
double or_bilinear(const double* I, int w, int h, double x, double y)
{
    int cx = 0, cy = 0;
    if (x < 0.0) { x = 0.0; cx = 1; }
    if (x > (double)(w - 1)) { x = (double)(w - 1); cx = 2; }
    if (y < 0.0) { y = 0.0; cy = 1; }
    if (y > (double)(h - 1)) { y = (double)(h - 1); cy = 2; }
    int x0 = (int)floor(x), y0 = (int)floor(y);
    int x1 = x0 + 1 < w ? x0 + 1 : w - 1;
    int y1 = y0 + 1 < h ? y0 + 1 : h - 1;
    double fx = x - x0, fy = y - y0;
    note(((int64_t)x0 << 2) | cx);
    note(((int64_t)y0 << 2) | cy);
    double top = (1.0 - fx) * I[(size_t)y0 * w + x0] + fx * I[(size_t)y0 * w + x1];
    double bot = (1.0 - fx) * I[(size_t)y1 * w + x0] + fx * I[(size_t)y1 * w + x1];
    return (1.0 - fy) * top + fy * bot;
}

/* or_bilinear and its derivatives d/dx, d/dy at (x, y): the slopes of the interpolant inside
 * its cell, 0 along a coordinate that is clamped (outside the image the value is constant). */
static double bilinear_grad(const double* I, int w, int h, double x, double y, double* dx, double* dy)
{
    int cx = 0, cy = 0;
    if (x < 0.0) { x = 0.0; cx = 1; }
    if (x > (double)(w - 1)) { x = (double)(w - 1); cx = 1; }
    if (y < 0.0) { y = 0.0; cy = 1; }
    if (y > (double)(h - 1)) { y = (double)(h - 1); cy = 1; }
    int x0 = (int)floor(x), y0 = (int)floor(y);
    int x1 = x0 + 1 < w ? x0 + 1 : w - 1;
    int y1 = y0 + 1 < h ? y0 + 1 : h - 1;
    double fx = x - x0, fy = y - y0;
    double a = I[(size_t)y0 * w + x0], b = I[(size_t)y0 * w + x1];
    double c = I[(size_t)y1 * w + x0], d = I[(size_t)y1 * w + x1];
    *dx = cx ? 0.0 : (1.0 - fy) * (b - a) + fy * (d - c);
    *dy = cy ? 0.0 : (1.0 - fx) * (c - a) + fx * (d - b);
    double top = (1.0 - fx) * a + fx * b, bot = (1.0 - fx) * c + fx * d;
    return (1.0 - fy) * top + fy * bot;
}

/* Bilinear interpolation of an interleaved 2-vector field (same rule as or_bilinear). */
static void bilinear_flow(const double* U, int w, int h, double x, double y, double out[2])
{
    int cx = 0, cy = 0;
    if (x < 0.0) { x = 0.0; cx = 1; }
    if (x > (double)(w - 1)) { x = (double)(w - 1); cx = 2; }
    if (y < 0.0) { y = 0.0; cy = 1; }
    if (y > (double)(h - 1)) { y = (double)(h - 1); cy = 2; }
    int x0 = (int)floor(x), y0 = (int)floor(y);
    int x1 = x0 + 1 < w ? x0 + 1 : w - 1;
    int y1 = y0 + 1 < h ? y0 + 1 : h - 1;
    double fx = x - x0, fy = y - y0;
    note(((int64_t)x0 << 2) | cx);
    note(((int64_t)y0 << 2) | cy);
    for (int k = 0; k < 2; k++) {
        double a = U[((size_t)y0 * w + x0) * 2 + k], b = U[((size_t)y0 * w + x1) * 2 + k];
        double c = U[((size_t)y1 * w + x0) * 2 + k], d = U[((size_t)y1 * w + x1) * 2 + k];
        out[k] = (1.0 - fy) * ((1.0 - fx) * a + fx * b) + fy * ((1.0 - fx) * c + fx * d);
    }
}

/* ---- pyramid (Sec. 3.1: downscaling quotient theta_sd = 2) ------------------------
 * [R2] Level s+1 is level s blurred with the separable binomial kernel [1 4 6 4 1]/16
 * (replicated border) and kept at even samples, so W_{s+1} = ceil(W_s / 2) and pixel
 * x of level s+1 sits at 2x of level s.  Written as the full 5x5 weighted sum. */
void or_pyr_down(const double* in, int w, int h, double* out)
{
    static const double k[5] = {1.0 / 16, 4.0 / 16, 6.0 / 16, 4.0 / 16, 1.0 / 16};
    int wo = (w + 1) / 2, ho = (h + 1) / 2;
    for (int y = 0; y < ho; y++)
        for (int x = 0; x < wo; x++) {
            double acc = 0.0;
            for (int j = -2; j <= 2; j++)
                for (int i = -2; i <= 2; i++)
                    acc += k[j + 2] * k[i + 2] *
                           in[(size_t)clampi(2 * y + j, 0, h - 1) * w + clampi(2 * x + i, 0, w - 1)];
            out[(size_t)y * wo + x] = acc;
        }
}

/* ---- image gradients (Sec. 3.1 "image pyramid including image gradients") --------
 * [R3] 3x3 Sobel with replicated border, divided by 8 so that a unit ramp has
 * derivative 1.  gx = d/dx (along columns), gy = d/dy (along rows). */
void or_sobel(const double* I, int w, int h, double* gx, double* gy)
{
    static const double sx[3][3] = {{-1, 0, 1}, {-2, 0, 2}, {-1, 0, 1}};
    static const double sy[3][3] = {{-1, -2, -1}, {0, 0, 0}, {1, 2, 1}};
    for (int y = 0; y < h; y++)
        for (int x = 0; x < w; x++) {
            double ax = 0.0, ay = 0.0;
            for (int j = -1; j <= 1; j++)
                for (int i = -1; i <= 1; i++) {
                    double v = I[(size_t)clampi(y + j, 0, h - 1) * w + clampi(x + i, 0, w - 1)];
                    ax += sx[j + 1][i + 1] * v;
                    ay += sy[j + 1][i + 1] * v;
                }
            gx[(size_t)y * w + x] = ax / 8.0;
            gy[(size_t)y * w + x] = ay / 8.0;
        }
}

/* ---- patch grid (Alg. 1 step 1) ----------------------------------------------------
 * [R5] The overlap theta_ov * theta_ps is floored to whole pixels, stride =
 * theta_ps - floor(theta_ov * theta_ps) (an explicit stride overrides).  Patch corners
 * along an axis of length L are min(i * stride, L - theta_ps), i = 0..ceil((L-ps)/stride),
 * which covers every pixel with no patch leaving the image. */
int or_stride(int ps, double overlap, int stride_override)
{
    if (stride_override > 0) return stride_override;
    int s = ps - (int)floor(overlap * ps);
    return s < 1 ? 1 : s;
}

int or_grid_n(int len, int ps, int stride)
{
    if (len < ps) return 0;
    return (len - ps + stride - 1) / stride + 1;
}

int or_grid_pos(int i, int len, int ps, int stride)
{
    int p = i * stride;
    return p < len - ps ? p : len - ps;
}

/* ---- levels (Sec. 3.1) -------------------------------------------------------------
 * [R4] theta_ss = ceil(log2(2 W / (f theta_ps))) with f = 8, lowered until the coarsest
 * level still holds one patch, and raised to theta_sf when it falls below it (Alg. 1 runs
 * s from theta_ss down to theta_sf, so a coarsest scale below the finest would process no
 * level).  Returns OR_OK and writes (ss, sf), or OR_ERR_TOO_SMALL. */
static int level_dim(int d, int s)
{
    for (int i = 0; i < s; i++) d = (d + 1) / 2;
    return d;
}

int or_levels(int W, int H, const or_params* p, int* ss_out, int* sf_out)
{
    int ps = p->patch_size, sf = p->finest_scale, ss = p->coarsest_scale;
    if (ps < 2 || sf < 0 || W < 1 || H < 1) return OR_ERR_INVALID;
    if (ss < 0) {
        double v = 2.0 * (double)W / (8.0 * (double)ps);
        ss = v <= 1.0 ? 0 : (int)ceil(log2(v));
        while (ss > sf && (level_dim(W, ss) < ps || level_dim(H, ss) < ps)) ss--;
        if (ss < sf) ss = sf;
    }
    if (ss < sf) return OR_ERR_TOO_SMALL;
    if (level_dim(W, ss) < ps || level_dim(H, ss) < ps) return OR_ERR_TOO_SMALL;
    *ss_out = ss;
    *sf_out = sf;
    return OR_OK;
}

/* ---- initial displacement (Alg. 1 step 2) ------------------------------------------
 * u_init = U_{s+1}(x / theta_sd) * theta_sd at the patch location x, with cscale =
 * theta_sd = 2.  [R6] x is the patch centre and U_{s+1} is interpolated bilinearly.
 * For an initial flow given at the same level cscale = 1.  No field: zero flow. */
static void init_at(const double* Uc, int wc, int hc, double cscale, double x, double y, double out[2])
{
    if (!Uc) {
        out[0] = out[1] = 0.0;
        return;
    }
    double v[2];
    bilinear_flow(Uc, wc, hc, x / cscale, y / cscale, v);
    out[0] = cscale * v[0];
    out[1] = cscale * v[1];
}

/* ---- inverse search of one level (Sec. 2.1, supplementary Sec. A) ------------------
 * For every patch i (row-major over the grid):
 *   T = I0 patch minus its mean (mean-normalisation, Sec. 2.1),
 *   S' = grad T (warp Jacobian = identity), H' = sum S'^T S'  (precomputed, Eq. solvereqinv),
 *   repeat theta_it times [R8: fixed count]:
 *     w(x) = I1(x + u) bilinear, w <- w - mean(w)                        [R10]
 *     du = H'^-1 sum S'^T (w - T)                                          (Eq. solvereqinv)
 *     u <- u - du                                  (inverse compositional update)
 *   outlier reset: |u - u_init|_2 > theta_ps  =>  u = u_init               (Alg. 1 step 4)
 * [R19] S' is the raw image gradient of I0 at the patch pixels (mean removal does not
 * change a gradient).  [R7] flat patches keep u_init.
 * frozen != NULL replaces the search by u = u_init + frozen[i] (no reset test): the
 * differentiable map's stop-gradient search, with increments recorded by a previous run.
 * uinit_out and status_out may be NULL.
 * [R20] dof = 1 (supplementary, depth from stereo: the vertical degree of freedom removed):
 * v stays at its initial value and u takes the scalar step du = sum S'_x e / sum S'_x^2; the
 * patch is flat when sum S'_x^2 <= 1e-6 tr(H') / 2.
 * [R21] norm / huber_b: the per-pixel error e = (w - mean w) - T is transformed by
 * or_robust_error before it enters sum S'^T e.
 * [R23] term_eps > 0 (supplementary Sec. C: iterations end early "for small residuals"): a patch
 * stops after the first update whose step |(du, dv)|_2 is at most term_eps (0: the fixed count
 * of R8).
 * [R24] polish > 0 with frozen increments: every patch with a nonzero increment restarts at
 * u_init + frozen and solves the search's stationarity condition
 *   g(u) = sum_q S'_q (w~_q(u) - T_q) = 0,   w~ = w - mean w,  w_q(u) = I1(x_q + u) bilinear
 * (the fixed point of the update: du = H'^-1 g) by Newton steps u <- u - J^-1 g with
 * J = dg/du = sum_q S'_q (grad w_q - mean grad w)^T (the bilinear interpolant's derivative,
 * 0 across a clamped coordinate), until a step is below 1e-13 px (at most `polish` steps;
 * whether it got there joins the decision trace; a patch that does not get there has no
 * solution and returns to u_init); then the reset test.  This is the converged
 * search, whose solution depends on the frames and not on where it started; the
 * differentiable form's implicit-function gradient is the derivative of this map. */
void or_search_level(const double* I0, const double* Ix, const double* Iy, const double* I1, int w, int h,
                     const double* Uc, int wc, int hc, double cscale, int ps, int stride, int iters,
                     const double* frozen, double* u_out, double* uinit_out, int* status_out, int dof, int norm,
                     double huber_b, double term_eps, int polish)
{
    int nx = or_grid_n(w, ps, stride), ny = or_grid_n(h, ps, stride), n = ps * ps;
    double* T = (double*)malloc(sizeof(double) * n);
    double* gx = (double*)malloc(sizeof(double) * n);
    double* gy = (double*)malloc(sizeof(double) * n);
    double* wv = (double*)malloc(sizeof(double) * n);
    double* T2x = (double*)malloc(sizeof(double) * n); /* polish: derivatives of w along x, y */
    double* T2y = (double*)malloc(sizeof(double) * n);
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            int k = j * nx + i;
            int px = or_grid_pos(i, w, ps, stride), py = or_grid_pos(j, h, ps, stride);
            double cx = px + 0.5 * (ps - 1), cy = py + 0.5 * (ps - 1);
            double ui[2];
            init_at(Uc, wc, hc, cscale, cx, cy, ui);
            if (uinit_out) {
                uinit_out[2 * k] = ui[0];
                uinit_out[2 * k + 1] = ui[1];
            }
            /* [R24] a zero frozen increment stands for a patch that was reset, flat or never moved:
             * it stays at u_init, polished or not */
            const int polishing = frozen && polish > 0 && (frozen[2 * k] != 0.0 || frozen[2 * k + 1] != 0.0);
            if (frozen && !polishing) {
                u_out[2 * k] = ui[0] + frozen[2 * k];
                u_out[2 * k + 1] = ui[1] + frozen[2 * k + 1];
                if (status_out) status_out[k] = OR_PATCH_OK;
                continue;
            }
            double mean0 = 0.0;
            for (int b = 0; b < ps; b++)
                for (int a = 0; a < ps; a++) mean0 += I0[(size_t)(py + b) * w + px + a];
            mean0 /= n;
            double h00 = 0.0, h01 = 0.0, h11 = 0.0;
            for (int b = 0; b < ps; b++)
                for (int a = 0; a < ps; a++) {
                    size_t o = (size_t)(py + b) * w + px + a;
                    int q = b * ps + a;
                    T[q] = I0[o] - mean0;
                    gx[q] = Ix[o];
                    gy[q] = Iy[o];
                    h00 += gx[q] * gx[q];
                    h01 += gx[q] * gy[q];
                    h11 += gy[q] * gy[q];
                }
            double u = ui[0], v = ui[1];
            if (polishing) {
                u += frozen[2 * k];
                v += frozen[2 * k + 1];
            }
            const int n_it = polishing ? polish : iters;
            double det = h00 * h11 - h01 * h01, tr = h00 + h11;
            int st = OR_PATCH_OK;
            const int flat = dof == 1 ? h00 <= OR_DEGENERATE_REL * 0.5 * tr
                                      : det <= OR_DEGENERATE_REL * (0.5 * tr) * (0.5 * tr);
            if (flat) {
                st = OR_PATCH_FLAT;
            } else {
                int converged = 0;
                for (int it = 0; polishing && it < n_it; it++) {
                    /* Newton step on g(u) = 0 */
                    double mw = 0.0, mgx = 0.0, mgy = 0.0;
                    for (int b = 0; b < ps; b++)
                        for (int a = 0; a < ps; a++) {
                            double X = px + a + u, Y = py + b + v, dx, dy;
                            double s = bilinear_grad(I1, w, h, X, Y, &dx, &dy);
                            int q = b * ps + a;
                            wv[q] = s;
                            T2x[q] = dx;
                            T2y[q] = dy;
                            mw += s;
                            mgx += dx;
                            mgy += dy;
                        }
                    mw /= n;
                    mgx /= n;
                    mgy /= n;
                    double g0 = 0.0, g1 = 0.0, j00 = 0.0, j01 = 0.0, j10 = 0.0, j11 = 0.0;
                    for (int q = 0; q < n; q++) {
                        double r = (wv[q] - mw) - T[q];
                        g0 += gx[q] * r;
                        g1 += gy[q] * r;
                        j00 += gx[q] * (T2x[q] - mgx);
                        j01 += gx[q] * (T2y[q] - mgy);
                        j10 += gy[q] * (T2x[q] - mgx);
                        j11 += gy[q] * (T2y[q] - mgy);
                    }
                    double du, dv = 0.0;
                    if (dof == 1) { /* [R20] v stays: the scalar root of g_x in u */
                        if (!(fabs(j00) > 0.0)) break;
                        du = g0 / j00;
                    } else {
                        double dj = j00 * j11 - j01 * j10;
                        if (!(fabs(dj) > 0.0)) break;
                        du = (j11 * g0 - j01 * g1) / dj;
                        dv = (j00 * g1 - j10 * g0) / dj;
                    }
                    u -= du;
                    v -= dv;
                    if (du * du + dv * dv <= 1e-26) {
                        converged = 1;
                        break;
                    }
                }
                for (int it = 0; !polishing && it < n_it; it++) {
                    double mw = 0.0;
                    for (int b = 0; b < ps; b++)
                        for (int a = 0; a < ps; a++) {
                            double s = or_bilinear(I1, w, h, px + a + u, py + b + v);
                            wv[b * ps + a] = s;
                            mw += s;
                        }
                    mw /= n;
                    double b0 = 0.0, b1 = 0.0;
                    for (int q = 0; q < n; q++) {
                        double r = or_robust_error((wv[q] - mw) - T[q], norm, huber_b);
                        b0 += gx[q] * r;
                        b1 += gy[q] * r;
                    }
                    double du, dv = 0.0;
                    if (dof == 1) {
                        du = b0 / h00;
                    } else {
                        du = (h11 * b0 - h01 * b1) / det;
                        dv = (h00 * b1 - h01 * b0) / det;
                    }
                    u -= du;
                    v -= dv;
                    if (term_eps > 0.0 && du * du + dv * dv <= term_eps * term_eps) break;
                }
                if (polishing) {
                    /* the solution's bilinear cell joins the trace: g is only piecewise smooth in
                     * u, so a root that crosses a cell boundary under a perturbation is a kink */
                    note(converged);
                    note((int64_t)floor(u));
                    note((int64_t)floor(v));
                    if (!converged) { /* no root found (Newton cycles or stalls): no solution */
                        u = ui[0];
                        v = ui[1];
                    }
                }
                double ex = u - ui[0], ey = v - ui[1];
                if (sqrt(ex * ex + ey * ey) > (double)ps) {
                    st = OR_PATCH_RESET;
                    u = ui[0];
                    v = ui[1];
                }
            }
            note(st);
            u_out[2 * k] = u;
            u_out[2 * k + 1] = v;
            if (status_out) status_out[k] = st;
        }
    free(T);
    free(gx);
    free(gy);
    free(T2x);
    free(T2y);
    free(wv);
}

/* ---- densification (Alg. 1 step 4, Eq. 3) ------------------------------------------
 * U(x) = (1/Z) sum_i lambda_{i,x} / max(1, |d_i(x)|) u_i,  d_i(x) = I1(x + u_i) - I0(x),
 * over the patches i that contain x, summed in row-major patch order.
 * [R11] d uses raw (not mean-normalised) intensities on the 0..255 scale.
 * A pixel no patch covers takes the initial flow (cannot happen on a valid grid). */
void or_densify_level(const double* I0, const double* I1, int w, int h, const double* u, int ps, int stride,
                      const double* Uc, int wc, int hc, double cscale, double* U)
{
    int nx = or_grid_n(w, ps, stride), ny = or_grid_n(h, ps, stride);
    for (int y = 0; y < h; y++)
        for (int x = 0; x < w; x++) {
            double nu = 0.0, nv = 0.0, Z = 0.0;
            for (int j = 0; j < ny; j++) {
                int py = or_grid_pos(j, h, ps, stride);
                if (y < py || y >= py + ps) continue;
                for (int i = 0; i < nx; i++) {
                    int px = or_grid_pos(i, w, ps, stride);
                    if (x < px || x >= px + ps) continue;
                    const double* ui = u + 2 * (j * nx + i);
                    double d = or_bilinear(I1, w, h, x + ui[0], y + ui[1]) - I0[(size_t)y * w + x];
                    double ad = fabs(d);
                    note(ad > 1.0);
                    double wt = 1.0 / (ad > 1.0 ? ad : 1.0);
                    nu += wt * ui[0];
                    nv += wt * ui[1];
                    Z += wt;
                }
            }
            double* o = U + 2 * ((size_t)y * w + x);
            if (Z > 0.0) {
                o[0] = nu / Z;
                o[1] = nv / Z;
            } else {
                init_at(Uc, wc, hc, cscale, x, y, o);
            }
        }
}

/* ---- densification with forward-backward consistency (supp. Sec. B (ii)) -----------
 * Both directions are searched; each direction's dense field merges its own patches with the
 * other direction's:
 *   U(x) = (1/Z) [ sum_i lambda_i,x / max(1, |d_i(x)|) u_i  -  sum_j mu_j,x / max(1, |e_j(x)|) u'_j ],
 *   Z = sum_i lambda_i,x / max(1, |d_i(x)|) + sum_j mu_j,x / max(1, |e_j(x)|),
 * the first sum as in Eq. 3 over the patches i of this direction (grid on I0, displacement u_i),
 * the second over the patches j of the other direction (grid on I1, displacement u'_j into I0).
 * [R22] mu_j,x is the bilinear footprint of patch j moved by u'_j ("bilinear interpolation for
 * the second term"): every template pixel q of the patch lands at q + u'_j in I0 and spreads
 * over its four neighbours with bilinear weights,
 *   mu_j,x = sum_q max(0, 1 - |x - q_x - u'_x|) max(0, 1 - |y - q_y - u'_y|)
 *          = (sum_qx max(0, 1 - |x - q_x - u'_x|)) (sum_qy max(0, 1 - |y - q_y - u'_y|)),
 * 1 inside the moved box, fading to 0 over one pixel beyond it (an integer move covers exactly
 * ps x ps pixels with weight 1; the weights of one patch always sum to ps^2).
 * e_j(x) = I0(x) - I1(x - u'_j), I1 being the template's frame, sampled bilinearly (clamped).
 * Contributions are summed patch by patch in row-major order of each grid, this direction's
 * first.  The other direction's field is this function with the roles of (I0, u) and (I1, u')
 * exchanged. */
void or_densify_level_fb(const double* I0, const double* I1, int w, int h, const double* u, const double* ub,
                         int ps, int stride, const double* Uc, int wc, int hc, double cscale, double* U)
{
    int nx = or_grid_n(w, ps, stride), ny = or_grid_n(h, ps, stride);
    size_t n = (size_t)w * h;
    double* acc = (double*)calloc(3 * n, sizeof(double)); /* per pixel: nu, nv, Z */
    /* this direction's patches containing x, in row-major patch order */
    for (int y = 0; y < h; y++)
        for (int x = 0; x < w; x++) {
            double* a = acc + 3 * ((size_t)y * w + x);
            for (int j = 0; j < ny; j++) {
                int py = or_grid_pos(j, h, ps, stride);
                if (y < py || y >= py + ps) continue;
                for (int i = 0; i < nx; i++) {
                    int px = or_grid_pos(i, w, ps, stride);
                    if (x < px || x >= px + ps) continue;
                    const double* ui = u + 2 * (j * nx + i);
                    double d = or_bilinear(I1, w, h, x + ui[0], y + ui[1]) - I0[(size_t)y * w + x];
                    double ad = fabs(d);
                    double wt = 1.0 / (ad > 1.0 ? ad : 1.0);
                    a[0] += wt * ui[0];
                    a[1] += wt * ui[1];
                    a[2] += wt;
                }
            }
        }
    /* then the other direction's patches, in row-major patch order: each visits the pixels its
     * footprint can reach (so every pixel still receives these contributions in patch order) */
    for (int j = 0; j < ny; j++) {
        int py = or_grid_pos(j, h, ps, stride);
        for (int i = 0; i < nx; i++) {
            int px = or_grid_pos(i, w, ps, stride);
            const double* uj = ub + 2 * (j * nx + i);
            if (!(fabs(uj[0]) < 1e6 && fabs(uj[1]) < 1e6)) continue; /* no frame reaches that far */
            int cx = px + (int)floor(uj[0]), cy = py + (int)floor(uj[1]);
            for (int y = cy - 1; y <= cy + ps + 1; y++) {
                if (y < 0 || y >= h) continue;
                double ly = 0.0;
                for (int qy = py; qy < py + ps; qy++) {
                    double t = 1.0 - fabs(y - qy - uj[1]);
                    if (t > 0.0) ly += t;
                }
                if (ly <= 0.0) continue;
                for (int x = cx - 1; x <= cx + ps + 1; x++) {
                    if (x < 0 || x >= w) continue;
                    double lx = 0.0;
                    for (int qx = px; qx < px + ps; qx++) {
                        double t = 1.0 - fabs(x - qx - uj[0]);
                        if (t > 0.0) lx += t;
                    }
                    if (lx <= 0.0) continue;
                    double e = I0[(size_t)y * w + x] - or_bilinear(I1, w, h, x - uj[0], y - uj[1]);
                    double ae = fabs(e);
                    double wt = lx * ly / (ae > 1.0 ? ae : 1.0);
                    double* a = acc + 3 * ((size_t)y * w + x);
                    a[0] -= wt * uj[0];
                    a[1] -= wt * uj[1];
                    a[2] += wt;
                }
            }
        }
    }
    for (int y = 0; y < h; y++)
        for (int x = 0; x < w; x++) {
            const double* a = acc + 3 * ((size_t)y * w + x);
            double* o = U + 2 * ((size_t)y * w + x);
            if (a[2] > 0.0) {
                o[0] = a[0] / a[2];
                o[1] = a[1] / a[2];
            } else {
                init_at(Uc, wc, hc, cscale, x, y, o);
            }
        }
    free(acc);
}

/* ---- variational refinement (Alg. 1 step 5, Sec. 2.3) ------------------------------
 * E(U) = int delta Psi(E_I) + gamma Psi(E_G) + alpha Psi(E_S),  Psi(a^2) = sqrt(a^2 + eps^2).
 * [R12] Discretisation: warp I1 once by U (bilinear, clamped); Ibar = (I0 + I1w)/2;
 * I_x, I_y = Sobel/8 of Ibar; I_z = I1w - I0; I_xx = Sobel_x(I_x), I_xy = Sobel_y(I_x),
 * I_yy = Sobel_y(I_y); I_xz = Sobel_x(I1w) - Sobel_x(I0), I_yz likewise.
 *   E_I = sum_c beta0 (I_x du + I_y dv + I_z)^2,        beta0 = 1/(I_x^2 + I_y^2 + 0.01)
 *   E_G = sum_c betax (I_xx du + I_xy dv + I_xz)^2 + betay (I_xy du + I_yy dv + I_yz)^2,
 *         betax = 1/(I_xx^2 + I_xy^2 + 0.01), betay = 1/(I_xy^2 + I_yy^2 + 0.01)
 *   E_S = |grad(u + du)|^2 + |grad(v + dv)|^2  (central differences, replicated border)
 * theta_vo lagged-nonlinearity iterations, each freezing psi = weight * Psi'(.) and running
 * theta_vi red-black SOR sweeps [R15] over the per-pixel 2x2 systems
 *   (A_p + sum_q w_pq I) d = b_p + sum_q w_pq (U_q + dU_q - U_p),  w_pq = (psiS_p + psiS_q)/2,
 * dU_p <- (1 - omega) dU_p + omega d, red ((x + y) even) pixels first.  Finally U += dU.
 * I0 and I1 hold C planes each. */
/* [R20] dof = 1: the increment dv stays 0; each SOR step solves the scalar equation
 * (A11 + sum w_pq) du = b1 + sum w_pq (U_q + dU_q - U_p). */
void or_refine_level(const double* I0, const double* I1, int w, int h, int C, double* U, int outer, int inner,
                     double delta, double gamma, double alpha, double omega, int dof)
{
    size_t n = (size_t)w * h;
    /* per channel: Ix Iy Iz Ixx Ixy Iyy Ixz Iyz b0 bx by */
    double* D = (double*)malloc(sizeof(double) * n * 11 * C);
    double* I1w = (double*)malloc(sizeof(double) * n);
    double* Ib = (double*)malloc(sizeof(double) * n);
    double* t0 = (double*)malloc(sizeof(double) * n);
    double* t1 = (double*)malloc(sizeof(double) * n);
    double* t2 = (double*)malloc(sizeof(double) * n);
    double* t3 = (double*)malloc(sizeof(double) * n);
    for (int c = 0; c < C; c++) {
        const double* P0 = I0 + n * c;
        const double* P1 = I1 + n * c;
        double* Dc = D + n * 11 * c;
        double *Ix = Dc, *Iy = Dc + n, *Iz = Dc + 2 * n, *Ixx = Dc + 3 * n, *Ixy = Dc + 4 * n, *Iyy = Dc + 5 * n;
        double *Ixz = Dc + 6 * n, *Iyz = Dc + 7 * n, *B0 = Dc + 8 * n, *Bx = Dc + 9 * n, *By = Dc + 10 * n;
        for (int y = 0; y < h; y++)
            for (int x = 0; x < w; x++) {
                size_t o = (size_t)y * w + x;
                I1w[o] = or_bilinear(P1, w, h, x + U[2 * o], y + U[2 * o + 1]);
                Ib[o] = 0.5 * (P0[o] + I1w[o]);
                Iz[o] = I1w[o] - P0[o];
            }
        or_sobel(Ib, w, h, Ix, Iy);
        or_sobel(Ix, w, h, Ixx, Ixy);
        or_sobel(Iy, w, h, t0, Iyy);
        or_sobel(I1w, w, h, t0, t1);
        or_sobel(P0, w, h, t2, t3);
        for (size_t o = 0; o < n; o++) {
            Ixz[o] = t0[o] - t2[o];
            Iyz[o] = t1[o] - t3[o];
            B0[o] = 1.0 / (Ix[o] * Ix[o] + Iy[o] * Iy[o] + OR_BETA_REG);
            Bx[o] = 1.0 / (Ixx[o] * Ixx[o] + Ixy[o] * Ixy[o] + OR_BETA_REG);
            By[o] = 1.0 / (Ixy[o] * Ixy[o] + Iyy[o] * Iyy[o] + OR_BETA_REG);
        }
    }
    double* dU = (double*)calloc(n * 2, sizeof(double));
    double* A = (double*)malloc(sizeof(double) * n * 6); /* A11 A12 A22 b1 b2 psiS */
    const double eps2 = OR_EPS * OR_EPS;
    for (int o_it = 0; o_it < outer; o_it++) {
        for (int y = 0; y < h; y++)
            for (int x = 0; x < w; x++) {
                size_t o = (size_t)y * w + x;
                double du = dU[2 * o], dv = dU[2 * o + 1];
                double EI = 0.0, EG = 0.0;
                for (int c = 0; c < C; c++) {
                    const double* Dc = D + n * 11 * c;
                    double Ix = Dc[o], Iy = Dc[n + o], Iz = Dc[2 * n + o], Ixx = Dc[3 * n + o];
                    double Ixy = Dc[4 * n + o], Iyy = Dc[5 * n + o], Ixz = Dc[6 * n + o], Iyz = Dc[7 * n + o];
                    double B0 = Dc[8 * n + o], Bx = Dc[9 * n + o], By = Dc[10 * n + o];
                    double eI = Ix * du + Iy * dv + Iz;
                    double eGx = Ixx * du + Ixy * dv + Ixz;
                    double eGy = Ixy * du + Iyy * dv + Iyz;
                    EI += B0 * eI * eI;
                    EG += Bx * eGx * eGx + By * eGy * eGy;
                }
                double psiI = delta / (2.0 * sqrt(EI + eps2));
                double psiG = gamma / (2.0 * sqrt(EG + eps2));
                double a11 = 0, a12 = 0, a22 = 0, b1 = 0, b2 = 0;
                for (int c = 0; c < C; c++) {
                    const double* Dc = D + n * 11 * c;
                    double Ix = Dc[o], Iy = Dc[n + o], Iz = Dc[2 * n + o], Ixx = Dc[3 * n + o];
                    double Ixy = Dc[4 * n + o], Iyy = Dc[5 * n + o], Ixz = Dc[6 * n + o], Iyz = Dc[7 * n + o];
                    double B0 = Dc[8 * n + o], Bx = Dc[9 * n + o], By = Dc[10 * n + o];
                    a11 += psiI * B0 * Ix * Ix + psiG * (Bx * Ixx * Ixx + By * Ixy * Ixy);
                    a12 += psiI * B0 * Ix * Iy + psiG * (Bx * Ixx * Ixy + By * Ixy * Iyy);
                    a22 += psiI * B0 * Iy * Iy + psiG * (Bx * Ixy * Ixy + By * Iyy * Iyy);
                    b1 -= psiI * B0 * Iz * Ix + psiG * (Bx * Ixz * Ixx + By * Iyz * Ixy);
                    b2 -= psiI * B0 * Iz * Iy + psiG * (Bx * Ixz * Ixy + By * Iyz * Iyy);
                }
                /* smoothness: central differences of u + du with replicated border */
                size_t xl = (size_t)y * w + clampi(x - 1, 0, w - 1), xr = (size_t)y * w + clampi(x + 1, 0, w - 1);
                size_t yu = (size_t)clampi(y - 1, 0, h - 1) * w + x, yd = (size_t)clampi(y + 1, 0, h - 1) * w + x;
                double ux = 0.5 * ((U[2 * xr] + dU[2 * xr]) - (U[2 * xl] + dU[2 * xl]));
                double vx = 0.5 * ((U[2 * xr + 1] + dU[2 * xr + 1]) - (U[2 * xl + 1] + dU[2 * xl + 1]));
                double uy = 0.5 * ((U[2 * yd] + dU[2 * yd]) - (U[2 * yu] + dU[2 * yu]));
                double vy = 0.5 * ((U[2 * yd + 1] + dU[2 * yd + 1]) - (U[2 * yu + 1] + dU[2 * yu + 1]));
                double ES = ux * ux + uy * uy + vx * vx + vy * vy;
                double* Ao = A + 6 * o;
                Ao[0] = a11;
                Ao[1] = a12;
                Ao[2] = a22;
                Ao[3] = b1;
                Ao[4] = b2;
                Ao[5] = alpha / (2.0 * sqrt(ES + eps2));
            }
        for (int it = 0; it < inner; it++)
            for (int color = 0; color < 2; color++)
                for (int y = 0; y < h; y++)
                    for (int x = 0; x < w; x++) {
                        if (((x + y) & 1) != color) continue;
                        size_t o = (size_t)y * w + x;
                        const double* Ao = A + 6 * o;
                        double sw = 0.0, r1 = Ao[3], r2 = Ao[4];
                        static const int nbx[4] = {-1, 1, 0, 0}, nby[4] = {0, 0, -1, 1};
                        for (int q = 0; q < 4; q++) {
                            int qx = x + nbx[q], qy = y + nby[q];
                            if (qx < 0 || qx >= w || qy < 0 || qy >= h) continue;
                            size_t oq = (size_t)qy * w + qx;
                            double wq = 0.5 * (Ao[5] + A[6 * oq + 5]);
                            sw += wq;
                            r1 += wq * (U[2 * oq] + dU[2 * oq] - U[2 * o]);
                            r2 += wq * (U[2 * oq + 1] + dU[2 * oq + 1] - U[2 * o + 1]);
                        }
                        double m11 = Ao[0] + sw, m12 = Ao[1], m22 = Ao[2] + sw;
                        double det = m11 * m22 - m12 * m12;
                        if (dof == 1) {
                            if (m11 > 0.0) dU[2 * o] = (1.0 - omega) * dU[2 * o] + omega * (r1 / m11);
                        } else if (det > 0.0) {
                            double d1 = (m22 * r1 - m12 * r2) / det;
                            double d2 = (m11 * r2 - m12 * r1) / det;
                            dU[2 * o] = (1.0 - omega) * dU[2 * o] + omega * d1;
                            dU[2 * o + 1] = (1.0 - omega) * dU[2 * o + 1] + omega * d2;
                        }
                    }
    }
    for (size_t o = 0; o < 2 * n; o++) U[o] += dU[o];
    free(D);
    free(I1w);
    free(Ib);
    free(t0);
    free(t1);
    free(t2);
    free(t3);
    free(dU);
    free(A);
}

/* ---- up-scaling (Sec. 3.1, last paragraph) -----------------------------------------
 * Uout(x) = factor * Uin(x / factor), bilinear with clamping. */
void or_upsample_flow(const double* Uin, int wi, int hi, double factor, double* Uout, int wo, int ho)
{
    for (int y = 0; y < ho; y++)
        for (int x = 0; x < wo; x++) {
            double v[2];
            bilinear_flow(Uin, wi, hi, x / factor, y / factor, v);
            Uout[2 * ((size_t)y * wo + x)] = factor * v[0];
            Uout[2 * ((size_t)y * wo + x) + 1] = factor * v[1];
        }
}

/* Total number of patches over levels ss..sf (coarsest first): the layout of `frozen`
 * and `record` in or_dis_flow. */
int or_total_patches(int W, int H, const or_params* p)
{
    int ss, sf;
    if (or_levels(W, H, p, &ss, &sf) != OR_OK) return -1;
    int stride = or_stride(p->patch_size, p->overlap, p->stride_override), tot = 0;
    for (int s = ss; s >= sf; s--)
        tot += or_grid_n(level_dim(W, s), p->patch_size, stride) * or_grid_n(level_dim(H, s), p->patch_size, stride);
    return tot;
}

/* ---- the whole method (Alg. 1) ----------------------------------------------------
 * I0, I1: C planes of H x W in [0,1]; flow_out: H x W x 2.
 * init_flow (optional): the flow that replaces U_{theta_ss + 1} = 0, given at the
 *   resolution of level theta_ss in that level's pixels (sampled with cscale = 1).
 * frozen / record (optional): per-patch increments u_i - u_init,i for every level,
 *   coarsest first (or_total_patches x 2).  record receives them (0 for reset and flat
 *   patches); frozen replays them instead of searching.
 * hash (optional): decision trace, see note().
 * [R1] intensities are scaled by intensity_scale; for C = 3 the search and the
 * densification use the channel mean, the refinement all channels (supp. Sec. B (i)). */
int or_dis_flow_fb(const double* I0, const double* I1, int W, int H, const or_params* p, const double* init_flow,
                   const double* frozen, double* record, double* flow_out, double* flow_b_out, uint64_t* hash)
{
    int C = p->channels, ss, sf;
    if (C != 1 && C != 3) return OR_ERR_INVALID;
    if ((p->dof != 1 && p->dof != 2) || p->norm < 0 || p->norm > 2 || !(p->huber_b > 0.0)) return OR_ERR_INVALID;
    /* [R22] forward-backward consistency starts both directions from zero and replays nothing */
    if (p->fb != 0 && p->fb != 1) return OR_ERR_INVALID;
    if (!(p->term_eps >= 0.0)) return OR_ERR_INVALID;
    if (p->fb && (init_flow || frozen || record)) return OR_ERR_INVALID;
    int rc = or_levels(W, H, p, &ss, &sf);
    if (rc != OR_OK) return rc;
    int ps = p->patch_size, stride = or_stride(ps, p->overlap, p->stride_override);
    t_hash = hash;
    int L = ss + 1;
    int* lw = (int*)malloc(sizeof(int) * L);
    int* lh = (int*)malloc(sizeof(int) * L);
    double** S0 = (double**)calloc(L, sizeof(double*));
    double** S1 = (double**)calloc(L, sizeof(double*));
    double** P0 = (double**)calloc((size_t)L * C, sizeof(double*)); /* [s*C + c] */
    double** P1 = (double**)calloc((size_t)L * C, sizeof(double*));
    for (int s = 0; s < L; s++) {
        lw[s] = level_dim(W, s);
        lh[s] = level_dim(H, s);
    }
    size_t n0 = (size_t)W * H;
    for (int c = 0; c < C; c++) {
        P0[c] = (double*)malloc(sizeof(double) * n0);
        P1[c] = (double*)malloc(sizeof(double) * n0);
        for (size_t o = 0; o < n0; o++) {
            P0[c][o] = p->intensity_scale * I0[n0 * c + o];
            P1[c][o] = p->intensity_scale * I1[n0 * c + o];
        }
    }
    S0[0] = (double*)malloc(sizeof(double) * n0);
    S1[0] = (double*)malloc(sizeof(double) * n0);
    for (size_t o = 0; o < n0; o++) {
        double a = 0.0, b = 0.0;
        for (int c = 0; c < C; c++) {
            a += P0[c][o];
            b += P1[c][o];
        }
        S0[0][o] = a / C;
        S1[0][o] = b / C;
    }
    for (int s = 1; s < L; s++) {
        size_t ns = (size_t)lw[s] * lh[s];
        S0[s] = (double*)malloc(sizeof(double) * ns);
        S1[s] = (double*)malloc(sizeof(double) * ns);
        or_pyr_down(S0[s - 1], lw[s - 1], lh[s - 1], S0[s]);
        or_pyr_down(S1[s - 1], lw[s - 1], lh[s - 1], S1[s]);
        if (p->refine)
            for (int c = 0; c < C; c++) {
                P0[s * C + c] = (double*)malloc(sizeof(double) * ns);
                P1[s * C + c] = (double*)malloc(sizeof(double) * ns);
                or_pyr_down(P0[(s - 1) * C + c], lw[s - 1], lh[s - 1], P0[s * C + c]);
                or_pyr_down(P1[(s - 1) * C + c], lw[s - 1], lh[s - 1], P1[s * C + c]);
            }
    }
    /* direction 0: I0 -> I1; direction 1 (forward-backward consistency): I1 -> I0 */
    const int ndir = p->fb ? 2 : 1;
    double* Uprev[2] = {NULL, NULL};
    int wprev = 0, hprev = 0, off = 0;
    for (int s = ss; s >= sf; s--) {
        int w = lw[s], h = lh[s];
        size_t ns = (size_t)w * h;
        int nx = or_grid_n(w, ps, stride), ny = or_grid_n(h, ps, stride), np = nx * ny;
        const double* A[2] = {S0[s], S1[s]};
        const double* B[2] = {S1[s], S0[s]};
        double* u[2] = {NULL, NULL};
        double* U[2] = {NULL, NULL};
        const double* Uc[2] = {Uprev[0], Uprev[1]};
        int wc = wprev, hc = hprev;
        double cs = 2.0;
        if (s == ss) {
            Uc[0] = init_flow;
            Uc[1] = NULL;
            wc = w;
            hc = h;
            cs = 1.0;
        }
        for (int d = 0; d < ndir; d++) {
            double* Ix = (double*)malloc(sizeof(double) * ns);
            double* Iy = (double*)malloc(sizeof(double) * ns);
            double* ui = (double*)malloc(sizeof(double) * 2 * np);
            u[d] = (double*)malloc(sizeof(double) * 2 * np);
            or_sobel(A[d], w, h, Ix, Iy);
            or_search_level(A[d], Ix, Iy, B[d], w, h, Uc[d], wc, hc, cs, ps, stride, p->grad_iters,
                            frozen ? frozen + 2 * off : NULL, u[d], ui, NULL, p->dof, p->norm, p->huber_b,
                            p->term_eps, p->polish);
            if (record && d == 0)
                for (int k = 0; k < 2 * np; k++) record[2 * off + k] = u[d][k] - ui[k];
            free(Ix);
            free(Iy);
            free(ui);
        }
        for (int d = 0; d < ndir; d++) {
            U[d] = (double*)malloc(sizeof(double) * 2 * ns);
            if (p->fb)
                or_densify_level_fb(A[d], B[d], w, h, u[d], u[1 - d], ps, stride, Uc[d], wc, hc, cs, U[d]);
            else
                or_densify_level(A[d], B[d], w, h, u[d], ps, stride, Uc[d], wc, hc, cs, U[d]);
        }
        if (p->refine)
            for (int d = 0; d < ndir; d++) {
                /* channel planes of level s, contiguous; direction 1 swaps the frames */
                double* Q0 = (double*)malloc(sizeof(double) * ns * C);
                double* Q1 = (double*)malloc(sizeof(double) * ns * C);
                for (int c = 0; c < C; c++) {
                    memcpy(Q0 + ns * c, (d ? P1 : P0)[s * C + c], sizeof(double) * ns);
                    memcpy(Q1 + ns * c, (d ? P0 : P1)[s * C + c], sizeof(double) * ns);
                }
                int outer = p->var_outer < 0 ? s + 1 : p->var_outer;
                or_refine_level(Q0, Q1, w, h, C, U[d], outer, p->var_inner, p->delta, p->gamma, p->alpha,
                                p->sor_omega, p->dof);
                free(Q0);
                free(Q1);
            }
        for (int d = 0; d < ndir; d++) {
            free(u[d]);
            free(Uprev[d]);
            Uprev[d] = U[d];
        }
        wprev = w;
        hprev = h;
        off += np;
    }
    if (flow_b_out && p->fb) or_upsample_flow(Uprev[1], wprev, hprev, (double)(1 << sf), flow_b_out, W, H);
    free(Uprev[1]);
    or_upsample_flow(Uprev[0], wprev, hprev, (double)(1 << sf), flow_out, W, H);
    free(Uprev[0]);
    for (int s = 0; s < L; s++) {
        free(S0[s]);
        free(S1[s]);
    }
    for (int k = 0; k < L * C; k++) {
        free(P0[k]);
        free(P1[k]);
    }
    free(S0);
    free(S1);
    free(P0);
    free(P1);
    free(lw);
    free(lh);
    t_hash = NULL;
    return OR_OK;
}

/* Alg. 1 on one pair; with p->fb the backward flow is computed alongside and dropped. */
int or_dis_flow(const double* I0, const double* I1, int W, int H, const or_params* p, const double* init_flow,
                const double* frozen, double* record, double* flow_out, uint64_t* hash)
{
    return or_dis_flow_fb(I0, I1, W, H, p, init_flow, frozen, record, flow_out, NULL, hash);
}

/* Photometric loss of the differentiable form: mean over channels and pixels of the
 * Charbonnier penalty sqrt((I1(x + U(x)) - I0(x))^2 + eps_c^2) on the [0,1] input scale.
 * [R18] eps_c is a parameter (the paper's eps = 0.001 by default).  hash (optional): the
 * bilinear cells and clampings of the loss's samples join the decision trace. */
double or_charbonnier_loss(const double* I0, const double* I1, int W, int H, int C, const double* flow, double eps_c,
                           uint64_t* hash)
{
    size_t n = (size_t)W * H;
    double acc = 0.0;
    t_hash = hash;
    for (int c = 0; c < C; c++)
        for (int y = 0; y < H; y++)
            for (int x = 0; x < W; x++) {
                size_t o = (size_t)y * W + x;
                double r = or_bilinear(I1 + n * c, W, H, x + flow[2 * o], y + flow[2 * o + 1]) - I0[n * c + o];
                acc += sqrt(r * r + eps_c * eps_c);
            }
    t_hash = NULL;
    return acc / (double)(n * C);
}
