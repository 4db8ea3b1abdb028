// Differentiable form of DIS (not in the paper): FP64 replay of the frozen-search map and its
// adjoint (reverse-mode derivative).
//
// The map: per level, u_i = u_init,i + Delta_i with the search increments Delta_i frozen
// (recorded by an FP32 forward call), u_init,i = cscale * Uc(c_i / cscale); U_d = densify(u)
// (Eq. 3); U = U_d + dU with dU from theta_vo x theta_vi unrolled red-black SOR sweeps
// (Sec. 2.3); the pyramid links the levels.  Its gradient depends on flow and residual
// differences at the 1e-6 level (Psi'(a^2) = 1 / (2 sqrt(a^2 + eps^2)) with eps = 0.001 has a
// second derivative of order 1e9 at a = 0), below the resolution of FP32 flow values, so the
// replay and the adjoint run in double precision: every kernel here computes in FP64.
//
// Every kernel works on one level of one pair.  Gradients that one output sends to several
// inputs are gathered by the input wherever the map is fixed by the geometry (SOR neighbours,
// central differences, Sobel transposes with clamped borders, the pyramid transpose), so those
// sums are deterministic and atomic-free.  The data-dependent scatters (the bilinear warp of I1
// by U in the refinement, the densification weights' samples of I1, the initial flow's samples
// of the coarser flow, the loss's samples of I1) accumulate in 64-bit fixed point: integer
// addition is associative, so the result does not depend on the order of the atomics.
#include <algorithm>

#include "dis_device.cuh"

namespace dis {

namespace {

// 2^48: resolution 3.6e-15, range +-32768.  The gradients scattered here are those of a mean
// photometric loss with respect to level images on the 0..255 scale (of order 1e-8) and flows;
// a gradient is a sum of dozens of contributions that largely cancel, so each contribution's
// rounding must stay far below it (at 2^-40 the sums of a few pixels erred by 1e-3 relative).
constexpr double kFix = 281474976710656.0;

__device__ __forceinline__ void fx_add(unsigned long long* p, double v)
{
    double d = v * kFix;
    d = fmin(fmax(d, -9.0e18), 9.0e18);
    atomicAdd(p, (unsigned long long)__double2ll_rn(d));
}

__device__ __forceinline__ double fx_get(const unsigned long long* p) { return (double)(long long)(*p) / kFix; }

// Sum of k[i + 1] over i in {-1, 0, 1} with clamp(x + i, 0, n - 1) == a  (x inside the image).
__device__ __forceinline__ double tw3(int a, int x, int n, double k0, double k1, double k2)
{
    double s = 0.0;
    if (max(x - 1, 0) == a) s += k0;
    if (x == a) s += k1;
    if (min(x + 1, n - 1) == a) s += k2;
    return s;
}

// Transpose of Sobel/8 (x: xdir = true) with replicated border, evaluated at (a, b).
__device__ double sobel_t(const double* __restrict__ G, int pitch, int w, int h, int a, int b, bool xdir)
{
    double acc = 0.0;
    for (int y = max(b - 1, 0); y <= min(b + 1, h - 1); ++y) {
        const double wy = xdir ? tw3(b, y, h, 1.0, 2.0, 1.0) : tw3(b, y, h, -1.0, 0.0, 1.0);
        if (wy == 0.0) continue;
        for (int x = max(a - 1, 0); x <= min(a + 1, w - 1); ++x) {
            const double wx = xdir ? tw3(a, x, w, -1.0, 0.0, 1.0) : tw3(a, x, w, 1.0, 2.0, 1.0);
            acc = fma(wx * wy, G[(long long)y * pitch + x], acc);
        }
    }
    return 0.125 * acc;
}

// Sobel/8 with replicated border at (x, y).
__device__ __forceinline__ double sobel_fwd(const double* __restrict__ P, int pitch, int w, int h, int x, int y,
                                            bool xdir)
{
    const int xl = max(x - 1, 0), xr = min(x + 1, w - 1);
    const double* ru = P + (long long)max(y - 1, 0) * pitch;
    const double* rc = P + (long long)y * pitch;
    const double* rd = P + (long long)min(y + 1, h - 1) * pitch;
    if (xdir) return 0.125 * ((ru[xr] - ru[xl]) + 2.0 * (rc[xr] - rc[xl]) + (rd[xr] - rd[xl]));
    return 0.125 * ((rd[xl] - ru[xl]) + 2.0 * (rd[x] - ru[x]) + (rd[xr] - ru[xr]));
}

// Clamped bilinear taps of I at (x + u, y + v): indices and weights, plus the value and its
// derivatives along u and v (zero along a clamped axis, where both taps coincide).
struct Taps {
    long long o00, o10, o01, o11;
    double ax, ay, val, du, dv;
};

template <class P>
__device__ __forceinline__ Taps taps_at(const P* __restrict__ I, int w, int h, int pitch, int x, int y, double u,
                                        double v)
{
    Taps t;
    const double uc = fmin(fmax(u, -1.0e7), 1.0e7), vc = fmin(fmax(v, -1.0e7), 1.0e7);
    const double fu = floor(uc), fv = floor(vc);
    t.ax = uc - fu;
    t.ay = vc - fv;
    const int xi = x + (int)fu, yi = y + (int)fv;
    const int x0 = clampi(xi, 0, w - 1), x1 = clampi(xi + 1, 0, w - 1);
    const int y0 = clampi(yi, 0, h - 1), y1 = clampi(yi + 1, 0, h - 1);
    t.o00 = (long long)y0 * pitch + x0;
    t.o10 = (long long)y0 * pitch + x1;
    t.o01 = (long long)y1 * pitch + x0;
    t.o11 = (long long)y1 * pitch + x1;
    const double a = I[t.o00], b = I[t.o10], c = I[t.o01], d = I[t.o11];
    const double top = fma(t.ax, b - a, a), bot = fma(t.ax, d - c, c);
    t.val = fma(t.ay, bot - top, top);
    t.du = (1.0 - t.ay) * (b - a) + t.ay * (d - c);
    t.dv = (1.0 - t.ax) * (c - a) + t.ax * (d - b);
    return t;
}

__device__ __forceinline__ void taps_scatter(unsigned long long* acc, const Taps& t, double g)
{
    fx_add(acc + t.o00, g * (1.0 - t.ax) * (1.0 - t.ay));
    fx_add(acc + t.o10, g * t.ax * (1.0 - t.ay));
    fx_add(acc + t.o01, g * (1.0 - t.ax) * t.ay);
    fx_add(acc + t.o11, g * t.ax * t.ay);
}

// Bilinear taps of a dense field at real (X, Y), clamped.
struct FlowTaps {
    long long i00, i10, i01, i11;
    double w00, w10, w01, w11;
};

__device__ __forceinline__ FlowTaps flow_taps(int w, int h, double X, double Y)
{
    FlowTaps t;
    X = fmin(fmax(X, 0.0), (double)(w - 1));
    Y = fmin(fmax(Y, 0.0), (double)(h - 1));
    const int x0 = (int)X, y0 = (int)Y, x1 = min(x0 + 1, w - 1), y1 = min(y0 + 1, h - 1);
    const double ax = X - x0, ay = Y - y0;
    t.i00 = (long long)y0 * w + x0;
    t.i10 = (long long)y0 * w + x1;
    t.i01 = (long long)y1 * w + x0;
    t.i11 = (long long)y1 * w + x1;
    t.w00 = (1.0 - ax) * (1.0 - ay);
    t.w10 = ax * (1.0 - ay);
    t.w01 = (1.0 - ax) * ay;
    t.w11 = ax * ay;
    return t;
}

__device__ __forceinline__ void cover_range(int q, int L_, int ps, int stride, int n, int& lo, int& hi, bool& last)
{
    const int t = q - ps + 1;
    lo = t <= 0 ? 0 : (t + stride - 1) / stride;
    hi = min(n - 2, q / stride);
    last = q >= L_ - ps;
}

}  // namespace

#define PIX_LOOP(W, H)                                                     \
    for (long long g = gtid(); g < (long long)(W) * (H); g += gstride()) { \
        const int y = (int)(g / (W)), x = (int)(g - (long long)y * (W));
#define PIX_END }
#define RS(k) (L.rs + (long long)(k)*L.plane)
#define GA(k) (L.ga + (long long)(k)*L.plane)

// ================================== FP64 replay =============================================
__global__ void __launch_bounds__(256) prep64_kernel(const float* __restrict__ I, int w, int h, int in_pitch,
                                                     double scale, double* S, int pitch)
{
    PIX_LOOP(w, h)
    S[(long long)y * pitch + x] = scale * (double)I[(long long)y * in_pitch + x];
    PIX_END
}

__global__ void __launch_bounds__(256) pyr64_kernel(const double* __restrict__ in, int win, int hin, int pin,
                                                    double* out, int wout, int hout, int pout)
{
    const double kw[5] = {0.0625, 0.25, 0.375, 0.25, 0.0625};
    PIX_LOOP(wout, hout)
    double acc = 0.0;
    for (int j = -2; j <= 2; ++j) {
        const double* row = in + (long long)clampi(2 * y + j, 0, hin - 1) * pin;
        double hsum = 0.0;
        for (int i = -2; i <= 2; ++i) hsum = fma(kw[i + 2], row[clampi(2 * x + i, 0, win - 1)], hsum);
        acc = fma(kw[j + 2], hsum, acc);
    }
    out[(long long)y * pout + x] = acc;
    PIX_END
}

// u_i = cscale * Uc(c_i / cscale) + Delta_i at the patch centre c_i (Uc null: zero).
__global__ void __launch_bounds__(256) uinit64_kernel(Dens64 A, int w, int h, const double2* __restrict__ Uc, int wc,
                                                      int hc, double cs, const float2* __restrict__ frozen, double2* pu)
{
    const long long np = (long long)A.nx * A.ny;
    for (long long k = gtid(); k < np; k += gstride()) {
        const int j = (int)(k / A.nx), i = (int)(k - (long long)j * A.nx);
        const int px = min(i * A.stride, w - A.ps), py = min(j * A.stride, h - A.ps);
        double ux = 0.0, uy = 0.0;
        if (Uc) {
            const FlowTaps t = flow_taps(wc, hc, (px + 0.5 * (A.ps - 1)) / cs, (py + 0.5 * (A.ps - 1)) / cs);
            ux = cs * (t.w00 * Uc[t.i00].x + t.w10 * Uc[t.i10].x + t.w01 * Uc[t.i01].x + t.w11 * Uc[t.i11].x);
            uy = cs * (t.w00 * Uc[t.i00].y + t.w10 * Uc[t.i10].y + t.w01 * Uc[t.i01].y + t.w11 * Uc[t.i11].y);
        }
        const float2 f = frozen[k];
        pu[k] = make_double2(ux + (double)f.x, uy + (double)f.y);
    }
}

__global__ void __launch_bounds__(256) densify64_kernel(const double* __restrict__ S0, const double* __restrict__ S1,
                                                        int w, int h, int pitch, Dens64 A,
                                                        const double2* __restrict__ Uc, int wc, int hc, double cs,
                                                        double2* Ud)
{
    PIX_LOOP(w, h)
    int ilo, ihi, jlo, jhi;
    bool il, jl;
    cover_range(x, w, A.ps, A.stride, A.nx, ilo, ihi, il);
    cover_range(y, h, A.ps, A.stride, A.ny, jlo, jhi, jl);
    const int jend = jhi + (jl ? 1 : 0), iend = ihi + (il ? 1 : 0);
    const double i0 = S0[(long long)y * pitch + x];
    double nu = 0.0, nv = 0.0, Z = 0.0;
    for (int jj = jlo; jj <= jend; ++jj) {
        const int j = jj > jhi ? A.ny - 1 : jj;
        for (int ii = ilo; ii <= iend; ++ii) {
            const int i = ii > ihi ? A.nx - 1 : ii;
            const double2 up = A.pu[(long long)j * A.nx + i];
            const double d = taps_at(S1, w, h, pitch, x, y, up.x, up.y).val - i0;
            const double wt = 1.0 / fmax(1.0, fabs(d));
            nu = fma(wt, up.x, nu);
            nv = fma(wt, up.y, nv);
            Z += wt;
        }
    }
    double2 r = make_double2(0.0, 0.0);
    if (Z > 0.0) {
        r = make_double2(nu / Z, nv / Z);
    } else if (Uc) {
        const FlowTaps t = flow_taps(wc, hc, x / cs, y / cs);
        r.x = cs * (t.w00 * Uc[t.i00].x + t.w10 * Uc[t.i10].x + t.w01 * Uc[t.i01].x + t.w11 * Uc[t.i11].x);
        r.y = cs * (t.w00 * Uc[t.i00].y + t.w10 * Uc[t.i10].y + t.w01 * Uc[t.i01].y + t.w11 * Uc[t.i11].y);
    }
    Ud[g] = r;
    PIX_END
}

// Refinement replay (the discretisation of the FP32 refinement kernels, in FP64).
__global__ void __launch_bounds__(256) ref64_prepare_kernel(Lvl64 L)
{
    PIX_LOOP(L.w, L.h)
    const long long o = (long long)y * L.pitch + x;
    const double2 U = L.U[g];
    RS(rs_mid(1, 0, 0))[o] = taps_at(L.S1, L.w, L.h, L.pitch, x, y, U.x, U.y).val;
    RS(rs_du(1, 0))[o] = 0.0;
    RS(rs_du(1, 1))[o] = 0.0;
    PIX_END
}

__global__ void __launch_bounds__(256) ref64_deriv1_kernel(Lvl64 L)
{
    PIX_LOOP(L.w, L.h)
    const int w = L.w, h = L.h, pitch = L.pitch;
    const long long o = (long long)y * pitch + x;
    const double* W1 = RS(rs_mid(1, 0, 0));
    const double sx0 = sobel_fwd(L.S0, pitch, w, h, x, y, true), sy0 = sobel_fwd(L.S0, pitch, w, h, x, y, false);
    const double sx1 = sobel_fwd(W1, pitch, w, h, x, y, true), sy1 = sobel_fwd(W1, pitch, w, h, x, y, false);
    RS(rs_mid(1, 0, 1))[o] = 0.5 * (sx0 + sx1);
    RS(rs_mid(1, 0, 2))[o] = 0.5 * (sy0 + sy1);
    RS(rs_mid(1, 0, 3))[o] = W1[o] - L.S0[o];
    RS(rs_mid(1, 0, 4))[o] = sx1 - sx0;
    RS(rs_mid(1, 0, 5))[o] = sy1 - sy0;
    PIX_END
}

__global__ void __launch_bounds__(256) ref64_deriv2_kernel(Lvl64 L)
{
    PIX_LOOP(L.w, L.h)
    const int w = L.w, h = L.h, pitch = L.pitch;
    const long long o = (long long)y * pitch + x;
    const double* Ixp = RS(rs_mid(1, 0, 1));
    const double* Iyp = RS(rs_mid(1, 0, 2));
    const double Ixx = sobel_fwd(Ixp, pitch, w, h, x, y, true), Ixy = sobel_fwd(Ixp, pitch, w, h, x, y, false);
    const double Iyy = sobel_fwd(Iyp, pitch, w, h, x, y, false);
    const double Ix = Ixp[o], Iy = Iyp[o];
    const double Iz = RS(rs_mid(1, 0, 3))[o], Ixz = RS(rs_mid(1, 0, 4))[o], Iyz = RS(rs_mid(1, 0, 5))[o];
    const double s0 = 1.0 / sqrt(Ix * Ix + Iy * Iy + 0.01);
    const double sx = 1.0 / sqrt(Ixx * Ixx + Ixy * Ixy + 0.01);
    const double sy = 1.0 / sqrt(Ixy * Ixy + Iyy * Iyy + 0.01);
    const double v[9] = {s0 * Ix, s0 * Iy, s0 * Iz, sx * Ixx, sx * Ixy, sx * Ixz, sy * Ixy, sy * Iyy, sy * Iyz};
    for (int k = 0; k < 9; ++k) RS(rs_dat(1, 0, k))[o] = v[k];
    PIX_END
}

__global__ void __launch_bounds__(256) ref64_weights_kernel(Lvl64 L)
{
    const double eps2 = 1.0e-6;
    PIX_LOOP(L.w, L.h)
    const int w = L.w, h = L.h, pitch = L.pitch;
    const long long o = (long long)y * pitch + x;
    const double* du_p = RS(rs_du(1, 0));
    const double* dv_p = RS(rs_du(1, 1));
    const double du = du_p[o], dv = dv_p[o];
    double d[9];
    for (int k = 0; k < 9; ++k) d[k] = RS(rs_dat(1, 0, k))[o];
    const double eI = fma(d[0], du, fma(d[1], dv, d[2]));
    const double eX = fma(d[3], du, fma(d[4], dv, d[5]));
    const double eY = fma(d[6], du, fma(d[7], dv, d[8]));
    const double psiI = L.delta / (2.0 * sqrt(eI * eI + eps2));
    const double psiG = L.gamma / (2.0 * sqrt(eX * eX + eY * eY + eps2));
    double* S = RS(rs_sys(1, 0)) + o;
    S[0] = psiI * d[0] * d[0] + psiG * (d[3] * d[3] + d[6] * d[6]);
    S[L.plane] = psiI * d[0] * d[1] + psiG * (d[3] * d[4] + d[6] * d[7]);
    S[2 * L.plane] = psiI * d[1] * d[1] + psiG * (d[4] * d[4] + d[7] * d[7]);
    S[3 * L.plane] = -(psiI * d[2] * d[0] + psiG * (d[5] * d[3] + d[8] * d[6]));
    S[4 * L.plane] = -(psiI * d[2] * d[1] + psiG * (d[5] * d[4] + d[8] * d[7]));
    const int xl = max(x - 1, 0), xr = min(x + 1, w - 1), yu = max(y - 1, 0), yd = min(y + 1, h - 1);
    const double2 Ul = L.U[(long long)y * w + xl], Ur = L.U[(long long)y * w + xr];
    const double2 Uu = L.U[(long long)yu * w + x], Ud = L.U[(long long)yd * w + x];
    const long long ol = (long long)y * pitch + xl, orr = (long long)y * pitch + xr;
    const long long ou = (long long)yu * pitch + x, od = (long long)yd * pitch + x;
    const double ux = 0.5 * ((Ur.x + du_p[orr]) - (Ul.x + du_p[ol]));
    const double vx = 0.5 * ((Ur.y + dv_p[orr]) - (Ul.y + dv_p[ol]));
    const double uy = 0.5 * ((Ud.x + du_p[od]) - (Uu.x + du_p[ou]));
    const double vy = 0.5 * ((Ud.y + dv_p[od]) - (Uu.y + dv_p[ou]));
    S[5 * L.plane] = L.alpha / (2.0 * sqrt(ux * ux + uy * uy + vx * vx + vy * vy + eps2));
    PIX_END
}

__global__ void __launch_bounds__(256) ref64_sor_kernel(Lvl64 L, int colour)
{
    const int w = L.w, h = L.h, pitch = L.pitch, hw = (w + 1) >> 1;
    const double* S = RS(rs_sys(1, 0));
    double* du_p = RS(rs_du(1, 0));
    double* dv_p = RS(rs_du(1, 1));
    const long long pl = L.plane;
    for (long long g = gtid(); g < (long long)h * hw; g += gstride()) {
        const int y = (int)(g / hw);
        const int x = 2 * (int)(g - (long long)y * hw) + ((y + colour) & 1);
        if (x >= w) continue;
        const long long o = (long long)y * pitch + x;
        const double psp = S[5 * pl + o];
        const double2 Up = L.U[(long long)y * w + x];
        double sw = 0.0, r1 = S[3 * pl + o], r2 = S[4 * pl + o];
        const int nxs[4] = {x - 1, x + 1, x, x}, nys[4] = {y, y, y - 1, y + 1};
        for (int q = 0; q < 4; ++q) {
            if (nxs[q] < 0 || nxs[q] >= w || nys[q] < 0 || nys[q] >= h) continue;
            const long long oq = (long long)nys[q] * pitch + nxs[q];
            const double wq = 0.5 * (psp + S[5 * pl + oq]);
            const double2 Uq = L.U[(long long)nys[q] * w + nxs[q]];
            sw += wq;
            r1 = fma(wq, (Uq.x + du_p[oq]) - Up.x, r1);
            r2 = fma(wq, (Uq.y + dv_p[oq]) - Up.y, r2);
        }
        const double m11 = S[o] + sw, m12 = S[pl + o], m22 = S[2 * pl + o] + sw;
        if (L.dof == 1) {  // stereo: the scalar x equation, dv stays
            if (m11 > 0.0) du_p[o] = (1.0 - L.omega) * du_p[o] + L.omega * (r1 / m11);
            continue;
        }
        const double det = m11 * m22 - m12 * m12;
        if (det > 0.0) {
            const double d1 = (m22 * r1 - m12 * r2) / det, d2 = (m11 * r2 - m12 * r1) / det;
            du_p[o] = (1.0 - L.omega) * du_p[o] + L.omega * d1;
            dv_p[o] = (1.0 - L.omega) * dv_p[o] + L.omega * d2;
        }
    }
}

// Uout = U + dU.
__global__ void __launch_bounds__(256) ref64_apply_kernel(Lvl64 L, double2* Uout)
{
    PIX_LOOP(L.w, L.h)
    const long long o = (long long)y * L.pitch + x;
    const double2 U = L.U[g];
    Uout[g] = make_double2(U.x + RS(rs_du(1, 0))[o], U.y + RS(rs_du(1, 1))[o]);
    PIX_END
}

// ================================== loss ====================================================
__global__ void __launch_bounds__(256) loss_kernel(const float* __restrict__ I0, const float* __restrict__ I1, int w,
                                                   int h, int pitch, int C, const float2* __restrict__ flow, double eps,
                                                   double inv_count, double* partials, float2* gflow, float* gI0,
                                                   unsigned long long* gI1acc)
{
    double local = 0.0;
    const long long plane = (long long)pitch * h;
    PIX_LOOP(w, h)
    const float2 f = flow[g];
    double gfx = 0.0, gfy = 0.0;
    for (int c = 0; c < C; ++c) {
        Taps t = taps_at(I1 + c * plane, w, h, pitch, x, y, (double)f.x, (double)f.y);
        const double r = t.val - (double)I0[c * plane + (long long)y * pitch + x];
        const double q = sqrt(r * r + eps * eps);
        local += q;
        const double gr = r / q * inv_count;
        gI0[c * plane + (long long)y * pitch + x] = (float)(-gr);
        t.o00 += c * plane;
        t.o10 += c * plane;
        t.o01 += c * plane;
        t.o11 += c * plane;
        taps_scatter(gI1acc, t, gr);
        gfx = fma(gr, t.du, gfx);
        gfy = fma(gr, t.dv, gfy);
    }
    gflow[g] = make_float2((float)gfx, (float)gfy);
    PIX_END
    // deterministic block partial: fixed shuffle tree, then warp sums in warp order
    __shared__ double ws[32];
    for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = local;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += ws[k];
        partials[blockIdx.x] = s;
    }
}

__global__ void loss_finalize_kernel(const double* partials, int n, double scale, double* out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < n; ++k) s += partials[k];
        out[0] = s * scale;
    }
}

// out = scale * fixed-point array (+ out when `accumulate`): float or double output.
template <class T>
__global__ void __launch_bounds__(256) fx_out_kernel(const unsigned long long* __restrict__ acc, int apitch, T* out,
                                                     int opitch, int w, int h, double scale, int accumulate)
{
    PIX_LOOP(w, h)
    const double v = scale * fx_get(acc + (long long)y * apitch + x);
    T* o = out + (long long)y * opitch + x;
    *o = accumulate ? (T)((double)*o + v) : (T)v;
    PIX_END
}

// ================================== adjoint =================================================
// Red-black SOR half-sweep, pixels p of `colour` (updated by the half-sweep): replace the
// increment's adjoint by (1 - omega) times itself, push omega * adjoint through d* = M^-1 r into
// b, A, the edge weights and U_p; store (M^-1 g, g_sumw) for the neighbours' gather.
__global__ void __launch_bounds__(256) sor_bwd_p_kernel(Lvl64 L, const double* __restrict__ st_du,
                                                        const double* __restrict__ st_dv, int colour)
{
    const int w = L.w, h = L.h, pitch = L.pitch, hw = (w + 1) >> 1;
    const long long pl = L.plane;
    const double* S = RS(rs_sys(1, 0));
    double* gS = GA(ADJ_GSYS);
    double* gdu = GA(ADJ_GDU);
    double* gdv = gdu + pl;
    double* T = GA(ADJ_GT);
    for (long long g = gtid(); g < (long long)h * hw; g += gstride()) {
        const int y = (int)(g / hw);
        const int x = 2 * (int)(g - (long long)y * hw) + ((y + colour) & 1);
        if (x >= w) continue;
        const long long o = (long long)y * pitch + x, f = (long long)y * w + x;
        const double psp = S[5 * pl + o];
        const double2 Up = L.U[f];
        double sw = 0.0, r1 = S[3 * pl + o], r2 = S[4 * pl + o];
        const int nxs[4] = {x - 1, x + 1, x, x}, nys[4] = {y, y, y - 1, y + 1};
        double wq[4], dxq[4], dyq[4];
        bool in[4];
        for (int q = 0; q < 4; ++q) {
            in[q] = nxs[q] >= 0 && nxs[q] < w && nys[q] >= 0 && nys[q] < h;
            wq[q] = dxq[q] = dyq[q] = 0.0;
            if (!in[q]) continue;
            const long long oq = (long long)nys[q] * pitch + nxs[q];
            const double2 Uq = L.U[(long long)nys[q] * w + nxs[q]];
            wq[q] = 0.5 * (psp + S[5 * pl + oq]);
            dxq[q] = (Uq.x + st_du[oq]) - Up.x;
            dyq[q] = (Uq.y + st_dv[oq]) - Up.y;
            sw += wq[q];
            r1 = fma(wq[q], dxq[q], r1);
            r2 = fma(wq[q], dyq[q], r2);
        }
        const double m11 = S[o] + sw, m12 = S[pl + o], m22 = S[2 * pl + o] + sw;
        double d1, d2, gr1, gr2;
        if (L.dof == 1) {
            // stereo: du = (1 - omega) du + omega r1 / m11; dv (and its adjoint) pass unchanged
            if (!(m11 > 0.0)) {
                T[o] = T[pl + o] = T[2 * pl + o] = 0.0;
                continue;
            }
            d1 = r1 / m11;
            d2 = 0.0;
            gr1 = L.omega * gdu[o] / m11;
            gr2 = 0.0;
            gdu[o] *= (1.0 - L.omega);
            gS[o] -= gr1 * d1;
            gS[3 * pl + o] += gr1;
        } else {
            const double det = m11 * m22 - m12 * m12;
            if (!(det > 0.0)) {
                T[o] = T[pl + o] = T[2 * pl + o] = 0.0;
                continue;
            }
            d1 = (m22 * r1 - m12 * r2) / det;
            d2 = (m11 * r2 - m12 * r1) / det;
            const double gd1 = L.omega * gdu[o], gd2 = L.omega * gdv[o];
            gr1 = (m22 * gd1 - m12 * gd2) / det;
            gr2 = (m11 * gd2 - m12 * gd1) / det;
            gdu[o] *= (1.0 - L.omega);
            gdv[o] *= (1.0 - L.omega);
            gS[o] -= gr1 * d1;
            gS[pl + o] -= gr1 * d2 + gr2 * d1;
            gS[2 * pl + o] -= gr2 * d2;
            gS[3 * pl + o] += gr1;
            gS[4 * pl + o] += gr2;
        }
        const double gsw = -(gr1 * d1 + gr2 * d2);
        double gps = 0.0, gux = 0.0, guy = 0.0;
        for (int q = 0; q < 4; ++q) {
            if (!in[q]) continue;
            gps += 0.5 * (gsw + gr1 * dxq[q] + gr2 * dyq[q]);
            gux -= wq[q] * gr1;
            guy -= wq[q] * gr2;
        }
        gS[5 * pl + o] += gps;
        L.gU[f].x += gux;
        L.gU[f].y += guy;
        T[o] = gr1;
        T[pl + o] = gr2;
        T[2 * pl + o] = gsw;
    }
}

// Pixels q of the other colour gather from their updated neighbours p the shares of the edge
// weight, increment and flow adjoints.
__global__ void __launch_bounds__(256) sor_bwd_q_kernel(Lvl64 L, const double* __restrict__ st_du,
                                                        const double* __restrict__ st_dv, int colour_q)
{
    const int w = L.w, h = L.h, pitch = L.pitch, hw = (w + 1) >> 1;
    const long long pl = L.plane;
    const double* S = RS(rs_sys(1, 0));
    double* gS = GA(ADJ_GSYS);
    double* gdu = GA(ADJ_GDU);
    double* gdv = gdu + pl;
    const double* T = GA(ADJ_GT);
    for (long long g = gtid(); g < (long long)h * hw; g += gstride()) {
        const int y = (int)(g / hw);
        const int x = 2 * (int)(g - (long long)y * hw) + ((y + colour_q) & 1);
        if (x >= w) continue;
        const long long o = (long long)y * pitch + x, f = (long long)y * w + x;
        const double psq = S[5 * pl + o];
        const double2 Uq = L.U[f];
        const double wxq = Uq.x + st_du[o], wyq = Uq.y + st_dv[o];
        const int nxs[4] = {x - 1, x + 1, x, x}, nys[4] = {y, y, y - 1, y + 1};
        double gps = 0.0, g1 = 0.0, g2 = 0.0;
        for (int q = 0; q < 4; ++q) {
            const int px = nxs[q], py = nys[q];
            if (px < 0 || px >= w || py < 0 || py >= h) continue;
            const long long op = (long long)py * pitch + px;
            const double gr1 = T[op], gr2 = T[pl + op], gsw = T[2 * pl + op];
            const double2 Up = L.U[(long long)py * w + px];
            const double wpq = 0.5 * (S[5 * pl + op] + psq);
            gps += 0.5 * (gsw + gr1 * (wxq - Up.x) + gr2 * (wyq - Up.y));
            g1 = fma(wpq, gr1, g1);
            g2 = fma(wpq, gr2, g2);
        }
        gS[5 * pl + o] += gps;
        gdu[o] += g1;
        gdv[o] += g2;
        L.gU[f].x += g1;
        L.gU[f].y += g2;
    }
}

// Lagged weights: from the adjoints of (A11 A12 A22 b1 b2 psiS) to the data values D, to the
// increment at the start of the outer pass (through E_I, E_G) and, for the smoothness term, to
// the central differences (stored for the gather below).
__global__ void __launch_bounds__(256) weights_bwd_kernel(Lvl64 L, const double* __restrict__ st_du,
                                                          const double* __restrict__ st_dv)
{
    const double eps2 = 1.0e-6;
    const long long pl = L.plane;
    PIX_LOOP(L.w, L.h)
    const int w = L.w, h = L.h, pitch = L.pitch;
    const long long o = (long long)y * pitch + x;
    double d[9];
    for (int k = 0; k < 9; ++k) d[k] = RS(rs_dat(1, 0, k))[o];
    const double du = st_du[o], dv = st_dv[o];
    const double eI = fma(d[0], du, fma(d[1], dv, d[2]));
    const double eX = fma(d[3], du, fma(d[4], dv, d[5]));
    const double eY = fma(d[6], du, fma(d[7], dv, d[8]));
    const double EI = eI * eI, EG = eX * eX + eY * eY;
    const double psiI = L.delta / (2.0 * sqrt(EI + eps2));
    const double psiG = L.gamma / (2.0 * sqrt(EG + eps2));
    const double* gS = GA(ADJ_GSYS) + o;
    const double gA11 = gS[0], gA12 = gS[pl], gA22 = gS[2 * pl], gb1 = gS[3 * pl], gb2 = gS[4 * pl], gps = gS[5 * pl];
    const double gpsiI = gA11 * d[0] * d[0] + gA12 * d[0] * d[1] + gA22 * d[1] * d[1] - gb1 * d[2] * d[0] -
                         gb2 * d[2] * d[1];
    const double gpsiG = gA11 * (d[3] * d[3] + d[6] * d[6]) + gA12 * (d[3] * d[4] + d[6] * d[7]) +
                         gA22 * (d[4] * d[4] + d[7] * d[7]) - gb1 * (d[5] * d[3] + d[8] * d[6]) -
                         gb2 * (d[5] * d[4] + d[8] * d[7]);
    double gd[9];
    gd[0] = psiI * (2.0 * gA11 * d[0] + gA12 * d[1] - gb1 * d[2]);
    gd[1] = psiI * (gA12 * d[0] + 2.0 * gA22 * d[1] - gb2 * d[2]);
    gd[2] = psiI * (-gb1 * d[0] - gb2 * d[1]);
    gd[3] = psiG * (2.0 * gA11 * d[3] + gA12 * d[4] - gb1 * d[5]);
    gd[4] = psiG * (gA12 * d[3] + 2.0 * gA22 * d[4] - gb2 * d[5]);
    gd[5] = psiG * (-gb1 * d[3] - gb2 * d[4]);
    gd[6] = psiG * (2.0 * gA11 * d[6] + gA12 * d[7] - gb1 * d[8]);
    gd[7] = psiG * (gA12 * d[6] + 2.0 * gA22 * d[7] - gb2 * d[8]);
    gd[8] = psiG * (-gb1 * d[6] - gb2 * d[7]);
    // psi = weight / (2 sqrt(E + eps^2))  ->  dpsi/dE = -psi / (2 (E + eps^2))
    const double geI = 2.0 * eI * gpsiI * (-psiI / (2.0 * (EI + eps2)));
    const double gEG = gpsiG * (-psiG / (2.0 * (EG + eps2)));
    const double geX = 2.0 * eX * gEG, geY = 2.0 * eY * gEG;
    gd[0] += geI * du;
    gd[1] += geI * dv;
    gd[2] += geI;
    gd[3] += geX * du;
    gd[4] += geX * dv;
    gd[5] += geX;
    gd[6] += geY * du;
    gd[7] += geY * dv;
    gd[8] += geY;
    for (int k = 0; k < 9; ++k) GA(ADJ_GD + k)[o] += gd[k];
    GA(ADJ_GDU)[o] += geI * d[0] + geX * d[3] + geY * d[6];
    GA(ADJ_GDU + 1)[o] += geI * d[1] + geX * d[4] + geY * d[7];
    // smoothness weight psiS = alpha / (2 sqrt(E_S + eps^2)), E_S from central differences of U + dU
    const int xl = max(x - 1, 0), xr = min(x + 1, w - 1), yu = max(y - 1, 0), yd = min(y + 1, h - 1);
    const double2 Ul = L.U[(long long)y * w + xl], Ur = L.U[(long long)y * w + xr];
    const double2 Uu = L.U[(long long)yu * w + x], Ud = L.U[(long long)yd * w + x];
    const long long ol = (long long)y * pitch + xl, orr = (long long)y * pitch + xr;
    const long long ou = (long long)yu * pitch + x, od = (long long)yd * pitch + x;
    const double ux = 0.5 * ((Ur.x + st_du[orr]) - (Ul.x + st_du[ol]));
    const double vx = 0.5 * ((Ur.y + st_dv[orr]) - (Ul.y + st_dv[ol]));
    const double uy = 0.5 * ((Ud.x + st_du[od]) - (Uu.x + st_du[ou]));
    const double vy = 0.5 * ((Ud.y + st_dv[od]) - (Uu.y + st_dv[ou]));
    const double ES = ux * ux + uy * uy + vx * vx + vy * vy;
    const double psS = L.alpha / (2.0 * sqrt(ES + eps2));
    const double gES = gps * (-psS / (2.0 * (ES + eps2)));
    // d(ux)/dW(xr).u = +1/2: the factor 2 of ux^2 and the 1/2 cancel
    double* T = GA(ADJ_GT) + o;
    T[0] = ux * gES;
    T[pl] = vx * gES;
    T[2 * pl] = uy * gES;
    T[3 * pl] = vy * gES;
    PIX_END
}

// Gather of the smoothness weights' central-difference adjoints onto U + dU.
__global__ void __launch_bounds__(256) smooth_bwd_kernel(Lvl64 L)
{
    const long long pl = L.plane;
    PIX_LOOP(L.w, L.h)
    const int w = L.w, h = L.h, pitch = L.pitch;
    const double* T = GA(ADJ_GT);
    double gx = 0.0, gy = 0.0;
    const int cx[5] = {x, x - 1, x + 1, x, x}, cy[5] = {y, y, y, y - 1, y + 1};
    for (int k = 0; k < 5; ++k) {
        const int px = cx[k], py = cy[k];
        if (px < 0 || px >= w || py < 0 || py >= h) continue;
        const long long op = (long long)py * pitch + px;
        if (py == y) {
            if (min(px + 1, w - 1) == x) {
                gx += T[op];
                gy += T[pl + op];
            }
            if (max(px - 1, 0) == x) {
                gx -= T[op];
                gy -= T[pl + op];
            }
        }
        if (px == x) {
            if (min(py + 1, h - 1) == y) {
                gx += T[2 * pl + op];
                gy += T[3 * pl + op];
            }
            if (max(py - 1, 0) == y) {
                gx -= T[2 * pl + op];
                gy -= T[3 * pl + op];
            }
        }
    }
    const long long o = (long long)y * pitch + x;
    GA(ADJ_GDU)[o] += gx;
    GA(ADJ_GDU + 1)[o] += gy;
    L.gU[g].x += gx;
    L.gU[g].y += gy;
    PIX_END
}

// D = (s0 Ix, s0 Iy, s0 Iz, sx Ixx, sx Ixy, sx Ixz, sy Ixy, sy Iyy, sy Iyz), s = (|.|^2 + 0.01)^-1/2.
__global__ void __launch_bounds__(256) deriv_bwd_local_kernel(Lvl64 L)
{
    const long long pl = L.plane;
    PIX_LOOP(L.w, L.h)
    const int w = L.w, h = L.h, pitch = L.pitch;
    const long long o = (long long)y * pitch + x;
    const double* Ixp = RS(rs_mid(1, 0, 1));
    const double* Iyp = RS(rs_mid(1, 0, 2));
    const double Ix = Ixp[o], Iy = Iyp[o];
    const double Iz = RS(rs_mid(1, 0, 3))[o], Ixz = RS(rs_mid(1, 0, 4))[o], Iyz = RS(rs_mid(1, 0, 5))[o];
    const double Ixx = sobel_fwd(Ixp, pitch, w, h, x, y, true), Ixy = sobel_fwd(Ixp, pitch, w, h, x, y, false);
    const double Iyy = sobel_fwd(Iyp, pitch, w, h, x, y, false);
    const double s0 = 1.0 / sqrt(Ix * Ix + Iy * Iy + 0.01);
    const double sx = 1.0 / sqrt(Ixx * Ixx + Ixy * Ixy + 0.01);
    const double sy = 1.0 / sqrt(Ixy * Ixy + Iyy * Iyy + 0.01);
    double gk[9];
    for (int k = 0; k < 9; ++k) gk[k] = GA(ADJ_GD + k)[o];
    const double gs0 = (gk[0] * Ix + gk[1] * Iy + gk[2] * Iz) * (-s0 * s0 * s0);
    const double gsx = (gk[3] * Ixx + gk[4] * Ixy + gk[5] * Ixz) * (-sx * sx * sx);
    const double gsy = (gk[6] * Ixy + gk[7] * Iyy + gk[8] * Iyz) * (-sy * sy * sy);
    double* G = GA(ADJ_GM) + o;  // gIx_l gIy_l gIz gIxx gIxy gIyy gIxz gIyz
    G[0] = s0 * gk[0] + gs0 * Ix;
    G[pl] = s0 * gk[1] + gs0 * Iy;
    G[2 * pl] = s0 * gk[2];
    G[3 * pl] = sx * gk[3] + gsx * Ixx;
    G[4 * pl] = sx * gk[4] + gsx * Ixy + sy * gk[6] + gsy * Ixy;
    G[5 * pl] = sy * gk[7] + gsy * Iyy;
    G[6 * pl] = sx * gk[5];
    G[7 * pl] = sy * gk[8];
    PIX_END
}

// I_xx = Sobel_x(I_x), I_xy = Sobel_y(I_x), I_yy = Sobel_y(I_y): transpose onto I_x, I_y.
__global__ void __launch_bounds__(256) deriv_bwd_second_kernel(Lvl64 L)
{
    const long long pl = L.plane;
    PIX_LOOP(L.w, L.h)
    const int w = L.w, h = L.h, pitch = L.pitch;
    const long long o = (long long)y * pitch + x;
    const double* G = GA(ADJ_GM);
    GA(ADJ_GIX)[o] = G[o] + sobel_t(G + 3 * pl, pitch, w, h, x, y, true) + sobel_t(G + 4 * pl, pitch, w, h, x, y, false);
    GA(ADJ_GIY)[o] = G[pl + o] + sobel_t(G + 5 * pl, pitch, w, h, x, y, false);
    PIX_END
}

// I_x, I_y = Sobel/8 of (I0 + I1w)/2, I_z = I1w - I0, I_xz / I_yz = Sobel/8 of I1w - I0.
__global__ void __launch_bounds__(256) deriv_bwd_first_kernel(Lvl64 L)
{
    const long long pl = L.plane;
    PIX_LOOP(L.w, L.h)
    const int w = L.w, h = L.h, pitch = L.pitch;
    const long long o = (long long)y * pitch + x;
    const double* G = GA(ADJ_GM);
    const double gbar = sobel_t(GA(ADJ_GIX), pitch, w, h, x, y, true) + sobel_t(GA(ADJ_GIY), pitch, w, h, x, y, false);
    const double gz = sobel_t(G + 6 * pl, pitch, w, h, x, y, true) + sobel_t(G + 7 * pl, pitch, w, h, x, y, false);
    const double gIz = G[2 * pl + o];
    GA(ADJ_GI1W)[o] = 0.5 * gbar + gIz + gz;
    L.gS0[o] += 0.5 * gbar - gIz - gz;
    PIX_END
}

// I1w(x) = I1(x + U(x)): scatter to I1 (fixed point), gather the flow derivative.
__global__ void __launch_bounds__(256) warp_bwd_kernel(Lvl64 L)
{
    PIX_LOOP(L.w, L.h)
    const long long o = (long long)y * L.pitch + x;
    const double gw = GA(ADJ_GI1W)[o];
    const double2 U = L.U[g];
    const Taps t = taps_at(L.S1, L.w, L.h, L.pitch, x, y, U.x, U.y);
    taps_scatter(L.gS1, t, gw);
    L.gU[g].x = fma(gw, t.du, L.gU[g].x);
    L.gU[g].y = fma(gw, t.dv, L.gU[g].y);
    PIX_END
}

// Densification, per pixel: U_d = N / Z; adjoints of N and Z (stored), of I0(x) and, through
// the weights' samples, of I1 (fixed point).
__global__ void __launch_bounds__(256) dens_bwd_pix_kernel(Lvl64 L, Dens64 A)
{
    PIX_LOOP(L.w, L.h)
    const int w = L.w, h = L.h, pitch = L.pitch;
    const long long o = (long long)y * pitch + x;
    int ilo, ihi, jlo, jhi;
    bool il, jl;
    cover_range(x, w, A.ps, A.stride, A.nx, ilo, ihi, il);
    cover_range(y, h, A.ps, A.stride, A.ny, jlo, jhi, jl);
    const int jend = jhi + (jl ? 1 : 0), iend = ihi + (il ? 1 : 0);
    const double i0 = L.S0[o];
    double nu = 0.0, nv = 0.0, Z = 0.0;
    for (int jj = jlo; jj <= jend; ++jj) {
        const int j = jj > jhi ? A.ny - 1 : jj;
        for (int ii = ilo; ii <= iend; ++ii) {
            const int i = ii > ihi ? A.nx - 1 : ii;
            const double2 up = A.pu[(long long)j * A.nx + i];
            const double d = taps_at(L.S1, w, h, pitch, x, y, up.x, up.y).val - i0;
            const double wt = 1.0 / fmax(1.0, fabs(d));
            nu = fma(wt, up.x, nu);
            nv = fma(wt, up.y, nv);
            Z += wt;
        }
    }
    double* T = GA(ADJ_GT);
    if (!(Z > 0.0)) {
        T[o] = T[L.plane + o] = T[2 * L.plane + o] = 0.0;
        continue;
    }
    const double2 gUd = A.gUd[g];
    const double gnx = gUd.x / Z, gny = gUd.y / Z;
    const double gZ = -(gUd.x * nu + gUd.y * nv) / (Z * Z);
    T[o] = gnx;
    T[L.plane + o] = gny;
    T[2 * L.plane + o] = gZ;
    double gi0 = 0.0;
    for (int jj = jlo; jj <= jend; ++jj) {
        const int j = jj > jhi ? A.ny - 1 : jj;
        for (int ii = ilo; ii <= iend; ++ii) {
            const int i = ii > ihi ? A.nx - 1 : ii;
            const double2 up = A.pu[(long long)j * A.nx + i];
            const Taps t = taps_at(L.S1, w, h, pitch, x, y, up.x, up.y);
            const double d = t.val - i0;
            const double ad = fabs(d);
            if (ad <= 1.0) continue;
            const double gwt = gnx * up.x + gny * up.y + gZ;
            const double gd = gwt * (d > 0.0 ? -1.0 : 1.0) / (ad * ad);
            gi0 -= gd;
            taps_scatter(L.gS1, t, gd);
        }
    }
    L.gS0[o] += gi0;
    PIX_END
}

// Densification, per patch (one warp): g u_i = sum over its pixels of w_i(x) gN(x) + g d_i(x)
// grad I1(x + u_i).
__global__ void __launch_bounds__(128) dens_bwd_patch_kernel(Lvl64 L, Dens64 A)
{
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long np = (long long)A.nx * A.ny;
    const int ps = A.ps, n = ps * ps;
    const double* T = GA(ADJ_GT);
    for (long long k = warp; k < np; k += nwarps) {
        const int j = (int)(k / A.nx), i = (int)(k - (long long)j * A.nx);
        const int px = min(i * A.stride, L.w - ps), py = min(j * A.stride, L.h - ps);
        const double2 up = A.pu[k];
        double gx = 0.0, gy = 0.0;
        for (int q = lane; q < n; q += 32) {
            const int x = px + q % ps, y = py + q / ps;
            const long long o = (long long)y * L.pitch + x;
            const double gnx = T[o], gny = T[L.plane + o], gZ = T[2 * L.plane + o];
            const Taps t = taps_at(L.S1, L.w, L.h, L.pitch, x, y, up.x, up.y);
            const double d = t.val - L.S0[o];
            const double ad = fabs(d);
            const double wt = 1.0 / fmax(1.0, ad);
            gx = fma(wt, gnx, gx);
            gy = fma(wt, gny, gy);
            if (ad > 1.0) {
                const double gwt = gnx * up.x + gny * up.y + gZ;
                const double gd = gwt * (d > 0.0 ? -1.0 : 1.0) / (ad * ad);
                gx = fma(gd, t.du, gx);
                gy = fma(gd, t.dv, gy);
            }
        }
        for (int o2 = 16; o2 > 0; o2 >>= 1) {
            gx += __shfl_xor_sync(0xffffffffu, gx, o2);
            gy += __shfl_xor_sync(0xffffffffu, gy, o2);
        }
        if (lane == 0) A.gpu[k] = make_double2(gx, gy);
    }
}

// u_init,i = cscale * Uc(c_i / cscale): scatter cscale * weights * g u_i onto Uc (fixed point,
// two components per pixel).
// Implicit-function gradient of the converged patch search.  At a patch's solution u the search
// is stationary: g(u) = sum_q S'_q (w~_q - T_q) = 0 with w~ = w - mean w, w_q = I1(x_q + u)
// (bilinear), T = I0 patch - its mean, S' = Sobel/8 of I0.  Hence du/dtheta = -J^-1 dg/dtheta,
// J = sum_q S'_q (grad w_q - mean grad w)^T, and for the patch's upstream gradient gu,
// lambda = -J^-T gu gives dL/dtheta = lambda . dg/dtheta:
//   I1 through w_q:      lambda . (S'_q - mean S')        (bilinear scatter at x_q + u)
//   I0 through T_q:     -lambda . (S'_q - mean S')
//   I0 through S'_q:     lambda_x r_q, lambda_y r_q       (Sobel transpose), r_q = w~_q - T_q.
// The solution does not depend on u_init, so the patch's gradient is consumed here (gpu = 0).
// dof 1 (stereo): g = sum S'_x (w~ - T) in u alone, J = its scalar derivative, lambda_y = 0; v is
// u_init's, and the solution u depends on it through g (the samples at x + (u, v)), so v's
// gradient gains lambda_x dg/dv = lambda_x sum S'_x (dw/dv - mean dw/dv) before it goes on to the
// initial-displacement transpose.
// A zero frozen increment marks a patch that was reset, flat or never moved: it stays at
// u_init and keeps its gradient for the initial-displacement transpose.  One warp per patch.
__global__ void __launch_bounds__(128) search_ift_bwd_kernel(Lvl64 L, Dens64 A, const float2* __restrict__ frozen,
                                                             unsigned long long* __restrict__ gS0acc, int dof)
{
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long np = (long long)A.nx * A.ny;
    const int ps = A.ps, n = ps * ps, w = L.w, h = L.h, pitch = L.pitch;
    for (long long k = warp; k < np; k += nwarps) {
        const float2 dz = frozen[k];
        if (dz.x == 0.0f && dz.y == 0.0f) continue;
        const int j = (int)(k / A.nx), i = (int)(k - (long long)j * A.nx);
        const int px = min(i * A.stride, w - ps), py = min(j * A.stride, h - ps);
        const double2 u = A.pu[k];
        // sums over the patch: I0, w, grad w, S', S' grad w^T
        double s[11] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
        for (int q = lane; q < n; q += 32) {
            const int x = px + q % ps, y = py + q / ps;
            const double gx = sobel_fwd(L.S0, pitch, w, h, x, y, true), gy = sobel_fwd(L.S0, pitch, w, h, x, y, false);
            const Taps t = taps_at(L.S1, w, h, pitch, x, y, u.x, u.y);
            s[0] += L.S0[(long long)y * pitch + x];
            s[1] += t.val;
            s[2] += t.du;
            s[3] += t.dv;
            s[4] += gx;
            s[5] += gy;
            s[6] += gx * t.du;
            s[7] += gx * t.dv;
            s[8] += gy * t.du;
            s[9] += gy * t.dv;
        }
#pragma unroll
        for (int m = 0; m < 10; ++m)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s[m] += __shfl_xor_sync(0xffffffffu, s[m], o);
        const double inv_n = 1.0 / n;
        const double mean0 = s[0] * inv_n, mw = s[1] * inv_n, mdu = s[2] * inv_n, mdv = s[3] * inv_n;
        const double msx = s[4] * inv_n, msy = s[5] * inv_n;
        const double j00 = s[6] - s[4] * mdu, j01 = s[7] - s[4] * mdv;  // J = sum S' (grad w - mean)^T
        const double j10 = s[8] - s[5] * mdu, j11 = s[9] - s[5] * mdv;
        const double2 gu = A.gpu[k];
        double lx, ly;
        if (dof == 1) {
            // stereo: g = sum S'_x (w~ - T) = 0 in u alone; v is u_init's and keeps its gradient
            if (!(fabs(j00) > 0.0)) continue;
            lx = -gu.x / j00;
            ly = 0.0;
        } else {
            const double det = j00 * j11 - j01 * j10;
            if (!(fabs(det) > 0.0)) continue;  // no solution to differentiate: keep the frozen rule
            // J^T lambda = -gu
            lx = -(j11 * gu.x - j10 * gu.y) / det;
            ly = -(-j01 * gu.x + j00 * gu.y) / det;
        }
        for (int q = lane; q < n; q += 32) {
            const int x = px + q % ps, y = py + q / ps;
            const double gx = sobel_fwd(L.S0, pitch, w, h, x, y, true), gy = sobel_fwd(L.S0, pitch, w, h, x, y, false);
            const Taps t = taps_at(L.S1, w, h, pitch, x, y, u.x, u.y);
            const double c = lx * (gx - msx) + ly * (gy - msy);
            taps_scatter(L.gS1, t, c);
            fx_add(gS0acc + (long long)y * pitch + x, -c);
            const double r = (t.val - mw) - (L.S0[(long long)y * pitch + x] - mean0);
            const double ax = 0.125 * lx * r, ay = 0.125 * ly * r;
            // Sobel transpose: Ix(x, y) = (1/8) sum kx I0(clamp(x + dx), clamp(y + dy)), likewise Iy
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const double kx = (double)dx * (dy == 0 ? 2.0 : 1.0), ky = (double)dy * (dx == 0 ? 2.0 : 1.0);
                    const double v = ax * kx + ay * ky;
                    if (v != 0.0)
                        fx_add(gS0acc + (long long)clampi(y + dy, 0, h - 1) * pitch + clampi(x + dx, 0, w - 1), v);
                }
        }
        if (lane == 0) A.gpu[k] = make_double2(0.0, dof == 1 ? fma(lx, j01, gu.y) : 0.0);
    }
}

__global__ void __launch_bounds__(256) uinit_bwd_kernel(Dens64 A, int w, int h, unsigned long long* gUc, int wc,
                                                        int hc, double cs)
{
    const long long np = (long long)A.nx * A.ny;
    for (long long k = gtid(); k < np; k += gstride()) {
        const int j = (int)(k / A.nx), i = (int)(k - (long long)j * A.nx);
        const int px = min(i * A.stride, w - A.ps), py = min(j * A.stride, h - A.ps);
        const FlowTaps t = flow_taps(wc, hc, (px + 0.5 * (A.ps - 1)) / cs, (py + 0.5 * (A.ps - 1)) / cs);
        const double2 gk = A.gpu[k];
        fx_add(gUc + 2 * t.i00, cs * t.w00 * gk.x);
        fx_add(gUc + 2 * t.i00 + 1, cs * t.w00 * gk.y);
        fx_add(gUc + 2 * t.i10, cs * t.w10 * gk.x);
        fx_add(gUc + 2 * t.i10 + 1, cs * t.w10 * gk.y);
        fx_add(gUc + 2 * t.i01, cs * t.w01 * gk.x);
        fx_add(gUc + 2 * t.i01 + 1, cs * t.w01 * gk.y);
        fx_add(gUc + 2 * t.i11, cs * t.w11 * gk.x);
        fx_add(gUc + 2 * t.i11 + 1, cs * t.w11 * gk.y);
    }
}

// Pyramid transpose: fine(a, b) += sum_{X, Y} Wx(a <- X) Wy(b <- Y) coarse(X, Y), with
// Wx(a <- X) = sum of k[i + 2] over i in -2..2 with clamp(2X + i) == a, k = [1 4 6 4 1] / 16.
__device__ __forceinline__ double tw5(int a, int X, int n)
{
    const double k[5] = {0.0625, 0.25, 0.375, 0.25, 0.0625};
    double s = 0.0;
    for (int i = -2; i <= 2; ++i)
        if (clampi(2 * X + i, 0, n - 1) == a) s += k[i + 2];
    return s;
}

__global__ void __launch_bounds__(256) pyr_bwd_kernel(const double* __restrict__ gc, int wc, int hc, int pc, double* gf,
                                                      int wf, int hf, int pf)
{
    PIX_LOOP(wf, hf)
    double acc = 0.0;
    for (int Y = max(0, (y - 2) / 2 - 1); Y <= min(hc - 1, (y + 2) / 2 + 1); ++Y) {
        const double wy = tw5(y, Y, hf);
        if (wy == 0.0) continue;
        for (int X = max(0, (x - 2) / 2 - 1); X <= min(wc - 1, (x + 2) / 2 + 1); ++X) {
            const double wx = tw5(x, X, wf);
            if (wx != 0.0) acc = fma(wx * wy, gc[(long long)Y * pc + X], acc);
        }
    }
    gf[(long long)y * pf + x] += acc;
    PIX_END
}

// Start of a level's refinement adjoint, U_out = U_d + dU: the flow adjoint goes to the
// increment planes and to the densified-flow adjoint.
__global__ void __launch_bounds__(256) start_flow_kernel(Lvl64 L, const double2* __restrict__ gin)
{
    PIX_LOOP(L.w, L.h)
    const double2 v = gin[g];
    const long long o = (long long)y * L.pitch + x;
    GA(ADJ_GDU)[o] = v.x;
    GA(ADJ_GDU + 1)[o] = v.y;
    L.gU[g] = v;
    PIX_END
}

// Final up-scaling (Sec. 3.1): out(x) = factor * in(x / factor), bilinear with clamping, and its
// transpose (fixed-point scatter into the coarse field's accumulator).
__global__ void __launch_bounds__(256) upsample64_kernel(const double2* __restrict__ in, int wi, int hi, double factor,
                                                         double2* out, int wo, int ho)
{
    PIX_LOOP(wo, ho)
    const FlowTaps t = flow_taps(wi, hi, x / factor, y / factor);
    const double2 a = in[t.i00], b = in[t.i10], c = in[t.i01], d = in[t.i11];
    out[g] = make_double2(factor * (t.w00 * a.x + t.w10 * b.x + t.w01 * c.x + t.w11 * d.x),
                          factor * (t.w00 * a.y + t.w10 * b.y + t.w01 * c.y + t.w11 * d.y));
    PIX_END
}

__global__ void __launch_bounds__(256) upsample_bwd_kernel(const double2* __restrict__ gout, int wo, int ho,
                                                           double factor, unsigned long long* gin, int wi, int hi)
{
    PIX_LOOP(wo, ho)
    const FlowTaps t = flow_taps(wi, hi, x / factor, y / factor);
    const double2 gk = gout[g];
    fx_add(gin + 2 * t.i00, factor * t.w00 * gk.x);
    fx_add(gin + 2 * t.i00 + 1, factor * t.w00 * gk.y);
    fx_add(gin + 2 * t.i10, factor * t.w10 * gk.x);
    fx_add(gin + 2 * t.i10 + 1, factor * t.w10 * gk.y);
    fx_add(gin + 2 * t.i01, factor * t.w01 * gk.x);
    fx_add(gin + 2 * t.i01 + 1, factor * t.w01 * gk.y);
    fx_add(gin + 2 * t.i11, factor * t.w11 * gk.x);
    fx_add(gin + 2 * t.i11 + 1, factor * t.w11 * gk.y);
    PIX_END
}

__global__ void __launch_bounds__(256) f2_to_d2_kernel(const float2* __restrict__ in, double2* out, long long n)
{
    for (long long g = gtid(); g < n; g += gstride()) out[g] = make_double2((double)in[g].x, (double)in[g].y);
}

__global__ void __launch_bounds__(256) d2_to_f2_kernel(const double2* __restrict__ in, float2* out, long long n)
{
    for (long long g = gtid(); g < n; g += gstride()) out[g] = make_float2((float)in[g].x, (float)in[g].y);
}

// out (float, pitch) = scale * in (double, pitch).
__global__ void __launch_bounds__(256) scale_out_kernel(const double* __restrict__ in, int ipitch, float* out,
                                                        int opitch, int w, int h, double scale)
{
    PIX_LOOP(w, h)
    out[(long long)y * opitch + x] = (float)(scale * in[(long long)y * ipitch + x]);
    PIX_END
}

// ================================== launchers ===============================================
static int grid_of(long long n, const LaunchCfg& lc)
{
    long long b = (n + 255) / 256;
    const long long cap = (long long)lc.sm_count * lc.max_blocks_256;
    return (int)std::max(1LL, std::min(b, cap));
}

#define LAUNCH(kernel, n, ...) kernel<<<grid_of((n), lc), 256, 0, s>>>(__VA_ARGS__)

cudaError_t launch_prep64(const float* I, int w, int h, int in_pitch, double scale, double* S, int pitch,
                          const LaunchCfg& lc, cudaStream_t s)
{
    LAUNCH(prep64_kernel, (long long)w * h, I, w, h, in_pitch, scale, S, pitch);
    return cudaGetLastError();
}

cudaError_t launch_pyr64(const double* in, int win, int hin, int pin, double* out, int wout, int hout, int pout,
                         const LaunchCfg& lc, cudaStream_t s)
{
    LAUNCH(pyr64_kernel, (long long)wout * hout, in, win, hin, pin, out, wout, hout, pout);
    return cudaGetLastError();
}

cudaError_t launch_uinit64(const Dens64& A, int w, int h, const double2* Uc, int wc, int hc, double cs,
                           const float2* frozen, double2* pu, const LaunchCfg& lc, cudaStream_t s)
{
    LAUNCH(uinit64_kernel, (long long)A.nx * A.ny, A, w, h, Uc, wc, hc, cs, frozen, pu);
    return cudaGetLastError();
}

cudaError_t launch_densify64(const double* S0, const double* S1, int w, int h, int pitch, const Dens64& A,
                             const double2* Uc, int wc, int hc, double cs, double2* Ud, const LaunchCfg& lc,
                             cudaStream_t s)
{
    LAUNCH(densify64_kernel, (long long)w * h, S0, S1, w, h, pitch, A, Uc, wc, hc, cs, Ud);
    return cudaGetLastError();
}

cudaError_t launch_ref64_prepare(const Lvl64& L, const LaunchCfg& lc, cudaStream_t s)
{
    const long long n = (long long)L.w * L.h;
    LAUNCH(ref64_prepare_kernel, n, L);
    LAUNCH(ref64_deriv1_kernel, n, L);
    LAUNCH(ref64_deriv2_kernel, n, L);
    return cudaGetLastError();
}

cudaError_t launch_ref64_weights(const Lvl64& L, const LaunchCfg& lc, cudaStream_t s)
{
    LAUNCH(ref64_weights_kernel, (long long)L.w * L.h, L);
    return cudaGetLastError();
}

cudaError_t launch_ref64_sor(const Lvl64& L, int colour, const LaunchCfg& lc, cudaStream_t s)
{
    LAUNCH(ref64_sor_kernel, (long long)L.h * ((L.w + 1) / 2), L, colour);
    return cudaGetLastError();
}

cudaError_t launch_ref64_apply(const Lvl64& L, double2* Uout, const LaunchCfg& lc, cudaStream_t s)
{
    LAUNCH(ref64_apply_kernel, (long long)L.w * L.h, L, Uout);
    return cudaGetLastError();
}

cudaError_t launch_loss(const float* I0, const float* I1, int w, int h, int pitch, int C, const float2* flow, float eps,
                        double* partials, int max_partials, double* loss_out, float2* gflow, float* gI0,
                        unsigned long long* gI1acc, const LaunchCfg& lc, cudaStream_t s)
{
    const long long n = (long long)w * h;
    int blocks = grid_of(n, lc);
    if (blocks > max_partials) blocks = max_partials;
    const double inv = 1.0 / (double)(n * C);
    loss_kernel<<<blocks, 256, 0, s>>>(I0, I1, w, h, pitch, C, flow, (double)eps, inv, partials, gflow, gI0, gI1acc);
    loss_finalize_kernel<<<1, 32, 0, s>>>(partials, blocks, inv, loss_out);
    return cudaGetLastError();
}

cudaError_t launch_fx_to_float(const unsigned long long* acc, int apitch, float* out, int opitch, int w, int h,
                               double scale, bool accumulate, const LaunchCfg& lc, cudaStream_t s)
{
    LAUNCH(fx_out_kernel<float>, (long long)w * h, acc, apitch, out, opitch, w, h, scale, accumulate ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_fx_to_double(const unsigned long long* acc, int apitch, double* out, int opitch, int w, int h,
                                double scale, bool accumulate, const LaunchCfg& lc, cudaStream_t s)
{
    LAUNCH(fx_out_kernel<double>, (long long)w * h, acc, apitch, out, opitch, w, h, scale, accumulate ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_sor_bwd(const Lvl64& L, const double* st_du, const double* st_dv, int colour, const LaunchCfg& lc,
                           cudaStream_t s)
{
    const long long n = (long long)L.h * ((L.w + 1) / 2);
    LAUNCH(sor_bwd_p_kernel, n, L, st_du, st_dv, colour);
    LAUNCH(sor_bwd_q_kernel, n, L, st_du, st_dv, 1 - colour);
    return cudaGetLastError();
}

cudaError_t launch_weights_bwd(const Lvl64& L, const double* st_du, const double* st_dv, const LaunchCfg& lc,
                               cudaStream_t s)
{
    const long long n = (long long)L.w * L.h;
    LAUNCH(weights_bwd_kernel, n, L, st_du, st_dv);
    LAUNCH(smooth_bwd_kernel, n, L);
    return cudaGetLastError();
}

cudaError_t launch_deriv_warp_bwd(const Lvl64& L, const LaunchCfg& lc, cudaStream_t s)
{
    const long long n = (long long)L.w * L.h;
    LAUNCH(deriv_bwd_local_kernel, n, L);
    LAUNCH(deriv_bwd_second_kernel, n, L);
    LAUNCH(deriv_bwd_first_kernel, n, L);
    LAUNCH(warp_bwd_kernel, n, L);
    return cudaGetLastError();
}

cudaError_t launch_start_flow(const Lvl64& L, const double2* g, const LaunchCfg& lc, cudaStream_t s)
{
    LAUNCH(start_flow_kernel, (long long)L.w * L.h, L, g);
    return cudaGetLastError();
}

cudaError_t launch_dens_bwd(const Lvl64& L, const Dens64& A, const LaunchCfg& lc, cudaStream_t s)
{
    LAUNCH(dens_bwd_pix_kernel, (long long)L.w * L.h, L, A);
    const long long np = (long long)A.nx * A.ny;
    const long long b = std::min((np * 32 + 127) / 128, (long long)lc.sm_count * 16);
    dens_bwd_patch_kernel<<<(int)std::max(1LL, b), 128, 0, s>>>(L, A);
    return cudaGetLastError();
}

cudaError_t launch_uinit_bwd(const Dens64& A, int w, int h, unsigned long long* gUc, int wc, int hc, double cs,
                             const LaunchCfg& lc, cudaStream_t s)
{
    LAUNCH(uinit_bwd_kernel, (long long)A.nx * A.ny, A, w, h, gUc, wc, hc, cs);
    return cudaGetLastError();
}

cudaError_t launch_search_ift_bwd(const Lvl64& L, const Dens64& A, const float2* frozen, unsigned long long* gS0acc,
                                  int dof, const LaunchCfg& lc, cudaStream_t s)
{
    const long long np = (long long)A.nx * A.ny;
    if (np <= 0) return cudaSuccess;
    const int blocks = (int)std::min<long long>((np * 32 + 127) / 128, (long long)lc.sm_count * 16);
    search_ift_bwd_kernel<<<blocks, 128, 0, s>>>(L, A, frozen, gS0acc, dof);
    return cudaGetLastError();
}

cudaError_t launch_pyr_bwd(const double* gc, int wc, int hc, int pc, double* gf, int wf, int hf, int pf,
                           const LaunchCfg& lc, cudaStream_t s)
{
    LAUNCH(pyr_bwd_kernel, (long long)wf * hf, gc, wc, hc, pc, gf, wf, hf, pf);
    return cudaGetLastError();
}

cudaError_t launch_upsample64(const double2* in, int wi, int hi, double factor, double2* out, int wo, int ho,
                              const LaunchCfg& lc, cudaStream_t s)
{
    LAUNCH(upsample64_kernel, (long long)wo * ho, in, wi, hi, factor, out, wo, ho);
    return cudaGetLastError();
}

cudaError_t launch_upsample_bwd(const double2* gout, int wo, int ho, double factor, unsigned long long* gin, int wi,
                                int hi, const LaunchCfg& lc, cudaStream_t s)
{
    LAUNCH(upsample_bwd_kernel, (long long)wo * ho, gout, wo, ho, factor, gin, wi, hi);
    return cudaGetLastError();
}

cudaError_t launch_f2_to_d2(const float2* in, double2* out, long long n, const LaunchCfg& lc, cudaStream_t s)
{
    LAUNCH(f2_to_d2_kernel, n, in, out, n);
    return cudaGetLastError();
}

cudaError_t launch_d2_to_f2(const double2* in, float2* out, long long n, const LaunchCfg& lc, cudaStream_t s)
{
    LAUNCH(d2_to_f2_kernel, n, in, out, n);
    return cudaGetLastError();
}

cudaError_t launch_scale_out(const double* in, int ipitch, float* out, int opitch, int w, int h, double scale,
                             const LaunchCfg& lc, cudaStream_t s)
{
    LAUNCH(scale_out_kernel, (long long)w * h, in, ipitch, out, opitch, w, h, scale);
    return cudaGetLastError();
}

}  // namespace dis
