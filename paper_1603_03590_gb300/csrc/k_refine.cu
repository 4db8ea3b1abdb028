// Variational refinement of DIS (Alg. 1 step 5, Sec. 2.3).
//
// Energy E = int delta Psi(E_I) + gamma Psi(E_G) + alpha Psi(E_S), Psi(a^2) = sqrt(a^2 + eps^2),
// eps = 0.001, with the normalised intensity term E_I = beta0 (I_x du + I_y dv + I_z)^2, the
// gradient term E_G = betax (I_xx du + I_xy dv + I_xz)^2 + betay (I_xy du + I_yy dv + I_yz)^2
// (beta = (|grad_2 .|^2 + 0.01)^-1), summed over channels inside each Psi, and the smoothness
// term E_S = |grad(u + du)|^2 + |grad(v + dv)|^2.  Discretisation: I1 warped once by U;
// first derivatives are Sobel/8 of (I0 + I1w)/2, second derivatives Sobel/8 of those,
// I_z = I1w - I0, I_xz / I_yz the Sobel/8 differences of I1w and I0; smoothness by central
// differences (replicated border) and 4-neighbour edge weights (psiS_p + psiS_q)/2.
// theta_vo lagged-nonlinearity passes each freeze psi = weight * Psi'(.) and run theta_vi
// red-black SOR sweeps (red = (x + y) even first) on the per-pixel 2x2 systems.
//
// Kernels (thread per pixel, flattened over all jobs of a phase):
//   warp     I1w = I1(x + U), dU = 0                                  (once per level)
//   deriv1   I_x, I_y, I_z, I_xz, I_yz                                 (once per level)
//   deriv2   I_xx, I_xy, I_yy, betas -> 9 data values per channel      (once per level)
//   weights  A (3), b (2), psiS from the data values and U + dU        (per outer pass)
//   sor      one colour of one sweep                                   (2 per sweep)
//   apply    U += dU                                                   (once per level)
#include <algorithm>

#include "dis_device.cuh"

namespace dis {

#define DIS_PIX_LOOP(BASE)                                                               \
    for (long long g = gtid(); g < total; g += gstride()) {                              \
        const LevelJob& J = job_ref(js, find_job(js, g, &LevelJob::BASE));               \
        const long long k = g - J.BASE;                                                  \
        const int w = J.w, h = J.h, pitch = J.pitch;                                     \
        const int y = (int)(k / w), x = (int)(k - (long long)y * w);                     \
        const long long o = (long long)y * pitch + x;                                    \
        (void)h;

#define DIS_PIX_END }

__global__ void __launch_bounds__(256) refine_warp_kernel(const __grid_constant__ Jobs<LevelJob> js, long long total)
{
    DIS_PIX_LOOP(pix_base)
    const float2 U = J.U[k];
    for (int c = 0; c < J.C; ++c)
        J.rs[rs_mid(J.C, c, 0) * J.plane + o] = sample_shift(J.P1 + c * J.plane, w, h, pitch, x, y, U.x, U.y);
    J.rs[rs_du(J.C, 0) * J.plane + o] = 0.0f;
    J.rs[rs_du(J.C, 1) * J.plane + o] = 0.0f;
    DIS_PIX_END
}

// Sobel/8 of plane P at (x, y) with replicated border.
__device__ __forceinline__ void sobel_at(const float* __restrict__ P, int pitch, int xl, int x, int xr,
                                         long long ru, long long rc, long long rd, float& gx, float& gy)
{
    const float a = P[ru + xl], b = P[ru + x], c = P[ru + xr];
    const float d = P[rc + xl], f = P[rc + xr];
    const float p = P[rd + xl], q = P[rd + x], s = P[rd + xr];
    gx = 0.125f * ((c - a) + 2.0f * (f - d) + (s - p));
    gy = 0.125f * ((p - a) + 2.0f * (q - b) + (s - c));
}

__global__ void __launch_bounds__(256) refine_deriv1_kernel(const __grid_constant__ Jobs<LevelJob> js, long long total)
{
    DIS_PIX_LOOP(pix_base)
    const int xl = max(x - 1, 0), xr = min(x + 1, w - 1);
    const long long ru = (long long)max(y - 1, 0) * pitch, rc = (long long)y * pitch,
                    rd = (long long)min(y + 1, h - 1) * pitch;
    for (int c = 0; c < J.C; ++c) {
        const float* P0 = J.P0 + c * J.plane;
        const float* W1 = J.rs + rs_mid(J.C, c, 0) * J.plane;
        float sx0, sy0, sx1, sy1;
        sobel_at(P0, pitch, xl, x, xr, ru, rc, rd, sx0, sy0);
        sobel_at(W1, pitch, xl, x, xr, ru, rc, rd, sx1, sy1);
        J.rs[rs_mid(J.C, c, 1) * J.plane + o] = 0.5f * (sx0 + sx1);
        J.rs[rs_mid(J.C, c, 2) * J.plane + o] = 0.5f * (sy0 + sy1);
        J.rs[rs_mid(J.C, c, 3) * J.plane + o] = W1[o] - P0[o];
        J.rs[rs_mid(J.C, c, 4) * J.plane + o] = sx1 - sx0;
        J.rs[rs_mid(J.C, c, 5) * J.plane + o] = sy1 - sy0;
    }
    DIS_PIX_END
}

__global__ void __launch_bounds__(256) refine_deriv2_kernel(const __grid_constant__ Jobs<LevelJob> js, long long total)
{
    DIS_PIX_LOOP(pix_base)
    const int xl = max(x - 1, 0), xr = min(x + 1, w - 1);
    const long long ru = (long long)max(y - 1, 0) * pitch, rc = (long long)y * pitch,
                    rd = (long long)min(y + 1, h - 1) * pitch;
    for (int c = 0; c < J.C; ++c) {
        const float* Ixp = J.rs + rs_mid(J.C, c, 1) * J.plane;
        const float* Iyp = J.rs + rs_mid(J.C, c, 2) * J.plane;
        float Ixx, Ixy, Iyx, Iyy;
        sobel_at(Ixp, pitch, xl, x, xr, ru, rc, rd, Ixx, Ixy);
        sobel_at(Iyp, pitch, xl, x, xr, ru, rc, rd, Iyx, Iyy);
        (void)Iyx;
        const float Ix = Ixp[o], Iy = Iyp[o];
        const float Iz = J.rs[rs_mid(J.C, c, 3) * J.plane + o];
        const float Ixz = J.rs[rs_mid(J.C, c, 4) * J.plane + o];
        const float Iyz = J.rs[rs_mid(J.C, c, 5) * J.plane + o];
        const float s0 = 1.0f / sqrtf(Ix * Ix + Iy * Iy + 0.01f);
        const float sx = 1.0f / sqrtf(Ixx * Ixx + Ixy * Ixy + 0.01f);
        const float sy = 1.0f / sqrtf(Ixy * Ixy + Iyy * Iyy + 0.01f);
        float* D = J.rs + rs_dat(J.C, c, 0) * J.plane + o;
        D[0 * J.plane] = s0 * Ix;
        D[1 * J.plane] = s0 * Iy;
        D[2 * J.plane] = s0 * Iz;
        D[3 * J.plane] = sx * Ixx;
        D[4 * J.plane] = sx * Ixy;
        D[5 * J.plane] = sx * Ixz;
        D[6 * J.plane] = sy * Ixy;
        D[7 * J.plane] = sy * Iyy;
        D[8 * J.plane] = sy * Iyz;
    }
    DIS_PIX_END
}

__global__ void __launch_bounds__(256) refine_weights_kernel(const __grid_constant__ Jobs<LevelJob> js,
                                                             long long total, float delta, float gamma, float alpha)
{
    const float eps2 = 1.0e-6f;
    DIS_PIX_LOOP(pix_base)
    const long long pl = J.plane;
    const float* du_p = J.rs + rs_du(J.C, 0) * pl;
    const float* dv_p = J.rs + rs_du(J.C, 1) * pl;
    const float du = du_p[o], dv = dv_p[o];
    float EI = 0.0f, EG = 0.0f;
    for (int c = 0; c < J.C; ++c) {
        const float* D = J.rs + rs_dat(J.C, c, 0) * pl + o;
        const float eI = fmaf(D[0], du, fmaf(D[pl], dv, D[2 * pl]));
        const float eX = fmaf(D[3 * pl], du, fmaf(D[4 * pl], dv, D[5 * pl]));
        const float eY = fmaf(D[6 * pl], du, fmaf(D[7 * pl], dv, D[8 * pl]));
        EI = fmaf(eI, eI, EI);
        EG = fmaf(eX, eX, fmaf(eY, eY, EG));
    }
    const float psiI = delta / (2.0f * sqrtf(EI + eps2));
    const float psiG = gamma / (2.0f * sqrtf(EG + eps2));
    float a11 = 0.0f, a12 = 0.0f, a22 = 0.0f, b1 = 0.0f, b2 = 0.0f;
    for (int c = 0; c < J.C; ++c) {
        const float* D = J.rs + rs_dat(J.C, c, 0) * pl + o;
        const float d0 = D[0], d1 = D[pl], d2 = D[2 * pl], d3 = D[3 * pl], d4 = D[4 * pl], d5 = D[5 * pl];
        const float d6 = D[6 * pl], d7 = D[7 * pl], d8 = D[8 * pl];
        a11 += psiI * d0 * d0 + psiG * (d3 * d3 + d6 * d6);
        a12 += psiI * d0 * d1 + psiG * (d3 * d4 + d6 * d7);
        a22 += psiI * d1 * d1 + psiG * (d4 * d4 + d7 * d7);
        b1 -= psiI * d2 * d0 + psiG * (d5 * d3 + d8 * d6);
        b2 -= psiI * d2 * d1 + psiG * (d5 * d4 + d8 * d7);
    }
    // smoothness: central differences of u + du, replicated border
    const int xl = max(x - 1, 0), xr = min(x + 1, w - 1), yu = max(y - 1, 0), yd = min(y + 1, h - 1);
    const long long fl = (long long)y * w + xl, fr = (long long)y * w + xr;
    const long long fu = (long long)yu * w + x, fd = (long long)yd * w + x;
    const long long ol = (long long)y * pitch + xl, orr = (long long)y * pitch + xr;
    const long long ou = (long long)yu * pitch + x, od = (long long)yd * pitch + x;
    const float2 Ul = J.U[fl], Ur = J.U[fr], Uu = J.U[fu], Ud = J.U[fd];
    const float ux = 0.5f * ((Ur.x + du_p[orr]) - (Ul.x + du_p[ol]));
    const float vx = 0.5f * ((Ur.y + dv_p[orr]) - (Ul.y + dv_p[ol]));
    const float uy = 0.5f * ((Ud.x + du_p[od]) - (Uu.x + du_p[ou]));
    const float vy = 0.5f * ((Ud.y + dv_p[od]) - (Uu.y + dv_p[ou]));
    const float ES = ux * ux + uy * uy + vx * vx + vy * vy;
    float* S = J.rs + rs_sys(J.C, 0) * pl + o;
    S[0] = a11;
    S[pl] = a12;
    S[2 * pl] = a22;
    S[3 * pl] = b1;
    S[4 * pl] = b2;
    S[5 * pl] = alpha / (2.0f * sqrtf(ES + eps2));
    DIS_PIX_END
}

// One colour of one red-black sweep: the pixels with (x + y) % 2 == colour.
__global__ void __launch_bounds__(256) refine_sor_kernel(const __grid_constant__ Jobs<LevelJob> js, long long total,
                                                         int colour, float omega)
{
    for (long long g = gtid(); g < total; g += gstride()) {
        const LevelJob& J = job_ref(js, find_job(js, g, &LevelJob::half_base));
        const long long k = g - J.half_base;
        const int w = J.w, h = J.h, pitch = J.pitch;
        const int hw = (w + 1) >> 1;
        const int y = (int)(k / hw);
        const int x = 2 * (int)(k - (long long)y * hw) + ((y + colour) & 1);
        if (x >= w) continue;
        const long long pl = J.plane;
        const long long o = (long long)y * pitch + x, f = (long long)y * w + x;
        const float* S = J.rs + rs_sys(J.C, 0) * pl;
        float* du_p = J.rs + rs_du(J.C, 0) * pl;
        float* dv_p = J.rs + rs_du(J.C, 1) * pl;
        const float ps_ = S[5 * pl + o];
        const float2 Up = J.U[f];
        float sw = 0.0f, r1 = S[3 * pl + o], r2 = S[4 * pl + o];
        const int nxs[4] = {x - 1, x + 1, x, x};
        const int nys[4] = {y, y, y - 1, y + 1};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int qx = nxs[q], qy = nys[q];
            if (qx < 0 || qx >= w || qy < 0 || qy >= h) continue;
            const long long oq = (long long)qy * pitch + qx;
            const float wq = 0.5f * (ps_ + S[5 * pl + oq]);
            const float2 Uq = J.U[(long long)qy * w + qx];
            sw += wq;
            r1 = fmaf(wq, (Uq.x + du_p[oq]) - Up.x, r1);
            r2 = fmaf(wq, (Uq.y + dv_p[oq]) - Up.y, r2);
        }
        const float m11 = S[o] + sw, m12 = S[pl + o], m22 = S[2 * pl + o] + sw;
        const float det = m11 * m22 - m12 * m12;
        if (det > 0.0f) {
            const float id = 1.0f / det;
            const float d1 = (m22 * r1 - m12 * r2) * id;
            const float d2 = (m11 * r2 - m12 * r1) * id;
            du_p[o] = (1.0f - omega) * du_p[o] + omega * d1;
            dv_p[o] = (1.0f - omega) * dv_p[o] + omega * d2;
        }
    }
}

__global__ void __launch_bounds__(256) refine_apply_kernel(const __grid_constant__ Jobs<LevelJob> js, long long total)
{
    DIS_PIX_LOOP(pix_base)
    float2 U = J.U[k];
    U.x += J.rs[rs_du(J.C, 0) * J.plane + o];
    U.y += J.rs[rs_du(J.C, 1) * J.plane + o];
    J.U[k] = U;
    DIS_PIX_END
}

cudaError_t launch_refine(const Jobs<LevelJob>& js, long long total_pix, long long total_half, const RefineArgs& a,
                          const LaunchCfg& lc, cudaStream_t s)
{
    if (total_pix <= 0) return cudaSuccess;
    const long long cap = (long long)lc.sm_count * lc.max_blocks_256;
    const int gp = (int)std::min<long long>((total_pix + 255) / 256, cap);
    const int gh = (int)std::min<long long>((total_half + 255) / 256, cap);
    refine_warp_kernel<<<gp, 256, 0, s>>>(js, total_pix);
    refine_deriv1_kernel<<<gp, 256, 0, s>>>(js, total_pix);
    refine_deriv2_kernel<<<gp, 256, 0, s>>>(js, total_pix);
    for (int ot = 0; ot < a.outer; ++ot) {
        refine_weights_kernel<<<gp, 256, 0, s>>>(js, total_pix, a.delta, a.gamma, a.alpha);
        for (int it = 0; it < a.inner; ++it) {
            refine_sor_kernel<<<gh, 256, 0, s>>>(js, total_half, 0, a.omega);
            refine_sor_kernel<<<gh, 256, 0, s>>>(js, total_half, 1, a.omega);
        }
    }
    refine_apply_kernel<<<gp, 256, 0, s>>>(js, total_pix);
    return cudaGetLastError();
}

// Single phases of the refinement, for the backward pass, which recomputes the forward states
// (derivatives, lagged weights, the increment before every half-sweep) level by level.
cudaError_t launch_refine_prepare(const Jobs<LevelJob>& js, long long total_pix, const LaunchCfg& lc, cudaStream_t s)
{
    const int gp = (int)std::min<long long>((total_pix + 255) / 256, (long long)lc.sm_count * lc.max_blocks_256);
    refine_warp_kernel<<<gp, 256, 0, s>>>(js, total_pix);
    refine_deriv1_kernel<<<gp, 256, 0, s>>>(js, total_pix);
    refine_deriv2_kernel<<<gp, 256, 0, s>>>(js, total_pix);
    return cudaGetLastError();
}

cudaError_t launch_refine_weights(const Jobs<LevelJob>& js, long long total_pix, const RefineArgs& a,
                                  const LaunchCfg& lc, cudaStream_t s)
{
    const int gp = (int)std::min<long long>((total_pix + 255) / 256, (long long)lc.sm_count * lc.max_blocks_256);
    refine_weights_kernel<<<gp, 256, 0, s>>>(js, total_pix, a.delta, a.gamma, a.alpha);
    return cudaGetLastError();
}

cudaError_t launch_refine_half_sweep(const Jobs<LevelJob>& js, long long total_half, int colour, float omega,
                                     const LaunchCfg& lc, cudaStream_t s)
{
    const int gh = (int)std::min<long long>((total_half + 255) / 256, (long long)lc.sm_count * lc.max_blocks_256);
    refine_sor_kernel<<<gh, 256, 0, s>>>(js, total_half, colour, omega);
    return cudaGetLastError();
}

}  // namespace dis
