// Variational refinement of DIS (Alg. 1 step 5, Sec. 2.3).
//
// Energy E = int delta Psi(E_I) + gamma Psi(E_G) + alpha Psi(E_S), Psi(a^2) = sqrt(a^2 + eps^2),
// eps = 0.001, with the normalised intensity term E_I = beta0 (I_x du + I_y dv + I_z)^2, the
// gradient term E_G = betax (I_xx du + I_xy dv + I_xz)^2 + betay (I_xy du + I_yy dv + I_yz)^2
// (beta = (|grad_2 .|^2 + 0.01)^-1), summed over channels inside each Psi, and the smoothness
// term E_S = |grad(u + du)|^2 + |grad(v + dv)|^2.  Discretisation: I1 warped once by U; with the
// mean image Ibar = (I0 + I1w)/2 and the temporal difference I_z = I1w - I0, first derivatives
// are Sobel/8 of Ibar, second derivatives Sobel/8 of those, I_xz / I_yz Sobel/8 of I_z (the
// difference of the two frames' Sobel derivatives); smoothness by central differences
// (replicated border) and 4-neighbour edge weights (psiS_p + psiS_q)/2.  theta_vo
// lagged-nonlinearity passes each freeze psi = weight * Psi'(.) and run theta_vi red-black SOR
// sweeps (red = (x + y) even first) on the per-pixel 2x2 systems.
//
// Every form starts with refine_prep (thread per pixel): I1w = I1(x + U) and the two planes per
// channel every later step derives its data from, Ibar and I_z.
//
// Fused form (the default): one launch per outer pass (or two, each with half of its
// half-sweeps and half the halo).  A block takes a 32x32 tile and, in shared memory,
//   - loads Ibar and I_z of the tile with a halo of K + 2 (K = the launch's half-sweeps),
//   - forms I_x, I_y on a halo of K + 1 and from them, per pixel of a halo of K, the nine data
//     values of each channel and the lagged 2x2 system (the increment at the pass start comes
//     from global memory),
//   - loads U and that increment on a halo of K + 1 and forms the smoothness weights,
//   - runs the K red-black half-sweeps with a block barrier between them (after half-sweep j
//     only pixels within K - 1 - j of the tile still need to be exact, so each sweeps a smaller
//     square), and writes the tile's increment.
// Nothing but Ibar, I_z, U and the increments crosses DRAM.
// Per-sweep form (dis_set_refine_fusion 0, or more than 5 sweeps per pass): thread-per-pixel
// kernels write I_x, I_y, then the data values, then per pass the systems and one launch per
// half-sweep.  Both forms share every arithmetic step (refine_dvals, refine_energy_acc,
// refine_psi, refine_system_acc, refine_smooth_weight, refine_sor_update), so they agree bit
// for bit.
#include <algorithm>
#include <stdint.h>
#include <type_traits>

#include "dis_device.cuh"

namespace dis {

// Planes of the refinement scratch (rs_mid slots of channel c): the mean image and I_z (every
// form), I_x and I_y (per-sweep form).  The fused form keeps its increments in rs_du, in the
// fifth and sixth intermediate planes of channel 0 and in the first two system planes.
__host__ __device__ inline int rp_bar(int C, int c) { return rs_mid(C, c, 0); }
__host__ __device__ inline int rp_iz(int C, int c) { return rs_mid(C, c, 1); }
__host__ __device__ inline int rp_ix(int C, int c) { return rs_mid(C, c, 2); }
__host__ __device__ inline int rp_iy(int C, int c) { return rs_mid(C, c, 3); }

#define DIS_PIX_LOOP(BASE)                                                               \
    for (long long g = gtid(); g < total; g += gstride()) {                              \
        const LevelJob& J = job_ref(js, find_job(js, g, &LevelJob::BASE));               \
        const int k = (int)(g - J.BASE); /* < w * h < 2^31 */                            \
        const int w = J.w, h = J.h, pitch = J.pitch;                                     \
        const int y = k / w, x = k - y * w;                                              \
        const long long o = (long long)y * pitch + x;                                    \
        (void)h;

#define DIS_PIX_END }

// ---------------------------------------------------------------- shared arithmetic
// Sobel/8 of a 3x3 neighbourhood v (row-major, centre v[4]).  (2 (f - d) is exact, so whether
// the compiler fuses it into the following add does not change the result.)
__device__ __forceinline__ float sobel_x9(const float (&v)[9])
{
    return 0.125f * (((v[2] - v[0]) + 2.0f * (v[5] - v[3])) + (v[8] - v[6]));
}
__device__ __forceinline__ float sobel_y9(const float (&v)[9])
{
    return 0.125f * (((v[6] - v[0]) + 2.0f * (v[7] - v[1])) + (v[8] - v[2]));
}

// The nine data values of one channel at a pixel, from the 3x3 neighbourhoods of I_x, I_y and
// I_z around it: sqrt(beta0) (I_x, I_y, I_z), sqrt(betax) (I_xx, I_xy, I_xz), sqrt(betay)
// (I_xy, I_yy, I_yz), with I_xx = Sobel_x(I_x), I_xy = Sobel_y(I_x), I_yy = Sobel_y(I_y).
__device__ __forceinline__ void refine_dvals(const float (&ix)[9], const float (&iy)[9], const float (&iz)[9],
                                             float (&d)[9])
{
    const float Ixx = sobel_x9(ix), Ixy = sobel_y9(ix), Iyy = sobel_y9(iy);
    const float Ixz = sobel_x9(iz), Iyz = sobel_y9(iz);
    const float Ix = ix[4], Iy = iy[4], Iz = iz[4];
    // sqrt(beta) by the hardware reciprocal square root (2 ulp): the normalisers only scale the
    // rows of the data terms
    const float s0 = rsqrtf(fmaf(Ix, Ix, fmaf(Iy, Iy, 0.01f)));
    const float sx = rsqrtf(fmaf(Ixx, Ixx, fmaf(Ixy, Ixy, 0.01f)));
    const float sy = rsqrtf(fmaf(Ixy, Ixy, fmaf(Iyy, Iyy, 0.01f)));
    d[0] = s0 * Ix;
    d[1] = s0 * Iy;
    d[2] = s0 * Iz;
    d[3] = sx * Ixx;
    d[4] = sx * Ixy;
    d[5] = sx * Ixz;
    d[6] = sy * Ixy;
    d[7] = sy * Iyy;
    d[8] = sy * Iyz;
}

// One channel's share of the data energies at increment (du, dv).
__device__ __forceinline__ void refine_energy_acc(const float (&d)[9], float du, float dv, float& EI, float& EG)
{
    const float eI = fmaf(d[0], du, fmaf(d[1], dv, d[2]));
    const float eX = fmaf(d[3], du, fmaf(d[4], dv, d[5]));
    const float eY = fmaf(d[6], du, fmaf(d[7], dv, d[8]));
    EI = fmaf(eI, eI, EI);
    EG = fmaf(eX, eX, fmaf(eY, eY, EG));
}

// Lagged weights psi = weight * Psi'(E) = weight / (2 sqrt(E + eps^2)) of the two data terms
// (hardware reciprocal square root, 2 ulp).
__device__ __forceinline__ void refine_psi(float EI, float EG, float delta, float gamma, float& psiI, float& psiG)
{
    const float eps2 = 1.0e-6f;
    psiI = (0.5f * delta) * rsqrtf(EI + eps2);
    psiG = (0.5f * gamma) * rsqrtf(EG + eps2);
}

// One channel's share of the 2x2 data system A dU = b with the weights psi frozen.
__device__ __forceinline__ void refine_system_acc(const float (&d)[9], float psiI, float psiG, float& a11, float& a12,
                                                  float& a22, float& b1, float& b2)
{
    const float p0 = __fmul_rn(psiI, d[0]), p1 = __fmul_rn(psiI, d[1]), p2 = __fmul_rn(psiI, d[2]);
    const float q3 = __fmul_rn(psiG, d[3]), q4 = __fmul_rn(psiG, d[4]), q5 = __fmul_rn(psiG, d[5]);
    const float q6 = __fmul_rn(psiG, d[6]), q7 = __fmul_rn(psiG, d[7]), q8 = __fmul_rn(psiG, d[8]);
    a11 = __fadd_rn(a11, fmaf(p0, d[0], fmaf(q3, d[3], __fmul_rn(q6, d[6]))));
    a12 = __fadd_rn(a12, fmaf(p0, d[1], fmaf(q3, d[4], __fmul_rn(q6, d[7]))));
    a22 = __fadd_rn(a22, fmaf(p1, d[1], fmaf(q4, d[4], __fmul_rn(q7, d[7]))));
    b1 = __fsub_rn(b1, fmaf(p2, d[0], fmaf(q5, d[3], __fmul_rn(q8, d[6]))));
    b2 = __fsub_rn(b2, fmaf(p2, d[1], fmaf(q5, d[4], __fmul_rn(q8, d[7]))));
}

// Smoothness weight alpha * Psi'(|grad(u + du)|^2) from the four central differences.
__device__ __forceinline__ float refine_smooth_weight(float ux, float uy, float vx, float vy, float alpha)
{
    const float ES = fmaf(ux, ux, fmaf(uy, uy, fmaf(vx, vx, __fmul_rn(vy, vy))));
    return (0.5f * alpha) * rsqrtf(ES + 1.0e-6f);
}

// Central difference 0.5 * ((U_r + dU_r) - (U_l + dU_l)) of one component.
__device__ __forceinline__ float refine_cdiff(float Ur, float dur, float Ul, float dul)
{
    return 0.5f * ((Ur + dur) - (Ul + dul));
}

// One SOR update of pixel p: neighbours q (left, right, up, down; `in[q]` false outside the
// image) with smoothness weights psq, flows Uq and increments dq; updates (du, dv) in place.
// dof 1 (stereo, the vertical degree of freedom removed): dv stays, du solves the scalar
// equation (a11 + sum w) du = b1 + sum w (Uq.x + duq - Up.x).
__device__ __forceinline__ void refine_sor_update(float a11, float a12, float a22, float b1, float b2, float ps_p,
                                                  const bool (&in)[4], const float (&psq)[4], const float2 (&Uq)[4],
                                                  const float (&duq)[4], const float (&dvq)[4], float2 Up,
                                                  float omega, int dof, float& du, float& dv)
{
    if (dof == 1) {
        float sw = 0.0f, r1 = b1;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (!in[q]) continue;
            const float wq = 0.5f * (ps_p + psq[q]);
            sw += wq;
            r1 = fmaf(wq, (Uq[q].x + duq[q]) - Up.x, r1);
        }
        const float m11 = a11 + sw;
        if (m11 > 0.0f) du = (1.0f - omega) * du + omega * __fdividef(r1, m11);
        return;
    }
    float sw = 0.0f, r1 = b1, r2 = b2;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if (!in[q]) continue;
        const float wq = 0.5f * (ps_p + psq[q]);
        sw += wq;
        r1 = fmaf(wq, (Uq[q].x + duq[q]) - Up.x, r1);
        r2 = fmaf(wq, (Uq[q].y + dvq[q]) - Up.y, r2);
    }
    const float m11 = a11 + sw, m12 = a12, m22 = a22 + sw;
    const float det = m11 * m22 - m12 * m12;
    if (det > 0.0f) {
        const float id = __fdividef(1.0f, det);  // hardware reciprocal (det < 2^126: the weights are bounded)
        const float d1 = (m22 * r1 - m12 * r2) * id;
        const float d2 = (m11 * r2 - m12 * r1) * id;
        du = (1.0f - omega) * du + omega * d1;
        dv = (1.0f - omega) * dv + omega * d2;
    }
}

// ---------------------------------------------------------------- thread-per-pixel kernels
// I1w = I1(x + U) per channel, then Ibar = (I0 + I1w)/2 and I_z = I1w - I0; zero_du: also
// zero the increment planes (the per-sweep form starts from them).
__global__ void __launch_bounds__(256) refine_prep_kernel(const __grid_constant__ Jobs<LevelJob> js, long long total,
                                                          int zero_du)
{
    DIS_PIX_LOOP(pix_base)
    const float2 U = J.U[k];
    for (int c = 0; c < J.C; ++c) {
        const float w1 = sample_shift(J.P1 + c * J.plane, w, h, pitch, x, y, U.x, U.y);
        const float p0 = J.P0[c * J.plane + o];
        J.rs[rp_bar(J.C, c) * J.plane + o] = 0.5f * (p0 + w1);
        J.rs[rp_iz(J.C, c) * J.plane + o] = w1 - p0;
    }
    if (zero_du) {
        J.rs[rs_du(J.C, 0) * J.plane + o] = 0.0f;
        J.rs[rs_du(J.C, 1) * J.plane + o] = 0.0f;
    }
    DIS_PIX_END
}

// 3x3 neighbourhood of plane P around (x, y), replicated border (xl, xr, row offsets clamped).
__device__ __forceinline__ void gather3x3(const float* __restrict__ P, int xl, int x, int xr, long long ru,
                                          long long rc, long long rd, float (&v)[9])
{
    v[0] = P[ru + xl], v[1] = P[ru + x], v[2] = P[ru + xr];
    v[3] = P[rc + xl], v[4] = P[rc + x], v[5] = P[rc + xr];
    v[6] = P[rd + xl], v[7] = P[rd + x], v[8] = P[rd + xr];
}

// Per-sweep form: I_x, I_y = Sobel/8 of the mean image.
__global__ void __launch_bounds__(256) refine_grad_kernel(const __grid_constant__ Jobs<LevelJob> js, long long total)
{
    DIS_PIX_LOOP(pix_base)
    const int xl = max(x - 1, 0), xr = min(x + 1, w - 1);
    const long long ru = (long long)max(y - 1, 0) * pitch, rc = (long long)y * pitch,
                    rd = (long long)min(y + 1, h - 1) * pitch;
    for (int c = 0; c < J.C; ++c) {
        float v[9];
        gather3x3(J.rs + rp_bar(J.C, c) * J.plane, xl, x, xr, ru, rc, rd, v);
        J.rs[rp_ix(J.C, c) * J.plane + o] = sobel_x9(v);
        J.rs[rp_iy(J.C, c) * J.plane + o] = sobel_y9(v);
    }
    DIS_PIX_END
}

// Per-sweep form: the nine data values per channel.
__global__ void __launch_bounds__(256) refine_data_kernel(const __grid_constant__ Jobs<LevelJob> js, long long total)
{
    DIS_PIX_LOOP(pix_base)
    const int xl = max(x - 1, 0), xr = min(x + 1, w - 1);
    const long long ru = (long long)max(y - 1, 0) * pitch, rc = (long long)y * pitch,
                    rd = (long long)min(y + 1, h - 1) * pitch;
    for (int c = 0; c < J.C; ++c) {
        float ix[9], iy[9], iz[9], d[9];
        gather3x3(J.rs + rp_ix(J.C, c) * J.plane, xl, x, xr, ru, rc, rd, ix);
        gather3x3(J.rs + rp_iy(J.C, c) * J.plane, xl, x, xr, ru, rc, rd, iy);
        gather3x3(J.rs + rp_iz(J.C, c) * J.plane, xl, x, xr, ru, rc, rd, iz);
        refine_dvals(ix, iy, iz, d);
        float* D = J.rs + rs_dat(J.C, c, 0) * J.plane + o;
#pragma unroll
        for (int q = 0; q < 9; ++q) D[q * J.plane] = d[q];
    }
    DIS_PIX_END
}

// Lagged data system of pixel o from the data planes (per-sweep form), channel order as in the
// fused form.
__device__ __forceinline__ void refine_data_system(const float* __restrict__ rs, int C, long long pl, long long o,
                                                   float du, float dv, float delta, float gamma, float& a11,
                                                   float& a12, float& a22, float& b1, float& b2)
{
    float EI = 0.0f, EG = 0.0f;
    for (int c = 0; c < C; ++c) {
        float d[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) d[q] = rs[(rs_dat(C, c, 0) + q) * pl + o];
        refine_energy_acc(d, du, dv, EI, EG);
    }
    float psiI, psiG;
    refine_psi(EI, EG, delta, gamma, psiI, psiG);
    a11 = a12 = a22 = b1 = b2 = 0.0f;
    for (int c = 0; c < C; ++c) {
        float d[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) d[q] = rs[(rs_dat(C, c, 0) + q) * pl + o];
        refine_system_acc(d, psiI, psiG, a11, a12, a22, b1, b2);
    }
}

__global__ void __launch_bounds__(256) refine_weights_kernel(const __grid_constant__ Jobs<LevelJob> js,
                                                             long long total, float delta, float gamma, float alpha)
{
    DIS_PIX_LOOP(pix_base)
    const long long pl = J.plane;
    const float* du_p = J.rs + rs_du(J.C, 0) * pl;
    const float* dv_p = J.rs + rs_du(J.C, 1) * pl;
    float a11, a12, a22, b1, b2;
    refine_data_system(J.rs, J.C, pl, o, du_p[o], dv_p[o], delta, gamma, a11, a12, a22, b1, b2);
    // smoothness: central differences of u + du, replicated border
    const int xl = max(x - 1, 0), xr = min(x + 1, w - 1), yu = max(y - 1, 0), yd = min(y + 1, h - 1);
    const long long fl = (long long)y * w + xl, fr = (long long)y * w + xr;
    const long long fu = (long long)yu * w + x, fd = (long long)yd * w + x;
    const long long ol = (long long)y * pitch + xl, orr = (long long)y * pitch + xr;
    const long long ou = (long long)yu * pitch + x, od = (long long)yd * pitch + x;
    const float2 Ul = J.U[fl], Ur = J.U[fr], Uu = J.U[fu], Ud = J.U[fd];
    const float ux = refine_cdiff(Ur.x, du_p[orr], Ul.x, du_p[ol]);
    const float vx = refine_cdiff(Ur.y, dv_p[orr], Ul.y, dv_p[ol]);
    const float uy = refine_cdiff(Ud.x, du_p[od], Uu.x, du_p[ou]);
    const float vy = refine_cdiff(Ud.y, dv_p[od], Uu.y, dv_p[ou]);
    float* S = J.rs + rs_sys(J.C, 0) * pl + o;
    S[0] = a11;
    S[pl] = a12;
    S[2 * pl] = a22;
    S[3 * pl] = b1;
    S[4 * pl] = b2;
    S[5 * pl] = refine_smooth_weight(ux, uy, vx, vy, alpha);
    DIS_PIX_END
}

// One colour of one red-black sweep: the pixels with (x + y) % 2 == colour.
__global__ void __launch_bounds__(256) refine_sor_kernel(const __grid_constant__ Jobs<LevelJob> js, long long total,
                                                         int colour, float omega, int dof)
{
    for (long long g = gtid(); g < total; g += gstride()) {
        const LevelJob& J = job_ref(js, find_job(js, g, &LevelJob::half_base));
        const int k = (int)(g - J.half_base);  // < h * ceil(w / 2) < 2^31
        const int w = J.w, h = J.h, pitch = J.pitch;
        const int hw = (w + 1) >> 1;
        const int y = k / hw;
        const int x = 2 * (k - y * hw) + ((y + colour) & 1);
        if (x >= w) continue;
        const long long pl = J.plane;
        const long long o = (long long)y * pitch + x, f = (long long)y * w + x;
        const float* S = J.rs + rs_sys(J.C, 0) * pl;
        float* du_p = J.rs + rs_du(J.C, 0) * pl;
        float* dv_p = J.rs + rs_du(J.C, 1) * pl;
        const int nxs[4] = {x - 1, x + 1, x, x};
        const int nys[4] = {y, y, y - 1, y + 1};
        bool in[4];
        float psq[4], duq[4], dvq[4];
        float2 Uq[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int qx = nxs[q], qy = nys[q];
            in[q] = qx >= 0 && qx < w && qy >= 0 && qy < h;
            const long long oq = in[q] ? (long long)qy * pitch + qx : o;
            psq[q] = S[5 * pl + oq];
            duq[q] = du_p[oq];
            dvq[q] = dv_p[oq];
            Uq[q] = J.U[in[q] ? (long long)qy * w + qx : f];
        }
        float du = du_p[o], dv = dv_p[o];
        refine_sor_update(S[o], S[pl + o], S[2 * pl + o], S[3 * pl + o], S[4 * pl + o], S[5 * pl + o], in, psq, Uq,
                          duq, dvq, J.U[f], omega, dof, du, dv);
        du_p[o] = du;
        dv_p[o] = dv;
    }
}

__global__ void __launch_bounds__(256) refine_apply_kernel(const __grid_constant__ Jobs<LevelJob> js, long long total,
                                                           int src)
{
    DIS_PIX_LOOP(pix_base)
    float2 U = J.U[k];
    U.x += J.rs[(long long)src * J.plane + o];
    U.y += J.rs[(long long)(src + 1) * J.plane + o];
    J.U[k] = U;
    DIS_PIX_END
}

// ---------------------------------------------------------------- fused pass kernel
constexpr int kTile = kRefineTile;

// Shared-memory geometry of a launch of K half-sweeps with C channels.  Regions are squares
// around the 32x32 tile with a margin: R0 (the systems, margin K), R1 (U and the increment,
// margin K + 1), B (I_x, I_y, margin K + 1) and A (Ibar, I_z, margin K + 2, rows padded so that
// each starts on a 16-byte boundary of the image row: OX columns before the region, WA floats per
// row).  R0 and R1 are stored colour by colour (all red pixels row by row, then all black ones),
// so that a half-sweep touches consecutive words; R1 reuses the space of A and B once the
// systems exist.  With three channels R0 has a fourth plane for the energies and the weights
// between the two passes over the channels.
template <int K, int C>
struct PassGeom {
    static constexpr int S0 = kTile + 2 * K;
    static constexpr int S1 = kTile + 2 * (K + 1);
    static constexpr int SB = S1;
    static constexpr int SA = kTile + 2 * (K + 2);
    static constexpr int OX = ((K + 2 + 3) / 4) * 4 - (K + 2);
    static constexpr int WA = ((OX + SA + 3) / 4) * 4;
    static constexpr int R0P = C == 1 ? 3 : 4;
    static constexpr size_t bytes_r0 = sizeof(float2) * R0P * S0 * S0;
    static constexpr size_t bytes_ab = sizeof(float) * 2 * ((size_t)WA * SA + (size_t)SB * SB);
    static constexpr size_t bytes_r1 = sizeof(float4) * S1 * S1;
    static constexpr size_t bytes = bytes_r0 + (bytes_ab > bytes_r1 ? bytes_ab : bytes_r1);
    // threads per block and resident blocks per SM: three blocks of 256 threads in 74 KB at
    // K <= 5 (gray), two of 448 threads in 113 KB at K = 10
    static constexpr int threads = K <= 5 ? 256 : 448;
    static constexpr int min_blocks = (K <= 5 && C == 1) ? 3 : 2;
};

// Index of local pixel (lx, ly) in a colour-split square region of even side S whose origin
// has colour parity p.
__device__ __forceinline__ int csplit(int lx, int ly, int S, int p)
{
    return ((lx + ly + p) & 1) * (S * S / 2) + ly * (S / 2) + (lx >> 1);
}

// PHASE 0: the whole pass (systems, K = 2 theta_vi half-sweeps).  PHASE 1 / 2: the first / second
// half of a pass split into two launches of K = theta_vi half-sweeps (half the halo).  Planes:
// `start` holds the increment at the pass start (-1: zero, the first pass), which fixes the
// lagged weights; PHASE 2 continues the sweeps from the first half's increment in `cur`; the
// tile's increment goes to `dst`.  j0: index of the launch's first half-sweep within the pass
// (its colour parity).
template <int K, int PHASE, int C>
__global__ void __launch_bounds__(PassGeom<K, C>::threads, PassGeom<K, C>::min_blocks)
    refine_pass_kernel(const __grid_constant__ Jobs<LevelJob> js, long long total_tiles, int start, int cur, int dst,
                       int j0, float delta, float gamma, float alpha, float omega, int dof)
{
    using G = PassGeom<K, C>;
    constexpr int NT = G::threads;
    constexpr int S0 = G::S0, S1 = G::S1, SB = G::SB, SA = G::SA, WA = G::WA;
    constexpr int HS0 = S0 / 2, HE0 = S0 * S0 / 2, HS1 = S1 / 2, HE1 = S1 * S1 / 2;
    constexpr int E0 = S0 * S0;
    extern __shared__ float4 sm4[];
    // R0 planes: (a11, a12) (a22, b1) as float2, then b2 and psiS as two float planes (a float
    // plane per value keeps the four neighbour reads of psiS in a sweep free of bank conflicts),
    // then, for three channels, (EI, EG)
    float2* r0 = reinterpret_cast<float2*>(sm4);
    float* rb2 = reinterpret_cast<float*>(r0 + 2 * E0);
    float* rps = rb2 + E0;
    float* Ab = reinterpret_cast<float*>(reinterpret_cast<char*>(sm4) + G::bytes_r0);
    float* Az = Ab + WA * SA;
    float* Bx = Az + WA * SA;
    float* By = Bx + SB * SB;
    float4* r1 = reinterpret_cast<float4*>(Ab);  // (U.x, U.y, du, dv), after the systems
    for (long long tile = blockIdx.x; tile < total_tiles; tile += gridDim.x) {
        const LevelJob& J = job_ref(js, find_job(js, tile, &LevelJob::tile_base));
        const long long tk = tile - J.tile_base;
        const int ty = (int)(tk / J.tiles_x), tx = (int)(tk - (long long)ty * J.tiles_x);
        const int w = J.w, h = J.h, pitch = J.pitch;
        const long long pl = J.plane;
        const float* rs = J.rs;
        const int bx0 = tx * kTile, by0 = ty * kTile;               // tile origin
        const int xa = bx0 - (K + 2) - G::OX, ya = by0 - (K + 2);  // region A (xa: multiple of 4)
        const int x1 = bx0 - (K + 1), y1 = by0 - (K + 1);          // regions B and R1
        const int x0 = bx0 - K, y0 = by0 - K;                      // region R0
        const int p1 = (x1 + y1) & 1;                              // colour parity of R1's and R0's origins
        const float* gds = start >= 0 ? rs + (long long)start * pl : nullptr;
        // A loads as float4 rows when it lies inside the image and the planes are 16-byte aligned
        const bool vec = xa >= 0 && ya >= 0 && xa + WA <= w && ya + SA <= h && (pitch & 3) == 0 &&
                         ((reinterpret_cast<uintptr_t>(rs) | (uintptr_t)(pl * 4)) & 15) == 0;
        // ---- lagged systems on R0, channel by channel (three channels: energies first, then
        // the systems, as in refine_data_system)
        for (int sweep_c = 0; sweep_c < (C == 1 ? 1 : 2); ++sweep_c) {
            for (int c = 0; c < C; ++c) {
                const float* Pb = rs + (long long)rp_bar(C, c) * pl;
                const float* Pz = rs + (long long)rp_iz(C, c) * pl;
                if (vec) {
                    constexpr int Q4 = WA / 4;
                    for (int t = threadIdx.x; t < 2 * SA * Q4; t += NT) {
                        const int z = t >= SA * Q4;
                        const int tt = t - z * SA * Q4;
                        const int ly = tt / Q4, q = tt - ly * Q4;
                        const float4 v =
                            __ldg(reinterpret_cast<const float4*>((z ? Pz : Pb) + (long long)(ya + ly) * pitch + xa) + q);
                        reinterpret_cast<float4*>(z ? Az : Ab)[ly * Q4 + q] = v;
                    }
                } else {
                    for (int t = threadIdx.x; t < 2 * SA * WA; t += NT) {
                        const int z = t >= SA * WA;
                        const int tt = t - z * SA * WA;
                        const int ly = tt / WA, lx = tt - ly * WA;
                        const long long o =
                            (long long)clampi(ya + ly, 0, h - 1) * pitch + clampi(xa + lx, 0, w - 1);
                        (z ? Az : Ab)[tt] = __ldg((z ? Pz : Pb) + o);
                    }
                }
                __syncthreads();
                // I_x, I_y on B, each at the clamped position (so that B holds the replicated
                // border of the first derivatives)
                for (int t = threadIdx.x; t < SB * SB; t += NT) {
                    const int ly = t / SB, lx = t - ly * SB;
                    const int ax = clampi(x1 + lx, 0, w - 1) - xa, ay = clampi(y1 + ly, 0, h - 1) - ya;
                    const float* p = Ab + (ay - 1) * WA + ax - 1;
                    const float v[9] = {p[0], p[1], p[2], p[WA], p[WA + 1], p[WA + 2], p[2 * WA], p[2 * WA + 1],
                                        p[2 * WA + 2]};
                    Bx[t] = sobel_x9(v);
                    By[t] = sobel_y9(v);
                }
                __syncthreads();
                for (int t = threadIdx.x; t < E0; t += NT) {
                    const int ly = t / S0, lx = t - ly * S0;
                    const int x = x0 + lx, y = y0 + ly;
                    if (x < 0 || x >= w || y < 0 || y >= h) continue;
                    const float* bx = Bx + ly * SB + lx;  // (x - 1, y - 1) in B
                    const float* by = By + ly * SB + lx;
                    const float* az = Az + (ly + 1) * WA + lx + 1 + G::OX;
                    const float ix[9] = {bx[0], bx[1], bx[2], bx[SB], bx[SB + 1], bx[SB + 2], bx[2 * SB],
                                         bx[2 * SB + 1], bx[2 * SB + 2]};
                    const float iy[9] = {by[0], by[1], by[2], by[SB], by[SB + 1], by[SB + 2], by[2 * SB],
                                         by[2 * SB + 1], by[2 * SB + 2]};
                    const float iz[9] = {az[0], az[1], az[2], az[WA], az[WA + 1], az[WA + 2], az[2 * WA],
                                         az[2 * WA + 1], az[2 * WA + 2]};
                    float d[9];
                    refine_dvals(ix, iy, iz, d);
                    float du = 0.0f, dv = 0.0f;
                    if (gds) {
                        const long long o = (long long)y * pitch + x;
                        du = gds[o];
                        dv = gds[pl + o];
                    }
                    const int ci = csplit(lx, ly, S0, p1);
                    if constexpr (C == 1) {
                        float EI = 0.0f, EG = 0.0f, psiI, psiG;
                        refine_energy_acc(d, du, dv, EI, EG);
                        refine_psi(EI, EG, delta, gamma, psiI, psiG);
                        float a11 = 0.0f, a12 = 0.0f, a22 = 0.0f, b1 = 0.0f, b2 = 0.0f;
                        refine_system_acc(d, psiI, psiG, a11, a12, a22, b1, b2);
                        r0[ci] = make_float2(a11, a12);
                        r0[E0 + ci] = make_float2(a22, b1);
                        rb2[ci] = b2;
                    } else if (sweep_c == 0) {
                        float2 e = c == 0 ? make_float2(0.0f, 0.0f) : r0[3 * E0 + ci];
                        refine_energy_acc(d, du, dv, e.x, e.y);
                        r0[3 * E0 + ci] = e;
                    } else {
                        const float2 e = r0[3 * E0 + ci];
                        float psiI, psiG;
                        refine_psi(e.x, e.y, delta, gamma, psiI, psiG);
                        float2 s01 = make_float2(0.0f, 0.0f), s23 = s01;
                        float s4 = 0.0f;
                        if (c > 0) {
                            s01 = r0[ci];
                            s23 = r0[E0 + ci];
                            s4 = rb2[ci];
                        }
                        refine_system_acc(d, psiI, psiG, s01.x, s01.y, s23.x, s23.y, s4);
                        r0[ci] = s01;
                        r0[E0 + ci] = s23;
                        rb2[ci] = s4;
                    }
                }
                __syncthreads();
            }
        }
        // ---- U and the increment at the pass start on R1 (zero outside the image, never used
        // there), then the smoothness weights on R0
        const float* gcur = PHASE == 2 ? rs + (long long)cur * pl : gds;
        for (int t = threadIdx.x; t < S1 * S1; t += NT) {
            const int ly = t / S1, lx = t - ly * S1;
            const int x = x1 + lx, y = y1 + ly;
            float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            if (x >= 0 && x < w && y >= 0 && y < h) {
                const float2 U = J.U[(long long)y * w + x];
                v.x = U.x;
                v.y = U.y;
                if (gds) {
                    const long long o = (long long)y * pitch + x;
                    v.z = gds[o];
                    v.w = gds[pl + o];
                }
            }
            r1[csplit(lx, ly, S1, p1)] = v;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < E0; t += NT) {
            const int ly = t / S0, lx = t - ly * S0;
            const int x = x0 + lx, y = y0 + ly;
            if (x < 0 || x >= w || y < 0 || y >= h) continue;
            const int c = (x + y) & 1;
            const int pos = (ly + 1) * HS1 + ((lx + 1) >> 1), oth = (1 - c) * HE1 + pos;
            const int odd = (lx + 1) & 1;
            const float4 me = r1[c * HE1 + pos];
            // replicated border: a clamped neighbour is the pixel itself
            const float4 L = x > 0 ? r1[oth - 1 + odd] : me;
            const float4 R = x < w - 1 ? r1[oth + odd] : me;
            const float4 Up = y > 0 ? r1[oth - HS1] : me;
            const float4 Dn = y < h - 1 ? r1[oth + HS1] : me;
            const float ux = refine_cdiff(R.x, R.z, L.x, L.z);
            const float vx = refine_cdiff(R.y, R.w, L.y, L.w);
            const float uy = refine_cdiff(Dn.x, Dn.z, Up.x, Up.z);
            const float vy = refine_cdiff(Dn.y, Dn.w, Up.y, Up.w);
            rps[c * HE0 + ly * HS0 + (lx >> 1)] = refine_smooth_weight(ux, uy, vx, vy, alpha);
        }
        if constexpr (PHASE == 2) {
            // the sweeps continue from the first half's increment
            __syncthreads();
            for (int t = threadIdx.x; t < S1 * S1; t += NT) {
                const int ly = t / S1, lx = t - ly * S1;
                const int x = x1 + lx, y = y1 + ly;
                if (x < 0 || x >= w || y < 0 || y >= h) continue;
                const long long o = (long long)y * pitch + x;
                float4& v = r1[csplit(lx, ly, S1, p1)];
                v.z = gcur[o];
                v.w = gcur[pl + o];
            }
        }
        __syncthreads();
        // ---- K half-sweeps, red ((x + y) even) first.  Half-sweep j covers the square of margin
        // m = K - 1 - j around the tile; pair pr = (ly, k) of that square covers pixels (2k, ly)
        // and (2k + 1, ly), of which the one of the current colour is updated.
        const bool interior = x1 >= 0 && y1 >= 0 && x1 + S1 <= w && y1 + S1 <= h;
        auto sweep = [&](auto inner_tag) {
            constexpr bool INNER = decltype(inner_tag)::value;  // no image border in R1
#pragma unroll
            for (int j = 0; j < K; ++j) {  // unrolled: the square's side is a constant
                const int colour = (j + j0) & 1;  // the second half of a pass continues the alternation
                const int m = K - 1 - j, side = kTile + 2 * m, prow = side / 2;
                const int xo = bx0 - m, yo = by0 - m;
                const int off = K + 1 - m;  // R1 position of the square's origin
                for (int pr = threadIdx.x; pr < side * prow; pr += NT) {
                    const int ly = pr / prow, k = pr - ly * prow;
                    const int y = yo + ly;
                    const int first = ((xo + y) & 1) ^ colour;
                    const int x = xo + 2 * k + first;
                    if (!INNER && (x < 0 || x >= w || y < 0 || y >= h)) continue;
                    const int lx1 = off + 2 * k + first, ly1 = off + ly;
                    const int pos1 = ly1 * HS1 + (lx1 >> 1), pos0 = (ly1 - 1) * HS0 + ((lx1 - 1) >> 1);
                    const int odd1 = lx1 & 1, odd0 = 1 - odd1;
                    const int i1 = colour * HE1 + pos1, o1 = (1 - colour) * HE1 + pos1;
                    const int i0 = colour * HE0 + pos0, o0 = (1 - colour) * HE0 + pos0;
                    const int n1[4] = {o1 - 1 + odd1, o1 + odd1, o1 - HS1, o1 + HS1};
                    const int n0[4] = {o0 - 1 + odd0, o0 + odd0, o0 - HS0, o0 + HS0};
                    const bool in[4] = {INNER || x > 0, INNER || x < w - 1, INNER || y > 0, INNER || y < h - 1};
                    float psq[4], duq[4], dvq[4];
                    float2 Uq[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float4 v = r1[INNER ? n1[q] : (in[q] ? n1[q] : i1)];
                        psq[q] = rps[INNER ? n0[q] : (in[q] ? n0[q] : i0)];
                        Uq[q] = make_float2(v.x, v.y);
                        duq[q] = v.z;
                        dvq[q] = v.w;
                    }
                    float4 me = r1[i1];
                    const float2 s01 = r0[i0], s23 = r0[E0 + i0];
                    const float s4 = rb2[i0], s5 = rps[i0];
                    float du = me.z, dv = me.w;
                    refine_sor_update(s01.x, s01.y, s23.x, s23.y, s4, s5, in, psq, Uq, duq, dvq,
                                      make_float2(me.x, me.y), omega, dof, du, dv);
                    me.z = du;
                    me.w = dv;
                    r1[i1] = me;
                }
                __syncthreads();
            }
        };
        if (interior)
            sweep(std::true_type{});
        else
            sweep(std::false_type{});
        // the tile's increments to `dst`
        float* odu = J.rs + (long long)dst * pl;
        float* odv = odu + pl;
        for (int t = threadIdx.x; t < kTile * kTile; t += NT) {
            const int ly = t / kTile, lx = t - ly * kTile;
            const int x = bx0 + lx, y = by0 + ly;
            if (x >= w || y >= h) continue;
            const float4 v = r1[csplit(lx + K + 1, ly + K + 1, S1, p1)];
            const long long o = (long long)y * pitch + x;
            odu[o] = v.z;
            odv[o] = v.w;
        }
        __syncthreads();  // shared memory is reloaded for the next tile
    }
}

template <int K, int PHASE, int C>
static cudaError_t pass_launch(const Jobs<LevelJob>& js, long long total_tiles, const RefineArgs& a, int start,
                               int cur, int dst, int j0, const LaunchCfg& lc, cudaStream_t s)
{
    using G = PassGeom<K, C>;
    constexpr size_t smem = G::bytes;
    static int occ = 0;
    if (occ == 0) {
        cudaError_t e =
            cudaFuncSetAttribute(refine_pass_kernel<K, PHASE, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, refine_pass_kernel<K, PHASE, C>, G::threads, smem) !=
                cudaSuccess ||
            occ < 1)
            occ = 1;
    }
    const int gt = (int)std::min<long long>(total_tiles, (long long)lc.sm_count * occ);
    refine_pass_kernel<K, PHASE, C><<<gt, G::threads, smem, s>>>(js, total_tiles, start, cur, dst, j0, a.delta,
                                                                 a.gamma, a.alpha, a.omega, a.dof);
    return cudaGetLastError();
}

// a.outer fused passes of KT half-sweeps, each in one launch (KC == KT) or in two launches of
// KC = KT / 2.  Increment planes: X = rs_du, Y = the fifth and sixth intermediate planes of
// channel 0, Z = the first two system planes (all free in this form).  One launch per pass
// alternates between X and Y; a split pass writes its first half to X and its result to the one
// of Y, Z that does not hold its start.  Returns the plane of the final increment (-1: none,
// a.outer == 0).
template <int KT, int KC, int C>
static cudaError_t launch_passes(const Jobs<LevelJob>& js, long long total_tiles, const RefineArgs& a, int& fin,
                                 const LaunchCfg& lc, cudaStream_t s)
{
    static_assert(KT == KC || KT == 2 * KC, "a pass runs in one or two launches");
    const int X = rs_du(C, 0), Y = rs_mid(C, 0, 4), Z = rs_sys(C, 0);
    int start = -1;
    for (int ot = 0; ot < a.outer; ++ot) {
        cudaError_t e;
        int dst;
        if constexpr (KC == KT) {
            dst = start == X ? Y : X;
            e = pass_launch<KC, 0, C>(js, total_tiles, a, start, -1, dst, 0, lc, s);
        } else {
            dst = start == Y ? Z : Y;
            e = pass_launch<KC, 1, C>(js, total_tiles, a, start, -1, X, 0, lc, s);
            if (e == cudaSuccess) e = pass_launch<KC, 2, C>(js, total_tiles, a, start, X, dst, KC, lc, s);
        }
        if (e != cudaSuccess) return e;
        start = dst;
    }
    fin = start;
    return cudaSuccess;
}

template <int C>
static cudaError_t launch_fused(const Jobs<LevelJob>& js, long long total_tiles, const RefineArgs& a, int chunks,
                                int& fin, const LaunchCfg& lc, cudaStream_t s)
{
    switch (a.inner * 10 + chunks) {
        case 11: return launch_passes<2, 2, C>(js, total_tiles, a, fin, lc, s);
        case 12: return launch_passes<2, 1, C>(js, total_tiles, a, fin, lc, s);
        case 21: return launch_passes<4, 4, C>(js, total_tiles, a, fin, lc, s);
        case 22: return launch_passes<4, 2, C>(js, total_tiles, a, fin, lc, s);
        case 31: return launch_passes<6, 6, C>(js, total_tiles, a, fin, lc, s);
        case 32: return launch_passes<6, 3, C>(js, total_tiles, a, fin, lc, s);
        case 41: return launch_passes<8, 8, C>(js, total_tiles, a, fin, lc, s);
        case 42: return launch_passes<8, 4, C>(js, total_tiles, a, fin, lc, s);
        case 51: return launch_passes<10, 10, C>(js, total_tiles, a, fin, lc, s);
        default: return launch_passes<10, 5, C>(js, total_tiles, a, fin, lc, s);
    }
}

cudaError_t launch_refine(const Jobs<LevelJob>& js, long long total_pix, long long total_half, long long total_tiles,
                          const RefineArgs& a, const LaunchCfg& lc, cudaStream_t s)
{
    if (total_pix <= 0) return cudaSuccess;
    const long long cap = (long long)lc.sm_count * lc.max_blocks_256;
    const int gp = (int)std::min<long long>((total_pix + 255) / 256, cap);
    const int gh = (int)std::min<long long>((total_half + 255) / 256, cap);
    // The fused form recomputes the halo: at 10 half-sweeps in one launch a block forms the
    // systems of 2.6x the tile's pixels and sweeps 1.5x on average; a pass split into two
    // launches of 5 forms them twice on 1.7x and sweeps 1.2x, at three blocks per SM instead of
    // two.  mode 1 takes one launch up to a.split_px pixels per launch, two above; mode 2 / 3
    // force one; mode 0 (and passes of more than five sweeps) run the per-sweep kernels.
    const bool fused = a.fused != 0 && a.inner > 0 && a.inner <= kRefineMaxFusedInner && total_tiles > 0;
    refine_prep_kernel<<<gp, 256, 0, s>>>(js, total_pix, fused ? 0 : 1);
    if (!fused) {
        refine_grad_kernel<<<gp, 256, 0, s>>>(js, total_pix);
        refine_data_kernel<<<gp, 256, 0, s>>>(js, total_pix);
        for (int ot = 0; ot < a.outer; ++ot) {
            refine_weights_kernel<<<gp, 256, 0, s>>>(js, total_pix, a.delta, a.gamma, a.alpha);
            for (int it = 0; it < a.inner; ++it) {
                refine_sor_kernel<<<gh, 256, 0, s>>>(js, total_half, 0, a.omega, a.dof);
                refine_sor_kernel<<<gh, 256, 0, s>>>(js, total_half, 1, a.omega, a.dof);
            }
        }
        refine_apply_kernel<<<gp, 256, 0, s>>>(js, total_pix, rs_du(a.C, 0));
        return cudaGetLastError();
    }
    const int chunks = (a.fused == 3 || (a.fused == 1 && total_pix > a.split_px)) ? 2 : 1;
    int fin = -1;
    cudaError_t e = a.C == 1 ? launch_fused<1>(js, total_tiles, a, chunks, fin, lc, s)
                             : launch_fused<3>(js, total_tiles, a, chunks, fin, lc, s);
    if (e != cudaSuccess) return e;
    if (fin >= 0) refine_apply_kernel<<<gp, 256, 0, s>>>(js, total_pix, fin);
    return cudaGetLastError();
}

}  // namespace dis
