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
// or, fused (the default), weights and all half-sweeps of one outer pass in one launch: each
// block loads a 32x32 tile with a halo as wide as the half-sweeps (K <= 10) into shared
// memory, computes the lagged weights there, runs the K red-black half-sweeps with a block
// barrier between them (the halo absorbs the values that go stale at the tile's edge: after
// half-sweep j only pixels within K - j of the tile are still exact) and writes the tile's
// increments to the other of two increment buffers.  The arithmetic is shared with the
// per-sweep kernels, so both forms give the same result bit for bit.
#include <algorithm>
#include <type_traits>

#include "dis_device.cuh"

namespace dis {

#define DIS_PIX_LOOP(BASE)                                                               \
    for (long long g = gtid(); g < total; g += gstride()) {                              \
        const LevelJob& J = job_ref(js, find_job(js, g, &LevelJob::BASE));               \
        const int k = (int)(g - J.BASE); /* < w * h < 2^31 */                            \
        const int w = J.w, h = J.h, pitch = J.pitch;                                     \
        const int y = k / w, x = k - y * w;                                              \
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

// Lagged data terms of pixel o at increment (du, dv): the 2x2 system A dU = b of the data
// energy with psi = weight * Psi'(.) frozen (summed over channels inside each Psi).
__device__ __forceinline__ void refine_data_system(const float* __restrict__ rs, int C, long long pl, long long o,
                                                   float du, float dv, float delta, float gamma, float& a11,
                                                   float& a12, float& a22, float& b1, float& b2)
{
    const float eps2 = 1.0e-6f;
    float EI = 0.0f, EG = 0.0f;
    for (int c = 0; c < C; ++c) {
        const float* D = rs + rs_dat(C, c, 0) * pl + o;
        const float eI = fmaf(D[0], du, fmaf(D[pl], dv, D[2 * pl]));
        const float eX = fmaf(D[3 * pl], du, fmaf(D[4 * pl], dv, D[5 * pl]));
        const float eY = fmaf(D[6 * pl], du, fmaf(D[7 * pl], dv, D[8 * pl]));
        EI = fmaf(eI, eI, EI);
        EG = fmaf(eX, eX, fmaf(eY, eY, EG));
    }
    const float psiI = delta / (2.0f * sqrtf(EI + eps2));
    const float psiG = gamma / (2.0f * sqrtf(EG + eps2));
    a11 = a12 = a22 = b1 = b2 = 0.0f;
    for (int c = 0; c < C; ++c) {
        const float* D = rs + rs_dat(C, c, 0) * pl + o;
        const float d0 = D[0], d1 = D[pl], d2 = D[2 * pl], d3 = D[3 * pl], d4 = D[4 * pl], d5 = D[5 * pl];
        const float d6 = D[6 * pl], d7 = D[7 * pl], d8 = D[8 * pl];
        a11 += psiI * d0 * d0 + psiG * (d3 * d3 + d6 * d6);
        a12 += psiI * d0 * d1 + psiG * (d3 * d4 + d6 * d7);
        a22 += psiI * d1 * d1 + psiG * (d4 * d4 + d7 * d7);
        b1 -= psiI * d2 * d0 + psiG * (d5 * d3 + d8 * d6);
        b2 -= psiI * d2 * d1 + psiG * (d5 * d4 + d8 * d7);
    }
}

// Smoothness weight alpha * Psi'(|grad(u + du)|^2) from the four central differences.
__device__ __forceinline__ float refine_smooth_weight(float ux, float uy, float vx, float vy, float alpha)
{
    const float ES = ux * ux + uy * uy + vx * vx + vy * vy;
    return alpha / (2.0f * sqrtf(ES + 1.0e-6f));
}

// Central difference 0.5 * ((U_r + dU_r) - (U_l + dU_l)) of one component.
__device__ __forceinline__ float refine_cdiff(float Ur, float dur, float Ul, float dul)
{
    return 0.5f * ((Ur + dur) - (Ul + dul));
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
        if (m11 > 0.0f) du = (1.0f - omega) * du + omega * (r1 * __frcp_rn(m11));
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
        const float id = __frcp_rn(det);  // the correctly rounded 1 / det
        const float d1 = (m22 * r1 - m12 * r2) * id;
        const float d2 = (m11 * r2 - m12 * r1) * id;
        du = (1.0f - omega) * du + omega * d1;
        dv = (1.0f - omega) * dv + omega * d2;
    }
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

// Weights and K half-sweeps of one outer pass on 32x32 tiles (see the header).  The increment
// is read from planes `src` (rs_du or rs_mid(C, 0, .)) and written to planes `dst`.
// Shared memory holds two square regions around the tile, each stored colour by colour (all
// red pixels row by row, then all black ones) so that a half-sweep reads and writes
// consecutive words: R1, halo K + 1, with U and the increment (du, dv) per pixel, and R0,
// halo K, with the systems (a11, a12), (a22, b1), (b2, psiS).  The half-sweeps cover the tile
// with a halo of K - 1 (the pixels whose neighbours all carry weights) as horizontal pixel
// pairs, one pixel of each colour, with a fixed pair-to-thread assignment.
constexpr int kOuterThreads = 448;  // 1250 swept pairs at K = 10: 3 per thread (2.8 on average)

// Index of local pixel (lx, ly) in a colour-split square region of even side S whose origin
// has colour parity p.
__device__ __forceinline__ int csplit(int lx, int ly, int S, int p)
{
    return ((lx + ly + p) & 1) * (S * S / 2) + ly * (S / 2) + (lx >> 1);
}

// PHASE 0: the whole pass (weights, K half-sweeps).  PHASE 1 / 2: the first / a later chunk of
// a pass split into launches of K half-sweeps each, which narrows the halo to K: the first
// computes the weights and also stores the tile's systems (rs_sys planes) for the later ones,
// which load them with their halo instead of recomputing them from an increment they no longer
// have.  j0: index of the chunk's first half-sweep in the pass (its colour parity).
template <int K, int PHASE>
__global__ void __launch_bounds__(kOuterThreads, 2) refine_outer_kernel(const __grid_constant__ Jobs<LevelJob> js,
                                                                        long long total_tiles, int src, int dst,
                                                                        int j0, float delta, float gamma,
                                                                        float alpha, float omega, int dof)
{
    extern __shared__ float4 sm4[];
    constexpr int T = kRefineTile;
    constexpr int H = K;                 // halo of the systems
    constexpr int S1 = T + 2 * (H + 1);  // side of R1
    constexpr int S0 = T + 2 * H;        // side of R0
    constexpr int S2 = T + 2 * (H - 1);  // side of the swept region (even)
    constexpr int E1 = S1 * S1, E0 = S0 * S0;
    constexpr int npairs = S2 * S2 / 2, pairs_row = S2 / 2;
    constexpr int HS1 = S1 / 2, HE1 = E1 / 2, HS0 = S0 / 2, HE0 = E0 / 2;  // half rows / halves
    float4* r1 = sm4;                                       // (U.x, U.y, du, dv)
    float2* r0 = reinterpret_cast<float2*>(sm4 + E1);       // 3 planes of E0 float2
    for (long long tile = blockIdx.x; tile < total_tiles; tile += gridDim.x) {
        const LevelJob& J = job_ref(js, find_job(js, tile, &LevelJob::tile_base));
        const long long tk = tile - J.tile_base;
        const int ty = (int)(tk / J.tiles_x), tx = (int)(tk - (long long)ty * J.tiles_x);
        const int w = J.w, h = J.h, pitch = J.pitch, C = J.C;
        const long long pl = J.plane;
        const float* rs = J.rs;
        const float2* Ug = J.U;
        const int x1 = tx * T - (H + 1), y1 = ty * T - (H + 1);  // origin of R1
        const int p1 = (x1 + y1) & 1;                            // colour parity of R1's origin (= R0's)
        const float* gdu = rs + (long long)src * pl;
        const float* gdv = gdu + pl;
        // U and the increments on R1 (zero outside the image, never used there)
#pragma unroll 2
        for (int t = threadIdx.x; t < E1; t += kOuterThreads) {
            const int ly = t / S1, lx = t - ly * S1;
            const int x = x1 + lx, y = y1 + ly;
            float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            if (x >= 0 && x < w && y >= 0 && y < h) {
                const float2 U = Ug[(long long)y * w + x];
                const long long o = (long long)y * pitch + x;
                v = make_float4(U.x, U.y, gdu[o], gdv[o]);
            }
            r1[csplit(lx, ly, S1, p1)] = v;
        }
        __syncthreads();
        // lagged weights on R0 (origin x1 + 1, y1 + 1: the same colour parity as R1).  In a
        // colour-split region a pixel (lx, ly) of colour c sits at c * half + ly * S/2 + lx/2;
        // its left / right neighbours (the other colour) at the same position minus 1 when lx
        // is even, plus 1 when lx is odd, and its upper / lower ones one half row away.
        float* gsys = J.rs + (long long)rs_sys(C, 0) * pl;
        if constexpr (PHASE == 2) {
            // the stored systems of the pass's first chunk, with their halo (loads batched)
#pragma unroll 4
            for (int t = threadIdx.x; t < E0; t += kOuterThreads) {
                const int ly = t / S0, lx = t - ly * S0;
                const int x = x1 + 1 + lx, y = y1 + 1 + ly;
                if (x < 0 || x >= w || y < 0 || y >= h) continue;
                const int c0 = ((x + y) & 1) * HE0 + ly * HS0 + (lx >> 1);
                const long long o = (long long)y * pitch + x;
                r0[c0] = make_float2(gsys[o], gsys[pl + o]);
                r0[E0 + c0] = make_float2(gsys[2 * pl + o], gsys[3 * pl + o]);
                r0[2 * E0 + c0] = make_float2(gsys[4 * pl + o], gsys[5 * pl + o]);
            }
        }
        for (int t = threadIdx.x; PHASE != 2 && t < E0; t += kOuterThreads) {
            const int ly = t / S0, lx = t - ly * S0;
            const int x = x1 + 1 + lx, y = y1 + 1 + ly;
            if (x < 0 || x >= w || y < 0 || y >= h) continue;
            const int c = (x + y) & 1;
            const int c0 = c * HE0 + ly * HS0 + (lx >> 1);
            const long long o = (long long)y * pitch + x;
            const int pos = (ly + 1) * HS1 + ((lx + 1) >> 1), oth = (1 - c) * HE1 + pos;
            const int odd = (lx + 1) & 1;
            const float4 me = r1[c * HE1 + pos];
            // replicated border: a clamped neighbour is the pixel itself
            const float4 L = x > 0 ? r1[oth - 1 + odd] : me;
            const float4 R = x < w - 1 ? r1[oth + odd] : me;
            const float4 Up = y > 0 ? r1[oth - HS1] : me;
            const float4 Dn = y < h - 1 ? r1[oth + HS1] : me;
            float a11, a12, a22, b1, b2;
            refine_data_system(rs, C, pl, o, me.z, me.w, delta, gamma, a11, a12, a22, b1, b2);
            const float ux = refine_cdiff(R.x, R.z, L.x, L.z);
            const float vx = refine_cdiff(R.y, R.w, L.y, L.w);
            const float uy = refine_cdiff(Dn.x, Dn.z, Up.x, Up.z);
            const float vy = refine_cdiff(Dn.y, Dn.w, Up.y, Up.w);
            const float psS = refine_smooth_weight(ux, uy, vx, vy, alpha);
            r0[c0] = make_float2(a11, a12);
            r0[E0 + c0] = make_float2(a22, b1);
            r0[2 * E0 + c0] = make_float2(b2, psS);
            if (PHASE == 1 && lx >= H && lx < H + T && ly >= H && ly < H + T) {
                // the tile's own systems, for the second half of the pass
                gsys[o] = a11;
                gsys[pl + o] = a12;
                gsys[2 * pl + o] = a22;
                gsys[3 * pl + o] = b1;
                gsys[4 * pl + o] = b2;
                gsys[5 * pl + o] = psS;
            }
        }
        __syncthreads();
        // K half-sweeps, red ((x + y) even) first.  Pair pr = (ly, k) covers swept pixels
        // (2k, ly) and (2k + 1, ly); the one of the current colour is lx = 2k + first.
        const int x2 = x1 + 2, y2 = y1 + 2;  // origin of the swept region
        const bool interior = x1 >= 0 && y1 >= 0 && x1 + S1 <= w && y1 + S1 <= h;
        auto sweep = [&](auto inner_tag) {
            constexpr bool INNER = decltype(inner_tag)::value;  // no image border in R1
            for (int j = 0; j < K; ++j) {
                const int colour = (j + j0) & 1;  // later chunks continue the pass's alternation
                for (int pr = threadIdx.x; pr < npairs; pr += kOuterThreads) {
                    const int ly = pr / pairs_row, k = pr - ly * pairs_row;
                    const int y = y2 + ly;
                    const int first = ((x2 + y) & 1) == colour ? 0 : 1;
                    const int x = x2 + 2 * k + first;
                    if (!INNER && (x < 0 || x >= w || y < 0 || y >= h)) continue;
                    // R1 position (2k + first + 2, ly + 2), R0 position (2k + first + 1, ly + 1)
                    const int pos1 = (ly + 2) * HS1 + k + 1, pos0 = (ly + 1) * HS0 + k + first;
                    const int i1 = colour * HE1 + pos1, o1 = (1 - colour) * HE1 + pos1;
                    const int i0 = colour * HE0 + pos0, o0 = (1 - colour) * HE0 + pos0;
                    const int n1[4] = {o1 - 1 + first, o1 + first, o1 - HS1, o1 + HS1};
                    const int n0[4] = {o0 - first, o0 + 1 - first, o0 - HS0, o0 + HS0};
                    const bool in[4] = {INNER || x > 0, INNER || x < w - 1, INNER || y > 0, INNER || y < h - 1};
                    float psq[4], duq[4], dvq[4];
                    float2 Uq[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float4 v = r1[INNER ? n1[q] : (in[q] ? n1[q] : i1)];
                        psq[q] = r0[2 * E0 + (INNER ? n0[q] : (in[q] ? n0[q] : i0))].y;
                        Uq[q] = make_float2(v.x, v.y);
                        duq[q] = v.z;
                        dvq[q] = v.w;
                    }
                    float4 me = r1[i1];
                    const float2 s01 = r0[i0], s23 = r0[E0 + i0], s45 = r0[2 * E0 + i0];
                    float du = me.z, dv = me.w;
                    refine_sor_update(s01.x, s01.y, s23.x, s23.y, s45.x, s45.y, in, psq, Uq, duq, dvq,
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
        // the tile's increments to the other buffer
        float* odu = J.rs + (long long)dst * pl;
        float* odv = odu + pl;
        for (int t = threadIdx.x; t < T * T; t += kOuterThreads) {
            const int ly = t / T, lx = t - ly * T;
            const int x = tx * T + lx, y = ty * T + ly;
            if (x >= w || y >= h) continue;
            const float4 v = r1[csplit(lx + H + 1, ly + H + 1, S1, p1)];
            const long long o = (long long)y * pitch + x;
            odu[o] = v.z;
            odv[o] = v.w;
        }
        __syncthreads();  // shared memory is reloaded for the next tile
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

template <int K, int PHASE>
static cudaError_t outer_launch(const Jobs<LevelJob>& js, long long total_tiles, const RefineArgs& a, int src, int dst,
                                int j0, const LaunchCfg& lc, cudaStream_t s)
{
    constexpr int S1 = kRefineTile + 2 * (K + 1), S0 = kRefineTile + 2 * K;
    constexpr size_t smem = sizeof(float4) * (size_t)S1 * S1 + sizeof(float2) * 3 * (size_t)S0 * S0;
    static int occ = 0;
    if (occ == 0) {
        cudaError_t e =
            cudaFuncSetAttribute(refine_outer_kernel<K, PHASE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, refine_outer_kernel<K, PHASE>, kOuterThreads, smem) !=
                cudaSuccess ||
            occ < 1)
            occ = 1;
    }
    const int gt = (int)std::min<long long>(total_tiles, (long long)lc.sm_count * occ);
    refine_outer_kernel<K, PHASE><<<gt, kOuterThreads, smem, s>>>(js, total_tiles, src, dst, j0, a.delta, a.gamma,
                                                                   a.alpha, a.omega, a.dof);
    return cudaGetLastError();
}

// a.outer fused passes of KT half-sweeps, each in one launch (KC == KT) or in KT / KC launches
// of KC; on return `src` names the planes holding the final increment.
template <int KT, int KC>
static cudaError_t launch_outer(const Jobs<LevelJob>& js, long long total_tiles, const RefineArgs& a, int& src,
                                int& dst, const LaunchCfg& lc, cudaStream_t s)
{
    static_assert(KT % KC == 0, "chunks divide the pass");
    for (int ot = 0; ot < a.outer; ++ot) {
        cudaError_t e = cudaSuccess;
        if constexpr (KC == KT) {
            e = outer_launch<KT, 0>(js, total_tiles, a, src, dst, 0, lc, s);
            std::swap(src, dst);
        } else {
            for (int j0 = 0; j0 < KT && e == cudaSuccess; j0 += KC) {
                e = j0 == 0 ? outer_launch<KC, 1>(js, total_tiles, a, src, dst, j0, lc, s)
                            : outer_launch<KC, 2>(js, total_tiles, a, src, dst, j0, lc, s);
                std::swap(src, dst);
            }
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_refine(const Jobs<LevelJob>& js, long long total_pix, long long total_half, long long total_tiles,
                          const RefineArgs& a, const LaunchCfg& lc, cudaStream_t s)
{
    if (total_pix <= 0) return cudaSuccess;
    const long long cap = (long long)lc.sm_count * lc.max_blocks_256;
    const int gp = (int)std::min<long long>((total_pix + 255) / 256, cap);
    const int gh = (int)std::min<long long>((total_half + 255) / 256, cap);
    refine_warp_kernel<<<gp, 256, 0, s>>>(js, total_pix);
    refine_deriv1_kernel<<<gp, 256, 0, s>>>(js, total_pix);
    refine_deriv2_kernel<<<gp, 256, 0, s>>>(js, total_pix);
    // the increment starts in rs_du (zeroed by the warp kernel); the fused passes alternate it
    // with the first two intermediate planes, which are free once deriv2 has run
    const int du_plane = rs_du(a.C, 0), mid_plane = rs_mid(a.C, 0, 0);
    // The fused form recomputes the halo: about 2.4x the swept pixels at 10 half-sweeps in one
    // launch, 1.6x when the pass is split in two launches of 5 (which also stores and reloads
    // the systems).  Measured on GB300 the single launch wins up to about 128 K pixels per
    // launch, the split pass above (and both beat the per-sweep kernels); mode 2 / 3 force one.
    const bool fused = a.fused != 0 && a.inner > 0 && a.inner <= kRefineMaxFusedInner && total_tiles > 0;
    if (!fused) {
        for (int ot = 0; ot < a.outer; ++ot) {
            refine_weights_kernel<<<gp, 256, 0, s>>>(js, total_pix, a.delta, a.gamma, a.alpha);
            for (int it = 0; it < a.inner; ++it) {
                refine_sor_kernel<<<gh, 256, 0, s>>>(js, total_half, 0, a.omega, a.dof);
                refine_sor_kernel<<<gh, 256, 0, s>>>(js, total_half, 1, a.omega, a.dof);
            }
        }
        refine_apply_kernel<<<gp, 256, 0, s>>>(js, total_pix, du_plane);
        return cudaGetLastError();
    }
    // chunks per pass: 1 (mode 2, or small launches in mode 1) or 2 (mode 3, or large launches in
    // mode 1).  (Chunks of one full sweep, halo 2, measured slower than both: each reloads the
    // systems.)
    const int chunks = (a.fused == 3 || (a.fused == 1 && total_pix > kRefineFusedMaxPixels)) ? 2 : 1;
    int src = du_plane, dst = mid_plane;
    cudaError_t e = cudaSuccess;
    switch (a.inner * 10 + chunks) {
        case 11: e = launch_outer<2, 2>(js, total_tiles, a, src, dst, lc, s); break;
        case 12: e = launch_outer<2, 1>(js, total_tiles, a, src, dst, lc, s); break;
        case 21: e = launch_outer<4, 4>(js, total_tiles, a, src, dst, lc, s); break;
        case 22: e = launch_outer<4, 2>(js, total_tiles, a, src, dst, lc, s); break;
        case 31: e = launch_outer<6, 6>(js, total_tiles, a, src, dst, lc, s); break;
        case 32: e = launch_outer<6, 3>(js, total_tiles, a, src, dst, lc, s); break;
        case 41: e = launch_outer<8, 8>(js, total_tiles, a, src, dst, lc, s); break;
        case 42: e = launch_outer<8, 4>(js, total_tiles, a, src, dst, lc, s); break;
        case 51: e = launch_outer<10, 10>(js, total_tiles, a, src, dst, lc, s); break;
        default: e = launch_outer<10, 5>(js, total_tiles, a, src, dst, lc, s); break;
    }
    if (e != cudaSuccess) return e;
    refine_apply_kernel<<<gp, 256, 0, s>>>(js, total_pix, src);
    return cudaGetLastError();
}

}  // namespace dis
