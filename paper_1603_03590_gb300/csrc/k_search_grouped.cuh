// Grouped form of the inverse-compositional patch search (Sec. 2.1; supplementary Sec. A, Eq.
// solvereqinv; Alg. 1 steps 1-3 and the outlier reset of step 4), shared by the flow search
// (k_search.cu) and its stereo and robust-norm modes (k_search_modes.cu).
//
// A group of LPP lanes (4, 8, 16 or 32) owns one patch; lane l of the group owns patch pixels
// l, l + LPP, ... (PPL of them).  The prologue stages the (ps+2)^2 window of I0 around the
// patch in shared memory, computes the Sobel/8 gradients S' = grad T of the mean-normalised
// template T, leaves T (in the window) and S' in shared memory (registers stay free for
// occupancy: 28 warps per SM at 12x12, 32 at 8x8) and forms, by group shuffle reductions, the 2x2 Hessian
// H' = sum S'^T S', sum S' and sum T.
//
// Iterations.  u is shared by the whole patch, so while the integer part of u stays in one cell
// every pixel samples I1 with the same fractional weights (ax, ay):
//   w''(x) = I1(x + u) - T(x) - m = t0 + ax t1 + ay (t2 + ax t3),
// t0 = a - T - m, t1 = b - a, t2 = c - a, t3 = d - c - b + a from the pixel's four taps a..d and a
// reference intensity m.  The patch sums the update needs therefore factor into twelve sums
// that depend on the cell only,
//   sum w'' = T0 + ax T1 + ay (T2 + ax T3),   T_k = sum t_k,
//   sum S' w'' = G0 + ax G1 + ay (G2 + ax G3), G_k = sum S' t_k,
// which are rebuilt only when the integer part of u changes: the group sums the raw taps
// (sum a .. sum d and their products with S', clamped at the border, reduced over the group)
// and forms the twelve from them, T0 = sum a - sum T - n m, T1 = sum b - sum a, ..., and
// G0 = sum S' a - sum S' T - m sum S', ...  Every other iteration costs a few scalar FMAs:
//   e = (sum w'' + sum T) / n (mean of the window minus m),  b = sum S' w'' - e sum S',
//   u <- u - H'^-1 b  (= sum S'^T (w - mean w - T), Eq. solvereqinv with mean-normalisation).
// m follows the window mean at every rebuild.
//
// Modes (template DOF, ROBUST):
// - DOF = 1, stereo (supplementary, depth from stereo: the vertical degree of freedom removed):
//   v keeps its initial value and u takes the scalar step u <- u - b_x / H'_xx, a patch being flat
//   when H'_xx <= 1e-6 tr(H') / 2; only the eight sums T_k, Gx_k are formed.
// - ROBUST (supplementary, robust error norms; norm 1 = L1, 2 = Huber with threshold b): the
//   error of every pixel, r = w - mean w - T, is transformed before it enters sum S' psi(r), so the
//   cell factorisation of the gradient sums no longer holds.  At a rebuild each lane keeps its
//   pixels' interpolation coefficients (a - T, b - a, c - a, d - c - b + a) in registers and the
//   group forms the four tap sums (the window mean still factors); every iteration then costs,
//   per pixel, the bilinear value (3 FMA), psi and two FMA, and one group reduction of b.
#pragma once
#include <climits>

#include "dis_device.cuh"

namespace dis {

constexpr int kSearchThreads = 128;  // threads per block of the grouped search

template <int LPP>
__device__ __forceinline__ float group_sum(float v, unsigned mask)
{
#pragma unroll
    for (int o = LPP / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o);
    return v;
}

// Sums the twelve cell sums Q over the LPP lanes of a group and leaves the totals in every
// lane of it.  For 16 lanes a transposed reduction halves the values each lane carries at
// every exchange (12 -> 6 -> 3 -> 2 or 1 -> 1), so that each sum ends complete in one lane, and
// 12 broadcasts return them: 24 shuffles instead of 48.  Other widths use the butterfly (the
// transposed form raised the register use of the 8-lane variants more than it saved).
// Sums N values over the LPP lanes of a group (butterfly), leaving the totals in every lane.
template <int LPP, int N>
__device__ __forceinline__ void group_sumN(float (&Q)[N], unsigned gmask)
{
#pragma unroll
    for (int o = LPP / 2; o > 0; o >>= 1)
#pragma unroll
        for (int q = 0; q < N; ++q) Q[q] += __shfl_xor_sync(gmask, Q[q], o);
}

template <int LPP>
__device__ __forceinline__ void group_sum12(float (&Q)[12], unsigned gmask, int gl, int gbase)
{
    if constexpr (LPP == 16) {
        const bool h8 = gl & 8, h4 = gl & 4, h2 = gl & 2, h1 = gl & 1;
        float a6[6];
#pragma unroll
        for (int k = 0; k < 6; ++k)
            a6[k] = (h8 ? Q[k + 6] : Q[k]) + __shfl_xor_sync(gmask, h8 ? Q[k] : Q[k + 6], 8);
        float a3[3];
#pragma unroll
        for (int k = 0; k < 3; ++k)
            a3[k] = (h4 ? a6[k + 3] : a6[k]) + __shfl_xor_sync(gmask, h4 ? a6[k] : a6[k + 3], 4);
        // three values over bit 1: the low lane keeps 0 and 1, the high lane keeps 2
        const float r0 = __shfl_xor_sync(gmask, h2 ? a3[0] : a3[2], 2);
        const float r1 = __shfl_xor_sync(gmask, h2 ? a3[1] : 0.0f, 2);
        const float w2a = (h2 ? a3[2] : a3[0]) + r0;
        const float w2b = h2 ? 0.0f : a3[1] + r1;
        const float w1 = (h1 ? w2b : w2a) + __shfl_xor_sync(gmask, h1 ? w2a : w2b, 1);
#pragma unroll
        for (int k = 0; k < 12; ++k)
            Q[k] = __shfl_sync(gmask, w1, gbase + 8 * (k / 6) + 4 * ((k % 6) / 3) + 2 * (k % 3 == 2) + (k % 3 == 1));
    } else {
#pragma unroll
        for (int o = LPP / 2; o > 0; o >>= 1)
#pragma unroll
            for (int q = 0; q < 12; ++q) Q[q] += __shfl_xor_sync(gmask, Q[q], o);
    }
}

// PSC: compile-time patch size (0: the runtime `ps_rt`).  MINB: resident blocks per SM the
// register allocation must allow (chosen per variant by measurement: the default 12x12 and 8x8
// variants run at 7 and 8 blocks, which spills a few registers (36 and 12 bytes per thread) and
// gains more in latency hiding than the spills cost).  GSM: template gradients in shared memory (else in
// registers; measured per variant, see launch_search).
// DOF / ROBUST: the modes above; `norm` (1 L1, 2 Huber) and `huber_b` are read by ROBUST only.
// TERM: term2 > 0 makes a patch stop after the first update whose squared step length is at most
// term2 (early termination on a small step; 0: the fixed count, ended early only where exact).
template <int LPP, int PPL, int PSC, int MINB, bool GSM, int DOF = 2, bool ROBUST = false, bool TERM = false>
__global__ void __launch_bounds__(kSearchThreads, MINB) search_kernel(const __grid_constant__ Jobs<LevelJob> js, long long total,
                                                     int ps_rt, int stride, int iters, int norm, float huber_b,
                                                     float term2, unsigned int* __restrict__ wq)
{
    static_assert(DOF == 1 || DOF == 2, "one or two degrees of freedom");
    extern __shared__ float smem[];
    constexpr int GPW = 32 / LPP;  // patches per warp
    const int ps = PSC ? PSC : ps_rt;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    const int grp = lane / LPP, gl = lane % LPP;
    const unsigned gmask = (LPP == 32) ? 0xffffffffu : (((1u << LPP) - 1u) << (grp * LPP));
    const int ws = ps + 2, n = ps * ps;
    float* win = smem + (wib * GPW + grp) * (ws * ws + (GSM ? 2 * n : 0));  // the group's I0 window,
    float* gxs = win + ws * ws;                                             // then (GSM) the template
    float* gys = gxs + n;                                                   // gradients
    // after the groups' regions, per thread: the offset ky * pitch + kx of each of its patch
    // pixels k = gl + LPP m (set per patch), so that a rebuild addresses a pixel's taps from the
    // cell's two row pointers
    int* offs = reinterpret_cast<int*>(smem + (kSearchThreads / LPP) * (ws * ws + (GSM ? 2 * n : 0))) + threadIdx.x;
    const float inv_n = 1.0f / (float)n;
    // Patch assignment.  Every group starts on patch (its index in the grid); with a work queue
    // it then takes the next unclaimed patch (patch costs vary several-fold with the texture and
    // the iterations to convergence, so a fixed stride leaves SMs idle at the end of the launch),
    // else it strides by the number of groups.  A patch's result does not depend on the group
    // that computes it.
    const long long ngroups = (long long)gridDim.x * wpb * GPW;
    long long g = ((long long)blockIdx.x * wpb + wib) * GPW + grp;
    while (g < total) {
        // claimed now, read after this patch: the atomic's latency hides behind the patch
        unsigned int qn = 0;
        if (wq && gl == 0) qn = atomicAdd(wq, 1u);
        const LevelJob& J = job_ref(js, find_job(js, g, &LevelJob::patch_base));
        const long long pk = g - J.patch_base;
        const int w = J.w, h = J.h, pitch = J.pitch;
        const int j = (int)(pk / J.nx), i = (int)(pk - (long long)j * J.nx);
        const int px = min(i * stride, w - ps), py = min(j * stride, h - ps);
        const float2 ui = init_flow_at(J.Uc, J.wc, J.hc, J.cscale, (float)px + 0.5f * (float)(ps - 1),
                                       (float)py + 0.5f * (float)(ps - 1));
        float u = ui.x, v = ui.y;
        int st = 0;
        if (J.frozen) {
            const float2 f = J.frozen[pk];
            u += f.x;
            v += f.y;
        } else {
            // ---- template window, gradients, Hessian (once per patch)
            for (int t = gl; t < ws * ws; t += LPP) {
                const int a = t % ws, b = t / ws;
                win[t] = __ldg(J.S0 + (long long)clampi(py - 1 + b, 0, h - 1) * pitch + clampi(px - 1 + a, 0, w - 1));
            }
            if constexpr (!ROBUST) {
#pragma unroll
                for (int m = 0; m < PPL; ++m) {
                    const int k = gl + LPP * m;
                    if (k < n) offs[m * kSearchThreads] = (k / ps) * pitch + k % ps;
                }
            }
            __syncwarp(gmask);
            float s0 = 0.0f, h00 = 0.0f, h01 = 0.0f, h11 = 0.0f, sgx = 0.0f, sgy = 0.0f, sT = 0.0f;
            float gxr[GSM ? 1 : PPL], gyr[GSM ? 1 : PPL];
#pragma unroll
            for (int m = 0; m < PPL; ++m) {
                const int k = gl + LPP * m;
                if (!GSM) gxr[GSM ? 0 : m] = gyr[GSM ? 0 : m] = 0.0f;
                if (k < n) {
                    const int kx = k % ps, ky = k / ps;
                    const float* c0 = win + ky * ws + kx;  // (x-1, y-1)
                    const float* c1 = c0 + ws;
                    const float* c2 = c1 + ws;
                    s0 += c1[1];
                    const float gx = 0.125f * ((c0[2] - c0[0]) + 2.0f * (c1[2] - c1[0]) + (c2[2] - c2[0]));
                    const float gy = 0.125f * ((c2[0] - c0[0]) + 2.0f * (c2[1] - c0[1]) + (c2[2] - c0[2]));
                    if (GSM) {
                        gxs[k] = gx;  // read back by this lane only
                        gys[k] = gy;
                    } else {
                        gxr[GSM ? 0 : m] = gx;
                        gyr[GSM ? 0 : m] = gy;
                    }
                    h00 = fmaf(gx, gx, h00);
                    h01 = fmaf(gx, gy, h01);
                    h11 = fmaf(gy, gy, h11);
                    sgx += gx;
                    sgy += gy;
                }
            }
            const float mean0 = group_sum<LPP>(s0, gmask) * inv_n;
            __syncwarp(gmask);  // every lane has read its gradient neighbourhood
            float sgxT = 0.0f, sgyT = 0.0f;
#pragma unroll
            for (int m = 0; m < PPL; ++m) {
                const int k = gl + LPP * m;
                if (k < n) {
                    const float tv = win[(k / ps + 1) * ws + k % ps + 1] - mean0;  // the template T
                    sT += tv;
                    sgxT = fmaf(GSM ? gxs[k] : gxr[GSM ? 0 : m], tv, sgxT);
                    sgyT = fmaf(GSM ? gys[k] : gyr[GSM ? 0 : m], tv, sgyT);
                }
            }
#pragma unroll
            for (int o = LPP / 2; o > 0; o >>= 1) {
                h00 += __shfl_xor_sync(gmask, h00, o);
                h11 += __shfl_xor_sync(gmask, h11, o);
                sgx += __shfl_xor_sync(gmask, sgx, o);
                if constexpr (!ROBUST) {
                    sT += __shfl_xor_sync(gmask, sT, o);
                    sgxT += __shfl_xor_sync(gmask, sgxT, o);
                }
                if constexpr (DOF == 2) {
                    h01 += __shfl_xor_sync(gmask, h01, o);
                    sgy += __shfl_xor_sync(gmask, sgy, o);
                    if constexpr (!ROBUST) sgyT += __shfl_xor_sync(gmask, sgyT, o);
                }
            }
            bool flat;
            float k00, k01 = 0.0f, k11 = 0.0f;  // H'^-1 (DOF 1: 1 / H'_xx)
            if constexpr (DOF == 2) {
                // 2x2 determinant with the product h01^2 split exactly (Kahan)
                const float p2 = h01 * h01;
                const float e2 = fmaf(h01, h01, -p2);
                const float det = fmaf(h00, h11, -p2) - e2;
                const float tr = 0.5f * (h00 + h11);
                flat = !(det > 1.0e-6f * tr * tr);
                const float idet = 1.0f / det;
                k00 = h11 * idet;
                k01 = -h01 * idet;
                k11 = h00 * idet;
            } else {
                flat = !(h00 > 1.0e-6f * (0.5f * (h00 + h11)));
                k00 = 1.0f / h00;
            }
            if (flat) {
                st = 2;
            } else if constexpr (ROBUST) {
                // per-pixel coefficients of the current cell: w - T = c0 + ax c1 + ay (c2 + ax c3)
                float c0[PPL], c1[PPL], c2[PPL], c3[PPL];
                float R[4];  // cell sums of the taps: sum w = R0 + ax R1 + ay (R2 + ax R3)
                int ciu = INT_MIN, civ = INT_MIN;
                float u1 = 0.0f, v1 = 0.0f;
                const float b2 = huber_b * huber_b, twob = 2.0f * huber_b;
                for (int it = 0; it < iters; ++it) {
                    const float uc = fminf(fmaxf(u, -1.0e7f), 1.0e7f);
                    const float vc = fminf(fmaxf(v, -1.0e7f), 1.0e7f);
                    const float fu = floorf(uc), fv = floorf(vc);
                    const float ax = uc - fu, ay = vc - fv;
                    const int iu = (int)fu, iv = (int)fv;
                    if (iu != ciu || iv != civ) {
                        ciu = iu;
                        civ = iv;
                        const int xi = px + iu, yi = py + iv;
                        const bool inside = xi >= 0 && yi >= 0 && xi + ps <= w - 1 && yi + ps <= h - 1;
#pragma unroll
                        for (int q = 0; q < 4; ++q) R[q] = 0.0f;
#pragma unroll
                        for (int m = 0; m < PPL; ++m) {
                            const int k = gl + LPP * m;
                            c0[m] = c1[m] = c2[m] = c3[m] = 0.0f;
                            if (k < n) {
                                const int kx = k % ps, ky = k / ps;
                                float tp[4];
                                if (inside) {
                                    const float* p = J.S1 + (long long)(yi + ky) * pitch + (xi + kx);
                                    tp[0] = __ldg(p);
                                    tp[1] = __ldg(p + 1);
                                    tp[2] = __ldg(p + pitch);
                                    tp[3] = __ldg(p + pitch + 1);
                                } else {
                                    const int x0 = clampi(xi + kx, 0, w - 1), x1 = clampi(xi + kx + 1, 0, w - 1);
                                    const float* r0 = J.S1 + (long long)clampi(yi + ky, 0, h - 1) * pitch;
                                    const float* r1 = J.S1 + (long long)clampi(yi + ky + 1, 0, h - 1) * pitch;
                                    tp[0] = __ldg(r0 + x0);
                                    tp[1] = __ldg(r0 + x1);
                                    tp[2] = __ldg(r1 + x0);
                                    tp[3] = __ldg(r1 + x1);
                                }
#pragma unroll
                                for (int q = 0; q < 4; ++q) R[q] += tp[q];
                                const float tv = win[(ky + 1) * ws + kx + 1] - mean0;  // the template T
                                c0[m] = tp[0] - tv;
                                c1[m] = tp[1] - tp[0];
                                c2[m] = tp[2] - tp[0];
                                c3[m] = (tp[3] - tp[2]) - (tp[1] - tp[0]);
                            }
                        }
                        group_sumN<LPP, 4>(R, gmask);
                        R[3] = (R[3] - R[2]) - (R[1] - R[0]);
                        R[1] -= R[0];
                        R[2] -= R[0];
                    }
                    const float mw = fmaf(ay, fmaf(ax, R[3], R[2]), fmaf(ax, R[1], R[0])) * inv_n;
                    float bq[DOF];
#pragma unroll
                    for (int d = 0; d < DOF; ++d) bq[d] = 0.0f;
#pragma unroll
                    for (int m = 0; m < PPL; ++m) {
                        const int k = gl + LPP * m;
                        if (k < n) {
                            const float r = fmaf(ay, fmaf(ax, c3[m], c2[m]), fmaf(ax, c1[m], c0[m])) - mw;
                            const float ar = fabsf(r);
                            // correctly rounded square roots: the L1 transform's slope is unbounded
                            // at e = 0, and an approximate root's few ulp measurably move the
                            // search of weakly textured patches
                            const float e = norm == 1 ? copysignf(sqrtf(ar), r)
                                                      : (ar < huber_b ? r : copysignf(sqrtf(fmaf(twob, ar, -b2)), r));
                            bq[0] = fmaf(GSM ? gxs[k] : gxr[GSM ? 0 : m], e, bq[0]);
                            if constexpr (DOF == 2) bq[DOF - 1] = fmaf(GSM ? gys[k] : gyr[GSM ? 0 : m], e, bq[DOF - 1]);
                        }
                    }
                    group_sumN<LPP, DOF>(bq, gmask);
                    float un, vn = v;
                    if constexpr (DOF == 2) {
                        un = u - fmaf(k00, bq[0], k01 * bq[DOF - 1]);
                        vn = v - fmaf(k01, bq[0], k11 * bq[DOF - 1]);
                    } else {
                        un = u - k00 * bq[0];
                    }
                    if (TERM && term2 > 0.0f && (un - u) * (un - u) + (vn - v) * (vn - v) <= term2) {
                        u = un;
                        v = vn;
                        break;
                    }
                    // the state is (u, v) alone: a repeat two iterates back is a 2-cycle
                    if (search_cycle_exit(u, v, un, vn, u1, v1, 2, iters - 1 - it)) break;
                }
            } else {
                constexpr int NQ = 4 + 4 * DOF;
                float Q[NQ];  // T0..T3, Gx0..Gx3, (DOF 2) Gy0..Gy3 of the current cell
                int ciu = INT_MIN, civ = INT_MIN;
                float mref = mean0, mcur = mean0;
                float u1 = 0.0f, v1 = 0.0f;  // the iterate before the current one
                int quiet = 0;               // 1 + iterations since the last rebuild
                for (int it = 0; it < iters; ++it) {
                    const float uc = fminf(fmaxf(u, -1.0e7f), 1.0e7f);
                    const float vc = fminf(fmaxf(v, -1.0e7f), 1.0e7f);
                    const float fu = floorf(uc), fv = floorf(vc);
                    const float ax = uc - fu, ay = vc - fv;
                    const int iu = (int)fu, iv = (int)fv;
                    if (iu != ciu || iv != civ) {
                        // the integer displacement moved: rebuild the cell sums from the taps
                        ciu = iu;
                        civ = iv;
                        mref = mcur;
                        quiet = 0;
                        const int xi = px + iu, yi = py + iv;
                        const bool inside = xi >= 0 && yi >= 0 && xi + ps <= w - 1 && yi + ps <= h - 1;
#pragma unroll
                        for (int q = 0; q < NQ; ++q) Q[q] = 0.0f;
                        // inside the image: the first pixel's top-left tap
                        const float* r0 = J.S1;
                        if (inside) r0 += (long long)yi * pitch + xi;
                        // raw tap sums: Q[t] = sum tap_t, Q[4 + t] = sum gx tap_t, Q[8 + t] = sum
                        // gy tap_t for the taps t = a, b, c, d; the cell sums follow below.  (Sums
                        // relative to the patch mean would be residual-sized, but cost 4 more adds
                        // per pixel, 6 % of the kernel; raw sums keep the search within 3e-4 px of
                        // the FP64 result.)
#pragma unroll
                        for (int m = 0; m < PPL; ++m) {
                            const int k = gl + LPP * m;
                            if (k < n) {
                                const float gx = GSM ? gxs[k] : gxr[GSM ? 0 : m];
                                float tp[4];
                                if (inside) {
                                    const int o = offs[m * kSearchThreads];
                                    tp[0] = __ldg(r0 + o);
                                    tp[1] = __ldg(r0 + o + 1);
                                    tp[2] = __ldg(r0 + (o + pitch));
                                    tp[3] = __ldg(r0 + (o + pitch) + 1);
                                } else {
                                    const int kx = k % ps, ky = k / ps;
                                    const int x0 = clampi(xi + kx, 0, w - 1), x1 = clampi(xi + kx + 1, 0, w - 1);
                                    const float* r0 = J.S1 + (long long)clampi(yi + ky, 0, h - 1) * pitch;
                                    const float* r1 = J.S1 + (long long)clampi(yi + ky + 1, 0, h - 1) * pitch;
                                    tp[0] = __ldg(r0 + x0);
                                    tp[1] = __ldg(r0 + x1);
                                    tp[2] = __ldg(r1 + x0);
                                    tp[3] = __ldg(r1 + x1);
                                }
#pragma unroll
                                for (int q = 0; q < 4; ++q) {
                                    Q[q] += tp[q];
                                    Q[4 + q] = fmaf(gx, tp[q], Q[4 + q]);
                                }
                                if constexpr (DOF == 2) {
                                    const float gy = GSM ? gys[k] : gyr[GSM ? 0 : m];
#pragma unroll
                                    for (int q = 0; q < 4; ++q) Q[NQ - 4 + q] = fmaf(gy, tp[q], Q[NQ - 4 + q]);
                                }
                            }
                        }
                        if constexpr (DOF == 2)
                            group_sum12<LPP>(Q, gmask, gl, grp * LPP);
                        else
                            group_sumN<LPP, NQ>(Q, gmask);
                        // cell sums over t = (a - T - mref, b - a, c - a, d - c - b + a)
#pragma unroll
                        for (int g3 = 0; g3 < NQ; g3 += 4) {
                            const float ra = Q[g3], rb = Q[g3 + 1], rc = Q[g3 + 2], rd = Q[g3 + 3];
                            Q[g3 + 1] = rb - ra;
                            Q[g3 + 2] = rc - ra;
                            Q[g3 + 3] = (rd - rc) - (rb - ra);
                        }
                        Q[0] = (Q[0] - sT) - (float)n * mref;
                        Q[4] = (Q[4] - sgxT) - mref * sgx;
                        if constexpr (DOF == 2) Q[NQ - 4] = (Q[NQ - 4] - sgyT) - mref * sgy;
                    }
                    const float A0 = fmaf(ay, fmaf(ax, Q[3], Q[2]), fmaf(ax, Q[1], Q[0]));
                    const float Ax = fmaf(ay, fmaf(ax, Q[7], Q[6]), fmaf(ax, Q[5], Q[4]));
                    const float e = (A0 + sT) * inv_n;  // mean of the window minus mref
                    const float b0 = fmaf(-e, sgx, Ax);
                    mcur = mref + e;
                    float un, vn = v;
                    if constexpr (DOF == 2) {
                        const float Ay = fmaf(ay, fmaf(ax, Q[NQ - 1], Q[NQ - 2]), fmaf(ax, Q[NQ - 3], Q[NQ - 4]));
                        const float b1 = fmaf(-e, sgy, Ay);
                        un = u - fmaf(k00, b0, k01 * b1);
                        vn = v - fmaf(k01, b0, k11 * b1);
                    } else {
                        un = u - k00 * b0;
                    }
                    if (TERM && term2 > 0.0f && (un - u) * (un - u) + (vn - v) * (vn - v) <= term2) {
                        u = un;
                        v = vn;
                        break;
                    }
                    ++quiet;
                    if (search_cycle_exit(u, v, un, vn, u1, v1, quiet, iters - 1 - it)) break;
                }
            }
            // outlier reset (Alg. 1 step 4); a flat patch is still at u_init
            const float ex = u - ui.x, ey = v - ui.y;
            if (ex * ex + ey * ey > (float)(ps * ps)) {
                st = 1;
                u = ui.x;
                v = ui.y;
            }
            __syncwarp(gmask);  // the window is rewritten by the next patch of this group
        }
        if (gl == 0) {
            J.pu[pk] = make_float2(u, v);
            if (J.pui) J.pui[pk] = ui;
            if (J.pst) J.pst[pk] = st;
            if (J.record) J.record[pk] = make_float2(u - ui.x, v - ui.y);
        }
        g = wq ? ngroups + (long long)__shfl_sync(gmask, qn, grp * LPP) : g + ngroups;
    }
    if (wq && gl == 0) {
        // this group claims nothing more; the last group to get here zeroes the queue for the
        // next launch (every other group's last claim is ordered before its count by the fence)
        __threadfence();
        if (atomicAdd(wq + 1, 1u) == (unsigned int)ngroups - 1u) {
            __threadfence();
            atomicExch(wq, 0u);
            atomicExch(wq + 1, 0u);
        }
    }
}

template <int LPP, int PPL, int PSC, int MINB = 1, bool GSM = true, int DOF = 2, bool ROBUST = false,
          bool TERM = false>
static cudaError_t launch_lp(const Jobs<LevelJob>& js, long long total, int ps, int stride, int iters,
                             const LaunchCfg& lc, cudaStream_t s, int norm = 0, float huber_b = 0.0f,
                             float term2 = 0.0f)
{
    const int threads = kSearchThreads, wpb = threads / 32, per_block = wpb * (32 / LPP);
    const size_t smem = (size_t)per_block * ((ps + 2) * (ps + 2) + (GSM ? 2 * ps * ps : 0)) * sizeof(float) +
                        (size_t)PPL * threads * sizeof(int);
    static int occ = 0;
    if (occ == 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, search_kernel<LPP, PPL, PSC, MINB, GSM, DOF, ROBUST, TERM>, threads,
                                                          smem) !=
                cudaSuccess ||
            occ < 1)
            occ = 1;
    }
    long long blocks = (total + per_block - 1) / per_block;
    const long long cap = (long long)lc.sm_count * occ;
    if (blocks > cap) blocks = cap;
    // the queue's 32-bit counters hold the patch count plus one claim per group
    unsigned int* wq = total + blocks * per_block < (1LL << 31) ? lc.wq : nullptr;
    search_kernel<LPP, PPL, PSC, MINB, GSM, DOF, ROBUST, TERM>
        <<<(int)blocks, threads, smem, s>>>(js, total, ps, stride, iters, norm, huber_b, term2, wq);
    return cudaGetLastError();
}

}  // namespace dis
