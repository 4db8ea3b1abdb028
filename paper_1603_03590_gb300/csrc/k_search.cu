// Inverse-compositional patch search of DIS (Sec. 2.1; supplementary Sec. A, Eq. solvereqinv;
// Alg. 1 steps 1-3 and the outlier reset of step 4).
//
// A group of LPP lanes (8, 16 or 32 by patch size) owns one patch; lane l of the group owns
// patch pixels l, l + LPP, ... (PPL of them).  The prologue stages the (ps+2)^2 window of I0
// around the patch in shared memory and computes, in registers, the Sobel/8 gradients
// S' = grad T of the mean-normalised template T and the 2x2 Hessian H' = sum S'^T S' (group
// shuffle reductions); sum T and sum S' are kept for the update below.
//
// Iterations.  u is shared by the whole patch, so every pixel samples I1 with the same
// fractional weights (ax, ay).  Each pixel keeps its four bilinear taps folded into
// t0..t3 with t0 = I1(tap) - T - m, m a reference intensity fixed at the last re-read, so that
//   w'' = t0 + ax t1 + ay (t2 + ax t3) = I1(x + u) - T(x) - m.
// The taps stay in registers and are re-read only when the integer part of u changes (the
// clamped taps also encode the image border); a converged patch iterates from registers:
// 3 FMA per sample.  With A0 = sum w'', A = sum S' w'' and e = (A0 + sum T) / n (= mean w - m):
//   b = sum S'^T (w - mean w - T) = A - e sum S',   u <- u - H'^-1 b,
// all terms being residual-sized, which keeps the FP32 sums accurate.
#include <climits>

#include "dis_device.cuh"

namespace dis {

template <int LPP>
__device__ __forceinline__ float group_sum(float v, unsigned mask)
{
#pragma unroll
    for (int o = LPP / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o);
    return v;
}

// PSC: compile-time patch size (0: the runtime `ps_rt`).
template <int LPP, int PPL, int PSC>
__global__ void __launch_bounds__(128) search_kernel(const __grid_constant__ Jobs<LevelJob> js, long long total,
                                                     int ps_rt, int stride, int iters)
{
    extern __shared__ float smem[];
    constexpr int GPW = 32 / LPP;  // patches per warp
    const int ps = PSC ? PSC : ps_rt;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    const int grp = lane / LPP, gl = lane % LPP;
    const unsigned gmask = (LPP == 32) ? 0xffffffffu : (((1u << LPP) - 1u) << (grp * LPP));
    const int ws = ps + 2, n = ps * ps;
    float* win = smem + (wib * GPW + grp) * ws * ws;
    const float inv_n = 1.0f / (float)n;
    const long long step = (long long)gridDim.x * wpb * GPW;
    for (long long g = ((long long)blockIdx.x * wpb + wib) * GPW + grp; g < total; g += step) {
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
            __syncwarp(gmask);
            float gx[PPL], gy[PPL];
            float s0 = 0.0f;
#pragma unroll
            for (int m = 0; m < PPL; ++m) {
                const int k = gl + LPP * m;
                gx[m] = gy[m] = 0.0f;
                if (k < n) {
                    const int kx = k % ps, ky = k / ps;
                    const float* c0 = win + ky * ws + kx;  // (x-1, y-1)
                    const float* c1 = c0 + ws;
                    const float* c2 = c1 + ws;
                    s0 += c1[1];
                    gx[m] = 0.125f * ((c0[2] - c0[0]) + 2.0f * (c1[2] - c1[0]) + (c2[2] - c2[0]));
                    gy[m] = 0.125f * ((c2[0] - c0[0]) + 2.0f * (c2[1] - c0[1]) + (c2[2] - c0[2]));
                }
            }
            const float mean0 = group_sum<LPP>(s0, gmask) * inv_n;
            float h00 = 0.0f, h01 = 0.0f, h11 = 0.0f, sgx = 0.0f, sgy = 0.0f, sT = 0.0f;
#pragma unroll
            for (int m = 0; m < PPL; ++m) {
                const int k = gl + LPP * m;
                if (k < n) sT += win[(k / ps + 1) * ws + k % ps + 1] - mean0;
                h00 = fmaf(gx[m], gx[m], h00);
                h01 = fmaf(gx[m], gy[m], h01);
                h11 = fmaf(gy[m], gy[m], h11);
                sgx += gx[m];
                sgy += gy[m];
            }
#pragma unroll
            for (int o = LPP / 2; o > 0; o >>= 1) {
                h00 += __shfl_xor_sync(gmask, h00, o);
                h01 += __shfl_xor_sync(gmask, h01, o);
                h11 += __shfl_xor_sync(gmask, h11, o);
                sgx += __shfl_xor_sync(gmask, sgx, o);
                sgy += __shfl_xor_sync(gmask, sgy, o);
                sT += __shfl_xor_sync(gmask, sT, o);
            }
            // 2x2 determinant with the product h01^2 split exactly (Kahan)
            const float p2 = h01 * h01;
            const float e2 = fmaf(h01, h01, -p2);
            const float det = fmaf(h00, h11, -p2) - e2;
            const float tr = 0.5f * (h00 + h11);
            if (!(det > 1.0e-6f * tr * tr)) {
                st = 2;
            } else {
                const float idet = 1.0f / det;
                const float k00 = h11 * idet, k01 = -h01 * idet, k11 = h00 * idet;  // H'^-1
                float t0[PPL], t1[PPL], t2[PPL], t3[PPL];
                int ciu = INT_MIN, civ = INT_MIN;
                float mref = mean0;  // reference intensity of the folded taps
                float mcur = mean0;  // latest estimate of the window mean
                for (int it = 0; it < iters; ++it) {
                    const float uc = fminf(fmaxf(u, -1.0e7f), 1.0e7f);
                    const float vc = fminf(fmaxf(v, -1.0e7f), 1.0e7f);
                    const float fu = floorf(uc), fv = floorf(vc);
                    const float ax = uc - fu, ay = vc - fv;
                    const int iu = (int)fu, iv = (int)fv;
                    if (iu != ciu || iv != civ) {
                        // the integer displacement moved: re-read the taps (clamped at the border)
                        ciu = iu;
                        civ = iv;
                        mref = mcur;
                        const int xi = px + iu, yi = py + iv;
                        const bool inside = xi >= 0 && yi >= 0 && xi + ps <= w - 1 && yi + ps <= h - 1;
#pragma unroll
                        for (int m = 0; m < PPL; ++m) {
                            const int k = gl + LPP * m;
                            float a = 0.0f, b = 0.0f, c = 0.0f, d = 0.0f, T = 0.0f;
                            if (k < n) {
                                const int kx = k % ps, ky = k / ps;
                                T = win[(ky + 1) * ws + kx + 1] - mean0;
                                if (inside) {
                                    const float* p = J.S1 + (long long)(yi + ky) * pitch + (xi + kx);
                                    a = __ldg(p);
                                    b = __ldg(p + 1);
                                    c = __ldg(p + pitch);
                                    d = __ldg(p + pitch + 1);
                                } else {
                                    const int x0 = clampi(xi + kx, 0, w - 1), x1 = clampi(xi + kx + 1, 0, w - 1);
                                    const float* r0 = J.S1 + (long long)clampi(yi + ky, 0, h - 1) * pitch;
                                    const float* r1 = J.S1 + (long long)clampi(yi + ky + 1, 0, h - 1) * pitch;
                                    a = __ldg(r0 + x0);
                                    b = __ldg(r0 + x1);
                                    c = __ldg(r1 + x0);
                                    d = __ldg(r1 + x1);
                                }
                                t0[m] = (a - T) - mref;
                            } else {
                                t0[m] = 0.0f;
                            }
                            t1[m] = b - a;
                            t2[m] = c - a;
                            t3[m] = (d - c) - (b - a);
                        }
                    }
                    // two partial sums per quantity halve the dependency chains
                    float A0a = 0.0f, A0b = 0.0f, Axa = 0.0f, Axb = 0.0f, Aya = 0.0f, Ayb = 0.0f;
#pragma unroll
                    for (int m = 0; m < PPL; ++m) {
                        if (gl + LPP * m < n) {
                            const float wv = fmaf(ay, fmaf(ax, t3[m], t2[m]), fmaf(ax, t1[m], t0[m]));
                            if (m & 1) {
                                A0b += wv;
                                Axb = fmaf(gx[m], wv, Axb);
                                Ayb = fmaf(gy[m], wv, Ayb);
                            } else {
                                A0a += wv;
                                Axa = fmaf(gx[m], wv, Axa);
                                Aya = fmaf(gy[m], wv, Aya);
                            }
                        }
                    }
                    float A0 = A0a + A0b, Ax = Axa + Axb, Ay = Aya + Ayb;
#pragma unroll
                    for (int o = LPP / 2; o > 0; o >>= 1) {
                        A0 += __shfl_xor_sync(gmask, A0, o);
                        Ax += __shfl_xor_sync(gmask, Ax, o);
                        Ay += __shfl_xor_sync(gmask, Ay, o);
                    }
                    const float e = (A0 + sT) * inv_n;  // mean of the window minus mref
                    const float b0 = fmaf(-e, sgx, Ax), b1 = fmaf(-e, sgy, Ay);
                    mcur = mref + e;
                    u -= fmaf(k00, b0, k01 * b1);
                    v -= fmaf(k01, b0, k11 * b1);
                }
                const float ex = u - ui.x, ey = v - ui.y;
                if (ex * ex + ey * ey > (float)(ps * ps)) {
                    st = 1;
                    u = ui.x;
                    v = ui.y;
                }
            }
            __syncwarp(gmask);  // the window is rewritten by the next patch of this group
        }
        if (gl == 0) {
            J.pu[pk] = make_float2(u, v);
            if (J.pui) J.pui[pk] = ui;
            if (J.pst) J.pst[pk] = st;
            if (J.record) J.record[pk] = make_float2(u - ui.x, v - ui.y);
        }
    }
}

template <int LPP, int PPL, int PSC>
static cudaError_t launch_lp(const Jobs<LevelJob>& js, long long total, int ps, int stride, int iters,
                             const LaunchCfg& lc, cudaStream_t s)
{
    const int threads = 128, wpb = threads / 32, per_block = wpb * (32 / LPP);
    const size_t smem = (size_t)per_block * (ps + 2) * (ps + 2) * sizeof(float);
    static int occ = 0;
    if (occ == 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, search_kernel<LPP, PPL, PSC>, threads, smem) !=
                cudaSuccess ||
            occ < 1)
            occ = 1;
    }
    long long blocks = (total + per_block - 1) / per_block;
    const long long cap = (long long)lc.sm_count * occ;
    if (blocks > cap) blocks = cap;
    search_kernel<LPP, PPL, PSC><<<(int)blocks, threads, smem, s>>>(js, total, ps, stride, iters);
    return cudaGetLastError();
}

// Lanes per patch by patch size: 8 up to 8x8 (<= 8 pixels per lane), 16 up to 12x12 (<= 9),
// 32 up to 16x16 (<= 8); the 8x8 and 12x12 patches of the presets get compile-time sizes and
// alternative group widths `lanes` (0 = the default) for the autotuner.
cudaError_t launch_search(const Jobs<LevelJob>& js, long long total, int ps, int stride, int iters,
                          const LaunchCfg& lc, cudaStream_t s, int lanes)
{
    if (total <= 0) return cudaSuccess;
    const int n = ps * ps;
    if (ps == 8) {
        switch (lanes) {
            case 4: return launch_lp<4, 16, 8>(js, total, ps, stride, iters, lc, s);
            case 16: return launch_lp<16, 4, 8>(js, total, ps, stride, iters, lc, s);
            case 32: return launch_lp<32, 2, 8>(js, total, ps, stride, iters, lc, s);
            default: return launch_lp<8, 8, 8>(js, total, ps, stride, iters, lc, s);
        }
    }
    if (ps == 12) {
        switch (lanes) {
            case 8: return launch_lp<8, 18, 12>(js, total, ps, stride, iters, lc, s);
            case 32: return launch_lp<32, 5, 12>(js, total, ps, stride, iters, lc, s);
            default: return launch_lp<16, 9, 12>(js, total, ps, stride, iters, lc, s);
        }
    }
    if (ps < 8) {
        switch ((n + 7) / 8) {
            case 1: return launch_lp<8, 1, 0>(js, total, ps, stride, iters, lc, s);
            case 2: return launch_lp<8, 2, 0>(js, total, ps, stride, iters, lc, s);
            case 3: return launch_lp<8, 3, 0>(js, total, ps, stride, iters, lc, s);
            case 4: return launch_lp<8, 4, 0>(js, total, ps, stride, iters, lc, s);
            case 5: return launch_lp<8, 5, 0>(js, total, ps, stride, iters, lc, s);
            default: return launch_lp<8, 7, 0>(js, total, ps, stride, iters, lc, s);
        }
    }
    if (ps < 12) {
        switch ((n + 15) / 16) {
            case 6: return launch_lp<16, 6, 0>(js, total, ps, stride, iters, lc, s);
            case 7: return launch_lp<16, 7, 0>(js, total, ps, stride, iters, lc, s);
            default: return launch_lp<16, 8, 0>(js, total, ps, stride, iters, lc, s);
        }
    }
    switch ((n + 31) / 32) {
        case 6: return launch_lp<32, 6, 0>(js, total, ps, stride, iters, lc, s);
        case 7: return launch_lp<32, 7, 0>(js, total, ps, stride, iters, lc, s);
        default: return launch_lp<32, 8, 0>(js, total, ps, stride, iters, lc, s);
    }
}

int search_lane_options(int ps, int* out)
{
    if (ps == 8) {
        out[0] = 8, out[1] = 4, out[2] = 16, out[3] = 32;
        return 4;
    }
    if (ps == 12) {
        out[0] = 16, out[1] = 8, out[2] = 32;
        return 3;
    }
    out[0] = 0;
    return 1;
}

}  // namespace dis
