// Inverse-compositional patch search of DIS (Sec. 2.1; supplementary Sec. A, Eq. solvereqinv;
// Alg. 1 steps 1-3 and the outlier reset of step 4).
//
// One warp per patch.  The prologue stages the (ps+2)^2 window of I0 around the patch in
// shared memory, computes the Sobel/8 gradients S' = grad T, the mean-normalised template T
// and the 2x2 Hessian H' = sum S'^T S' (reduced with warp shuffles), all kept in registers.
// Each of the theta_it iterations samples I1 bilinearly at x + u (one fractional weight pair
// for the whole patch), removes the sample mean, and reduces b = sum S'^T (w - T) across the
// warp; u <- u - H'^-1 b.  Lane l owns patch pixels l, l + 32, ... (M = ceil(ps^2 / 32)).
#include "dis_device.cuh"

namespace dis {

template <int M>
__global__ void __launch_bounds__(256) search_kernel(const __grid_constant__ Jobs<LevelJob> js, long long total,
                                                     int ps, int stride, int iters)
{
    extern __shared__ float smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    const int ws = ps + 2, n = ps * ps;
    float* win = smem + wib * ws * ws;
    const float inv_n = 1.0f / (float)n;
    int kx[M], ky[M];
#pragma unroll
    for (int m = 0; m < M; ++m) {
        const int k = lane + 32 * m;
        kx[m] = k < n ? k % ps : 0;
        ky[m] = k < n ? k / ps : 0;
    }
    for (long long g = (long long)blockIdx.x * wpb + wib; g < total; g += (long long)gridDim.x * wpb) {
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
            // ---- template, gradients, Hessian (computed once per patch)
            for (int t = lane; t < ws * ws; t += 32) {
                const int a = t % ws, b = t / ws;
                win[t] = __ldg(J.S0 + (long long)clampi(py - 1 + b, 0, h - 1) * pitch + clampi(px - 1 + a, 0, w - 1));
            }
            __syncwarp();
            float T[M], gx[M], gy[M];
            float s0 = 0.0f;
#pragma unroll
            for (int m = 0; m < M; ++m) {
                if (lane + 32 * m < n) {
                    const float* c0 = win + ky[m] * ws + kx[m];  // (x-1, y-1)
                    const float* c1 = c0 + ws;
                    const float* c2 = c1 + ws;
                    T[m] = c1[1];
                    s0 += c1[1];
                    gx[m] = 0.125f * ((c0[2] - c0[0]) + 2.0f * (c1[2] - c1[0]) + (c2[2] - c2[0]));
                    gy[m] = 0.125f * ((c2[0] - c0[0]) + 2.0f * (c2[1] - c0[1]) + (c2[2] - c0[2]));
                } else {
                    T[m] = gx[m] = gy[m] = 0.0f;
                }
            }
            __syncwarp();
            const float mean0 = warp_sum(s0) * inv_n;
            float h00 = 0.0f, h01 = 0.0f, h11 = 0.0f;
#pragma unroll
            for (int m = 0; m < M; ++m) {
                if (lane + 32 * m < n) T[m] -= mean0;
                h00 = fmaf(gx[m], gx[m], h00);
                h01 = fmaf(gx[m], gy[m], h01);
                h11 = fmaf(gy[m], gy[m], h11);
            }
            h00 = warp_sum(h00);
            h01 = warp_sum(h01);
            h11 = warp_sum(h11);
            // 2x2 determinant with the product h01^2 split exactly (Kahan)
            const float p2 = h01 * h01;
            const float e2 = fmaf(h01, h01, -p2);
            const float det = fmaf(h00, h11, -p2) - e2;
            const float tr = 0.5f * (h00 + h11);
            if (!(det > 1.0e-6f * tr * tr)) {
                st = 2;
            } else {
                const float idet = 1.0f / det;
                for (int it = 0; it < iters; ++it) {
                    const float uc = fminf(fmaxf(u, -1.0e7f), 1.0e7f);
                    const float vc = fminf(fmaxf(v, -1.0e7f), 1.0e7f);
                    const float fu = floorf(uc), fv = floorf(vc);
                    const float ax = uc - fu, ay = vc - fv;
                    const int xi = px + (int)fu, yi = py + (int)fv;
                    float wv[M];
                    float sw = 0.0f;
                    if (xi >= 0 && yi >= 0 && xi + ps <= w - 1 && yi + ps <= h - 1) {
                        const float* base = J.S1 + (long long)yi * pitch + xi;
#pragma unroll
                        for (int m = 0; m < M; ++m) {
                            if (lane + 32 * m < n) {
                                const float* p = base + ky[m] * pitch + kx[m];
                                const float a = __ldg(p), b = __ldg(p + 1), c = __ldg(p + pitch), d = __ldg(p + pitch + 1);
                                const float top = fmaf(ax, b - a, a), bot = fmaf(ax, d - c, c);
                                wv[m] = fmaf(ay, bot - top, top);
                                sw += wv[m];
                            } else {
                                wv[m] = 0.0f;
                            }
                        }
                    } else {
#pragma unroll
                        for (int m = 0; m < M; ++m) {
                            if (lane + 32 * m < n) {
                                const int x0 = clampi(xi + kx[m], 0, w - 1), x1 = clampi(xi + kx[m] + 1, 0, w - 1);
                                const int y0 = clampi(yi + ky[m], 0, h - 1), y1 = clampi(yi + ky[m] + 1, 0, h - 1);
                                const float* r0 = J.S1 + (long long)y0 * pitch;
                                const float* r1 = J.S1 + (long long)y1 * pitch;
                                const float a = __ldg(r0 + x0), b = __ldg(r0 + x1), c = __ldg(r1 + x0), d = __ldg(r1 + x1);
                                const float top = fmaf(ax, b - a, a), bot = fmaf(ax, d - c, c);
                                wv[m] = fmaf(ay, bot - top, top);
                                sw += wv[m];
                            } else {
                                wv[m] = 0.0f;
                            }
                        }
                    }
                    const float mw = warp_sum(sw) * inv_n;
                    float b0 = 0.0f, b1 = 0.0f;
#pragma unroll
                    for (int m = 0; m < M; ++m) {
                        const float r = (lane + 32 * m < n) ? (wv[m] - mw) - T[m] : 0.0f;
                        b0 = fmaf(gx[m], r, b0);
                        b1 = fmaf(gy[m], r, b1);
                    }
                    b0 = warp_sum(b0);
                    b1 = warp_sum(b1);
                    u -= (h11 * b0 - h01 * b1) * idet;
                    v -= (h00 * b1 - h01 * b0) * idet;
                }
                const float ex = u - ui.x, ey = v - ui.y;
                if (ex * ex + ey * ey > (float)(ps * ps)) {
                    st = 1;
                    u = ui.x;
                    v = ui.y;
                }
            }
        }
        if (lane == 0) {
            J.pu[pk] = make_float2(u, v);
            if (J.pui) J.pui[pk] = ui;
            if (J.pst) J.pst[pk] = st;
            if (J.record) J.record[pk] = make_float2(u - ui.x, v - ui.y);
        }
    }
}

template <int M>
static cudaError_t launch_m(const Jobs<LevelJob>& js, long long total, int ps, int stride, int iters,
                            const LaunchCfg& lc, cudaStream_t s)
{
    const int threads = 256, wpb = threads / 32;
    const size_t smem = (size_t)wpb * (ps + 2) * (ps + 2) * sizeof(float);
    static int occ = 0;
    if (occ == 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, search_kernel<M>, threads, smem) != cudaSuccess ||
            occ < 1)
            occ = 1;
    }
    long long blocks = (total + wpb - 1) / wpb;
    const long long cap = (long long)lc.sm_count * occ;
    if (blocks > cap) blocks = cap;
    search_kernel<M><<<(int)blocks, threads, smem, s>>>(js, total, ps, stride, iters);
    return cudaGetLastError();
}

cudaError_t launch_search(const Jobs<LevelJob>& js, long long total, int ps, int stride, int iters,
                          const LaunchCfg& lc, cudaStream_t s)
{
    if (total <= 0) return cudaSuccess;
    switch ((ps * ps + 31) / 32) {
        case 1: return launch_m<1>(js, total, ps, stride, iters, lc, s);
        case 2: return launch_m<2>(js, total, ps, stride, iters, lc, s);
        case 3: return launch_m<3>(js, total, ps, stride, iters, lc, s);
        case 4: return launch_m<4>(js, total, ps, stride, iters, lc, s);
        case 5: return launch_m<5>(js, total, ps, stride, iters, lc, s);
        case 6: return launch_m<6>(js, total, ps, stride, iters, lc, s);
        case 7: return launch_m<7>(js, total, ps, stride, iters, lc, s);
        case 8: return launch_m<8>(js, total, ps, stride, iters, lc, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace dis
