// Inverse-compositional patch search, warp-cooperative form (Sec. 2.1; supplementary Sec. A,
// Eq. solvereqinv; Alg. 1 steps 1-3 and the outlier reset of step 4).
//
// The arithmetic per patch is that of the grouped form in k_search.cu: while the integer part
// of u stays in one cell, the sums of one update factor into twelve cell sums T_k, Gx_k, Gy_k
// over t = (a - T - m, b - a, c - a, d - c - b + a) (taps a..d, template T, reference m), and
// every iteration costs a few scalar FMAs on them; the sums are rebuilt when the cell changes.
//
// Work split.  A warp owns G patches, a group of 32/G lanes per patch.  Each group runs the
// prologue of its patch (window staged in shared memory, Sobel/8 gradients, mean, H', sum S',
// sum T) and the scalar updates.  The template T and its gradients of all G patches stay in
// shared memory, so that a rebuild of the cell sums can be shared by the whole warp: for every
// patch whose integer displacement moved, the 32 lanes take pixels lane, lane + 32, ... and a
// transposed shuffle reduction (13 exchanges for 12 sums, then 12 broadcasts) hands the totals
// to the patch's group.  A rebuild thus costs ps^2 / 32 pixels per lane whatever G is, while the
// scalar update is shared by G patches per warp instruction: larger G trades scalar work
// against fewer warps in flight.
#include <climits>

#include "dis_device.cuh"

namespace dis {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kCoopWarps = 4;

struct CoopDesc {
    const float* S1;
    int pitch, w, h, px, py;
};

__host__ __device__ constexpr int coop_holder_lane(int k)
{
    return 16 * (k / 6) + 8 * ((k % 6) / 3) + 4 * ((k % 3) == 2) + 2 * ((k % 3) == 1);
}

// Sums P over the warp; the twelve totals end in Q of the lanes for which `take` holds.
__device__ __forceinline__ void coop_sum12(float (&P)[12], int lane, bool take, float (&Q)[12])
{
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4, b1 = lane & 2;
    float w6[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const float send = b4 ? P[k] : P[k + 6];
        const float keep = b4 ? P[k + 6] : P[k];
        w6[k] = keep + __shfl_xor_sync(kFull, send, 16);
    }
    float w3[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float send = b3 ? w6[k] : w6[k + 3];
        const float keep = b3 ? w6[k + 3] : w6[k];
        w3[k] = keep + __shfl_xor_sync(kFull, send, 8);
    }
    // three values over the bit-2 pair: the low lane keeps 0 and 1, the high lane keeps 2
    const float s0 = b2 ? w3[0] : w3[2];
    const float s1 = b2 ? w3[1] : 0.0f;
    const float r0 = __shfl_xor_sync(kFull, s0, 4);
    const float r1 = __shfl_xor_sync(kFull, s1, 4);
    const float w2a = (b2 ? w3[2] : w3[0]) + r0;
    const float w2b = b2 ? 0.0f : w3[1] + r1;
    float w1 = (b1 ? w2b : w2a) + __shfl_xor_sync(kFull, b1 ? w2a : w2b, 2);
    w1 += __shfl_xor_sync(kFull, w1, 1);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        const float v = __shfl_sync(kFull, w1, coop_holder_lane(k));
        if (take) Q[k] = v;
    }
}

template <int LPP>
__device__ __forceinline__ float coop_group_sum(float v)
{
#pragma unroll
    for (int o = LPP / 2; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

template <int PS, int G, int MINB>
__global__ void __launch_bounds__(kCoopWarps * 32, MINB)
    search_coop_kernel(const __grid_constant__ Jobs<LevelJob> js, long long total, int stride, int iters)
{
    constexpr int LPP = 32 / G, N = PS * PS, WS = PS + 2, PPL = (N + LPP - 1) / LPP;
    constexpr int RPL = (N + 31) / 32;  // pixels per lane in a rebuild
    __shared__ float s_tpl[kCoopWarps][G][3][N];  // T, gx, gy of each patch of the warp
    __shared__ float s_win[kCoopWarps][G][WS * WS];
    __shared__ CoopDesc s_desc[kCoopWarps][G];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int grp = lane / LPP, gl = lane % LPP;
    float* win = s_win[wib][grp];
    float(*tpl)[3][N] = s_tpl[wib];
    const float inv_n = 1.0f / (float)N;
    const long long step = (long long)gridDim.x * kCoopWarps * G;
    for (long long g0 = ((long long)blockIdx.x * kCoopWarps + wib) * G; g0 < total; g0 += step) {
        const bool valid = g0 + grp < total;
        const long long g = valid ? g0 + grp : total - 1;
        const LevelJob& J = job_ref(js, find_job(js, g, &LevelJob::patch_base));
        const long long pk = g - J.patch_base;
        const int w = J.w, h = J.h, pitch = J.pitch;
        const int j = (int)(pk / J.nx), i = (int)(pk - (long long)j * J.nx);
        const int px = min(i * stride, w - PS), py = min(j * stride, h - PS);
        const float2 ui = init_flow_at(J.Uc, J.wc, J.hc, J.cscale, (float)px + 0.5f * (float)(PS - 1),
                                       (float)py + 0.5f * (float)(PS - 1));
        float u = ui.x, v = ui.y;
        int st = 0;
        bool run = false;
        float k00 = 0.0f, k01 = 0.0f, k11 = 0.0f, sgx = 0.0f, sgy = 0.0f, sT = 0.0f, mref = 0.0f, mcur = 0.0f;
        float Q[12];
#pragma unroll
        for (int q = 0; q < 12; ++q) Q[q] = 0.0f;
        int ciu = INT_MIN, civ = INT_MIN;
        const bool frozen = J.frozen != nullptr;
        if (valid && frozen) {
            const float2 f = J.frozen[pk];
            u += f.x;
            v += f.y;
        }
        // ---- prologue of the group's patch (groups of frozen or missing patches idle along)
        if (valid && !frozen) {
            for (int t = gl; t < WS * WS; t += LPP) {
                const int a = t % WS, b = t / WS;
                win[t] = __ldg(J.S0 + (long long)clampi(py - 1 + b, 0, h - 1) * pitch + clampi(px - 1 + a, 0, w - 1));
            }
        }
        __syncwarp();
        float h00 = 0.0f, h01 = 0.0f, h11 = 0.0f, s0 = 0.0f;
        if (valid && !frozen) {
#pragma unroll
            for (int m = 0; m < PPL; ++m) {
                const int k = gl + LPP * m;
                if (k < N) s0 += win[(k / PS + 1) * WS + k % PS + 1];
            }
        }
        const float mean0 = coop_group_sum<LPP>(s0) * inv_n;
        if (valid && !frozen) {
#pragma unroll
            for (int m = 0; m < PPL; ++m) {
                const int k = gl + LPP * m;
                if (k < N) {
                    const int kx = k % PS, ky = k / PS;
                    const float* c0 = win + ky * WS + kx;  // (x-1, y-1)
                    const float* c1 = c0 + WS;
                    const float* c2 = c1 + WS;
                    const float gx = 0.125f * ((c0[2] - c0[0]) + 2.0f * (c1[2] - c1[0]) + (c2[2] - c2[0]));
                    const float gy = 0.125f * ((c2[0] - c0[0]) + 2.0f * (c2[1] - c0[1]) + (c2[2] - c0[2]));
                    const float T = c1[1] - mean0;
                    tpl[grp][0][k] = T;
                    tpl[grp][1][k] = gx;
                    tpl[grp][2][k] = gy;
                    sT += T;
                    h00 = fmaf(gx, gx, h00);
                    h01 = fmaf(gx, gy, h01);
                    h11 = fmaf(gy, gy, h11);
                    sgx += gx;
                    sgy += gy;
                }
            }
        }
        h00 = coop_group_sum<LPP>(h00);
        h01 = coop_group_sum<LPP>(h01);
        h11 = coop_group_sum<LPP>(h11);
        sgx = coop_group_sum<LPP>(sgx);
        sgy = coop_group_sum<LPP>(sgy);
        sT = coop_group_sum<LPP>(sT);
        if (valid && !frozen) {
            // 2x2 determinant with the product h01^2 split exactly (Kahan)
            const float p2 = h01 * h01;
            const float e2 = fmaf(h01, h01, -p2);
            const float det = fmaf(h00, h11, -p2) - e2;
            const float tr = 0.5f * (h00 + h11);
            if (!(det > 1.0e-6f * tr * tr)) {
                st = 2;
            } else {
                const float idet = 1.0f / det;
                k00 = h11 * idet;
                k01 = -h01 * idet;
                k11 = h00 * idet;
                run = true;
                mref = mcur = mean0;
            }
            if (gl == 0) s_desc[wib][grp] = CoopDesc{J.S1, pitch, w, h, px, py};
        }
        __syncwarp();
        bool live = run;           // still iterating (a fixed point or a 2-cycle ends it early)
        float u1 = 0.0f, v1 = 0.0f;  // the iterate before the current one
        int quiet = 0;               // 1 + iterations since the last rebuild
        if (__any_sync(kFull, live)) {
            for (int it = 0; it < iters; ++it) {
                float ax = 0.0f, ay = 0.0f;
                int iu = 0, iv = 0;
                bool need = false;
                if (live) {
                    const float uc = fminf(fmaxf(u, -1.0e7f), 1.0e7f);
                    const float vc = fminf(fmaxf(v, -1.0e7f), 1.0e7f);
                    const float fu = floorf(uc), fv = floorf(vc);
                    ax = uc - fu;
                    ay = vc - fv;
                    iu = (int)fu;
                    iv = (int)fv;
                    need = iu != ciu || iv != civ;
                }
                unsigned pend = __ballot_sync(kFull, need && gl == 0);
                while (pend) {
                    // the integer displacement of patch `sg` moved: the warp rebuilds its sums
                    const int sl = __ffs(pend) - 1, sg = sl / LPP;
                    pend &= pend - 1;
                    const int siu = __shfl_sync(kFull, iu, sl), siv = __shfl_sync(kFull, iv, sl);
                    const float sref = __shfl_sync(kFull, mcur, sl);
                    const CoopDesc d = s_desc[wib][sg];
                    const int xi = d.px + siu, yi = d.py + siv;
                    const bool inside = xi >= 0 && yi >= 0 && xi + PS <= d.w - 1 && yi + PS <= d.h - 1;
                    float P[12];
#pragma unroll
                    for (int q = 0; q < 12; ++q) P[q] = 0.0f;
#pragma unroll
                    for (int m = 0; m < RPL; ++m) {
                        const int k = lane + 32 * m;
                        if (k < N) {
                            const int ky = k / PS, kx = k - ky * PS;
                            const float T = tpl[sg][0][k], gx = tpl[sg][1][k], gy = tpl[sg][2][k];
                            float a, b, c, dd;
                            if (inside) {
                                const float* p = d.S1 + (long long)(yi + ky) * d.pitch + (xi + kx);
                                a = __ldg(p);
                                b = __ldg(p + 1);
                                c = __ldg(p + d.pitch);
                                dd = __ldg(p + d.pitch + 1);
                            } else {
                                const int x0 = clampi(xi + kx, 0, d.w - 1), x1 = clampi(xi + kx + 1, 0, d.w - 1);
                                const float* r0 = d.S1 + (long long)clampi(yi + ky, 0, d.h - 1) * d.pitch;
                                const float* r1 = d.S1 + (long long)clampi(yi + ky + 1, 0, d.h - 1) * d.pitch;
                                a = __ldg(r0 + x0);
                                b = __ldg(r0 + x1);
                                c = __ldg(r1 + x0);
                                dd = __ldg(r1 + x1);
                            }
                            const float t[4] = {(a - T) - sref, b - a, c - a, (dd - c) - (b - a)};
#pragma unroll
                            for (int q = 0; q < 4; ++q) {
                                P[q] += t[q];
                                P[4 + q] = fmaf(gx, t[q], P[4 + q]);
                                P[8 + q] = fmaf(gy, t[q], P[8 + q]);
                            }
                        }
                    }
                    const bool mine = grp == sg;
                    coop_sum12(P, lane, mine, Q);
                    if (mine) {
                        ciu = siu;
                        civ = siv;
                        mref = sref;
                        quiet = 0;
                    }
                }
                if (live) {
                    const float A0 = fmaf(ay, fmaf(ax, Q[3], Q[2]), fmaf(ax, Q[1], Q[0]));
                    const float Ax = fmaf(ay, fmaf(ax, Q[7], Q[6]), fmaf(ax, Q[5], Q[4]));
                    const float Ay = fmaf(ay, fmaf(ax, Q[11], Q[10]), fmaf(ax, Q[9], Q[8]));
                    const float e = (A0 + sT) * inv_n;  // mean of the window minus mref
                    const float b0 = fmaf(-e, sgx, Ax), b1 = fmaf(-e, sgy, Ay);
                    mcur = mref + e;
                    const float un = u - fmaf(k00, b0, k01 * b1);
                    const float vn = v - fmaf(k01, b0, k11 * b1);
                    ++quiet;
                    if (search_cycle_exit(u, v, un, vn, u1, v1, quiet, iters - 1 - it)) live = false;
                }
                if (!__any_sync(kFull, live)) break;
            }
        }
        if (run) {
            const float ex = u - ui.x, ey = v - ui.y;
            if (ex * ex + ey * ey > (float)(PS * PS)) {
                st = 1;
                u = ui.x;
                v = ui.y;
            }
        }
        if (valid && gl == 0) {
            J.pu[pk] = make_float2(u, v);
            if (J.pui) J.pui[pk] = ui;
            if (J.pst) J.pst[pk] = st;
            if (J.record) J.record[pk] = make_float2(u - ui.x, v - ui.y);
        }
        __syncwarp();  // shared memory is rewritten for the next G patches
    }
}

template <int PS, int G, int MINB>
cudaError_t launch_coop(const Jobs<LevelJob>& js, long long total, int stride, int iters, const LaunchCfg& lc,
                        cudaStream_t s)
{
    constexpr int threads = kCoopWarps * 32;
    static int occ = 0;
    if (occ == 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, search_coop_kernel<PS, G, MINB>, threads, 0) !=
                cudaSuccess ||
            occ < 1)
            occ = 1;
    }
    long long blocks = (total + kCoopWarps * G - 1) / (kCoopWarps * G);
    const long long cap = (long long)lc.sm_count * occ;
    if (blocks > cap) blocks = cap;
    search_coop_kernel<PS, G, MINB><<<(int)blocks, threads, 0, s>>>(js, total, stride, iters);
    return cudaGetLastError();
}

}  // namespace

bool search_coop_supported(int ps, int g) { return (ps == 8 && (g == 2 || g == 4 || g == 8)) || (ps == 12 && (g == 2 || g == 4)); }

cudaError_t launch_search_coop(const Jobs<LevelJob>& js, long long total, int ps, int stride, int iters, int g,
                               const LaunchCfg& lc, cudaStream_t s)
{
    if (total <= 0) return cudaSuccess;
    if (ps == 8) {
        if (g == 2) return launch_coop<8, 2, 6>(js, total, stride, iters, lc, s);
        if (g == 8) return launch_coop<8, 8, 6>(js, total, stride, iters, lc, s);
        return launch_coop<8, 4, 6>(js, total, stride, iters, lc, s);
    }
    if (g == 2) return launch_coop<12, 2, 6>(js, total, stride, iters, lc, s);
    return launch_coop<12, 4, 5>(js, total, stride, iters, lc, s);
}

}  // namespace dis
