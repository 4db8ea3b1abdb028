// Inverse-compositional patch search, lane-per-patch form (Sec. 2.1; supplementary Sec. A,
// Eq. solvereqinv; Alg. 1 steps 1-3 and the outlier reset of step 4).
//
// The arithmetic per patch is that of the grouped form in k_search.cu: while the integer part
// of u stays in one cell, every pixel samples I1 with the same fractional weights (ax, ay), so
// the sums of one update factor into twelve cell sums
//   T_k = sum t_k,  Gx_k = sum gx t_k,  Gy_k = sum gy t_k,
//   t = (a - T - m, b - a, c - a, d - c - b + a)  from the pixel's four taps a..d,
// with T = I0 - mean(I0 over the patch) the template, (gx, gy) its Sobel/8 gradients and m a
// reference intensity; the update is
//   e = (A_T + sum T) / n,  b = A_G - e sum S',  u <- u - H'^-1 b,
// A = Q0 + ax Q1 + ay (Q2 + ax Q3) for each of the three sums, and m follows the window mean
// at every rebuild so that all sums stay residual-sized.
//
// Work split.  Each lane owns one patch for the whole search and runs its scalar update alone,
// so one warp instruction advances 32 patches.  The prologue (patch mean, gradients, H', sum S',
// sum T and the cell sums of the starting cell) is a serial loop per lane over its own patch.
// When a patch's integer displacement changes, the whole warp rebuilds that patch's cell sums:
// every lane takes pixels lane, lane + 32, ... of the pending patch, and a transposed shuffle
// reduction (13 exchanges for 12 sums, then 12 broadcasts) leaves the totals in the owner lane.
// Pending patches of one iteration are rebuilt one after the other.  Only the patches that
// actually changed cell pay for a rebuild, which is what makes this form cheaper than the
// grouped one, where a whole warp pays whenever any of its patches rebuilds.
#include <algorithm>
#include <climits>

#include "dis_device.cuh"

namespace dis {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kWarpsPerBlock = 4;

struct PatchDesc {
    const float* S0;
    const float* S1;
    const float4* tpl;
    const float4* tap;
    int pitch, w, h, px, py;
    float mean0;
};

// I0 at (x, y) and its Sobel/8 gradients with replicated border (x, y inside the image; the
// neighbours are clamped unless `inner` says the 3x3 neighbourhood is inside).
__device__ __forceinline__ void template_at(const float* __restrict__ S0, int pitch, int w, int h, int x, int y,
                                            bool inner, float& c, float& gx, float& gy)
{
    int xl = x - 1, xr = x + 1, yu = y - 1, yd = y + 1;
    if (!inner) {
        xl = max(xl, 0);
        xr = min(xr, w - 1);
        yu = max(yu, 0);
        yd = min(yd, h - 1);
    }
    const float* ru = S0 + (long long)yu * pitch;
    const float* rc = S0 + (long long)y * pitch;
    const float* rd = S0 + (long long)yd * pitch;
    const float a = __ldg(ru + xl), b = __ldg(ru + x), cc = __ldg(ru + xr);
    const float d = __ldg(rc + xl), f = __ldg(rc + xr);
    const float p = __ldg(rd + xl), q = __ldg(rd + x), s = __ldg(rd + xr);
    c = __ldg(rc + x);
    gx = 0.125f * ((cc - a) + 2.0f * (f - d) + (s - p));
    gy = 0.125f * ((p - a) + 2.0f * (q - b) + (s - cc));
}

// The four bilinear taps of I1 at integer (x, y): (x, y), (x+1, y), (x, y+1), (x+1, y+1),
// clamped to the image unless `inside` says all of them are inside.
__device__ __forceinline__ void taps_at(const float* __restrict__ S1, int pitch, int w, int h, int x, int y,
                                        bool inside, float& a, float& b, float& c, float& d)
{
    if (inside) {
        const float* p = S1 + (long long)y * pitch + x;
        a = __ldg(p);
        b = __ldg(p + 1);
        c = __ldg(p + pitch);
        d = __ldg(p + pitch + 1);
    } else {
        const int x0 = clampi(x, 0, w - 1), x1 = clampi(x + 1, 0, w - 1);
        const float* r0 = S1 + (long long)clampi(y, 0, h - 1) * pitch;
        const float* r1 = S1 + (long long)clampi(y + 1, 0, h - 1) * pitch;
        a = __ldg(r0 + x0);
        b = __ldg(r0 + x1);
        c = __ldg(r1 + x0);
        d = __ldg(r1 + x1);
    }
}

// Template value, gradients and the four taps of patch pixel (x, y) of I0 / (xt, yt) of I1:
// from the search planes when PLANES (tap plane valid when `tin`: the pixel's taps start inside
// the image), else from the images.  Both give the same values bit for bit.
template <bool PLANES>
__device__ __forceinline__ void fetch_pixel(const PatchDesc& d, int x, int y, int xt, int yt, bool inner, bool tin,
                                            float& c, float& gx, float& gy, float& a, float& b, float& cc, float& dd)
{
    if (PLANES) {
        const float4 t = __ldg(d.tpl + (long long)y * d.pitch + x);
        c = t.x;
        gx = t.y;
        gy = t.z;
        if (tin) {
            const float4 q = __ldg(d.tap + (long long)yt * d.pitch + xt);
            a = q.x;
            b = q.y;
            cc = q.z;
            dd = q.w;
        } else {
            taps_at(d.S1, d.pitch, d.w, d.h, xt, yt, false, a, b, cc, dd);
        }
    } else {
        template_at(d.S0, d.pitch, d.w, d.h, x, y, inner, c, gx, gy);
        taps_at(d.S1, d.pitch, d.w, d.h, xt, yt, tin, a, b, cc, dd);
    }
}

// Whether the taps of a patch whose top-left tap is (xi, yi) may be taken without clamping:
// from the tap plane, every tap start inside the image; from the image, all four taps inside.
template <bool PLANES>
__device__ __forceinline__ bool taps_inside(int xi, int yi, int ps, int w, int h)
{
    return PLANES ? (xi >= 0 && yi >= 0 && xi + ps <= w && yi + ps <= h)
                  : (xi >= 0 && yi >= 0 && xi + ps <= w - 1 && yi + ps <= h - 1);
}

// Adds one pixel's terms to the twelve cell sums.
__device__ __forceinline__ void cell_acc(float (&P)[12], float a, float b, float c, float d, float T, float gx,
                                         float gy, float mref)
{
    const float t[4] = {(a - T) - mref, b - a, c - a, (d - c) - (b - a)};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        P[q] += t[q];
        P[4 + q] = fmaf(gx, t[q], P[4 + q]);
        P[8 + q] = fmaf(gy, t[q], P[8 + q]);
    }
}

// Lane holding sum k after the transposed reduction (lane bits 4..1 select 6/3/2/1 blocks).
__host__ __device__ constexpr int holder_lane(int k)
{
    return 16 * (k / 6) + 8 * ((k % 6) / 3) + 4 * ((k % 3) == 2) + 2 * ((k % 3) == 1);
}

// Sums P over the 32 lanes of the warp and returns the twelve totals in lane `dst` (Q of the
// other lanes is left unchanged).  Each exchange level halves the values a lane carries.
__device__ __forceinline__ void warp_sum12_to(float (&P)[12], int lane, int dst, float (&Q)[12])
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
        const float v = __shfl_sync(kFull, w1, holder_lane(k));
        if (lane == dst) Q[k] = v;
    }
}

template <int PSC, int MINB, bool PLANES>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, MINB)
    search_lane_kernel(const __grid_constant__ Jobs<LevelJob> js, long long total, int ps_rt, int stride, int iters)
{
    __shared__ PatchDesc desc[kWarpsPerBlock][32];
    const int ps = PSC ? PSC : ps_rt;
    const int n = ps * ps;
    const float inv_n = 1.0f / (float)n;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    PatchDesc* D = desc[wib];
    const long long wstep = (long long)gridDim.x * kWarpsPerBlock * 32;
    for (long long g0 = ((long long)blockIdx.x * kWarpsPerBlock + wib) * 32; g0 < total; g0 += wstep) {
        const bool valid = g0 + lane < total;
        const long long g = valid ? g0 + lane : total - 1;
        const int jb = find_job(js, g, &LevelJob::patch_base);
        const LevelJob& J = job_ref(js, jb);
        const long long pk = g - J.patch_base;
        const int w = J.w, h = J.h, pitch = J.pitch;
        const int j = (int)(pk / J.nx), i = (int)(pk - (long long)j * J.nx);
        const int px = min(i * stride, w - ps), py = min(j * stride, h - ps);
        const float2 ui = init_flow_at(J.Uc, J.wc, J.hc, J.cscale, (float)px + 0.5f * (float)(ps - 1),
                                       (float)py + 0.5f * (float)(ps - 1));
        float u = ui.x, v = ui.y;
        int st = 0;
        bool run = false;
        float k00 = 0.0f, k01 = 0.0f, k11 = 0.0f, sgx = 0.0f, sgy = 0.0f, sT = 0.0f, mref = 0.0f, mcur = 0.0f;
        float Q[12];
#pragma unroll
        for (int q = 0; q < 12; ++q) Q[q] = 0.0f;
        int ciu = INT_MIN, civ = INT_MIN;
        if (valid && J.frozen) {
            const float2 f = J.frozen[pk];
            u += f.x;
            v += f.y;
        } else if (valid) {
            // ---- prologue: mean, gradients, H', sums, cell sums of the starting cell
            const PatchDesc me{J.S0, J.S1, J.tpl, J.tap, pitch, w, h, px, py, 0.0f};
            const bool inner = px >= 1 && py >= 1 && px + ps <= w - 1 && py + ps <= h - 1;
            float s0 = 0.0f;
            for (int b = 0; b < ps; ++b) {
                const float* row = me.S0 + (long long)(py + b) * pitch + px;
                float rsum = 0.0f;
#pragma unroll
                for (int a = 0; a < (PSC ? PSC : 16); ++a)
                    if (PSC || a < ps) rsum += __ldg(row + a);
                s0 += rsum;
            }
            const float mean0 = s0 * inv_n;
            const float uc = fminf(fmaxf(u, -1.0e7f), 1.0e7f);
            const float vc = fminf(fmaxf(v, -1.0e7f), 1.0e7f);
            const int iu = (int)floorf(uc), iv = (int)floorf(vc);
            const int xi = px + iu, yi = py + iv;
            const bool tin = taps_inside<PLANES>(xi, yi, ps, w, h);
            float P[12];
#pragma unroll
            for (int q = 0; q < 12; ++q) P[q] = 0.0f;
            float h00 = 0.0f, h01 = 0.0f, h11 = 0.0f;
            for (int b = 0; b < ps; ++b) {
#pragma unroll 1
                for (int a = 0; a < ps; ++a) {
                    float c, gx, gy, ta, tb, tc, td;
                    fetch_pixel<PLANES>(me, px + a, py + b, xi + a, yi + b, inner, tin, c, gx, gy, ta, tb, tc, td);
                    const float T = c - mean0;
                    sT += T;
                    h00 = fmaf(gx, gx, h00);
                    h01 = fmaf(gx, gy, h01);
                    h11 = fmaf(gy, gy, h11);
                    sgx += gx;
                    sgy += gy;
                    cell_acc(P, ta, tb, tc, td, T, gx, gy, mean0);
                }
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
                k00 = h11 * idet;
                k01 = -h01 * idet;
                k11 = h00 * idet;
                run = true;
#pragma unroll
                for (int q = 0; q < 12; ++q) Q[q] = P[q];
                ciu = iu;
                civ = iv;
                mref = mcur = mean0;
            }
            D[lane] = PatchDesc{J.S0, J.S1, J.tpl, J.tap, pitch, w, h, px, py, mean0};
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
                unsigned pend = __ballot_sync(kFull, need);
                while (pend) {
                    // the integer displacement of patch `src` moved: the warp rebuilds its sums
                    const int src = __ffs(pend) - 1;
                    pend &= pend - 1;
                    const int siu = __shfl_sync(kFull, iu, src), siv = __shfl_sync(kFull, iv, src);
                    const float sref = __shfl_sync(kFull, mcur, src);
                    const PatchDesc d = D[src];
                    const bool inner = d.px >= 1 && d.py >= 1 && d.px + ps <= d.w - 1 && d.py + ps <= d.h - 1;
                    const int xi = d.px + siu, yi = d.py + siv;
                    const bool tin = taps_inside<PLANES>(xi, yi, ps, d.w, d.h);
                    float P[12];
#pragma unroll
                    for (int q = 0; q < 12; ++q) P[q] = 0.0f;
#pragma unroll 2
                    for (int m = 0; m < (PSC ? (PSC * PSC + 31) / 32 : 8); ++m) {
                        const int k = lane + 32 * m;
                        if (k < n) {
                            const int ky = k / ps, kx = k - ky * ps;
                            float c, gx, gy, ta, tb, tc, td;
                            fetch_pixel<PLANES>(d, d.px + kx, d.py + ky, xi + kx, yi + ky, inner, tin, c, gx, gy, ta, tb,
                                                tc, td);
                            cell_acc(P, ta, tb, tc, td, c - d.mean0, gx, gy, sref);
                        }
                    }
                    warp_sum12_to(P, lane, src, Q);
                    if (lane == src) {
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
            if (ex * ex + ey * ey > (float)(ps * ps)) {
                st = 1;
                u = ui.x;
                v = ui.y;
            }
        }
        if (valid) {
            J.pu[pk] = make_float2(u, v);
            if (J.pui) J.pui[pk] = ui;
            if (J.pst) J.pst[pk] = st;
            if (J.record) J.record[pk] = make_float2(u - ui.x, v - ui.y);
        }
        __syncwarp();  // the descriptors are rewritten for the next 32 patches
    }
}

template <int PSC, int MINB, bool PLANES>
cudaError_t launch_lane(const Jobs<LevelJob>& js, long long total, int ps, int stride, int iters, const LaunchCfg& lc,
                        cudaStream_t s)
{
    constexpr int threads = kWarpsPerBlock * 32;
    static int occ = 0;
    if (occ == 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, search_lane_kernel<PSC, MINB, PLANES>, threads, 0) !=
                cudaSuccess ||
            occ < 1)
            occ = 1;
    }
    long long blocks = (total + threads - 1) / threads;
    const long long cap = (long long)lc.sm_count * occ;
    if (blocks > cap) blocks = cap;
    search_lane_kernel<PSC, MINB, PLANES><<<(int)blocks, threads, 0, s>>>(js, total, ps, stride, iters);
    return cudaGetLastError();
}

template <bool PLANES>
cudaError_t launch_lane_ps(const Jobs<LevelJob>& js, long long total, int ps, int stride, int iters,
                           const LaunchCfg& lc, cudaStream_t s)
{
    if (ps == 8) return launch_lane<8, 6, PLANES>(js, total, ps, stride, iters, lc, s);
    if (ps == 12) return launch_lane<12, 6, PLANES>(js, total, ps, stride, iters, lc, s);
    return launch_lane<0, 5, PLANES>(js, total, ps, stride, iters, lc, s);
}

// (I0, gx, gy, 0) and the taps (x, y), (x+1, y), (x, y+1), (x+1, y+1) of I1, clamped to the
// image, for every pixel of a level: the per-pixel data of the search in two 16-byte loads.
__global__ void __launch_bounds__(256) search_planes_kernel(const __grid_constant__ Jobs<LevelJob> js, long long total)
{
    for (long long g = gtid(); g < total; g += gstride()) {
        const LevelJob& J = job_ref(js, find_job(js, g, &LevelJob::pix_base));
        const long long k = g - J.pix_base;
        const int w = J.w, h = J.h, pitch = J.pitch;
        const int y = (int)(k / w), x = (int)(k - (long long)y * w);
        float c, gx, gy, a, b, cc, d;
        template_at(J.S0, pitch, w, h, x, y, false, c, gx, gy);
        taps_at(J.S1, pitch, w, h, x, y, false, a, b, cc, d);
        const long long o = (long long)y * pitch + x;
        const_cast<float4*>(J.tpl)[o] = make_float4(c, gx, gy, 0.0f);
        const_cast<float4*>(J.tap)[o] = make_float4(a, b, cc, d);
    }
}

}  // namespace

cudaError_t launch_search_lane(const Jobs<LevelJob>& js, long long total, int ps, int stride, int iters,
                               const LaunchCfg& lc, cudaStream_t s, bool planes)
{
    if (total <= 0) return cudaSuccess;
    return planes ? launch_lane_ps<true>(js, total, ps, stride, iters, lc, s)
                  : launch_lane_ps<false>(js, total, ps, stride, iters, lc, s);
}

cudaError_t launch_search_planes(const Jobs<LevelJob>& js, long long total_pix, const LaunchCfg& lc, cudaStream_t s)
{
    if (total_pix <= 0) return cudaSuccess;
    const int blocks = (int)std::min<long long>((total_pix + 255) / 256, (long long)lc.sm_count * lc.max_blocks_256);
    search_planes_kernel<<<blocks, 256, 0, s>>>(js, total_pix);
    return cudaGetLastError();
}

}  // namespace dis
