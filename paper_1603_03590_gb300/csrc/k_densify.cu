// Densification of DIS (Alg. 1 step 4, Eq. 3):
//   U(x) = sum_i w_i(x) u_i / sum_i w_i(x),  w_i(x) = 1 / max(1, |I1(x + u_i) - I0(x)|),
// over the patches i that contain x.  Thread per pixel; the covering patches follow from
// the grid arithmetic (corners min(i * stride, W - ps)), so every pixel gathers its own
// contributions in row-major patch order: no atomics, deterministic.
//
// With forward-backward consistency (supplementary Sec. B (ii)) each direction's field also
// takes the other direction's patches j through their bilinear footprint moved by u'_j:
// weight mu_j(x) / max(1, |I0(x) - I1(x - u'_j)|), displacement -u'_j, where mu_j(x) is the sum
// of the bilinear weights that the patch's template pixels q, landing at q + u'_j, give x (1
// inside the moved box, fading to 0 over one pixel around it).  Those footprints sit anywhere,
// so they are found by lists per 32 x 32 tile (count, scan, fill), and each tile block
// accumulates the listed patches' contributions per pixel in 64-bit fixed point: every term is
// rounded to an integer multiple of 2^-k (k from the largest |u'| of the tile, so that a term
// fits 31 bits and no sum of terms can overflow), and integer sums do not depend on the order in
// which the (atomically listed) patches arrive, so the result is deterministic.  Only 32-bit
// conversions run per term (64-bit ones would run on the slow FP64 pipe).
#include <algorithm>

#include "dis_device.cuh"

namespace dis {

// Range [lo, hi] of regular grid indices (those below n - 1, at i * stride) whose patch
// covers coordinate q, and whether the last patch (at L - ps) covers it.  SC: compile-time
// stride (0: the runtime `stride`), so that the divisions become multiplications.
template <int SC>
__device__ __forceinline__ void cover_range(int q, int L, int ps, int stride_rt, int n, int& lo, int& hi, bool& last)
{
    const int stride = SC ? SC : stride_rt;
    const int t = q - ps + 1;
    lo = t <= 0 ? 0 : (t + stride - 1) / stride;
    hi = min(n - 2, q / stride);
    last = q >= L - ps;
}

// Eq. 3 sums of pixel (x, y) over the job's own covering patches, in row-major patch order.
template <int SC>
__device__ __forceinline__ void own_sums(const LevelJob& J, int x, int y, int ps, int stride, float& nu, float& nv,
                                         float& Z)
{
    const int w = J.w, h = J.h, pitch = J.pitch, nx = J.nx, ny = J.ny;
    int ilo, ihi, jlo, jhi;
    bool ilast, jlast;
    cover_range<SC>(x, w, ps, stride, nx, ilo, ihi, ilast);
    cover_range<SC>(y, h, ps, stride, ny, jlo, jhi, jlast);
    const float i0 = __ldg(J.S0 + (long long)y * pitch + x);
    nu = nv = Z = 0.0f;
    const int jend = jhi + (jlast ? 1 : 0), iend = ihi + (ilast ? 1 : 0);
    for (int jj = jlo; jj <= jend; ++jj) {
        const int j = jj > jhi ? ny - 1 : jj;
        for (int ii = ilo; ii <= iend; ++ii) {
            const int i = ii > ihi ? nx - 1 : ii;
            const float2 up = J.pu[(long long)j * nx + i];
            const float d = sample_shift(J.S1, w, h, pitch, x, y, up.x, up.y) - i0;
            const float wt = __frcp_rn(fmaxf(1.0f, fabsf(d)));  // the correctly rounded 1 / max(1, |d|)
            nu = fmaf(wt, up.x, nu);
            nv = fmaf(wt, up.y, nv);
            Z += wt;
        }
    }
}

template <int SC>
__global__ void __launch_bounds__(256) densify_kernel(const __grid_constant__ Jobs<LevelJob> js, long long total,
                                                      int ps, int stride)
{
    for (long long g = gtid(); g < total; g += gstride()) {
        const LevelJob& J = job_ref(js, find_job(js, g, &LevelJob::pix_base));
        const int k = (int)(g - J.pix_base);  // < w * h < 2^31
        const int w = J.w;
        const int y = k / w, x = k - y * w;
        float nu, nv, Z;
        own_sums<SC>(J, x, y, ps, stride, nu, nv, Z);
        float2 r;
        if (Z > 0.0f) {
            r = make_float2(nu / Z, nv / Z);
        } else {
            r = init_flow_at(J.Uc, J.wc, J.hc, J.cscale, (float)x, (float)y);
        }
        J.U[k] = r;
    }
}

// ---- forward-backward consistency ------------------------------------------------------

constexpr int kFbTile = kRefineTile;  // the lists use the refinement tiles of each job
static_assert(kFbTile == 32, "tile indexing below assumes 32 x 32 tiles");

// Integer box [x0, x1] x [y0, y1] of the pixels that the footprint of patch pk of job K, moved
// by its displacement u, reaches (p - 1 < x - u < p + ps in both coordinates: p + floor(u) to
// p + ps - 1 + ceil(u)), clipped to the frame; false when it is empty or |u| is beyond any frame
// (or not a number).  (px, py): the patch corner.
__device__ __forceinline__ bool moved_box(const LevelJob& K, long long pk, int ps, int stride, float2& u, int& px,
                                          int& py, int& x0, int& x1, int& y0, int& y1)
{
    u = K.pu[pk];
    if (!(fabsf(u.x) <= 1.0e6f && fabsf(u.y) <= 1.0e6f)) return false;
    const int j = (int)(pk / K.nx), i = (int)(pk - (long long)j * K.nx);
    px = min(i * stride, K.w - ps);
    py = min(j * stride, K.h - ps);
    x0 = max(px + (int)floorf(u.x), 0);
    x1 = min(px + ps - 1 + (int)ceilf(u.x), K.w - 1);
    y0 = max(py + (int)floorf(u.y), 0);
    y1 = min(py + ps - 1 + (int)ceilf(u.y), K.h - 1);
    return x0 <= x1 && y0 <= y1;
}

// One coordinate of the footprint: sum over m = 0 .. ps-1 of max(0, 1 - |a - m|), a = k - u the
// pixel's offset from the patch corner minus the displacement: 1 on [0, ps - 1], linear to 0 on
// the unit intervals on either side.
__device__ __forceinline__ float footprint_1d(int k, float u, int ps)
{
    const float a = (float)k - u;
    return fminf(1.0f, fmaxf(0.0f, fminf(a + 1.0f, (float)ps - a)));
}

__global__ void __launch_bounds__(256) fb_clear_kernel(const __grid_constant__ Jobs<LevelJob> js, long long total)
{
    for (long long g = gtid(); g < total; g += gstride()) {
        const LevelJob& J = job_ref(js, find_job(js, g, &LevelJob::tile_base));
        const long long t = g - J.tile_base;
        J.fb_cnt[t] = 0;
        J.fb_cur[t] = 0;
    }
}

// FILL = false: count, per tile of the partner, the patches whose moved box meets it;
// FILL = true: append each patch to those tiles' lists.
template <bool FILL>
__global__ void __launch_bounds__(256) fb_list_kernel(const __grid_constant__ Jobs<LevelJob> js, long long total,
                                                      int ps, int stride)
{
    for (long long g = gtid(); g < total; g += gstride()) {
        const LevelJob& K = job_ref(js, find_job(js, g, &LevelJob::patch_base));
        const long long pk = g - K.patch_base;
        const LevelJob& P = job_ref(js, K.partner);
        float2 u;
        int px, py, x0, x1, y0, y1;
        if (!moved_box(K, pk, ps, stride, u, px, py, x0, x1, y0, y1)) continue;
        for (int ty = y0 / kFbTile; ty <= y1 / kFbTile; ++ty)
            for (int tx = x0 / kFbTile; tx <= x1 / kFbTile; ++tx) {
                const long long t = (long long)ty * P.tiles_x + tx;
                if (FILL)
                    P.fb_list[P.fb_cnt[t] + atomicAdd(&P.fb_cur[t], 1)] = (int)pk;
                else
                    atomicAdd(&P.fb_cnt[t], 1);
            }
    }
}

// One block per job: exclusive scan of the tile counts into offsets (in place); the fill
// cursors restart at 0.
__global__ void __launch_bounds__(1024) fb_scan_kernel(const __grid_constant__ Jobs<LevelJob> js, int njobs)
{
    __shared__ int wsum[32];
    __shared__ int carry_s;
    for (int jb = blockIdx.x; jb < njobs; jb += gridDim.x) {
        const LevelJob& J = job_ref(js, jb);
        const long long n = (long long)J.tiles_x * ((J.h + kFbTile - 1) / kFbTile);
        if (threadIdx.x == 0) carry_s = 0;
        __syncthreads();
        for (long long base = 0; base < n; base += blockDim.x) {
            const long long t = base + threadIdx.x;
            const int v = t < n ? J.fb_cnt[t] : 0;
            int incl = v;
            const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            if (lane == 31) wsum[wid] = incl;
            __syncthreads();
            if (wid == 0) {
                int ws = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, ws, o);
                    if (lane >= o) ws += y;
                }
                wsum[lane] = ws;  // inclusive prefix of the warp sums
            }
            __syncthreads();
            const int carry = carry_s;
            const int before = (wid > 0 ? wsum[wid - 1] : 0) + incl - v;
            if (t < n) J.fb_cnt[t] = carry + before;
            __syncthreads();
            if (threadIdx.x == blockDim.x - 1) carry_s = carry + before + v;
            __syncthreads();
        }
    }
}

constexpr int kFbThreads = 512;  // one warp per bin
constexpr int kFbChunk = 512;    // listed patches staged in shared memory at a time
constexpr int kFbBin = 8;        // 8 x 8 pixel bins: 16 per tile
constexpr int kFbStrip = kFbBin * kFbBin / (kFbThreads / 16);  // pixels per thread (a row strip)

// One block (512 threads) per tile of a job.  Warp b owns bin b; its lane l the 1 x 2 pixel
// strip (2 (l & 3), l / 4) of the bin.  The partner's listed patches are staged in chunks;
// each is entered in the bins its (tile-clipped) footprint meets, and each thread then visits
// only its bin's patches, accumulating its pixels' contributions in 64-bit fixed point in
// registers (the order in which patches enter a bin does not matter).
template <int SC>
__global__ void __launch_bounds__(kFbThreads, 2) densify_fb_kernel(const __grid_constant__ Jobs<LevelJob> js,
                                                                   long long total, int ps, int stride)
{
    constexpr int NB = (kFbTile / kFbBin) * (kFbTile / kFbBin);
    constexpr int SPR = kFbBin / kFbStrip;  // strips per bin row
    static_assert(kFbThreads / 32 == NB && SPR * kFbStrip == kFbBin, "one warp per bin, whole strips");
    __shared__ float2 eu[kFbChunk];
    __shared__ int2 epos[kFbChunk];
    __shared__ int4 ebox[kFbChunk];  // footprint clipped to the tile, tile coordinates
    __shared__ short blist[NB][kFbChunk];
    __shared__ int bcnt[NB];
    __shared__ float red[kFbThreads / 32];
    const int bin = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int bx0 = (bin % (kFbTile / kFbBin)) * kFbBin, by0 = (bin / (kFbTile / kFbBin)) * kFbBin;
    const int sx = bx0 + kFbStrip * (lane % SPR), sy = by0 + lane / SPR;  // the strip's first pixel (tile coordinates)
    for (long long g = blockIdx.x; g < total; g += gridDim.x) {
        const LevelJob& J = job_ref(js, find_job(js, g, &LevelJob::tile_base));
        const LevelJob& P = job_ref(js, J.partner);
        const long long t = g - J.tile_base;
        const int tx = (int)(t % J.tiles_x), ty = (int)(t / J.tiles_x);
        const int X0 = tx * kFbTile, Y0 = ty * kFbTile;
        const int tw = min(kFbTile, J.w - X0), th = min(kFbTile, J.h - Y0);
        const int beg = J.fb_cnt[t], L = J.fb_cur[t];  // after the fill the cursor holds the count
        // the largest |u'| of the listed patches bounds every term
        float m = 0.0f;
        for (int e = threadIdx.x; e < L; e += blockDim.x) {
            const float2 u = P.pu[J.fb_list[beg + e]];
            m = fmaxf(m, fmaxf(fabsf(u.x), fabsf(u.y)));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
        __syncthreads();
        m = 0.0f;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) m = fmaxf(m, red[k]);
        // |w u'| <= m < 2^ex: terms scaled by 2^kn stay below 2^30 (w <= 1: 2^kz = 2^30 too), so
        // each converts to a 32-bit integer and a sum of fewer than 2^33 of them fits 64 bits
        const int ex = ((__float_as_int(m + 1.0f) >> 23) & 0xff) - 126;  // m + 1 < 2^ex (m + 1 >= 1 is normal)
        const int kn = 30 - ex, kz = 30;
        const float sn = ldexpf(1.0f, kn), sz = ldexpf(1.0f, kz);
        // this thread's pixels
        const int y = Y0 + sy;
        const bool row_in = sy < th;
        float i0[kFbStrip];
        long long au[kFbStrip], av[kFbStrip], az[kFbStrip];
#pragma unroll
        for (int k = 0; k < kFbStrip; ++k) {
            i0[k] = (row_in && sx + k < tw) ? __ldg(J.S0 + (long long)y * J.pitch + X0 + sx + k) : 0.0f;
            au[k] = av[k] = az[k] = 0;
        }
        for (int c0 = 0; c0 < L; c0 += kFbChunk) {
            const int nc = min(kFbChunk, L - c0);
            __syncthreads();  // the previous chunk is consumed
            if (threadIdx.x < NB) bcnt[threadIdx.x] = 0;
            __syncthreads();
            if ((int)threadIdx.x < nc) {
                float2 u;
                int px, py, x0, x1, y0, y1;
                const bool ok =
                    moved_box(P, J.fb_list[beg + c0 + threadIdx.x], ps, stride, u, px, py, x0, x1, y0, y1);
                const int4 b = make_int4(max(x0, X0) - X0, min(x1, X0 + tw - 1) - X0, max(y0, Y0) - Y0,
                                         min(y1, Y0 + th - 1) - Y0);
                eu[threadIdx.x] = u;
                epos[threadIdx.x] = make_int2(px, py);
                ebox[threadIdx.x] = b;
                if (ok && b.x <= b.y && b.z <= b.w)
                    for (int qy = b.z / kFbBin; qy <= b.w / kFbBin; ++qy)
                        for (int qx = b.x / kFbBin; qx <= b.y / kFbBin; ++qx) {
                            const int q = qy * (kFbTile / kFbBin) + qx;
                            blist[q][atomicAdd(&bcnt[q], 1)] = (short)threadIdx.x;
                        }
            }
            __syncthreads();
            const int nb = bcnt[bin];
            for (int k = 0; k < nb; ++k) {
                const int e = blist[bin][k];
                const int4 b = ebox[e];
                if (!row_in || sy < b.z || sy > b.w) continue;
                const float2 u = eu[e];
                const int2 pc = epos[e];
                const float ly = footprint_1d(y - pc.y, u.y, ps);
#pragma unroll
                for (int q = 0; q < kFbStrip; ++q) {
                    const int lx = sx + q;
                    if (lx < b.x || lx > b.y) continue;
                    const int x = X0 + lx;
                    const float d = i0[q] - sample_shift(J.S1, J.w, J.h, J.pitch, x, y, -u.x, -u.y);
                    const float wt = footprint_1d(x - pc.x, u.x, ps) * ly * __frcp_rn(fmaxf(1.0f, fabsf(d)));
                    au[q] += __float2int_rn((-wt * u.x) * sn);
                    av[q] += __float2int_rn((-wt * u.y) * sn);
                    az[q] += __float2int_rn(wt * sz);
                }
            }
        }
        const float in_ = ldexpf(1.0f, -kn), iz = ldexpf(1.0f, -kz);
#pragma unroll
        for (int q = 0; q < kFbStrip; ++q) {
            if (!row_in || sx + q >= tw) continue;
            const int x = X0 + sx + q;
            float nu, nv, Z;
            own_sums<SC>(J, x, y, ps, stride, nu, nv, Z);
            const float Zt = Z + __ll2float_rn(az[q]) * iz;
            float2 r;
            if (Zt > 0.0f) {
                r = make_float2((nu + __ll2float_rn(au[q]) * in_) / Zt, (nv + __ll2float_rn(av[q]) * in_) / Zt);
            } else {
                r = init_flow_at(J.Uc, J.wc, J.hc, J.cscale, (float)x, (float)y);
            }
            J.U[(long long)y * J.w + x] = r;
        }
        __syncthreads();  // red and bcnt are rewritten for the next tile
    }
}

long long fb_scratch_ints(int w, int h, int ps, int stride)
{
    const long long tiles = (long long)((w + kFbTile - 1) / kFbTile) * ((h + kFbTile - 1) / kFbTile);
    const long long nx = w < ps ? 0 : (w - ps + stride - 1) / stride + 1;
    const long long ny = h < ps ? 0 : (h - ps + stride - 1) / stride + 1;
    return 2 * tiles + 4 * nx * ny;  // a footprint (at most 17 wide) meets at most 2 x 2 tiles
}

cudaError_t launch_densify_fb(const Jobs<LevelJob>& js, long long total_patches, long long total_tiles, int njobs,
                              int ps, int stride, const LaunchCfg& lc, cudaStream_t s)
{
    if (total_tiles <= 0) return cudaSuccess;
    auto grid = [&](long long items, long long per_block_cap) {
        long long b = (items + 255) / 256;
        const long long cap = (long long)lc.sm_count * per_block_cap;
        return (int)std::max<long long>(1, std::min(b, cap));
    };
    fb_clear_kernel<<<grid(total_tiles, lc.max_blocks_256), 256, 0, s>>>(js, total_tiles);
    if (total_patches > 0) fb_list_kernel<false><<<grid(total_patches, lc.max_blocks_256), 256, 0, s>>>(js, total_patches, ps, stride);
    fb_scan_kernel<<<std::min(njobs, lc.sm_count * 2), 1024, 0, s>>>(js, njobs);
    if (total_patches > 0) fb_list_kernel<true><<<grid(total_patches, lc.max_blocks_256), 256, 0, s>>>(js, total_patches, ps, stride);
    const int gt = (int)std::min<long long>(total_tiles, (long long)lc.sm_count * 4);
    switch (stride) {
        case 3: densify_fb_kernel<3><<<gt, kFbThreads, 0, s>>>(js, total_tiles, ps, stride); break;
        case 4: densify_fb_kernel<4><<<gt, kFbThreads, 0, s>>>(js, total_tiles, ps, stride); break;
        case 5: densify_fb_kernel<5><<<gt, kFbThreads, 0, s>>>(js, total_tiles, ps, stride); break;
        case 6: densify_fb_kernel<6><<<gt, kFbThreads, 0, s>>>(js, total_tiles, ps, stride); break;
        default: densify_fb_kernel<0><<<gt, kFbThreads, 0, s>>>(js, total_tiles, ps, stride); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_densify(const Jobs<LevelJob>& js, long long total, int ps, int stride, const LaunchCfg& lc,
                           cudaStream_t s)
{
    if (total <= 0) return cudaSuccess;
    long long b = (total + 255) / 256;
    const long long cap = (long long)lc.sm_count * lc.max_blocks_256;
    if (b > cap) b = cap;
    switch (stride) {  // the strides of the presets
        case 3: densify_kernel<3><<<(int)b, 256, 0, s>>>(js, total, ps, stride); break;
        case 4: densify_kernel<4><<<(int)b, 256, 0, s>>>(js, total, ps, stride); break;
        case 5: densify_kernel<5><<<(int)b, 256, 0, s>>>(js, total, ps, stride); break;
        case 6: densify_kernel<6><<<(int)b, 256, 0, s>>>(js, total, ps, stride); break;
        default: densify_kernel<0><<<(int)b, 256, 0, s>>>(js, total, ps, stride); break;
    }
    return cudaGetLastError();
}

}  // namespace dis
