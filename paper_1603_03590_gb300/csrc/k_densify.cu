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
#include <climits>

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
            const float wt = __fdividef(1.0f, fmaxf(1.0f, fabsf(d)));  // 1 / max(1, |d|), hardware reciprocal
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

// Tiled form for the strides of the presets: a block per band of 32 x 8 pixels (a quarter of one
// of the job's 32 x 32 refinement tiles), a thread per pixel.  Every pixel of a patch samples I1
// with the patch's displacement, so the parts of the bilinear sample that depend on the patch
// alone (the clamped displacement's floor and fraction) and the patch flow are staged once per
// band for all patches that cover it, instead of once per (pixel, patch); so is, for a patch whose
// four taps stay inside the frame at every pixel of the band, the offset of its taps from the
// pixel (then no pixel clamps them).  Each pixel then runs the loop of own_sums over the staged
// patches in the same row-major order with the same operations on the same samples: the result
// equals densify_kernel's bit for bit.  Covering patches per band and
// axis: at most (30 + ps) / stride + 1 regular ones and the last one, so at most 17 for
// ps <= 16 and stride >= 3.
constexpr int kDensTile = kRefineTile;
constexpr int kDensRows = 8;  // rows of a band
constexpr int kDensBands = kDensTile / kDensRows;
constexpr int kDensAxis = 18;
constexpr int kDensThreads = kDensTile * kDensRows;

struct DensPatch {
    float ax, ay, u, v;  // fraction of the clamped displacement, patch flow
};
constexpr int kOutside = INT_MIN;  // a staged patch whose taps leave the frame somewhere in the band

template <int SC>
__global__ void __launch_bounds__(kDensThreads) densify_tile_kernel(const __grid_constant__ Jobs<LevelJob> js,
                                                                    long long bands, int ps)
{
    constexpr int stride = SC;
    static_assert(SC >= 3, "the staged table holds kDensAxis patches per axis");
    __shared__ DensPatch tab[kDensAxis * kDensAxis];
    __shared__ int2 cell[kDensAxis * kDensAxis];  // integer part of the clamped displacement
    __shared__ int offs[kDensAxis * kDensAxis];   // tap offset from the pixel, or kOutside
    for (long long g = blockIdx.x; g < bands; g += gridDim.x) {
        const long long t = g / kDensBands;
        const LevelJob& J = job_ref(js, find_job(js, t, &LevelJob::tile_base));
        const int tk = (int)(t - J.tile_base);
        const int w = J.w, h = J.h, pitch = J.pitch, nx = J.nx, ny = J.ny;
        const int tx0 = (tk % J.tiles_x) * kDensTile;
        const int ty0 = (tk / J.tiles_x) * kDensTile + (int)(g % kDensBands) * kDensRows;
        if (ty0 >= h) continue;  // a band below the frame in the last row of tiles (uniform)
        const int tx1 = min(tx0 + kDensTile, w) - 1, ty1 = min(ty0 + kDensRows, h) - 1;
        // regular patches covering the band's columns / rows, then the last one
        int ib, ie, jb, je, d0, d1;
        bool lx, ly, l0;
        cover_range<SC>(tx0, w, ps, stride, nx, ib, d0, l0);
        cover_range<SC>(tx1, w, ps, stride, nx, d1, ie, lx);
        cover_range<SC>(ty0, h, ps, stride, ny, jb, d0, l0);
        cover_range<SC>(ty1, h, ps, stride, ny, d1, je, ly);
        const int nreg_x = max(0, ie - ib + 1), nreg_y = max(0, je - jb + 1);
        const int tw = nreg_x + (lx ? 1 : 0), th = nreg_y + (ly ? 1 : 0);
        for (int q = threadIdx.x; q < tw * th; q += kDensThreads) {
            const int a = q % tw, b = q / tw;
            const int i = a < nreg_x ? ib + a : nx - 1, j = b < nreg_y ? jb + b : ny - 1;
            const float2 up = J.pu[(long long)j * nx + i];
            // the patch-only part of sample_shift
            const float uc = fminf(fmaxf(up.x, -1.0e7f), 1.0e7f);
            const float vc = fminf(fmaxf(up.y, -1.0e7f), 1.0e7f);
            const float fu = floorf(uc), fv = floorf(vc);
            tab[q] = DensPatch{uc - fu, vc - fv, up.x, up.y};
            const int cx = (int)fu, cy = (int)fv;
            cell[q] = make_int2(cx, cy);
            // every pixel of the band samples rows y + cy, y + cy + 1 and columns x + cx, x + cx + 1
            const bool inside = tx0 + cx >= 0 && tx1 + cx + 1 <= w - 1 && ty0 + cy >= 0 && ty1 + cy + 1 <= h - 1;
            offs[q] = inside ? cy * pitch + cx : kOutside;  // |cy| < h: no overflow when inside
        }
        __syncthreads();
        const int x = tx0 + (int)(threadIdx.x % kDensTile), y = ty0 + (int)(threadIdx.x / kDensTile);
        if (x <= tx1 && y <= ty1) {
            int ilo, ihi, jlo, jhi;
            bool ilast, jlast;
            cover_range<SC>(x, w, ps, stride, nx, ilo, ihi, ilast);
            cover_range<SC>(y, h, ps, stride, ny, jlo, jhi, jlast);
            const float i0 = __ldg(J.S0 + (long long)y * pitch + x);
            const float* s1px = J.S1 + (long long)y * pitch + x;
            float nu = 0.0f, nv = 0.0f, Z = 0.0f;
            const int jend = jhi + (jlast ? 1 : 0), iend = ihi + (ilast ? 1 : 0);
            for (int jj = jlo; jj <= jend; ++jj) {
                const int row = (jj > jhi ? nreg_y : jj - jb) * tw;
                for (int ii = ilo; ii <= iend; ++ii) {
                    const int q = row + (ii > ihi ? nreg_x : ii - ib);
                    const DensPatch P = tab[q];
                    const int off = offs[q];
                    float pa, pb, pc, pd;
                    if (off != kOutside) {
                        const float* p = s1px + off;
                        pa = __ldg(p);
                        pb = __ldg(p + 1);
                        pc = __ldg(p + pitch);
                        pd = __ldg(p + pitch + 1);
                    } else {
                        const int2 c = cell[q];
                        const int xi = x + c.x, yi = y + c.y;
                        const int x0 = clampi(xi, 0, w - 1), x1 = clampi(xi + 1, 0, w - 1);
                        const int y0 = clampi(yi, 0, h - 1), y1 = clampi(yi + 1, 0, h - 1);
                        const float* r0 = J.S1 + (long long)y0 * pitch;
                        const float* r1 = J.S1 + (long long)y1 * pitch;
                        pa = __ldg(r0 + x0);
                        pb = __ldg(r0 + x1);
                        pc = __ldg(r1 + x0);
                        pd = __ldg(r1 + x1);
                    }
                    const float top = fmaf(P.ax, pb - pa, pa), bot = fmaf(P.ax, pd - pc, pc);
                    const float d = fmaf(P.ay, bot - top, top) - i0;
                    const float wt = __fdividef(1.0f, fmaxf(1.0f, fabsf(d)));  // as in own_sums
                    nu = fmaf(wt, P.u, nu);
                    nv = fmaf(wt, P.v, nv);
                    Z += wt;
                }
            }
            float2 r;
            if (Z > 0.0f) {
                r = make_float2(nu / Z, nv / Z);
            } else {
                r = init_flow_at(J.Uc, J.wc, J.hc, J.cscale, (float)x, (float)y);
            }
            J.U[(long long)y * w + x] = r;
        }
        __syncthreads();  // the table is rewritten for the next band
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

constexpr int kFbBin = 16;       // 16 x 16 pixel bins: 4 per tile
constexpr int kFbThreads = 32 * (kFbTile / kFbBin) * (kFbTile / kFbBin);  // one warp per bin
constexpr int kFbChunk = kFbThreads;  // listed patches staged in shared memory at a time

// One block (a warp per bin) per tile of a job; warp b owns the 16 x 16 pixel bin b and its
// accumulators.  The partner's listed patches are staged in chunks and entered in the bins their
// (tile-clipped) footprints meet; each warp then takes its bin's patches one after another and
// spreads the lanes over the rectangle the footprint covers in the bin, so that a lane adds to
// one pixel's shared-memory accumulators with a plain read-modify-write (no other lane or warp
// touches that pixel meanwhile).  Sums are 64-bit fixed point: the order in which the patches
// enter a bin (atomic) does not change them.
template <int SC>
__global__ void __launch_bounds__(kFbThreads, 6) densify_fb_kernel(const __grid_constant__ Jobs<LevelJob> js,
                                                                   long long total, int ps, int stride,
                                                                   unsigned int* __restrict__ wq)
{
    constexpr int NB = (kFbTile / kFbBin) * (kFbTile / kFbBin);
    constexpr int NP = kFbTile * kFbTile;
    static_assert(kFbThreads / 32 == NB, "one warp per bin");
    __shared__ float2 eu[kFbChunk];
    __shared__ int2 epos[kFbChunk];
    __shared__ int4 ebox[kFbChunk];  // footprint clipped to the tile, tile coordinates
    __shared__ short blist[NB][kFbChunk];
    __shared__ int bcnt[NB];
    __shared__ long long acc[3][NP];  // fixed-point sums per tile pixel: -w u'_x, -w u'_y, w
    __shared__ float s0[NP];          // the tile of I0
    __shared__ float red[kFbThreads / 32];
    __shared__ long long next_tile;
    const int bin = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int bx0 = (bin % (kFbTile / kFbBin)) * kFbBin, by0 = (bin / (kFbTile / kFbBin)) * kFbBin;
    // Tiles differ in how many partner footprints their lists hold, so with a work queue (the
    // search's counters, free while this kernel runs) each block claims its next tile when it
    // starts the current one; else the grid stride.  A tile's result does not depend on the block.
    long long g = blockIdx.x;
    while (g < total) {
        unsigned int qn = 0;
        if (wq && threadIdx.x == 0) qn = atomicAdd(wq, 1u);
        const LevelJob& J = job_ref(js, find_job(js, g, &LevelJob::tile_base));
        const LevelJob& P = job_ref(js, J.partner);
        const long long t = g - J.tile_base;
        const int tx = (int)(t % J.tiles_x), ty = (int)(t / J.tiles_x);
        const int X0 = tx * kFbTile, Y0 = ty * kFbTile;
        const int tw = min(kFbTile, J.w - X0), th = min(kFbTile, J.h - Y0);
        const int beg = J.fb_cnt[t], L = J.fb_cur[t];  // after the fill the cursor holds the count
        for (int q = threadIdx.x; q < NP; q += blockDim.x) {
            const int ly = q / kFbTile, lx = q - ly * kFbTile;
            acc[0][q] = acc[1][q] = acc[2][q] = 0;
            s0[q] = (lx < tw && ly < th) ? __ldg(J.S0 + (long long)(Y0 + ly) * J.pitch + X0 + lx) : 0.0f;
        }
        // the largest |u'| of the listed patches bounds every term
        float m = 0.0f;
        for (int e = threadIdx.x; e < L; e += blockDim.x) {
            const float2 u = P.pu[J.fb_list[beg + e]];
            m = fmaxf(m, fmaxf(fabsf(u.x), fabsf(u.y)));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) red[bin] = m;
        __syncthreads();
        m = 0.0f;
        for (int k = 0; k < NB; ++k) m = fmaxf(m, red[k]);
        // |w u'| <= m < 2^ex: terms scaled by 2^kn stay below 2^30 (w <= 1: 2^kz = 2^30 too), so
        // each converts to a 32-bit integer and a sum of fewer than 2^33 of them fits 64 bits
        const int ex = ((__float_as_int(m + 1.0f) >> 23) & 0xff) - 126;  // m + 1 < 2^ex (m + 1 >= 1 is normal)
        const int kn = 30 - ex, kz = 30;
        const float sn = ldexpf(1.0f, kn), sz = ldexpf(1.0f, kz);
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
                const int rx0 = max(b.x, bx0), rx1 = min(b.y, bx0 + kFbBin - 1);
                const int ry0 = max(b.z, by0), ry1 = min(b.w, by0 + kFbBin - 1);
                const int rw = rx1 - rx0 + 1, n = rw * (ry1 - ry0 + 1);
                const unsigned inv_rw = (65536u + (unsigned)rw - 1u) / (unsigned)rw;  // r / rw = (r inv_rw) >> 16 for r < 256
                const float2 u = eu[e];
                const int2 pc = epos[e];
                // the sample I1(x - u'): the same cell offset and weights for every pixel of the patch
                const float fu = floorf(-u.x), fv = floorf(-u.y);
                const float ax = -u.x - fu, ay = -u.y - fv;
                const int ox = (int)fu, oy = (int)fv;
                const float su = (-u.x) * sn, sv = (-u.y) * sn;
                for (int r = lane; r < n; r += 32) {
                    const int dy = (int)(((unsigned)r * inv_rw) >> 16);
                    const int lx = rx0 + (r - dy * rw), ly = ry0 + dy;
                    const int x = X0 + lx, y = Y0 + ly, a = ly * kFbTile + lx;
                    const int xi = x + ox, yi = y + oy;
                    const int x0 = clampi(xi, 0, J.w - 1), x1 = clampi(xi + 1, 0, J.w - 1);
                    const float* r0 = J.S1 + (long long)clampi(yi, 0, J.h - 1) * J.pitch;
                    const float* r1 = J.S1 + (long long)clampi(yi + 1, 0, J.h - 1) * J.pitch;
                    const float p00 = __ldg(r0 + x0), p01 = __ldg(r0 + x1), p10 = __ldg(r1 + x0), p11 = __ldg(r1 + x1);
                    const float top = fmaf(ax, p01 - p00, p00), bot = fmaf(ax, p11 - p10, p10);
                    const float d = s0[a] - fmaf(ay, bot - top, top);
                    const float wt = footprint_1d(x - pc.x, u.x, ps) * footprint_1d(y - pc.y, u.y, ps) *
                                     __fdividef(1.0f, fmaxf(1.0f, fabsf(d)));
                    acc[0][a] += __float2int_rn(wt * su);
                    acc[1][a] += __float2int_rn(wt * sv);
                    acc[2][a] += __float2int_rn(wt * sz);
                }
                __syncwarp();  // the next patch's rectangle may overlap this one's pixels
            }
        }
        __syncthreads();
        const float in_ = ldexpf(1.0f, -kn), iz = ldexpf(1.0f, -kz);
        for (int q = threadIdx.x; q < tw * th; q += blockDim.x) {
            const int ly = q / tw, lx = q - ly * tw;
            const int x = X0 + lx, y = Y0 + ly, a = ly * kFbTile + lx;
            float nu, nv, Z;
            own_sums<SC>(J, x, y, ps, stride, nu, nv, Z);
            const float Zt = Z + __ll2float_rn(acc[2][a]) * iz;
            float2 r;
            if (Zt > 0.0f) {
                r = make_float2((nu + __ll2float_rn(acc[0][a]) * in_) / Zt, (nv + __ll2float_rn(acc[1][a]) * in_) / Zt);
            } else {
                r = init_flow_at(J.Uc, J.wc, J.hc, J.cscale, (float)x, (float)y);
            }
            J.U[(long long)y * J.w + x] = r;
        }
        if (threadIdx.x == 0) next_tile = wq ? (long long)gridDim.x + qn : g + gridDim.x;
        __syncthreads();  // the accumulators, red, bcnt and next_tile are rewritten for the next tile
        g = next_tile;
    }
    if (wq && threadIdx.x == 0) {
        // the last block to finish zeroes the queue for the next launch
        __threadfence();
        if (atomicAdd(wq + 1, 1u) == gridDim.x - 1u) {
            __threadfence();
            atomicExch(wq, 0u);
            atomicExch(wq + 1, 0u);
        }
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
    // with the queue one block per resident slot (6 per SM), else two waves of them
    unsigned int* wq = total_tiles + (long long)lc.sm_count * 12 < (1LL << 31) ? lc.wq : nullptr;
    const int gt = (int)std::min<long long>(total_tiles, (long long)lc.sm_count * (wq ? 6 : 12));
    switch (stride) {
        case 3: densify_fb_kernel<3><<<gt, kFbThreads, 0, s>>>(js, total_tiles, ps, stride, wq); break;
        case 4: densify_fb_kernel<4><<<gt, kFbThreads, 0, s>>>(js, total_tiles, ps, stride, wq); break;
        case 5: densify_fb_kernel<5><<<gt, kFbThreads, 0, s>>>(js, total_tiles, ps, stride, wq); break;
        case 6: densify_fb_kernel<6><<<gt, kFbThreads, 0, s>>>(js, total_tiles, ps, stride, wq); break;
        default: densify_fb_kernel<0><<<gt, kFbThreads, 0, s>>>(js, total_tiles, ps, stride, wq); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_densify(const Jobs<LevelJob>& js, long long total, long long tiles, int ps, int stride,
                           const LaunchCfg& lc, cudaStream_t s)
{
    if (total <= 0) return cudaSuccess;
    if (tiles > 0 && stride >= 3 && stride <= 6 && (30 + ps) / stride + 2 <= kDensAxis) {
        const long long bands = tiles * kDensBands;
        long long b = bands;
        const long long cap = (long long)lc.sm_count * 4;
        if (b > cap) b = cap;
        switch (stride) {
            case 3: densify_tile_kernel<3><<<(int)b, kDensThreads, 0, s>>>(js, bands, ps); break;
            case 4: densify_tile_kernel<4><<<(int)b, kDensThreads, 0, s>>>(js, bands, ps); break;
            case 5: densify_tile_kernel<5><<<(int)b, kDensThreads, 0, s>>>(js, bands, ps); break;
            default: densify_tile_kernel<6><<<(int)b, kDensThreads, 0, s>>>(js, bands, ps); break;
        }
        return cudaGetLastError();
    }
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
