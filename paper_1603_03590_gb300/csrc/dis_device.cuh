// Device helpers of the DIS kernels: job lookup and bilinear sampling.
#pragma once

#include "dis_internal.cuh"

namespace dis {

// Job owning flattened item `item` (jobs sorted by their base).
template <class J>
__device__ __forceinline__ int find_job(const Jobs<J>& js, long long item, long long J::*base)
{
    if (js.dev == nullptr) return 0;
    int lo = 0, hi = js.n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (js.dev[mid].*base <= item)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

template <class J>
__device__ __forceinline__ const J& job_ref(const Jobs<J>& js, int i)
{
    return js.dev ? js.dev[i] : js.one;
}

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return min(max(v, lo), hi); }

// I(x + u, y + v) for integer (x, y) and real (u, v), with the coordinate clamped to the image
// before interpolating.  Splitting u into floor and fraction keeps the weights exact; clamping
// both integer taps reproduces the clamped-coordinate rule exactly (outside the image both taps
// are the border pixel).
__device__ __forceinline__ float sample_shift(const float* __restrict__ I, int w, int h, int pitch, int x, int y,
                                              float u, float v)
{
    const float uc = fminf(fmaxf(u, -1.0e7f), 1.0e7f);
    const float vc = fminf(fmaxf(v, -1.0e7f), 1.0e7f);
    const float fu = floorf(uc), fv = floorf(vc);
    const float ax = uc - fu, ay = vc - fv;
    const int xi = x + (int)fu, yi = y + (int)fv;
    const int x0 = clampi(xi, 0, w - 1), x1 = clampi(xi + 1, 0, w - 1);
    const int y0 = clampi(yi, 0, h - 1), y1 = clampi(yi + 1, 0, h - 1);
    const float* r0 = I + (long long)y0 * pitch;
    const float* r1 = I + (long long)y1 * pitch;
    const float a = __ldg(r0 + x0), b = __ldg(r0 + x1), c = __ldg(r1 + x0), d = __ldg(r1 + x1);
    const float top = fmaf(ax, b - a, a), bot = fmaf(ax, d - c, c);
    return fmaf(ay, bot - top, top);
}

// Bilinear value of a dense (w*h) float2 field at real (X, Y), clamped to the field.
__device__ __forceinline__ float2 sample_flow(const float2* __restrict__ F, int w, int h, float X, float Y)
{
    X = fminf(fmaxf(X, 0.0f), (float)(w - 1));
    Y = fminf(fmaxf(Y, 0.0f), (float)(h - 1));
    const int x0 = (int)X, y0 = (int)Y;
    const int x1 = min(x0 + 1, w - 1), y1 = min(y0 + 1, h - 1);
    const float ax = X - (float)x0, ay = Y - (float)y0;
    const float2 a = __ldg(F + (long long)y0 * w + x0), b = __ldg(F + (long long)y0 * w + x1);
    const float2 c = __ldg(F + (long long)y1 * w + x0), d = __ldg(F + (long long)y1 * w + x1);
    float2 r;
    const float tx = fmaf(ax, b.x - a.x, a.x), bx = fmaf(ax, d.x - c.x, c.x);
    const float ty = fmaf(ax, b.y - a.y, a.y), by = fmaf(ax, d.y - c.y, c.y);
    r.x = fmaf(ay, bx - tx, tx);
    r.y = fmaf(ay, by - ty, ty);
    return r;
}

// Initial displacement at real position (X, Y) of the level: cscale * Uc((X, Y) / cscale).
__device__ __forceinline__ float2 init_flow_at(const float2* Uc, int wc, int hc, float cscale, float X, float Y)
{
    if (Uc == nullptr) return make_float2(0.0f, 0.0f);
    const float2 v = sample_flow(Uc, wc, hc, X / cscale, Y / cscale);
    return make_float2(cscale * v.x, cscale * v.y);
}

// Advances a patch search by one accepted update (u, v) -> (un, vn) and reports whether every
// later iteration is already known.  The update is a deterministic function of u, v and the
// current cell sums, so: if it leaves (u, v) unchanged, all later iterations repeat it (fixed
// point); if it returns to the iterate before the current one (u1, v1) without a rebuild of
// the cell sums in between (quiet >= 2), the search alternates between the two points and the
// last iterate follows from the parity of the `left` iterations still to run.  Either way
// (u, v) is set to the result of the full iteration count, bit for bit.
__device__ __forceinline__ bool search_cycle_exit(float& u, float& v, float un, float vn, float& u1, float& v1,
                                                  int quiet, int left)
{
    if (un == u && vn == v) return true;
    if (quiet >= 2 && un == u1 && vn == v1) {
        if ((left & 1) == 0) {
            u = un;
            v = vn;
        }
        return true;
    }
    u1 = u;
    v1 = v;
    u = un;
    v = vn;
    return false;
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Grid-stride helpers.
__device__ __forceinline__ long long gtid() { return (long long)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ long long gstride() { return (long long)gridDim.x * blockDim.x; }

}  // namespace dis
