// Pyramid and resampling kernels of DIS (Sec. 3.1: image pyramid with theta_sd = 2 and
// image gradients; up-scaling of the flow to full resolution).  All are streaming stencils
// bound by memory bandwidth, with read-only loads through L1.
#include "dis_device.cuh"

namespace dis {

// Work split of the batched kernels below: one output row (preparation, up-scaling) or one band
// of output rows (pyramid) per block iteration.  The job is found once per row or band (a
// search over the jobs' first units, `base`), not once per pixel, and the block's threads cover
// the row with several pixels per thread in flight.

// Level 0: multiply the caller's [0,1] frames by intensity_scale, write the channel mean
// (the search image) and, for colour input, the scaled channel planes.
__global__ void __launch_bounds__(256) prep_kernel(const __grid_constant__ Jobs<PrepJob> js, long long rows)
{
    for (long long r = blockIdx.x; r < rows; r += gridDim.x) {
        const PrepJob& J = job_ref(js, find_job(js, r, &PrepJob::base));
        const int y = (int)(r - J.base), w = J.w, C = J.C;
        const long long io = (long long)y * J.in_pitch, oo = (long long)y * J.out_pitch;
        const float inv = 1.0f / (float)C;
        const float scale = J.scale;
        for (int x4 = 4 * threadIdx.x; x4 < w; x4 += 4 * blockDim.x) {
            float a[4] = {0.0f, 0.0f, 0.0f, 0.0f}, b[4] = {0.0f, 0.0f, 0.0f, 0.0f};
            const int nq = min(4, w - x4);
            for (int c = 0; c < C; ++c) {
                const float* __restrict__ p0 = J.I0 + c * J.in_plane + io + x4;
                const float* __restrict__ p1 = J.I1 + c * J.in_plane + io + x4;
                float v0[4], v1[4];
                if (J.vec && nq == 4) {
                    const float4 q0 = __ldg(reinterpret_cast<const float4*>(p0));
                    const float4 q1 = __ldg(reinterpret_cast<const float4*>(p1));
                    v0[0] = q0.x, v0[1] = q0.y, v0[2] = q0.z, v0[3] = q0.w;
                    v1[0] = q1.x, v1[1] = q1.y, v1[2] = q1.z, v1[3] = q1.w;
                } else {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        v0[q] = q < nq ? __ldg(p0 + q) : 0.0f;
                        v1[q] = q < nq ? __ldg(p1 + q) : 0.0f;
                    }
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    v0[q] *= scale;
                    v1[q] *= scale;
                    a[q] += v0[q];
                    b[q] += v1[q];
                }
                if (J.P0) {
                    float* o0 = J.P0 + c * J.out_plane + oo + x4;
                    float* o1 = J.P1 + c * J.out_plane + oo + x4;
                    for (int q = 0; q < nq; ++q) {
                        o0[q] = v0[q];
                        o1[q] = v1[q];
                    }
                }
            }
            float* s0 = J.S0 + oo + x4;
            float* s1 = J.S1 + oo + x4;
            if (nq == 4) {  // output rows start on 128-byte boundaries
                reinterpret_cast<float4*>(s0)[0] = make_float4(a[0] * inv, a[1] * inv, a[2] * inv, a[3] * inv);
                reinterpret_cast<float4*>(s1)[0] = make_float4(b[0] * inv, b[1] * inv, b[2] * inv, b[3] * inv);
            } else {
                for (int q = 0; q < nq; ++q) {
                    s0[q] = a[q] * inv;
                    s1[q] = b[q] * inv;
                }
            }
        }
    }
}

// One pyramid step: out(x, y) = sum_{i,j} k_i k_j in(2x + i, 2y + j), k = [1 4 6 4 1] / 16,
// indices clamped (replicated border).  Rows are blurred first, then the column.  A block
// iteration is a band of J.band (<= kPyrBand) output rows by kPyrChunk output columns of one
// plane: the horizontal blurs of the band's 2 band + 3 input rows are computed once into
// shared memory (an input row serves up to three output rows), then every output sums five of
// them, in the same order as a per-pixel evaluation.  The host picks the band height per call:
// the tallest band that still gives every SM several units.
constexpr int kPyrBand = 8, kPyrChunk = 256;

__global__ void __launch_bounds__(kPyrChunk) pyr_down_kernel(const __grid_constant__ Jobs<PyrJob> js, long long units)
{
    __shared__ float hb[2 * kPyrBand + 3][kPyrChunk];
    const float kw[5] = {0.0625f, 0.25f, 0.375f, 0.25f, 0.0625f};
    const int xx = threadIdx.x;
    for (long long u = blockIdx.x; u < units; u += gridDim.x) {
        const PyrJob& J = job_ref(js, find_job(js, u, &PyrJob::base));
        const int bh = J.band;
        const int bands = (J.hout + bh - 1) / bh, chunks = (J.wout + kPyrChunk - 1) / kPyrChunk;
        const int rr = (int)(u - J.base);
        const int p = rr / (bands * chunks), rem = rr - p * (bands * chunks);
        const int band = rem / chunks, cx = rem - band * chunks;
        const int y0 = band * bh, ny = min(bh, J.hout - y0);
        const int x = cx * kPyrChunk + xx;
        const bool on = x < J.wout;
        const float* __restrict__ in = J.in + p * J.in_plane;
        const int win = J.win;
        if (bh == 1) {  // one output row: its five input rows' blurs are used once, no staging
            if (on) {
                const int xs[5] = {clampi(2 * x - 2, 0, win - 1), clampi(2 * x - 1, 0, win - 1), min(2 * x, win - 1),
                                   clampi(2 * x + 1, 0, win - 1), clampi(2 * x + 2, 0, win - 1)};
                float acc = 0.0f;
#pragma unroll
                for (int j = 0; j < 5; ++j) {
                    const float* row = in + (long long)clampi(2 * y0 + j - 2, 0, J.hin - 1) * J.pin;
                    float h = kw[0] * __ldg(row + xs[0]);
#pragma unroll
                    for (int i = 1; i < 5; ++i) h = fmaf(kw[i], __ldg(row + xs[i]), h);
                    acc = fmaf(kw[j], h, acc);
                }
                J.out[p * J.out_plane + (long long)y0 * J.pout + x] = acc;
            }
            continue;  // uniform over the block: no barrier is skipped by part of it
        }
        if (on) {
            const int xs[5] = {clampi(2 * x - 2, 0, win - 1), clampi(2 * x - 1, 0, win - 1), min(2 * x, win - 1),
                               clampi(2 * x + 1, 0, win - 1), clampi(2 * x + 2, 0, win - 1)};
            for (int jr = 0; jr < 2 * ny + 3; ++jr) {
                const float* row = in + (long long)clampi(2 * y0 - 2 + jr, 0, J.hin - 1) * J.pin;
                float h = kw[0] * __ldg(row + xs[0]);
#pragma unroll
                for (int i = 1; i < 5; ++i) h = fmaf(kw[i], __ldg(row + xs[i]), h);
                hb[jr][xx] = h;
            }
        }
        __syncthreads();
        if (on) {
            float* out = J.out + p * J.out_plane + (long long)y0 * J.pout + x;
            for (int yy = 0; yy < ny; ++yy) {
                float acc = 0.0f;
#pragma unroll
                for (int j = 0; j < 5; ++j) acc = fmaf(kw[j], hb[2 * yy + j][xx], acc);
                out[(long long)yy * J.pout] = acc;
            }
        }
        __syncthreads();  // hb is refilled by the next band
    }
}

long long pyr_units(int wout, int hout, int nplanes, int band)
{
    return (long long)nplanes * ((hout + band - 1) / band) * ((wout + kPyrChunk - 1) / kPyrChunk);
}

int pyr_band(long long units_at_full_band, long long units_at_band2, int sm_count)
{
    const long long want = 4LL * sm_count;  // units that keep every SM busy for a few rounds
    return units_at_full_band >= want ? kPyrBand : units_at_band2 >= want ? 2 : 1;
}

// Sobel / 8 with replicated border (standalone form of the operator the search computes in
// its prologue).
__global__ void __launch_bounds__(256) sobel_kernel(const float* __restrict__ in, int w, int h, int pitch,
                                                    float* __restrict__ gx, float* __restrict__ gy, int out_pitch)
{
    const long long total = (long long)w * h;
    for (long long g = gtid(); g < total; g += gstride()) {
        const int y = (int)(g / w), x = (int)(g - (long long)y * w);
        const int xl = max(x - 1, 0), xr = min(x + 1, w - 1);
        const float* ru = in + (long long)max(y - 1, 0) * pitch;
        const float* rc = in + (long long)y * pitch;
        const float* rd = in + (long long)min(y + 1, h - 1) * pitch;
        const float a = __ldg(ru + xl), b = __ldg(ru + x), c = __ldg(ru + xr);
        const float d = __ldg(rc + xl), f = __ldg(rc + xr);
        const float p = __ldg(rd + xl), q = __ldg(rd + x), s = __ldg(rd + xr);
        gx[(long long)y * out_pitch + x] = 0.125f * ((c - a) + 2.0f * (f - d) + (s - p));
        gy[(long long)y * out_pitch + x] = 0.125f * ((p - a) + 2.0f * (q - b) + (s - c));
    }
}

// Uout(x) = factor * Uin(x / factor), bilinear with clamping (Sec. 3.1, last paragraph).  A
// block row is one output row.
__global__ void __launch_bounds__(256) upsample_kernel(const __grid_constant__ Jobs<UpJob> js, long long rows)
{
    for (long long r = blockIdx.x; r < rows; r += gridDim.x) {
        const UpJob& J = job_ref(js, find_job(js, r, &UpJob::base));
        const int y = (int)(r - J.base);
        float2* out = J.out + (long long)y * J.wo;
        const float fy = (float)y / J.factor;
#pragma unroll 4
        for (int x = threadIdx.x; x < J.wo; x += blockDim.x) {
            const float2 v = sample_flow(J.in, J.wi, J.hi, (float)x / J.factor, fy);
            out[x] = make_float2(J.factor * v.x, J.factor * v.y);
        }
    }
}

static int grid_rows(long long rows, const LaunchCfg& lc)
{
    const long long cap = (long long)lc.sm_count * lc.max_blocks_256;
    return (int)(rows < 1 ? 1 : rows < cap ? rows : cap);
}

static int grid_for(long long total, int threads, const LaunchCfg& lc)
{
    long long b = (total + threads - 1) / threads;
    const long long cap = (long long)lc.sm_count * lc.max_blocks_256;
    if (b > cap) b = cap;
    return (int)(b < 1 ? 1 : b);
}

cudaError_t launch_prep(const Jobs<PrepJob>& js, long long rows, const LaunchCfg& lc, cudaStream_t s)
{
    if (rows <= 0) return cudaSuccess;
    prep_kernel<<<grid_rows(rows, lc), 256, 0, s>>>(js, rows);
    return cudaGetLastError();
}

cudaError_t launch_pyr_down(const Jobs<PyrJob>& js, long long units, const LaunchCfg& lc, cudaStream_t s)
{
    if (units <= 0) return cudaSuccess;
    pyr_down_kernel<<<grid_rows(units, lc), kPyrChunk, 0, s>>>(js, units);
    return cudaGetLastError();
}

cudaError_t launch_sobel(const float* in, int w, int h, int pitch, float* gx, float* gy, int out_pitch,
                         const LaunchCfg& lc, cudaStream_t s)
{
    const long long total = (long long)w * h;
    if (total <= 0) return cudaSuccess;
    sobel_kernel<<<grid_for(total, 256, lc), 256, 0, s>>>(in, w, h, pitch, gx, gy, out_pitch);
    return cudaGetLastError();
}

cudaError_t launch_upsample(const Jobs<UpJob>& js, long long rows, const LaunchCfg& lc, cudaStream_t s)
{
    if (rows <= 0) return cudaSuccess;
    upsample_kernel<<<grid_rows(rows, lc), 256, 0, s>>>(js, rows);
    return cudaGetLastError();
}

LaunchCfg query_launch_cfg()
{
    LaunchCfg lc;
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&lc.sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || lc.sm_count <= 0)
        lc.sm_count = 152;
    lc.max_blocks_256 = 8;
    return lc;
}

}  // namespace dis
