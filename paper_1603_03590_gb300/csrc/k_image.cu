// Pyramid and resampling kernels of DIS (Sec. 3.1: image pyramid with theta_sd = 2 and
// image gradients; up-scaling of the flow to full resolution).  All are streaming stencils
// bound by memory bandwidth: thread per output pixel, read-only loads through L1.
#include "dis_device.cuh"

namespace dis {

// Level 0: multiply the caller's [0,1] frames by intensity_scale, write the channel mean
// (the search image) and, for colour input, the scaled channel planes.
__global__ void __launch_bounds__(256) prep_kernel(const __grid_constant__ Jobs<PrepJob> js, long long total)
{
    for (long long g = gtid(); g < total; g += gstride()) {
        const PrepJob& J = job_ref(js, find_job(js, g, &PrepJob::base));
        const int k = (int)(g - J.base);  // < w * h < 2^31
        const int y = k / J.w, x = k - y * J.w;
        const long long io = (long long)y * J.in_pitch + x, oo = (long long)y * J.out_pitch + x;
        float a = 0.0f, b = 0.0f;
        for (int c = 0; c < J.C; ++c) {
            const float v0 = J.scale * __ldg(J.I0 + c * J.in_plane + io);
            const float v1 = J.scale * __ldg(J.I1 + c * J.in_plane + io);
            if (J.P0) {
                J.P0[c * J.out_plane + oo] = v0;
                J.P1[c * J.out_plane + oo] = v1;
            }
            a += v0;
            b += v1;
        }
        const float inv = 1.0f / (float)J.C;
        J.S0[oo] = a * inv;
        J.S1[oo] = b * inv;
    }
}

// One pyramid step: out(x, y) = sum_{i,j} k_i k_j in(2x + i, 2y + j), k = [1 4 6 4 1] / 16,
// indices clamped (replicated border).  Rows are blurred first, then the column.
__global__ void __launch_bounds__(256) pyr_down_kernel(const __grid_constant__ Jobs<PyrJob> js, long long total)
{
    for (long long g = gtid(); g < total; g += gstride()) {
        const PyrJob& J = job_ref(js, find_job(js, g, &PyrJob::base));
        const int k = (int)(g - J.base);  // < planes * w * h < 2^31
        const int npix = J.wout * J.hout;
        const int p = k / npix;
        const int r = k - p * npix;
        const int y = r / J.wout, x = r - y * J.wout;
        const float* in = J.in + p * J.in_plane;
        const int xs[5] = {clampi(2 * x - 2, 0, J.win - 1), clampi(2 * x - 1, 0, J.win - 1), min(2 * x, J.win - 1),
                           clampi(2 * x + 1, 0, J.win - 1), clampi(2 * x + 2, 0, J.win - 1)};
        const float kw[5] = {0.0625f, 0.25f, 0.375f, 0.25f, 0.0625f};
        float acc = 0.0f;
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            const float* row = in + (long long)clampi(2 * y + j - 2, 0, J.hin - 1) * J.pin;
            float h = kw[0] * __ldg(row + xs[0]);
#pragma unroll
            for (int i = 1; i < 5; ++i) h = fmaf(kw[i], __ldg(row + xs[i]), h);
            acc = fmaf(kw[j], h, acc);
        }
        J.out[p * J.out_plane + (long long)y * J.pout + x] = acc;
    }
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

// Uout(x) = factor * Uin(x / factor), bilinear with clamping (Sec. 3.1, last paragraph).
__global__ void __launch_bounds__(256) upsample_kernel(const __grid_constant__ Jobs<UpJob> js, long long total)
{
    for (long long g = gtid(); g < total; g += gstride()) {
        const UpJob& J = job_ref(js, find_job(js, g, &UpJob::base));
        const int k = (int)(g - J.base);  // < w * h < 2^31
        const int y = k / J.wo, x = k - y * J.wo;
        const float2 v = sample_flow(J.in, J.wi, J.hi, (float)x / J.factor, (float)y / J.factor);
        J.out[k] = make_float2(J.factor * v.x, J.factor * v.y);
    }
}

static int grid_for(long long total, int threads, const LaunchCfg& lc)
{
    long long b = (total + threads - 1) / threads;
    const long long cap = (long long)lc.sm_count * lc.max_blocks_256;
    if (b > cap) b = cap;
    return (int)(b < 1 ? 1 : b);
}

cudaError_t launch_prep(const Jobs<PrepJob>& js, long long total, const LaunchCfg& lc, cudaStream_t s)
{
    if (total <= 0) return cudaSuccess;
    prep_kernel<<<grid_for(total, 256, lc), 256, 0, s>>>(js, total);
    return cudaGetLastError();
}

cudaError_t launch_pyr_down(const Jobs<PyrJob>& js, long long total, const LaunchCfg& lc, cudaStream_t s)
{
    if (total <= 0) return cudaSuccess;
    pyr_down_kernel<<<grid_for(total, 256, lc), 256, 0, s>>>(js, total);
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

cudaError_t launch_upsample(const Jobs<UpJob>& js, long long total, const LaunchCfg& lc, cudaStream_t s)
{
    if (total <= 0) return cudaSuccess;
    upsample_kernel<<<grid_for(total, 256, lc), 256, 0, s>>>(js, total);
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
