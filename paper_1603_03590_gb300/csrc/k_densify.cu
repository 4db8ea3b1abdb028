// Densification of DIS (Alg. 1 step 4, Eq. 3):
//   U(x) = sum_i w_i(x) u_i / sum_i w_i(x),  w_i(x) = 1 / max(1, |I1(x + u_i) - I0(x)|),
// over the patches i that contain x.  Thread per pixel; the covering patches follow from
// the grid arithmetic (corners min(i * stride, W - ps)), so every pixel gathers its own
// contributions in row-major patch order: no atomics, deterministic.
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

template <int SC>
__global__ void __launch_bounds__(256) densify_kernel(const __grid_constant__ Jobs<LevelJob> js, long long total,
                                                      int ps, int stride)
{
    for (long long g = gtid(); g < total; g += gstride()) {
        const LevelJob& J = job_ref(js, find_job(js, g, &LevelJob::pix_base));
        const int k = (int)(g - J.pix_base);  // < w * h < 2^31
        const int w = J.w, h = J.h, pitch = J.pitch, nx = J.nx, ny = J.ny;
        const int y = k / w, x = k - y * w;
        int ilo, ihi, jlo, jhi;
        bool ilast, jlast;
        cover_range<SC>(x, w, ps, stride, nx, ilo, ihi, ilast);
        cover_range<SC>(y, h, ps, stride, ny, jlo, jhi, jlast);
        const float i0 = __ldg(J.S0 + (long long)y * pitch + x);
        float nu = 0.0f, nv = 0.0f, Z = 0.0f;
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
        float2 r;
        if (Z > 0.0f) {
            r = make_float2(nu / Z, nv / Z);
        } else {
            r = init_flow_at(J.Uc, J.wc, J.hc, J.cscale, (float)x, (float)y);
        }
        J.U[k] = r;
    }
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
