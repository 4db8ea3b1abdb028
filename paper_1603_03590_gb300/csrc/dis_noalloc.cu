// Variational refinement of one level without any device allocation (no counterpart in the
// paper).
//
// dis_refine_level takes its per-pixel scratch (derivatives, 2x2 systems, increments) from a
// handle, whose arena dis_create allocates with cudaMalloc.  Some callers cannot do that:
// code running inside a host application that owns the whole device-memory budget through its
// own pool, or a latency-critical loop where cudaMalloc / cudaFree are not allowed because
// they may synchronise the device.  dis_refine_level_noalloc serves them: the scratch is the
// file-scope device array below, reserved when the library is loaded, so the call itself
// allocates nothing.  The caller still owns the images and the flow.
//
// Host code cannot hand `g_refine_scratch` to a kernel: in host code that name denotes a
// host-side stand-in, not device memory.  The device address is looked up once per device
// with cudaGetSymbolAddress (with that device current) on the first call made on it, cached,
// and passed to the kernels.  cudaDeviceReset destroys the array with the context, so the
// cached address of a device is not valid after a reset of that device.
#include <cmath>
#include <mutex>
#include <string>

#include "../../include/dis.h"
#include "dis_internal.cuh"

namespace {

__device__ __align__(256) float g_refine_scratch[DIS_NOALLOC_SCRATCH_FLOATS];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
float* g_scratch_addr[kMaxDevices] = {};

dis_status noalloc_fail(dis_status st, const std::string& msg)
{
    dis::set_thread_error(msg);
    return st;
}

}  // namespace

extern "C" dis_status dis_refine_level_noalloc(const float* I0, const float* I1, int w, int h, int64_t pitch,
                                               int channels, float* U, int outer, int inner, float delta,
                                               float gamma, float alpha, float omega, void* stream)
{
    if (!I0 || !I1 || !U || w < 1 || h < 1 || pitch < w || channels < 1 || channels > 3 || outer < 0 || inner < 0 ||
        !std::isfinite(delta) || !std::isfinite(gamma) || !std::isfinite(alpha) || !(omega > 0.0f && omega < 2.0f))
        return noalloc_fail(DIS_ERR_INVALID_ARG, "dis_refine_level_noalloc: bad pointer, size, pitch or parameter");
    // bound each factor before the product, so that it cannot wrap: any level that fits the
    // array has pitch * h below 2^22
    if (pitch > (int64_t)DIS_NOALLOC_SCRATCH_FLOATS || h > (int)DIS_NOALLOC_SCRATCH_FLOATS ||
        (unsigned long long)pitch * (unsigned long long)h > (unsigned long long)DIS_NOALLOC_SCRATCH_FLOATS)
        return noalloc_fail(DIS_ERR_INVALID_ARG,
                            "dis_refine_level_noalloc: pitch * height above the fixed scratch of " +
                                std::to_string((unsigned long long)DIS_NOALLOC_SCRATCH_FLOATS) + " floats");
    const unsigned long long need =
        (unsigned long long)dis::rs_planes(channels) * (unsigned long long)pitch * (unsigned long long)h;
    if (need > (unsigned long long)DIS_NOALLOC_SCRATCH_FLOATS)
        return noalloc_fail(DIS_ERR_INVALID_ARG,
                            "dis_refine_level_noalloc: level needs " + std::to_string(need) +
                                " scratch floats ((15 * channels + 8) * pitch * height), more than the fixed " +
                                std::to_string((unsigned long long)DIS_NOALLOC_SCRATCH_FLOATS));
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(DIS_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(DIS_ERR_NOT_SUPPORTED, "device ordinal above 63");
    float* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_scratch_addr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_refine_scratch);
            if (e != cudaSuccess)
                return noalloc_fail(DIS_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            g_scratch_addr[dev] = static_cast<float*>(p);
        }
        scratch = g_scratch_addr[dev];
    }
    dis::LevelJob J = {};
    J.P0 = I0;
    J.P1 = I1;
    J.w = w;
    J.h = h;
    J.pitch = (int)pitch;
    J.plane = (long long)pitch * h;
    J.C = channels;
    J.U = reinterpret_cast<float2*>(U);
    J.rs = scratch;  // every plane is written before it is read; the increments are zeroed first
    long long tiles = 0;
    dis::set_refine_tiles(J, tiles);
    dis::RefineArgs a{outer, inner, delta, gamma, alpha, omega};
    a.fused = 1;  // launch form 1 with its default threshold: one fused launch per outer pass
    a.C = channels;
    e = dis::launch_refine(dis::single_job(J), (long long)w * h, (long long)h * ((w + 1) / 2), tiles, a,
                           dis::stage_launch_cfg(), (cudaStream_t)stream);
    if (e != cudaSuccess) return noalloc_fail(DIS_ERR_CUDA, std::string("dis_refine_level_noalloc: ") + cudaGetErrorString(e));
    return DIS_OK;
}
