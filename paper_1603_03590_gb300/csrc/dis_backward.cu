// Host side of the differentiable form (not in the paper): the photometric loss, the FP64
// replay of the frozen-search DIS map and its backward pass through the pyramid, the initial
// displacements, densification (Eq. 3) and the unrolled red-black SOR of the variational
// refinement (Sec. 2.3).
//
// The replay starts from the caller's frames, initial flow and recorded increments and runs in
// double precision; the backward repeats it, then, per level (finest first), recomputes the
// refinement's derivatives, lagged weights and the increment before every half-sweep (stored
// in the caller's workspace) and runs the adjoint kernels in reverse order.  No device memory
// is allocated: everything lives in the caller's workspace.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <initializer_list>
#include <string>
#include <vector>

#include "../../include/dis.h"
#include "dis_host.h"
#include "dis_internal.cuh"

using namespace dis_host;

namespace {

constexpr size_t kAl = 256;
size_t al(size_t v) { return (v + kAl - 1) / kAl * kAl; }

struct BwdLayout {
    int ss = 0, sf = 0;
    std::vector<int> w, h, pitch, outer, np;
    // accumulators first (one memset): per level gS0, gS1acc, gUacc, gS0acc, then gInit
    std::vector<size_t> gS0, gS1acc, gUacc, gS0acc;
    size_t gInit = 0, acc_end = 0;
    // per level state
    std::vector<size_t> S0, S1, Ud, U, pu, gS1f, gU;
    size_t init64 = 0, rs = 0, ga = 0, states = 0, gUd = 0, gpu = 0, total = 0;
};

dis_status layout(int W, int H, const dis_params& p, BwdLayout& L, std::string& err)
{
    dis_status st = levels_of(W, H, p, L.ss, L.sf, err);
    if (st != DIS_OK) return st;
    const int n = L.ss + 1, ps = p.patch_size, stride = stride_of_params(p);
    size_t max_states = 0;
    for (int s = 0; s < n; ++s) {
        const int w = level_dim_of(W, s), h = level_dim_of(H, s);
        L.w.push_back(w);
        L.h.push_back(h);
        L.pitch.push_back(pitch_of_w(w));
        L.outer.push_back(p.refine ? (p.var_outer < 0 ? s + 1 : p.var_outer) : 0);
        L.np.push_back(grid_count(w, ps, stride) * grid_count(h, ps, stride));
        max_states = std::max(max_states, (size_t)L.outer[s] * 2 * p.var_inner * 2 * L.pitch[s] * h);
    }
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = al(off + bytes);
        return o;
    };
    for (int s = 0; s < n; ++s) {
        const size_t plane = (size_t)L.pitch[s] * L.h[s], pix = (size_t)L.w[s] * L.h[s];
        L.gS0.push_back(take(sizeof(double) * plane));
        L.gS1acc.push_back(take(sizeof(unsigned long long) * plane));
        L.gUacc.push_back(take(sizeof(unsigned long long) * 2 * pix));
        L.gS0acc.push_back(take(sizeof(unsigned long long) * plane));
    }
    L.gInit = take(sizeof(unsigned long long) * 2 * L.w[L.ss] * L.h[L.ss]);
    L.acc_end = off;
    for (int s = 0; s < n; ++s) {
        const size_t plane = (size_t)L.pitch[s] * L.h[s], pix = (size_t)L.w[s] * L.h[s];
        L.S0.push_back(take(sizeof(double) * plane));
        L.S1.push_back(take(sizeof(double) * plane));
        L.Ud.push_back(take(sizeof(double) * 2 * pix));
        L.U.push_back(take(sizeof(double) * 2 * pix));
        L.pu.push_back(take(sizeof(double) * 2 * std::max(1, L.np[s])));
        L.gS1f.push_back(take(sizeof(double) * plane));
        L.gU.push_back(take(sizeof(double) * 2 * pix));
    }
    const size_t plane0 = (size_t)L.pitch[0] * L.h[0], pix0 = (size_t)L.w[0] * L.h[0];
    L.init64 = take(sizeof(double) * 2 * L.w[L.ss] * L.h[L.ss]);
    L.rs = take(sizeof(double) * dis::rs_planes(1) * plane0);
    L.ga = take(sizeof(double) * dis::ADJ_PLANES * plane0);
    L.states = take(sizeof(double) * std::max<size_t>(1, max_states));
    L.gUd = take(sizeof(double) * 2 * pix0);
    L.gpu = take(sizeof(double) * 2 * std::max(1, L.np[0]));
    L.total = off;
    return DIS_OK;
}

struct Ctx {
    const BwdLayout& L;
    char* ws;
    const dis_params& p;
    const dis::LaunchCfg& lc;
    cudaStream_t s;
    double* D(size_t off) const { return reinterpret_cast<double*>(ws + off); }
    double2* D2(size_t off) const { return reinterpret_cast<double2*>(ws + off); }
    unsigned long long* U64(size_t off) const { return reinterpret_cast<unsigned long long*>(ws + off); }
    dis::Lvl64 level(int s) const
    {
        dis::Lvl64 v = {};
        v.S0 = D(L.S0[s]);
        v.S1 = D(L.S1[s]);
        v.U = D2(L.Ud[s]);
        v.rs = D(L.rs);
        v.ga = D(L.ga);
        v.gS0 = D(L.gS0[s]);
        v.gS1 = U64(L.gS1acc[s]);
        v.gU = D2(L.gUd);
        v.plane = (long long)L.pitch[s] * L.h[s];
        v.w = L.w[s];
        v.h = L.h[s];
        v.pitch = L.pitch[s];
        v.delta = p.delta;
        v.gamma = p.gamma;
        v.alpha = p.alpha;
        v.omega = p.sor_omega;
        v.dof = p.dof;
        return v;
    }
    dis::Dens64 dens(int s) const
    {
        dis::Dens64 a = {};
        a.pu = D2(L.pu[s]);
        a.gpu = D2(L.gpu);
        a.gUd = D2(L.gUd);
        a.ps = p.patch_size;
        a.stride = stride_of_params(p);
        a.nx = grid_count(L.w[s], a.ps, a.stride);
        a.ny = grid_count(L.h[s], a.ps, a.stride);
        return a;
    }
};

// FP64 forward of the frozen map: level images, patch flows, densified and refined flows.
cudaError_t replay(const Ctx& c, const float* I0, const float* I1, long long pitch, const float* init,
                   const float* frozen)
{
    const BwdLayout& L = c.L;
    cudaError_t e = dis::launch_prep64(I0, L.w[0], L.h[0], (int)pitch, c.p.intensity_scale, c.D(L.S0[0]), L.pitch[0],
                                       c.lc, c.s);
    if (e == cudaSuccess)
        e = dis::launch_prep64(I1, L.w[0], L.h[0], (int)pitch, c.p.intensity_scale, c.D(L.S1[0]), L.pitch[0], c.lc, c.s);
    for (int s = 1; s <= L.ss && e == cudaSuccess; ++s) {
        e = dis::launch_pyr64(c.D(L.S0[s - 1]), L.w[s - 1], L.h[s - 1], L.pitch[s - 1], c.D(L.S0[s]), L.w[s], L.h[s],
                              L.pitch[s], c.lc, c.s);
        if (e == cudaSuccess)
            e = dis::launch_pyr64(c.D(L.S1[s - 1]), L.w[s - 1], L.h[s - 1], L.pitch[s - 1], c.D(L.S1[s]), L.w[s],
                                  L.h[s], L.pitch[s], c.lc, c.s);
    }
    if (init && e == cudaSuccess)
        e = dis::launch_f2_to_d2(reinterpret_cast<const float2*>(init), c.D2(L.init64), (long long)L.w[L.ss] * L.h[L.ss],
                                 c.lc, c.s);
    long long off = 0;
    for (int s = L.ss; s >= L.sf && e == cudaSuccess; --s) {
        const int w = L.w[s], h = L.h[s];
        const double2* Uc = nullptr;
        int wc = w, hc = h;
        double cs = 1.0;
        if (s == L.ss) {
            Uc = init ? c.D2(L.init64) : nullptr;
        } else {
            Uc = c.D2(L.U[s + 1]);
            wc = L.w[s + 1];
            hc = L.h[s + 1];
            cs = 2.0;
        }
        const dis::Dens64 A = c.dens(s);
        e = dis::launch_uinit64(A, w, h, Uc, wc, hc, cs, reinterpret_cast<const float2*>(frozen) + off, c.D2(L.pu[s]),
                                c.lc, c.s);
        off += L.np[s];
        if (e == cudaSuccess)
            e = dis::launch_densify64(c.D(L.S0[s]), c.D(L.S1[s]), w, h, L.pitch[s], A, Uc, wc, hc, cs, c.D2(L.Ud[s]),
                                      c.lc, c.s);
        if (e != cudaSuccess) break;
        if (c.p.refine) {
            const dis::Lvl64 lv = c.level(s);
            e = dis::launch_ref64_prepare(lv, c.lc, c.s);
            for (int o = 0; o < L.outer[s] && e == cudaSuccess; ++o) {
                e = dis::launch_ref64_weights(lv, c.lc, c.s);
                for (int k = 0; k < 2 * c.p.var_inner && e == cudaSuccess; ++k) e = dis::launch_ref64_sor(lv, k & 1, c.lc, c.s);
            }
            if (e == cudaSuccess) e = dis::launch_ref64_apply(lv, c.D2(L.U[s]), c.lc, c.s);
        } else {
            e = cudaMemcpyAsync(c.D2(L.U[s]), c.D2(L.Ud[s]), sizeof(double2) * w * h, cudaMemcpyDeviceToDevice, c.s);
        }
    }
    if (e == cudaSuccess && L.sf > 0)  // final up-scaling to full resolution (Sec. 3.1)
        e = dis::launch_upsample64(c.D2(L.U[L.sf]), L.w[L.sf], L.h[L.sf], (double)(1 << L.sf), c.D2(L.U[0]), L.w[0],
                                   L.h[0], c.lc, c.s);
    return e;
}

dis_status check_common(dis_handle* hd, const float* I0, const float* I1, int W, int H, int64_t pitch,
                        const dis_params* p, const float* frozen, void* workspace, int64_t workspace_bytes,
                        BwdLayout& L)
{
    if (!hd) return set_fail(nullptr, DIS_ERR_INVALID_ARG, "handle is NULL");
    std::string err;
    dis_status st = validate_params(p, err);
    if (st != DIS_OK) return set_fail(hd, st, err);
    if (p->channels != 1) return set_fail(hd, DIS_ERR_NOT_SUPPORTED, "differentiable form: grayscale (channels = 1) only");
    if (p->fb) return set_fail(hd, DIS_ERR_NOT_SUPPORTED, "differentiable form: no forward-backward consistency");
    if (p->search_grad && p->norm != 0)
        return set_fail(hd, DIS_ERR_NOT_SUPPORTED, "implicit search gradient: L2 search norm only");
    if (!I0 || !I1 || !frozen || !workspace || W < 1 || H < 1 || pitch < W)
        return set_fail(hd, DIS_ERR_INVALID_ARG, "differentiable form: bad pointer, size or pitch");
    if ((st = layout(W, H, *p, L, err)) != DIS_OK) return set_fail(hd, st, err);
    if ((int64_t)L.total > workspace_bytes)
        return set_fail(hd, DIS_ERR_INVALID_ARG, "workspace smaller than dis_backward_workspace_bytes");
    return DIS_OK;
}

// The backward pass of one pair (the chain of launches dis_backward issues).
cudaError_t backward(const Ctx& c, const float* I0, const float* I1, int W, int H, int64_t pitch, const float* init_flow,
                     const float* frozen, const float* grad_flow, float* grad_I0, float* grad_I1, int64_t grad_pitch,
                     float* grad_init_flow)
{
    const BwdLayout& L = c.L;
    cudaStream_t s = c.s;
    const dis::LaunchCfg& lc = c.lc;
    cudaError_t e = cudaMemsetAsync(c.ws, 0, L.acc_end, s);
    if (e == cudaSuccess) e = replay(c, I0, I1, pitch, init_flow, frozen);
    if (e == cudaSuccess)
        e = dis::launch_f2_to_d2(reinterpret_cast<const float2*>(grad_flow), c.D2(L.gU[0]), (long long)W * H, lc, s);
    if (e == cudaSuccess && L.sf > 0)  // the final up-scaling's transpose into level theta_sf
        e = dis::launch_upsample_bwd(c.D2(L.gU[0]), W, H, (double)(1 << L.sf), c.U64(L.gUacc[L.sf]), L.w[L.sf],
                                     L.h[L.sf], lc, s);
    for (int sl = L.sf; sl <= L.ss && e == cudaSuccess; ++sl) {
        const int w = L.w[sl], h = L.h[sl];
        const long long plane = (long long)L.pitch[sl] * h;
        if (sl > 0) e = dis::launch_fx_to_double(c.U64(L.gUacc[sl]), 2 * w, c.D(L.gU[sl]), 2 * w, 2 * w, h, 1.0, false, lc, s);
        const dis::Lvl64 lv = c.level(sl);
        if (c.p.refine && e == cudaSuccess) {
            const int outer = L.outer[sl], inner = c.p.var_inner;
            double* du = lv.rs + (long long)dis::rs_du(1, 0) * plane;  // du and dv planes are adjacent
            const size_t st_bytes = sizeof(double) * 2 * plane;
            double* states = c.D(L.states);
            auto state = [&](int o, int k) { return states + ((size_t)o * 2 * inner + k) * 2 * plane; };
            // forward recompute of this level, saving the increment before every half-sweep
            e = dis::launch_ref64_prepare(lv, lc, s);
            for (int o = 0; o < outer && e == cudaSuccess; ++o) {
                e = dis::launch_ref64_weights(lv, lc, s);
                for (int k = 0; k < 2 * inner && e == cudaSuccess; ++k) {
                    e = cudaMemcpyAsync(state(o, k), du, st_bytes, cudaMemcpyDeviceToDevice, s);
                    if (e == cudaSuccess) e = dis::launch_ref64_sor(lv, k & 1, lc, s);
                }
            }
            // adjoint of U_out = U_d + dU
            if (e == cudaSuccess) e = cudaMemsetAsync(lv.ga + (long long)dis::ADJ_GD * plane, 0, sizeof(double) * 9 * plane, s);
            if (e == cudaSuccess) e = dis::launch_start_flow(lv, c.D2(L.gU[sl]), lc, s);
            for (int o = outer - 1; o >= 0 && e == cudaSuccess; --o) {
                if (inner > 0)
                    e = cudaMemcpyAsync(du, state(o, 0), st_bytes, cudaMemcpyDeviceToDevice, s);
                else  // no sweep: the increment stays 0
                    e = cudaMemsetAsync(du, 0, st_bytes, s);
                if (e == cudaSuccess) e = dis::launch_ref64_weights(lv, lc, s);
                if (e == cudaSuccess)
                    e = cudaMemsetAsync(lv.ga + (long long)dis::ADJ_GSYS * plane, 0, sizeof(double) * 6 * plane, s);
                for (int k = 2 * inner - 1; k >= 0 && e == cudaSuccess; --k) {
                    const double* sd = state(o, k);
                    e = dis::launch_sor_bwd(lv, sd, sd + plane, k & 1, lc, s);
                }
                if (e == cudaSuccess) {
                    const double* s0 = inner > 0 ? state(o, 0) : du;
                    e = dis::launch_weights_bwd(lv, s0, s0 + plane, lc, s);
                }
            }
            if (e == cudaSuccess) e = dis::launch_deriv_warp_bwd(lv, lc, s);
        } else if (e == cudaSuccess) {
            e = cudaMemcpyAsync(c.D2(L.gUd), c.D2(L.gU[sl]), sizeof(double2) * w * h, cudaMemcpyDeviceToDevice, s);
        }
        const dis::Dens64 A = c.dens(sl);
        if (e == cudaSuccess) e = dis::launch_dens_bwd(lv, A, lc, s);
        if (e == cudaSuccess && c.p.search_grad) {
            long long off = 0;  // increments of coarser levels come first
            for (int q = L.ss; q > sl; --q) off += L.np[q];
            e = dis::launch_search_ift_bwd(lv, A, reinterpret_cast<const float2*>(frozen) + off, c.U64(L.gS0acc[sl]),
                                           c.p.dof, lc, s);
        }
        if (e == cudaSuccess) {
            if (sl < L.ss)
                e = dis::launch_uinit_bwd(A, w, h, c.U64(L.gUacc[sl + 1]), L.w[sl + 1], L.h[sl + 1], 2.0, lc, s);
            else if (grad_init_flow)
                e = dis::launch_uinit_bwd(A, w, h, c.U64(L.gInit), w, h, 1.0, lc, s);
        }
    }
    // level images: fixed point -> double, then the pyramid transpose down to level 0
    for (int sl = 0; sl <= L.ss && e == cudaSuccess; ++sl) {
        e = dis::launch_fx_to_double(c.U64(L.gS1acc[sl]), L.pitch[sl], c.D(L.gS1f[sl]), L.pitch[sl], L.w[sl], L.h[sl],
                                     1.0, false, lc, s);
        if (e == cudaSuccess && c.p.search_grad)
            e = dis::launch_fx_to_double(c.U64(L.gS0acc[sl]), L.pitch[sl], c.D(L.gS0[sl]), L.pitch[sl], L.w[sl],
                                         L.h[sl], 1.0, true, lc, s);
    }
    for (int sl = L.ss; sl >= 1 && e == cudaSuccess; --sl) {
        e = dis::launch_pyr_bwd(c.D(L.gS0[sl]), L.w[sl], L.h[sl], L.pitch[sl], c.D(L.gS0[sl - 1]), L.w[sl - 1],
                                L.h[sl - 1], L.pitch[sl - 1], lc, s);
        if (e == cudaSuccess)
            e = dis::launch_pyr_bwd(c.D(L.gS1f[sl]), L.w[sl], L.h[sl], L.pitch[sl], c.D(L.gS1f[sl - 1]), L.w[sl - 1],
                                    L.h[sl - 1], L.pitch[sl - 1], lc, s);
    }
    if (e == cudaSuccess)
        e = dis::launch_scale_out(c.D(L.gS0[0]), L.pitch[0], grad_I0, (int)grad_pitch, W, H, c.p.intensity_scale, lc, s);
    if (e == cudaSuccess)
        e = dis::launch_scale_out(c.D(L.gS1f[0]), L.pitch[0], grad_I1, (int)grad_pitch, W, H, c.p.intensity_scale, lc, s);
    if (e == cudaSuccess && grad_init_flow)
        e = dis::launch_fx_to_float(c.U64(L.gInit), 2 * L.w[L.ss], grad_init_flow, 2 * L.w[L.ss], 2 * L.w[L.ss],
                                    L.h[L.ss], 1.0, false, lc, s);
    return e;
}

// The key of a differentiable-form call: its kind, every pointer and size, the parameters.
std::vector<int64_t> call_key(int kind, std::initializer_list<int64_t> args, const dis_params& p)
{
    std::vector<int64_t> k{kind};
    k.insert(k.end(), args);
    const int32_t* pw = reinterpret_cast<const int32_t*>(&p);  // every field is 4 bytes wide
    for (size_t i = 0; i < sizeof(dis_params) / 4; ++i) k.push_back(pw[i]);
    return k;
}

int64_t ptr_key(const void* q) { return (int64_t)reinterpret_cast<uintptr_t>(q); }

// Runs record(stream) on `s`.  The differentiable form is a chain of several hundred short
// launches whose issue, not their work, bounds a call; a call seen before (same key) is
// captured once into a CUDA graph on the handle's capture stream and replayed with one launch
// from then on.  A key seen for the first time launches directly, so callers whose buffers
// change at every call pay no capture.
template <class Record>
cudaError_t run_graphed(dis_handle* hd, const std::vector<int64_t>& key, cudaStream_t s, Record&& record)
{
    if (!hd->use_graphs) {
        hd->last_kernels = -1;
        return record(s);
    }
    for (auto& g : hd->bwd_graphs)
        if (g.key == key) {
            hd->last_kernels = g.kernels;
            return cudaGraphLaunch(g.exec, s);
        }
    auto seen = std::find(hd->bwd_seen.begin(), hd->bwd_seen.end(), key);
    if (seen == hd->bwd_seen.end()) {
        if (hd->bwd_seen.size() >= 16) hd->bwd_seen.erase(hd->bwd_seen.begin());
        hd->bwd_seen.push_back(key);
        hd->last_kernels = -1;
        return record(s);
    }
    hd->bwd_seen.erase(seen);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(hd->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    const cudaError_t le = record(hd->cap_stream);
    e = cudaStreamEndCapture(hd->cap_stream, &graph);
    if (le != cudaSuccess || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return le != cudaSuccess ? le : e;
    }
    const int kernels = graph_kernel_nodes(graph);
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return e;
    if (hd->bwd_graphs.size() >= 8) {
        cudaGraphExecDestroy(hd->bwd_graphs.front().exec);
        hd->bwd_graphs.erase(hd->bwd_graphs.begin());
    }
    hd->bwd_graphs.push_back({key, exec, kernels});
    hd->last_kernels = kernels;
    return cudaGraphLaunch(exec, s);
}

}  // namespace

extern "C" {

int64_t dis_backward_workspace_bytes(int width, int height, const dis_params* p)
{
    std::string e;
    if (validate_params(p, e) != DIS_OK || width < 1 || height < 1) return -1;
    BwdLayout L;
    if (layout(width, height, *p, L, e) != DIS_OK) return -1;
    return (int64_t)L.total;
}

int64_t dis_photometric_loss_scratch_bytes(int width, int height, int64_t pitch, int channels)
{
    if (width < 1 || height < 1 || pitch < width || channels < 1) return -1;
    return (int64_t)(al(sizeof(unsigned long long) * (size_t)pitch * height * channels) + sizeof(double) * 2048);
}

dis_status dis_photometric_loss(const float* I0, const float* I1, int w, int h, int64_t pitch, int channels,
                                const float* flow, float eps, double* loss_out, float* grad_flow, float* grad_I0,
                                float* grad_I1, void* scratch, int64_t scratch_bytes, void* stream)
{
    if (!I0 || !I1 || !flow || !loss_out || !grad_flow || !grad_I0 || !grad_I1 || !scratch || w < 1 || h < 1 ||
        pitch < w || channels < 1 || channels > 3 || !(eps > 0.0f))
        return set_fail(nullptr, DIS_ERR_INVALID_ARG, "dis_photometric_loss: bad pointer, size or eps");
    const int64_t need = dis_photometric_loss_scratch_bytes(w, h, pitch, channels);
    if (scratch_bytes < need) return set_fail(nullptr, DIS_ERR_INVALID_ARG, "dis_photometric_loss: scratch too small");
    cudaStream_t s = (cudaStream_t)stream;
    const dis::LaunchCfg lc = dis::stage_launch_cfg();
    auto* acc = static_cast<unsigned long long*>(scratch);
    const size_t acc_bytes = al(sizeof(unsigned long long) * (size_t)pitch * h * channels);
    auto* partials = reinterpret_cast<double*>(static_cast<char*>(scratch) + acc_bytes);
    cudaError_t e = cudaMemsetAsync(acc, 0, acc_bytes, s);
    if (e == cudaSuccess)
        e = dis::launch_loss(I0, I1, w, h, (int)pitch, channels, reinterpret_cast<const float2*>(flow), eps, partials,
                             2048, loss_out, reinterpret_cast<float2*>(grad_flow), grad_I0, acc, lc, s);
    if (e == cudaSuccess)
        e = dis::launch_fx_to_float(acc, (int)pitch, grad_I1, (int)pitch, w, h * channels, 1.0, false, lc, s);
    return e == cudaSuccess ? DIS_OK : set_cuda_fail(nullptr, e, "dis_photometric_loss");
}

dis_status dis_replay_flow(dis_handle* hd, const float* I0, const float* I1, int W, int H, int64_t pitch,
                           const dis_params* p, const float* init_flow, const float* frozen, float* flow_out,
                           void* workspace, int64_t workspace_bytes, void* stream)
{
    BwdLayout L;
    dis_status st = check_common(hd, I0, I1, W, H, pitch, p, frozen, workspace, workspace_bytes, L);
    if (st != DIS_OK) return st;
    if (!flow_out) return set_fail(hd, DIS_ERR_INVALID_ARG, "dis_replay_flow: flow_out is NULL");
    const auto key = call_key(0, {ptr_key(I0), ptr_key(I1), W, H, pitch, ptr_key(init_flow), ptr_key(frozen),
                                  ptr_key(flow_out), ptr_key(workspace)}, *p);
    const cudaError_t e = run_graphed(hd, key, (cudaStream_t)stream, [&](cudaStream_t s) {
        const Ctx c{L, static_cast<char*>(workspace), *p, hd->lc, s};
        cudaError_t e = replay(c, I0, I1, pitch, init_flow, frozen);
        if (e == cudaSuccess)
            e = dis::launch_d2_to_f2(c.D2(L.U[0]), reinterpret_cast<float2*>(flow_out), (long long)W * H, c.lc, s);
        return e;
    });
    return e == cudaSuccess ? DIS_OK : set_cuda_fail(hd, e, "dis_replay_flow");
}

dis_status dis_backward(dis_handle* hd, const float* I0, const float* I1, int W, int H, int64_t pitch,
                        const dis_params* p, const float* init_flow, const float* frozen, const float* grad_flow,
                        float* grad_I0, float* grad_I1, int64_t grad_pitch, float* grad_init_flow, void* workspace,
                        int64_t workspace_bytes, void* stream)
{
    BwdLayout L;
    dis_status st = check_common(hd, I0, I1, W, H, pitch, p, frozen, workspace, workspace_bytes, L);
    if (st != DIS_OK) return st;
    if (!grad_flow || !grad_I0 || !grad_I1 || grad_pitch < W || (grad_init_flow && !init_flow))
        return set_fail(hd, DIS_ERR_INVALID_ARG, "dis_backward: bad gradient pointer or pitch");
    const auto key = call_key(1, {ptr_key(I0), ptr_key(I1), W, H, pitch, ptr_key(init_flow), ptr_key(frozen),
                                  ptr_key(grad_flow), ptr_key(grad_I0), ptr_key(grad_I1), grad_pitch,
                                  ptr_key(grad_init_flow), ptr_key(workspace)}, *p);
    const cudaError_t e = run_graphed(hd, key, (cudaStream_t)stream, [&](cudaStream_t s) {
        return backward(Ctx{L, static_cast<char*>(workspace), *p, hd->lc, s}, I0, I1, W, H, pitch, init_flow, frozen,
                        grad_flow, grad_I0, grad_I1, grad_pitch, grad_init_flow);
    });
    return e == cudaSuccess ? DIS_OK : set_cuda_fail(hd, e, "dis_backward");
}

}  // extern "C"
