// Host side of the DIS library: parameter validation, level arithmetic, the device arena,
// the per-call plan (job tables for every phase), CUDA-graph caching, and the C ABI
// declared in include/dis.h.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/dis.h"
#include "dis_host.h"
#include "dis_internal.cuh"

using dis::Jobs;
using dis::LevelJob;
using dis::PrepJob;
using dis::PyrJob;
using dis::UpJob;

namespace {

thread_local std::string g_err = "no error";

constexpr int kMaxPatch = 16;
constexpr size_t kAlign = 256;

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }
int pitch_of(int w) { return (w + 31) / 32 * 32; }
int level_dim(int d, int s)
{
    for (int i = 0; i < s; ++i) d = (d + 1) / 2;
    return d;
}

// ---- parameters -------------------------------------------------------------------------
struct Resolved {
    int ps, stride, iters, ss, sf, refine, inner, outer_fixed, C;
    float delta, gamma, alpha, omega, scale;
};

bool finite(float v) { return std::isfinite(v); }

// stride = ps - floor(ov * ps) (Alg. 1 step 1: the overlap is floored to whole pixels).  The
// product ov * ps is formed in double from the float parameter, with a 1e-4 guard so that a
// decimal overlap such as 0.7 (0.69999999 in float) floors like its decimal value.
int stride_of(const dis_params& p)
{
    if (p.stride_override > 0) return p.stride_override;
    const int ov = (int)std::floor((double)p.overlap * (double)p.patch_size + 1e-4);
    return std::max(1, p.patch_size - ov);
}

dis_status validate(const dis_params* p, std::string& err)
{
    if (!p) {
        err = "params is NULL";
        return DIS_ERR_INVALID_ARG;
    }
    if (p->struct_size != sizeof(dis_params)) {
        err = "params.struct_size != sizeof(dis_params) (call dis_default_params first)";
        return DIS_ERR_INVALID_ARG;
    }
    if (p->patch_size < 2 || p->patch_size > kMaxPatch) {
        err = "patch_size must be in [2, 16]";
        return DIS_ERR_INVALID_ARG;
    }
    if (!(p->overlap >= 0.0f && p->overlap < 1.0f)) {
        err = "overlap must be in [0, 1)";
        return DIS_ERR_INVALID_ARG;
    }
    if (p->stride_override < 0 || p->grad_iters < 0 || p->grad_iters > (1 << 24) || p->finest_scale < 0 ||
        p->finest_scale > 30 || p->coarsest_scale < -1 || p->coarsest_scale > 30 || p->var_inner < 0 ||
        p->var_inner > (1 << 16) || p->var_outer < -1 || p->var_outer > (1 << 16)) {
        err = "an iteration count, scale or stride is out of range";
        return DIS_ERR_INVALID_ARG;
    }
    if (p->channels != 1 && p->channels != 3) {
        err = "channels must be 1 or 3";
        return DIS_ERR_INVALID_ARG;
    }
    if (!finite(p->delta) || !finite(p->gamma) || !finite(p->alpha) || p->delta < 0 || p->gamma < 0 ||
        p->alpha < 0 || !(p->sor_omega > 0.0f && p->sor_omega < 2.0f) || !finite(p->intensity_scale) ||
        p->intensity_scale <= 0.0f) {
        err = "refinement weights must be finite and >= 0, sor_omega in (0, 2), intensity_scale > 0";
        return DIS_ERR_INVALID_ARG;
    }
    if (p->dof != 1 && p->dof != 2) {
        err = "dof must be 1 (stereo) or 2 (optical flow)";
        return DIS_ERR_INVALID_ARG;
    }
    if (p->norm < 0 || p->norm > 2 || !finite(p->huber_b) || !(p->huber_b > 0.0f)) {
        err = "norm must be 0 (L2), 1 (L1) or 2 (Huber), huber_b finite and > 0";
        return DIS_ERR_INVALID_ARG;
    }
    if (p->fb != 0 && p->fb != 1) {
        err = "fb must be 0 or 1";
        return DIS_ERR_INVALID_ARG;
    }
    if (!finite(p->term_eps) || p->term_eps < 0.0f) {
        err = "term_eps must be finite and >= 0";
        return DIS_ERR_INVALID_ARG;
    }
    if (p->search_grad != 0 && p->search_grad != 1) {
        err = "search_grad must be 0 or 1";
        return DIS_ERR_INVALID_ARG;
    }
    return DIS_OK;
}

// theta_ss = ceil(log2(2 W / (f theta_ps))), f = 8 (Sec. 3.1), lowered until the coarsest
// level holds a patch and raised to theta_sf if below it (Alg. 1 loops from theta_ss down
// to theta_sf); an explicit theta_ss that cannot hold a patch is refused.
dis_status resolve_levels(int W, int H, const dis_params& p, int& ss, int& sf, std::string& err)
{
    const int ps = p.patch_size;
    sf = p.finest_scale;
    ss = p.coarsest_scale;
    if (ss < 0) {
        const double v = 2.0 * (double)W / (8.0 * (double)ps);
        ss = v <= 1.0 ? 0 : (int)std::ceil(std::log2(v));
        while (ss > sf && (level_dim(W, ss) < ps || level_dim(H, ss) < ps)) --ss;
        ss = std::max(ss, sf);
    }
    if (ss < sf || level_dim(W, ss) < ps || level_dim(H, ss) < ps) {
        err = "image too small: the coarsest processed level cannot hold one patch";
        return DIS_ERR_TOO_SMALL;
    }
    return DIS_OK;
}

int grid_n(int L, int ps, int stride) { return L < ps ? 0 : (L - ps + stride - 1) / stride + 1; }

}  // namespace

namespace {

dis_status fail(dis_handle* h, dis_status st, const std::string& msg)
{
    if (h)
        h->err = msg;
    else
        g_err = msg;
    return st;
}

dis_status cuda_fail(dis_handle* h, cudaError_t e, const char* what)
{
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    return fail(h, DIS_ERR_CUDA, m);
}

// ---- plan: job tables of every phase of one call ----------------------------------------
struct PairIn {
    const float* I0;
    const float* I1;
    int w, h;
    long long pitch;
    float* flow;
    const float* init;
    const float* frozen;
    float* record;
    float* ckpt;
    float* flow_b = nullptr;  // forward-backward consistency: the backward flow (nullable)
};

struct Phase {
    enum Kind { PREP, PYR, LEVEL, UP } kind;
    size_t off;  // byte offset of the table in the job blob
    int n;
    long long total, total2, total3;
    int s;
    long long total4 = 0;  // refinement tiles of a LEVEL phase
};

struct Plan {
    std::vector<char> blob;
    std::vector<Phase> phases;
    std::vector<int64_t> key;
    bool graphable = true;
    // checkpoint copies (single pair): per level (dst, src, bytes)
    struct Copy {
        int s;
        void* dst;
        const void* src;
        size_t bytes;
    };
    std::vector<Copy> copies;
};

template <class J>
size_t push_table(std::vector<char>& blob, const std::vector<J>& t)
{
    size_t off = align_up(blob.size(), 16);
    blob.resize(off + sizeof(J) * t.size());
    if (!t.empty()) std::memcpy(blob.data() + off, t.data(), sizeof(J) * t.size());
    return off;
}

dis_status build_plan(dis_handle* hd, const std::vector<PairIn>& pairs, const dis_params& p, Plan& plan)
{
    const int C = p.channels, ps = p.patch_size, stride = stride_of(p);
    const bool refine = p.refine != 0;
    const int n = (int)pairs.size();
    std::vector<int> ss(n), sf(n);
    int max_ss = 0, fsf = p.finest_scale;
    for (int i = 0; i < n; ++i) {
        std::string e;
        dis_status st = resolve_levels(pairs[i].w, pairs[i].h, p, ss[i], sf[i], e);
        if (st != DIS_OK) return fail(hd, st, "pair " + std::to_string(i) + ": " + e);
        if (ss[i] >= hd->levels) return fail(hd, DIS_ERR_INVALID_ARG, "coarsest scale exceeds the handle's pyramid");
        max_ss = std::max(max_ss, ss[i]);
    }
    const bool colour_planes = (C == 3) && refine;
    const int nplanes = colour_planes ? 2 + 2 * C : 2;
    // forward-backward consistency: pair i's backward direction uses slot n + i (its flows,
    // patches and scratch) and reads the forward direction's pyramid with the frames exchanged
    const bool fb = p.fb != 0;
    if (fb) {
        if (2 * n > hd->max_batch)
            return fail(hd, DIS_ERR_INVALID_ARG, "forward-backward consistency takes two pair slots per pair (2 n > max_batch)");
        for (int i = 0; i < n; ++i)
            if (pairs[i].init || pairs[i].frozen || pairs[i].record || pairs[i].ckpt)
                return fail(hd, DIS_ERR_NOT_SUPPORTED,
                            "forward-backward consistency: no initial flow, recorded or frozen increments, checkpoints");
    }
    plan.blob.clear();
    plan.phases.clear();
    plan.copies.clear();
    plan.key.clear();
    plan.graphable = true;
    plan.key.push_back(n);
    const int32_t* pw = reinterpret_cast<const int32_t*>(&p);
    for (size_t i = 0; i < sizeof(dis_params) / 4; ++i) plan.key.push_back(pw[i]);
    plan.key.push_back(hd->search_lanes[p.patch_size]);
    plan.key.push_back(hd->refine_fused);
    plan.key.push_back(hd->refine_split_px);
    plan.key.push_back(hd->probe_kind);
    plan.key.push_back(hd->lc.wq != nullptr);
    plan.key.push_back(hd->probe_level);

    auto slot = [&](int i) { return hd->arena + (size_t)i * hd->slot_bytes; };
    auto img = [&](int i, int s) { return reinterpret_cast<float*>(slot(i) + hd->off_img[s]); };
    auto lw = [&](int i, int s) { return level_dim(pairs[i].w, s); };
    auto lh = [&](int i, int s) { return level_dim(pairs[i].h, s); };
    auto Uof = [&](int i, int s) -> float2* {
        if (s == 0 && sf[i] == 0) return reinterpret_cast<float2*>(pairs[i].flow);
        return reinterpret_cast<float2*>(slot(i) + hd->off_U[s]);
    };
    auto Ubof = [&](int i, int s) -> float2* {  // the backward direction's flows
        if (s == 0 && sf[i] == 0 && pairs[i].flow_b) return reinterpret_cast<float2*>(pairs[i].flow_b);
        return reinterpret_cast<float2*>(slot(n + i) + hd->off_U[s]);
    };

    // level 0 preparation
    {
        std::vector<PrepJob> t(n);
        long long base = 0;
        for (int i = 0; i < n; ++i) {
            PrepJob& J = t[i];
            std::memset(&J, 0, sizeof(J));
            const int w = pairs[i].w, h = pairs[i].h, pit = pitch_of(w);
            J.I0 = pairs[i].I0;
            J.I1 = pairs[i].I1;
            J.in_plane = pairs[i].pitch * (long long)h;
            J.in_pitch = (int)pairs[i].pitch;
            J.S0 = img(i, 0);
            J.S1 = J.S0 + (long long)pit * h;
            J.P0 = colour_planes ? J.S1 + (long long)pit * h : nullptr;
            J.P1 = colour_planes ? J.P0 + (long long)C * pit * h : nullptr;
            J.out_plane = (long long)pit * h;
            J.out_pitch = pit;
            J.w = w;
            J.h = h;
            J.C = C;
            J.scale = p.intensity_scale;
            J.vec = ((reinterpret_cast<uintptr_t>(J.I0) | reinterpret_cast<uintptr_t>(J.I1)) & 15) == 0 &&
                    pairs[i].pitch % 4 == 0;
            J.base = base;
            base += h;
            plan.key.push_back(w);
            plan.key.push_back(h);
            plan.key.push_back(pairs[i].pitch);
            plan.key.push_back((pairs[i].init ? 1 : 0) | (pairs[i].frozen ? 2 : 0) | (pairs[i].record ? 4 : 0) |
                               (pairs[i].flow_b ? 8 : 0));
        }
        plan.phases.push_back({Phase::PREP, push_table(plan.blob, t), n, base, 0, 0, 0});
    }
    // pyramid
    for (int s = 1; s <= max_ss; ++s) {
        std::vector<PyrJob> t;
        long long base = 0;
        for (int i = 0; i < n; ++i) {
            if (ss[i] < s) continue;
            PyrJob J;
            std::memset(&J, 0, sizeof(J));
            J.win = lw(i, s - 1);
            J.hin = lh(i, s - 1);
            J.pin = pitch_of(J.win);
            J.wout = lw(i, s);
            J.hout = lh(i, s);
            J.pout = pitch_of(J.wout);
            J.in = img(i, s - 1);
            J.out = img(i, s);
            J.in_plane = (long long)J.pin * J.hin;
            J.out_plane = (long long)J.pout * J.hout;
            J.nplanes = nplanes;
            t.push_back(J);
        }
        long long u8 = 0, u2 = 0;
        for (const PyrJob& J : t) {
            u8 += dis::pyr_units(J.wout, J.hout, J.nplanes, 8);
            u2 += dis::pyr_units(J.wout, J.hout, J.nplanes, 2);
        }
        const int band = dis::pyr_band(u8, u2, hd->lc.sm_count);
        for (PyrJob& J : t) {
            J.band = band;
            J.base = base;
            base += dis::pyr_units(J.wout, J.hout, J.nplanes, band);
        }
        plan.phases.push_back({Phase::PYR, push_table(plan.blob, t), (int)t.size(), base, 0, 0, s});
    }
    // per-level chain
    for (int s = max_ss; s >= fsf; --s) {
        std::vector<LevelJob> t;
        long long pb = 0, xb = 0, hb = 0, tb = 0;
        for (int i = 0; i < n; ++i) {
            if (ss[i] < s) continue;
            LevelJob J;
            std::memset(&J, 0, sizeof(J));
            const int w = lw(i, s), h = lh(i, s), pit = pitch_of(w);
            J.w = w;
            J.h = h;
            J.pitch = pit;
            J.plane = (long long)pit * h;
            J.S0 = img(i, s);
            J.S1 = J.S0 + J.plane;
            J.P0 = colour_planes ? J.S1 + J.plane : J.S0;
            J.P1 = colour_planes ? J.P0 + (long long)C * J.plane : J.S1;
            J.C = C;
            if (s == ss[i]) {
                J.Uc = reinterpret_cast<const float2*>(pairs[i].init);
                J.wc = w;
                J.hc = h;
                J.cscale = 1.0f;
            } else {
                J.Uc = Uof(i, s + 1);
                J.wc = lw(i, s + 1);
                J.hc = lh(i, s + 1);
                J.cscale = 2.0f;
            }
            J.U = Uof(i, s);
            J.pu = reinterpret_cast<float2*>(slot(i) + hd->off_pu[s]);
            J.pui = nullptr;
            J.pst = nullptr;
            J.nx = grid_n(w, ps, stride);
            J.ny = grid_n(h, ps, stride);
            // increments of earlier (coarser) levels come first in frozen / record
            long long before = 0;
            for (int q = ss[i]; q > s; --q)
                before += (long long)grid_n(lw(i, q), ps, stride) * grid_n(lh(i, q), ps, stride);
            J.frozen = pairs[i].frozen ? reinterpret_cast<const float2*>(pairs[i].frozen) + before : nullptr;
            J.record = pairs[i].record ? reinterpret_cast<float2*>(pairs[i].record) + before : nullptr;
            J.rs = reinterpret_cast<float*>(slot(i) + hd->off_rs);
            // the search planes live in the refinement scratch, which the level's refinement
            // overwrites only after its search (8 of its 15 C + 8 planes)
            J.tpl = reinterpret_cast<const float4*>(J.rs);
            J.tap = J.tpl + J.plane;
            J.patch_base = pb;
            J.pix_base = xb;
            J.half_base = hb;
            dis::set_refine_tiles(J, tb);
            J.partner = -1;
            pb += (long long)J.nx * J.ny;
            xb += (long long)w * h;
            hb += (long long)h * ((w + 1) / 2);
            if (fb) {
                // the lists of this direction's tiles, in its refinement scratch (free between
                // the search and the refinement)
                const long long tiles = dis::refine_tiles(w, h);
                J.fb_cnt = reinterpret_cast<int*>(J.rs);
                J.fb_cur = J.fb_cnt + tiles;
                J.fb_list = J.fb_cur + tiles;
                LevelJob B = J;
                B.S0 = J.S1;
                B.S1 = J.S0;
                B.P0 = J.P1;
                B.P1 = J.P0;
                if (s == ss[i]) {
                    B.Uc = nullptr;
                } else {
                    B.Uc = Ubof(i, s + 1);
                }
                B.U = Ubof(i, s);
                B.pu = reinterpret_cast<float2*>(slot(n + i) + hd->off_pu[s]);
                B.rs = reinterpret_cast<float*>(slot(n + i) + hd->off_rs);
                B.tpl = reinterpret_cast<const float4*>(B.rs);
                B.tap = B.tpl + B.plane;
                B.fb_cnt = reinterpret_cast<int*>(B.rs);
                B.fb_cur = B.fb_cnt + tiles;
                B.fb_list = B.fb_cur + tiles;
                B.patch_base = pb;
                B.pix_base = xb;
                B.half_base = hb;
                dis::set_refine_tiles(B, tb);
                pb += (long long)B.nx * B.ny;
                xb += (long long)w * h;
                hb += (long long)h * ((w + 1) / 2);
                J.partner = (int)t.size() + 1;
                B.partner = (int)t.size();
                t.push_back(J);
                t.push_back(B);
                continue;
            }
            t.push_back(J);
            if (pairs[i].ckpt) {
                long long cb = 0;
                for (int q = ss[i]; q > s; --q) cb += (long long)lw(i, q) * lh(i, q) * 2;
                plan.copies.push_back({s, pairs[i].ckpt + cb, J.U, sizeof(float2) * (size_t)w * h});
                plan.graphable = false;
            }
        }
        plan.phases.push_back({Phase::LEVEL, push_table(plan.blob, t), (int)t.size(), pb, xb, hb, s, tb});
    }
    // final up-scaling
    if (fsf > 0) {
        std::vector<UpJob> t(n);
        long long base = 0;
        for (int i = 0; i < n; ++i) {
            UpJob& J = t[i];
            std::memset(&J, 0, sizeof(J));
            J.in = Uof(i, fsf);
            J.wi = lw(i, fsf);
            J.hi = lh(i, fsf);
            J.out = reinterpret_cast<float2*>(pairs[i].flow);
            J.wo = pairs[i].w;
            J.ho = pairs[i].h;
            J.factor = (float)(1 << fsf);
            J.base = base;
            base += J.ho;
        }
        for (int i = 0; fb && i < n; ++i) {
            if (!pairs[i].flow_b) continue;
            UpJob J;
            std::memset(&J, 0, sizeof(J));
            J.in = Ubof(i, fsf);
            J.wi = lw(i, fsf);
            J.hi = lh(i, fsf);
            J.out = reinterpret_cast<float2*>(pairs[i].flow_b);
            J.wo = pairs[i].w;
            J.ho = pairs[i].h;
            J.factor = (float)(1 << fsf);
            J.base = base;
            base += J.ho;
            t.push_back(J);
        }
        plan.phases.push_back({Phase::UP, push_table(plan.blob, t), (int)t.size(), base, 0, 0, fsf});
    }
    if (plan.blob.size() > hd->jobs_bytes) return fail(hd, DIS_ERR_INVALID_ARG, "job tables exceed the handle's job region");
    return DIS_OK;
}

// One traced launcher call: events on both sides of it on the launching stream.
struct TraceRec {
    int kind, level;
    cudaEvent_t a, b;
};

cudaError_t record_plan(dis_handle* hd, const Plan& plan, const dis_params& p, cudaStream_t s,
                        std::vector<TraceRec>* tr = nullptr)
{
    const int ps = p.patch_size, stride = stride_of(p);
    cudaError_t e = cudaSuccess;
    // runs one launcher call, bracketed by events when tracing
    auto traced = [&](int kind, int level, auto&& launch) -> cudaError_t {
        if (!tr && kind == hd->probe_kind && level == hd->probe_level) {
            // external event nodes when captured into a graph, plain records otherwise
            cudaError_t ce = cudaEventRecordWithFlags(hd->probe_a, s, cudaEventRecordExternal);
            if (ce == cudaSuccess) ce = launch();
            if (ce == cudaSuccess) ce = cudaEventRecordWithFlags(hd->probe_b, s, cudaEventRecordExternal);
            if (ce == cudaSuccess) hd->probe_armed = true;
            return ce;
        }
        if (!tr) return launch();
        TraceRec r{kind, level, nullptr, nullptr};
        cudaError_t ce = cudaEventCreate(&r.a);
        if (ce == cudaSuccess) ce = cudaEventCreate(&r.b);
        if (ce == cudaSuccess) ce = cudaEventRecord(r.a, s);
        if (ce == cudaSuccess) ce = launch();
        if (ce == cudaSuccess) ce = cudaEventRecord(r.b, s);
        tr->push_back(r);
        return ce;
    };
    for (const Phase& ph : plan.phases) {
        const char* tab = hd->jobs_cur + ph.off;
        switch (ph.kind) {
            case Phase::PREP:
                e = traced(DIS_LAUNCH_PREP, 0, [&] {
                    return dis::launch_prep(dis::device_jobs(reinterpret_cast<const PrepJob*>(tab), ph.n), ph.total,
                                            hd->lc, s);
                });
                break;
            case Phase::PYR:
                e = traced(DIS_LAUNCH_PYRAMID, ph.s, [&] {
                    return dis::launch_pyr_down(dis::device_jobs(reinterpret_cast<const PyrJob*>(tab), ph.n), ph.total,
                                                hd->lc, s);
                });
                break;
            case Phase::LEVEL: {
                auto js = dis::device_jobs(reinterpret_cast<const LevelJob*>(tab), ph.n);
                const int lanes = hd->search_lanes[ps];
                if (lanes == 1 && p.dof == 2 && p.norm == 0 && p.term_eps == 0.0f)
                    e = traced(DIS_LAUNCH_SEARCH_PLANES, ph.s,
                               [&] { return dis::launch_search_planes(js, ph.total2, hd->lc, s); });
                if (e == cudaSuccess)
                    e = traced(DIS_LAUNCH_SEARCH, ph.s, [&] {
                        if (p.dof != 2 || p.norm != 0 || p.term_eps > 0.0f)
                            return dis::launch_search_mode(js, ph.total, ps, stride, p.grad_iters, p.dof, p.norm,
                                                           p.huber_b, p.term_eps, lanes, hd->lc, s);
                        return dis::launch_search(js, ph.total, ps, stride, p.grad_iters, hd->lc, s, lanes, lanes == 1);
                    });
                if (e == cudaSuccess)
                    e = traced(DIS_LAUNCH_DENSIFY, ph.s, [&] {
                        if (p.fb)
                            return dis::launch_densify_fb(js, ph.total, ph.total4, ph.n, ps, stride, hd->lc, s);
                        return dis::launch_densify(js, ph.total2, ph.total4, ps, stride, hd->lc, s);
                    });
                for (const auto& c : plan.copies)
                    if (e == cudaSuccess && c.s == ph.s) e = cudaMemcpyAsync(c.dst, c.src, c.bytes, cudaMemcpyDeviceToDevice, s);
                if (e == cudaSuccess && p.refine) {
                    dis::RefineArgs a;
                    a.outer = p.var_outer < 0 ? ph.s + 1 : p.var_outer;
                    a.inner = p.var_inner;
                    a.delta = p.delta;
                    a.gamma = p.gamma;
                    a.alpha = p.alpha;
                    a.omega = p.sor_omega;
                    a.fused = hd->refine_fused;
                    a.split_px = hd->refine_split_px;
                    a.C = p.channels;
                    a.dof = p.dof;
                    e = traced(DIS_LAUNCH_REFINE, ph.s,
                               [&] { return dis::launch_refine(js, ph.total2, ph.total3, ph.total4, a, hd->lc, s); });
                }
                break;
            }
            case Phase::UP:
                e = traced(DIS_LAUNCH_UPSAMPLE, ph.s, [&] {
                    return dis::launch_upsample(dis::device_jobs(reinterpret_cast<const UpJob*>(tab), ph.n), ph.total,
                                                hd->lc, s);
                });
                break;
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Stream-ordered upload of the job tables when they changed (from a pinned buffer whose
// previous copy has completed).
dis_status upload_jobs(dis_handle* hd, const Plan& plan, cudaStream_t s)
{
    cudaError_t e;
    int slot = -1;
    for (int k = 0; k < dis_handle::kJobSlots && slot < 0; ++k)
        if (hd->jobs_ok[k] && hd->jobs_blob[k] == plan.blob) slot = k;
    if (slot >= 0) {
        // resident: a call on another stream than the upload's waits for that upload
        if (hd->jobs_stream[slot] != s && (e = cudaStreamWaitEvent(s, hd->jobs_ev[slot], 0)) != cudaSuccess)
            return cuda_fail(hd, e, "job table wait");
    } else {
        slot = 0;  // replace the least recently used table
        for (int k = 1; k < dis_handle::kJobSlots; ++k)
            if (hd->jobs_stamp[k] < hd->jobs_stamp[slot]) slot = k;
        char* pin = hd->jobs_pinned + (size_t)slot * hd->jobs_bytes;
        if ((e = cudaEventSynchronize(hd->jobs_ev[slot])) != cudaSuccess) return cuda_fail(hd, e, "job upload wait");
        std::memcpy(pin, plan.blob.data(), plan.blob.size());
        if ((e = cudaMemcpyAsync(hd->jobs_dev + (size_t)slot * hd->jobs_bytes, pin, plan.blob.size(),
                                 cudaMemcpyHostToDevice, s)) != cudaSuccess)
            return cuda_fail(hd, e, "job upload");
        if ((e = cudaEventRecord(hd->jobs_ev[slot], s)) != cudaSuccess) return cuda_fail(hd, e, "job upload event");
        hd->jobs_blob[slot] = plan.blob;
        hd->jobs_ok[slot] = true;
        hd->jobs_stream[slot] = s;
    }
    hd->jobs_stamp[slot] = ++hd->jobs_clock;
    hd->jobs_slot = slot;
    hd->jobs_cur = hd->jobs_dev + (size_t)slot * hd->jobs_bytes;
    return DIS_OK;
}

}  // namespace

// The kernel nodes of a captured graph: the kernels every replay of it launches.
int dis_host::graph_kernel_nodes(cudaGraph_t graph)
{
    size_t nn = 0;
    int kernels = 0;
    if (cudaGraphGetNodes(graph, nullptr, &nn) == cudaSuccess && nn > 0) {
        std::vector<cudaGraphNode_t> nodes(nn);
        if (cudaGraphGetNodes(graph, nodes.data(), &nn) == cudaSuccess)
            for (size_t k = 0; k < nn; ++k) {
                cudaGraphNodeType ty;
                if (cudaGraphNodeGetType(nodes[k], &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++kernels;
            }
    }
    return kernels;
}

namespace {

dis_status run_plan(dis_handle* hd, const Plan& plan, const dis_params& p, cudaStream_t s)
{
    cudaError_t e;
    dis_status ust = upload_jobs(hd, plan, s);
    if (ust != DIS_OK) return ust;
    if (!hd->use_graphs || !plan.graphable) {
        hd->last_kernels = -1;
        if ((e = record_plan(hd, plan, p, s)) != cudaSuccess) return cuda_fail(hd, e, "kernel launch");
        return DIS_OK;
    }
    cudaGraphExec_t exec = nullptr;
    int kernels = -1;
    // a graph's kernels read the job table of one slot
    std::vector<int64_t> key = plan.key;
    key.push_back(hd->jobs_slot);
    for (auto& g : hd->graphs)
        if (g.key == key) {
            exec = g.exec;
            kernels = g.kernels;
        }
    if (!exec) {
        cudaGraph_t graph = nullptr;
        if ((e = cudaStreamBeginCapture(hd->cap_stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
            return cuda_fail(hd, e, "graph capture begin");
        cudaError_t le = record_plan(hd, plan, p, hd->cap_stream);
        e = cudaStreamEndCapture(hd->cap_stream, &graph);
        if (le != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return cuda_fail(hd, le, "kernel launch (capture)");
        }
        if (e != cudaSuccess) return cuda_fail(hd, e, "graph capture end");
        kernels = dis_host::graph_kernel_nodes(graph);
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(hd, e, "graph instantiate");
        if (hd->graphs.size() >= 8) {
            cudaGraphExecDestroy(hd->graphs.front().exec);
            hd->graphs.erase(hd->graphs.begin());
        }
        hd->graphs.push_back({key, exec, kernels});
    }
    if ((e = cudaGraphLaunch(exec, s)) != cudaSuccess) return cuda_fail(hd, e, "graph launch");
    hd->last_kernels = kernels;
    return DIS_OK;
}

dis_status check_pair(dis_handle* hd, const PairIn& q, int idx)
{
    const std::string tag = "pair " + std::to_string(idx) + ": ";
    if (!q.I0 || !q.I1 || !q.flow) return fail(hd, DIS_ERR_INVALID_ARG, tag + "null image or flow pointer");
    if (q.w < 1 || q.h < 1 || q.w > hd->max_w || q.h > hd->max_h)
        return fail(hd, DIS_ERR_INVALID_ARG, tag + "size outside [1, handle max]");
    if (q.pitch < q.w || q.pitch > (1LL << 30)) return fail(hd, DIS_ERR_INVALID_ARG, tag + "pitch < width");
    return DIS_OK;
}

}  // namespace

// ---- C ABI ------------------------------------------------------------------------------
extern "C" {

void dis_default_params(dis_params* p, int preset)
{
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->struct_size = sizeof(dis_params);
    p->patch_size = 8;
    p->overlap = 0.3f;
    p->stride_override = 0;
    p->grad_iters = 16;
    p->coarsest_scale = -1;
    p->finest_scale = 0;
    p->refine = 1;
    p->var_outer = -1;
    p->var_inner = 5;
    p->delta = 5.0f;
    p->gamma = 10.0f;
    p->alpha = 10.0f;
    p->sor_omega = 1.6f;
    p->intensity_scale = 255.0f;
    p->channels = 1;
    p->dof = 2;
    p->norm = 0;
    p->huber_b = 5.0f;
    int stereo = 0;
    if (preset >= DIS_PRESET_STEREO_OP1 && preset <= DIS_PRESET_STEREO_DENSE) {
        stereo = 1;
        preset = preset == DIS_PRESET_STEREO_DENSE ? DIS_PRESET_DENSE : preset - DIS_PRESET_STEREO_OP1 + DIS_PRESET_OP1;
    }
    switch (preset) {
        case DIS_PRESET_OP1: p->finest_scale = 3; p->grad_iters = 16; p->patch_size = 8; p->overlap = 0.30f; p->refine = 0; break;
        case DIS_PRESET_OP2: p->finest_scale = 3; p->grad_iters = 12; p->patch_size = 8; p->overlap = 0.40f; break;
        case DIS_PRESET_OP3: p->finest_scale = 1; p->grad_iters = 16; p->patch_size = 12; p->overlap = 0.75f; break;
        case DIS_PRESET_OP4: p->finest_scale = 0; p->grad_iters = 256; p->patch_size = 12; p->overlap = 0.75f; break;
        case DIS_PRESET_FAST: p->finest_scale = 2; p->grad_iters = 16; p->patch_size = 8; p->overlap = 0.30f; p->refine = 0; break;
        case DIS_PRESET_MEDIUM: p->finest_scale = 0; p->grad_iters = 32; p->patch_size = 8; p->overlap = 0.50f; break;
        case DIS_PRESET_DENSE: p->finest_scale = 0; p->grad_iters = 128; p->patch_size = 12; p->overlap = 0.75f; break;
        default: break;
    }
    if (stereo) {  // supplementary, depth from stereo: the same operating points, theta_it halved
        p->dof = 1;
        p->grad_iters /= 2;
    }
}

dis_status dis_levels(int width, int height, const dis_params* p, int* coarsest, int* finest, int64_t* total_patches)
{
    std::string e;
    dis_status st = validate(p, e);
    if (st != DIS_OK) return fail(nullptr, st, e);
    if (width < 1 || height < 1) return fail(nullptr, DIS_ERR_INVALID_ARG, "size must be positive");
    int ss, sf;
    if ((st = resolve_levels(width, height, *p, ss, sf, e)) != DIS_OK) return fail(nullptr, st, e);
    const int stride = stride_of(*p);
    int64_t tot = 0;
    for (int s = ss; s >= sf; --s)
        tot += (int64_t)grid_n(level_dim(width, s), p->patch_size, stride) *
               grid_n(level_dim(height, s), p->patch_size, stride);
    if (coarsest) *coarsest = ss;
    if (finest) *finest = sf;
    if (total_patches) *total_patches = tot;
    return DIS_OK;
}

dis_status dis_create(dis_handle** out, int max_w, int max_h, int max_batch, int channels)
{
    if (!out) return fail(nullptr, DIS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    // the kernels index a pair's pixels (and up to 8 planes of a level-1 image) with 32-bit
    // integers: at most 2^30 pixels per frame
    if (max_w < 1 || max_h < 1 || max_batch < 1 || (channels != 1 && channels != 3) || max_w > (1 << 16) ||
        max_h > (1 << 16) || max_batch > 4096 || (long long)max_w * max_h > (1LL << 30))
        return fail(nullptr, DIS_ERR_INVALID_ARG, "invalid handle size");
    dis_handle* h = new dis_handle();
    h->max_w = max_w;
    h->max_h = max_h;
    h->max_batch = max_batch;
    h->C = channels;
    cudaGetDevice(&h->device);
    // pyramid depth: until both dimensions are 1
    int L = 1;
    for (int w = max_w, hh = max_h; w > 1 || hh > 1; w = (w + 1) / 2, hh = (hh + 1) / 2) ++L;
    h->levels = L;
    const int nplanes = channels == 3 ? 2 + 2 * channels : 2;
    size_t off = 0;
    for (int s = 0; s < L; ++s) {
        const size_t w = level_dim(max_w, s), hh = level_dim(max_h, s), pit = pitch_of((int)w);
        h->off_img.push_back(off);
        off = align_up(off + sizeof(float) * nplanes * pit * hh, kAlign);
        h->off_U.push_back(off);
        off = align_up(off + sizeof(float) * 2 * w * hh, kAlign);
        h->off_pu.push_back(off);
        off = align_up(off + sizeof(float) * 2 * w * hh, kAlign);
        h->off_pui.push_back(off);
        off = align_up(off + sizeof(float) * 2 * w * hh, kAlign);
        h->off_pst.push_back(off);
        off = align_up(off + sizeof(int) * w * hh, kAlign);
    }
    h->off_rs = off;
    h->rs_floats = (size_t)dis::rs_planes(channels) * pitch_of(max_w) * max_h;
    off = align_up(off + sizeof(float) * h->rs_floats, kAlign);
    h->slot_bytes = off;
    h->jobs_bytes = align_up((size_t)max_batch * (4 + 2 * L) * 256 + 4096, kAlign);
    h->arena_bytes = h->slot_bytes * max_batch + dis_handle::kJobSlots * h->jobs_bytes + kAlign;  // + the work queue
    cudaError_t e = cudaMalloc(&h->arena, h->arena_bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return fail(nullptr, DIS_ERR_OUT_OF_MEMORY, std::string("arena allocation failed: ") + cudaGetErrorString(e));
    }
    h->jobs_dev = h->arena + h->slot_bytes * max_batch;
    unsigned int* wq = (unsigned int*)(h->jobs_dev + dis_handle::kJobSlots * h->jobs_bytes);
    // zeroed before dis_create returns: the caller's stream may be one that does not wait for
    // the legacy default stream, on which cudaMemset runs
    if ((e = cudaMemset(wq, 0, 2 * sizeof(unsigned int))) != cudaSuccess ||
        (e = cudaStreamSynchronize(nullptr)) != cudaSuccess) {
        cudaGetLastError();
        dis_destroy(h);
        return fail(nullptr, DIS_ERR_CUDA, std::string("handle setup failed: ") + cudaGetErrorString(e));
    }
    e = cudaMallocHost(&h->jobs_pinned, dis_handle::kJobSlots * h->jobs_bytes);
    for (int k = 0; k < dis_handle::kJobSlots && e == cudaSuccess; ++k)
        e = cudaEventCreateWithFlags(&h->jobs_ev[k], cudaEventDisableTiming);
    if (e != cudaSuccess || (e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking)) != cudaSuccess) {
        dis_destroy(h);
        return fail(nullptr, DIS_ERR_CUDA, std::string("handle setup failed: ") + cudaGetErrorString(e));
    }
    for (int k = 0; k < dis_handle::kJobSlots; ++k) cudaEventRecord(h->jobs_ev[k], h->cap_stream);
    h->lc = dis::query_launch_cfg();
    h->lc.wq = h->wq = wq;
    const char* ng = std::getenv("DIS_NO_GRAPH");
    h->use_graphs = !(ng && ng[0] == '1');
    *out = h;
    return DIS_OK;
}

void dis_destroy(dis_handle* h)
{
    if (!h) return;
    if (h->cap_stream) cudaStreamSynchronize(h->cap_stream);
    for (int k = 0; k < dis_handle::kJobSlots; ++k)
        if (h->jobs_ev[k]) cudaEventSynchronize(h->jobs_ev[k]);
    for (auto& g : h->graphs) cudaGraphExecDestroy(g.exec);
    for (auto& g : h->bwd_graphs) cudaGraphExecDestroy(g.exec);
    if (h->probe_a) cudaEventDestroy(h->probe_a);
    if (h->probe_b) cudaEventDestroy(h->probe_b);
    if (h->hs.cs_in) cudaStreamSynchronize(h->hs.cs_in);
    if (h->hs.cs_out) cudaStreamSynchronize(h->hs.cs_out);
    for (int b = 0; b < 2; ++b) {
        if (h->hs.ev_in[b]) cudaEventDestroy(h->hs.ev_in[b]);
        if (h->hs.ev_out[b]) cudaEventDestroy(h->hs.ev_out[b]);
        if (h->hs.ev_done[b]) cudaEventDestroy(h->hs.ev_done[b]);
    }
    if (h->hs.buf) cudaFree(h->hs.buf);
    if (h->hs.cs_in) cudaStreamDestroy(h->hs.cs_in);
    if (h->hs.cs_out) cudaStreamDestroy(h->hs.cs_out);
    if (h->arena) cudaFree(h->arena);
    if (h->jobs_pinned) cudaFreeHost(h->jobs_pinned);
    for (int k = 0; k < dis_handle::kJobSlots; ++k)
        if (h->jobs_ev[k]) cudaEventDestroy(h->jobs_ev[k]);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    delete h;
}

const char* dis_last_error_string(const dis_handle* h) { return h ? h->err.c_str() : g_err.c_str(); }

int64_t dis_arena_bytes(const dis_handle* h) { return h ? (int64_t)h->arena_bytes : 0; }

dis_status dis_compute_flow_ex(dis_handle* hd, const float* I0, const float* I1, int w, int hgt, int64_t pitch,
                               const dis_params* p, const float* init_flow, const float* frozen_in,
                               float* record_out, float* checkpoints, float* flow_out, void* stream)
{
    if (!hd) return fail(nullptr, DIS_ERR_INVALID_ARG, "handle is NULL");
    std::string e;
    dis_status st = validate(p, e);
    if (st != DIS_OK) return fail(hd, st, e);
    if (p->channels != hd->C) return fail(hd, DIS_ERR_INVALID_ARG, "params.channels differs from the handle's");
    PairIn q{I0, I1, w, hgt, pitch, flow_out, init_flow, frozen_in, record_out, checkpoints};
    if ((st = check_pair(hd, q, 0)) != DIS_OK) return st;
    Plan plan;
    if ((st = build_plan(hd, {q}, *p, plan)) != DIS_OK) return st;
    return run_plan(hd, plan, *p, (cudaStream_t)stream);
}

dis_status dis_compute_flow(dis_handle* hd, const float* I0, const float* I1, int w, int hgt, int64_t pitch,
                            const dis_params* p, float* flow_out, void* stream)
{
    return dis_compute_flow_ex(hd, I0, I1, w, hgt, pitch, p, nullptr, nullptr, nullptr, nullptr, flow_out, stream);
}

dis_status dis_compute_flow_fb(dis_handle* hd, const float* I0, const float* I1, int w, int hgt, int64_t pitch,
                               const dis_params* p, float* flow_out, float* flow_b_out, void* stream)
{
    if (!hd) return fail(nullptr, DIS_ERR_INVALID_ARG, "handle is NULL");
    std::string e;
    dis_status st = validate(p, e);
    if (st != DIS_OK) return fail(hd, st, e);
    if (p->channels != hd->C) return fail(hd, DIS_ERR_INVALID_ARG, "params.channels differs from the handle's");
    dis_params q = *p;
    q.fb = 1;
    PairIn in{I0, I1, w, hgt, pitch, flow_out, nullptr, nullptr, nullptr, nullptr, flow_b_out};
    if ((st = check_pair(hd, in, 0)) != DIS_OK) return st;
    Plan plan;
    if ((st = build_plan(hd, {in}, q, plan)) != DIS_OK) return st;
    return run_plan(hd, plan, q, (cudaStream_t)stream);
}

dis_status dis_compute_flow_batched(dis_handle* hd, const dis_pair* pairs, int n, const dis_params* p, void* stream)
{
    if (!hd) return fail(nullptr, DIS_ERR_INVALID_ARG, "handle is NULL");
    std::string e;
    dis_status st = validate(p, e);
    if (st != DIS_OK) return fail(hd, st, e);
    if (p->channels != hd->C) return fail(hd, DIS_ERR_INVALID_ARG, "params.channels differs from the handle's");
    if (!pairs || n < 1 || n > hd->max_batch) return fail(hd, DIS_ERR_INVALID_ARG, "pairs NULL or n outside [1, max_batch]");
    std::vector<PairIn> v;
    v.reserve(n);
    for (int i = 0; i < n; ++i) {
        PairIn q{pairs[i].I0, pairs[i].I1, pairs[i].width, pairs[i].height, (long long)pairs[i].pitch,
                 pairs[i].flow_out, nullptr, nullptr, nullptr, nullptr};
        if ((st = check_pair(hd, q, i)) != DIS_OK) return st;
        v.push_back(q);
    }
    Plan plan;
    if ((st = build_plan(hd, v, *p, plan)) != DIS_OK) return st;
    return run_plan(hd, plan, *p, (cudaStream_t)stream);
}

dis_status dis_compute_flow_batched_host(dis_handle* hd, const dis_pair* pairs, int n, const dis_params* p,
                                        void* stream)
{
    if (!hd) return fail(nullptr, DIS_ERR_INVALID_ARG, "handle is NULL");
    std::string e;
    dis_status st = validate(p, e);
    if (st != DIS_OK) return fail(hd, st, e);
    if (p->channels != hd->C) return fail(hd, DIS_ERR_INVALID_ARG, "params.channels differs from the handle's");
    if (!pairs || n < 1 || n > hd->max_batch) return fail(hd, DIS_ERR_INVALID_ARG, "pairs NULL or n outside [1, max_batch]");
    const int C = p->channels;
    // staging layout of one half: per pair I0, I1 (C planes of pitch x height) and the flow
    std::vector<size_t> off_in(n), off_out(n);
    size_t half = 0;
    for (int i = 0; i < n; ++i) {
        PairIn q{pairs[i].I0, pairs[i].I1, pairs[i].width, pairs[i].height, (long long)pairs[i].pitch,
                 pairs[i].flow_out, nullptr, nullptr, nullptr, nullptr};
        if ((st = check_pair(hd, q, i)) != DIS_OK) return st;
        off_in[i] = half;
        half = align_up(half + 2 * sizeof(float) * (size_t)C * q.pitch * q.h, kAlign);
        off_out[i] = half;
        half = align_up(half + sizeof(float) * 2 * (size_t)q.w * q.h, kAlign);
    }
    cudaStream_t s = (cudaStream_t)stream;
    auto& H = hd->hs;
    cudaError_t ce = cudaSuccess;
    if (!H.cs_in) {
        ce = cudaStreamCreateWithFlags(&H.cs_in, cudaStreamNonBlocking);
        if (ce == cudaSuccess) ce = cudaStreamCreateWithFlags(&H.cs_out, cudaStreamNonBlocking);
        for (int b = 0; b < 2 && ce == cudaSuccess; ++b) {
            ce = cudaEventCreateWithFlags(&H.ev_in[b], cudaEventDisableTiming);
            if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&H.ev_out[b], cudaEventDisableTiming);
            if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&H.ev_done[b], cudaEventDisableTiming);
        }
        if (ce != cudaSuccess) return cuda_fail(hd, ce, "host staging setup");
    }
    if (half > H.half_bytes) {
        // grow: every earlier call must be done with the old staging
        if ((ce = cudaStreamSynchronize(H.cs_in)) != cudaSuccess || (ce = cudaStreamSynchronize(H.cs_out)) != cudaSuccess ||
            (ce = cudaStreamSynchronize(s)) != cudaSuccess)
            return cuda_fail(hd, ce, "host staging wait");
        if (H.buf) cudaFree(H.buf);
        H.buf = nullptr;
        H.half_bytes = 0;
        H.used[0] = H.used[1] = false;
        if ((ce = cudaMalloc(&H.buf, 2 * half)) != cudaSuccess) {
            H.buf = nullptr;
            return fail(hd, DIS_ERR_OUT_OF_MEMORY, "host staging allocation failed");
        }
        H.half_bytes = half;
    }
    const int b = H.next;
    char* base = H.buf + (size_t)b * H.half_bytes;
    // frames in, once the previous computation on this half has read its frames
    if (H.used[b]) ce = cudaStreamWaitEvent(H.cs_in, H.ev_out[b], 0);
    std::vector<dis_pair> dev(n);
    for (int i = 0; i < n && ce == cudaSuccess; ++i) {
        const size_t frame = sizeof(float) * (size_t)C * pairs[i].pitch * pairs[i].height;
        float* d0 = reinterpret_cast<float*>(base + off_in[i]);
        float* d1 = reinterpret_cast<float*>(base + off_in[i] + frame);
        ce = cudaMemcpyAsync(d0, pairs[i].I0, frame, cudaMemcpyHostToDevice, H.cs_in);
        if (ce == cudaSuccess) ce = cudaMemcpyAsync(d1, pairs[i].I1, frame, cudaMemcpyHostToDevice, H.cs_in);
        dev[i] = pairs[i];
        dev[i].I0 = d0;
        dev[i].I1 = d1;
        dev[i].flow_out = reinterpret_cast<float*>(base + off_out[i]);
    }
    if (ce == cudaSuccess) ce = cudaEventRecord(H.ev_in[b], H.cs_in);
    // compute once the frames are in and the previous flows of this half are out
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(s, H.ev_in[b], 0);
    if (ce == cudaSuccess && H.used[b]) ce = cudaStreamWaitEvent(s, H.ev_done[b], 0);
    if (ce != cudaSuccess) return cuda_fail(hd, ce, "host frames copy");
    if ((st = dis_compute_flow_batched(hd, dev.data(), n, p, stream)) != DIS_OK) return st;
    // flows out once computed
    ce = cudaEventRecord(H.ev_out[b], s);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(H.cs_out, H.ev_out[b], 0);
    for (int i = 0; i < n && ce == cudaSuccess; ++i)
        ce = cudaMemcpyAsync(pairs[i].flow_out, dev[i].flow_out, sizeof(float) * 2 * (size_t)pairs[i].width * pairs[i].height,
                             cudaMemcpyDeviceToHost, H.cs_out);
    if (ce == cudaSuccess) ce = cudaEventRecord(H.ev_done[b], H.cs_out);
    if (ce != cudaSuccess) return cuda_fail(hd, ce, "host flows copy");
    H.used[b] = true;
    H.last = b;
    H.next = b ^ 1;
    return DIS_OK;
}

dis_status dis_host_flows_ready(dis_handle* hd, void* stream)
{
    if (!hd) return fail(nullptr, DIS_ERR_INVALID_ARG, "handle is NULL");
    if (hd->hs.last < 0) return DIS_OK;
    cudaError_t ce = cudaStreamWaitEvent((cudaStream_t)stream, hd->hs.ev_done[hd->hs.last], 0);
    return ce == cudaSuccess ? DIS_OK : cuda_fail(hd, ce, "dis_host_flows_ready");
}

dis_status dis_trace_batched(dis_handle* hd, const dis_pair* pairs, int n, const dis_params* p, void* stream,
                             dis_launch_record* out, int cap, int* count)
{
    if (!hd) return fail(nullptr, DIS_ERR_INVALID_ARG, "handle is NULL");
    if (count) *count = 0;
    std::string e;
    dis_status st = validate(p, e);
    if (st != DIS_OK) return fail(hd, st, e);
    if (p->channels != hd->C) return fail(hd, DIS_ERR_INVALID_ARG, "params.channels differs from the handle's");
    if (!pairs || n < 1 || n > hd->max_batch) return fail(hd, DIS_ERR_INVALID_ARG, "pairs NULL or n outside [1, max_batch]");
    if (cap < 0 || (cap > 0 && !out)) return fail(hd, DIS_ERR_INVALID_ARG, "out NULL with cap > 0");
    std::vector<PairIn> v;
    for (int i = 0; i < n; ++i) {
        PairIn q{pairs[i].I0, pairs[i].I1, pairs[i].width, pairs[i].height, (long long)pairs[i].pitch,
                 pairs[i].flow_out, nullptr, nullptr, nullptr, nullptr};
        if ((st = check_pair(hd, q, i)) != DIS_OK) return st;
        v.push_back(q);
    }
    Plan plan;
    if ((st = build_plan(hd, v, *p, plan)) != DIS_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = upload_jobs(hd, plan, s)) != DIS_OK) return st;
    std::vector<TraceRec> tr;
    cudaError_t ce = record_plan(hd, plan, *p, s, &tr);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    int k = 0;
    for (const TraceRec& r : tr) {
        float ms = 0.0f;
        if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, r.a, r.b);
        if (k < cap) out[k] = dis_launch_record{r.kind, r.level, ms};
        ++k;
        if (r.a) cudaEventDestroy(r.a);
        if (r.b) cudaEventDestroy(r.b);
    }
    if (ce != cudaSuccess) return cuda_fail(hd, ce, "dis_trace_batched");
    if (count) *count = k;
    return DIS_OK;
}

dis_status dis_set_refine_fusion(dis_handle* hd, int fused)
{
    if (!hd) return fail(nullptr, DIS_ERR_INVALID_ARG, "handle is NULL");
    if (fused < 0 || fused > 3) return fail(hd, DIS_ERR_INVALID_ARG, "dis_set_refine_fusion: mode must be 0 to 3");
    hd->refine_fused = fused;
    return DIS_OK;
}

dis_status dis_set_refine_split(dis_handle* hd, int64_t pixels)
{
    if (!hd) return fail(nullptr, DIS_ERR_INVALID_ARG, "handle is NULL");
    hd->refine_split_px = pixels < 0 ? dis::kRefineSplitNever : std::min<long long>(pixels, dis::kRefineSplitNever);
    return DIS_OK;
}

dis_status dis_get_refine_split(const dis_handle* hd, int64_t* pixels)
{
    if (!hd || !pixels) return fail(const_cast<dis_handle*>(hd), DIS_ERR_INVALID_ARG, "dis_get_refine_split: NULL argument");
    *pixels = hd->refine_split_px >= dis::kRefineSplitNever ? -1 : hd->refine_split_px;
    return DIS_OK;
}

dis_status dis_set_work_queue(dis_handle* hd, int on)
{
    if (!hd) return fail(nullptr, DIS_ERR_INVALID_ARG, "handle is NULL");
    if (on != 0 && on != 1) return fail(hd, DIS_ERR_INVALID_ARG, "dis_set_work_queue: on must be 0 or 1");
    hd->lc.wq = on ? hd->wq : nullptr;
    return DIS_OK;
}

dis_status dis_set_probe(dis_handle* hd, int kind, int level)
{
    if (!hd) return fail(nullptr, DIS_ERR_INVALID_ARG, "handle is NULL");
    if (kind > DIS_LAUNCH_UPSAMPLE || level < 0) return fail(hd, DIS_ERR_INVALID_ARG, "dis_set_probe: bad kind or level");
    if (kind >= 0 && !hd->probe_a) {
        cudaError_t e = cudaEventCreate(&hd->probe_a);
        if (e == cudaSuccess) e = cudaEventCreate(&hd->probe_b);
        if (e != cudaSuccess) return cuda_fail(hd, e, "dis_set_probe");
    }
    hd->probe_kind = kind < 0 ? -1 : kind;
    hd->probe_level = level;
    hd->probe_armed = false;
    return DIS_OK;
}

dis_status dis_probe_ms(dis_handle* hd, float* ms)
{
    if (!hd || !ms) return fail(hd, DIS_ERR_INVALID_ARG, "handle or ms is NULL");
    if (hd->probe_kind < 0 || !hd->probe_armed)
        return fail(hd, DIS_ERR_INVALID_ARG, "dis_probe_ms: no call has run the probed launch group");
    cudaError_t e = cudaEventSynchronize(hd->probe_b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, hd->probe_a, hd->probe_b);
    if (e != cudaSuccess) return cuda_fail(hd, e, "dis_probe_ms");
    return DIS_OK;
}

// ---- per-stage entry points -------------------------------------------------------------
static dis::LaunchCfg stage_lc()
{
    static thread_local bool init = false;
    static thread_local dis::LaunchCfg lc;
    if (!init) {
        lc = dis::query_launch_cfg();
        init = true;
    }
    return lc;
}

dis_status dis_pyr_down(const float* in, int w, int h, int64_t in_pitch, float* out, int64_t out_pitch, void* stream)
{
    if (!in || !out || w < 1 || h < 1 || in_pitch < w || out_pitch < (w + 1) / 2 || (long long)w * h > (1LL << 30))
        return fail(nullptr, DIS_ERR_INVALID_ARG, "dis_pyr_down: bad pointer, size or pitch");
    PyrJob J;
    std::memset(&J, 0, sizeof(J));
    J.in = in;
    J.out = out;
    J.win = w;
    J.hin = h;
    J.pin = (int)in_pitch;
    J.wout = (w + 1) / 2;
    J.hout = (h + 1) / 2;
    J.pout = (int)out_pitch;
    J.nplanes = 1;
    const dis::LaunchCfg lc = stage_lc();
    J.band = dis::pyr_band(dis::pyr_units(J.wout, J.hout, 1, 8), dis::pyr_units(J.wout, J.hout, 1, 2), lc.sm_count);
    cudaError_t e = dis::launch_pyr_down(dis::single_job(J), dis::pyr_units(J.wout, J.hout, 1, J.band), lc,
                                         (cudaStream_t)stream);
    return e == cudaSuccess ? DIS_OK : cuda_fail(nullptr, e, "dis_pyr_down");
}

dis_status dis_sobel(const float* in, int w, int h, int64_t pitch, float* gx, float* gy, int64_t out_pitch,
                     void* stream)
{
    if (!in || !gx || !gy || w < 1 || h < 1 || pitch < w || out_pitch < w)
        return fail(nullptr, DIS_ERR_INVALID_ARG, "dis_sobel: bad pointer, size or pitch");
    cudaError_t e = dis::launch_sobel(in, w, h, (int)pitch, gx, gy, (int)out_pitch, stage_lc(), (cudaStream_t)stream);
    return e == cudaSuccess ? DIS_OK : cuda_fail(nullptr, e, "dis_sobel");
}

static bool level_args_ok(int w, int h, int64_t pitch, int ps, int stride, const float* Uc, int wc, int hc, float cscale)
{
    if (w < 1 || h < 1 || pitch < w || ps < 2 || ps > kMaxPatch || stride < 1 || w < ps || h < ps) return false;
    if ((long long)w * h > (1LL << 30)) return false;  // 32-bit pixel indices
    if (Uc && (wc < 1 || hc < 1 || !(cscale > 0.0f))) return false;
    return true;
}

// A search variant of patch size ps: one of the flow search's forms, or (mode) one of the group
// widths of the stereo and robust-norm searches.
static bool variant_ok(int ps, int v, bool mode)
{
    int opts[8];
    const int n = mode ? dis::search_mode_options(ps, opts) : dis::search_lane_options(ps, opts);
    for (int k = 0; k < n; ++k)
        if (opts[k] == v) return true;
    return false;
}

dis_status dis_search_level_ex2(const float* I0, const float* I1, int w, int h, int64_t pitch, const float* Uc,
                                int wc, int hc, float cscale, int ps, int stride, int iters, int variant, int dof,
                                int norm, float huber_b, float term_eps, float* u_out, float* uinit_out,
                                int* status_out, void* stream)
{
    if (!I0 || !I1 || !u_out || iters < 0 || !level_args_ok(w, h, pitch, ps, stride, Uc, wc, hc, cscale))
        return fail(nullptr, DIS_ERR_INVALID_ARG, "dis_search_level: bad pointer, size, pitch or grid");
    if ((dof != 1 && dof != 2) || norm < 0 || norm > 2 || !finite(huber_b) || !(huber_b > 0.0f) ||
        !finite(term_eps) || term_eps < 0.0f)
        return fail(nullptr, DIS_ERR_INVALID_ARG, "dis_search_level: dof, norm, huber_b or term_eps out of range");
    const bool mode = dof != 2 || norm != 0 || term_eps > 0.0f;
    if (variant != 0 && !variant_ok(ps, variant, mode))
        return fail(nullptr, DIS_ERR_INVALID_ARG, "dis_search_level: not a search variant of this patch size");
    LevelJob J;
    std::memset(&J, 0, sizeof(J));
    J.S0 = I0;
    J.S1 = I1;
    J.w = w;
    J.h = h;
    J.pitch = (int)pitch;
    J.Uc = reinterpret_cast<const float2*>(Uc);
    J.wc = wc;
    J.hc = hc;
    J.cscale = cscale;
    J.pu = reinterpret_cast<float2*>(u_out);
    J.pui = reinterpret_cast<float2*>(uinit_out);
    J.pst = status_out;
    J.nx = grid_n(w, ps, stride);
    J.ny = grid_n(h, ps, stride);
    J.C = 1;
    const long long np = (long long)J.nx * J.ny;
    cudaError_t e = mode ? dis::launch_search_mode(dis::single_job(J), np, ps, stride, iters, dof, norm, huber_b,
                                                   term_eps, variant, stage_lc(), (cudaStream_t)stream)
                        : dis::launch_search(dis::single_job(J), np, ps, stride, iters, stage_lc(),
                                             (cudaStream_t)stream, variant, false);
    return e == cudaSuccess ? DIS_OK : cuda_fail(nullptr, e, "dis_search_level");
}

dis_status dis_search_level_ex(const float* I0, const float* I1, int w, int h, int64_t pitch, const float* Uc, int wc,
                               int hc, float cscale, int ps, int stride, int iters, int variant, float* u_out,
                               float* uinit_out, int* status_out, void* stream)
{
    return dis_search_level_ex2(I0, I1, w, h, pitch, Uc, wc, hc, cscale, ps, stride, iters, variant, 2, 0, 5.0f,
                                0.0f, u_out, uinit_out, status_out, stream);
}

dis_status dis_search_level(const float* I0, const float* I1, int w, int h, int64_t pitch, const float* Uc, int wc,
                            int hc, float cscale, int ps, int stride, int iters, float* u_out, float* uinit_out,
                            int* status_out, void* stream)
{
    return dis_search_level_ex(I0, I1, w, h, pitch, Uc, wc, hc, cscale, ps, stride, iters, 0, u_out, uinit_out,
                               status_out, stream);
}

dis_status dis_densify_level_fb(dis_handle* hd, const float* I0, const float* I1, int w, int h, int64_t pitch,
                                const float* u, const float* ub, int ps, int stride, float* U_out, float* Ub_out,
                                void* stream)
{
    if (!hd) return fail(nullptr, DIS_ERR_INVALID_ARG, "handle is NULL");
    if (!I0 || !I1 || !u || !ub || !U_out || !Ub_out || !level_args_ok(w, h, pitch, ps, stride, nullptr, 0, 0, 1.0f))
        return fail(hd, DIS_ERR_INVALID_ARG, "dis_densify_level_fb: bad pointer, size, pitch or grid");
    if (hd->max_batch < 2 || w > hd->max_w || h > hd->max_h ||
        (size_t)dis::fb_scratch_ints(w, h, ps, stride) > hd->rs_floats)
        return fail(hd, DIS_ERR_INVALID_ARG, "dis_densify_level_fb: needs a handle of two pairs of at least w x h");
    // two jobs, each the other's partner: the forward one on (I0, I1) with patch flows u, the
    // backward one on (I1, I0) with ub; the lists live in the scratch of slots 0 and 1
    LevelJob J[2];
    for (int k = 0; k < 2; ++k) {
        LevelJob& A = J[k];
        std::memset(&A, 0, sizeof(A));
        A.S0 = k ? I1 : I0;
        A.S1 = k ? I0 : I1;
        A.w = w;
        A.h = h;
        A.pitch = (int)pitch;
        A.wc = w;
        A.hc = h;
        A.cscale = 1.0f;
        A.pu = reinterpret_cast<float2*>(const_cast<float*>(k ? ub : u));
        A.U = reinterpret_cast<float2*>(k ? Ub_out : U_out);
        A.nx = grid_n(w, ps, stride);
        A.ny = grid_n(h, ps, stride);
        A.C = 1;
        A.patch_base = (long long)k * A.nx * A.ny;
        A.pix_base = (long long)k * w * h;
        long long tb = (long long)k * dis::refine_tiles(w, h);
        dis::set_refine_tiles(A, tb);
        A.rs = reinterpret_cast<float*>(hd->arena + (size_t)k * hd->slot_bytes + hd->off_rs);
        const long long tiles = dis::refine_tiles(w, h);
        A.fb_cnt = reinterpret_cast<int*>(A.rs);
        A.fb_cur = A.fb_cnt + tiles;
        A.fb_list = A.fb_cur + tiles;
        A.partner = 1 - k;
    }
    Plan plan;
    plan.blob.resize(sizeof(J));
    std::memcpy(plan.blob.data(), J, sizeof(J));
    cudaStream_t s = (cudaStream_t)stream;
    dis_status st = upload_jobs(hd, plan, s);
    if (st != DIS_OK) return st;
    const long long np = (long long)J[0].nx * J[0].ny;
    cudaError_t e = dis::launch_densify_fb(dis::device_jobs(reinterpret_cast<const LevelJob*>(hd->jobs_cur), 2), 2 * np,
                                           2 * dis::refine_tiles(w, h), 2, ps, stride, hd->lc, s);
    return e == cudaSuccess ? DIS_OK : cuda_fail(hd, e, "dis_densify_level_fb");
}

dis_status dis_densify_level(const float* I0, const float* I1, int w, int h, int64_t pitch, const float* u, int ps,
                             int stride, const float* Uc, int wc, int hc, float cscale, float* U_out, void* stream)
{
    if (!I0 || !I1 || !u || !U_out || !level_args_ok(w, h, pitch, ps, stride, Uc, wc, hc, cscale))
        return fail(nullptr, DIS_ERR_INVALID_ARG, "dis_densify_level: bad pointer, size, pitch or grid");
    LevelJob J;
    std::memset(&J, 0, sizeof(J));
    J.S0 = I0;
    J.S1 = I1;
    J.w = w;
    J.h = h;
    J.pitch = (int)pitch;
    J.Uc = reinterpret_cast<const float2*>(Uc);
    J.wc = wc;
    J.hc = hc;
    J.cscale = cscale;
    J.pu = reinterpret_cast<float2*>(const_cast<float*>(u));
    J.U = reinterpret_cast<float2*>(U_out);
    J.nx = grid_n(w, ps, stride);
    J.ny = grid_n(h, ps, stride);
    J.C = 1;
    long long tiles = 0;
    dis::set_refine_tiles(J, tiles);
    cudaError_t e = dis::launch_densify(dis::single_job(J), (long long)w * h, tiles, ps, stride, stage_lc(),
                                        (cudaStream_t)stream);
    return e == cudaSuccess ? DIS_OK : cuda_fail(nullptr, e, "dis_densify_level");
}

dis_status dis_refine_level_ex(dis_handle* hd, const float* I0, const float* I1, int w, int h, int64_t pitch,
                               int channels, float* U, int outer, int inner, float delta, float gamma, float alpha,
                               float omega, int dof, void* stream)
{
    if (!hd) return fail(nullptr, DIS_ERR_INVALID_ARG, "handle is NULL");
    if (!I0 || !I1 || !U || w < 1 || h < 1 || pitch < w || channels < 1 || channels > 3 || outer < 0 || inner < 0 ||
        !finite(delta) || !finite(gamma) || !finite(alpha) || !(omega > 0.0f && omega < 2.0f) ||
        (dof != 1 && dof != 2))
        return fail(hd, DIS_ERR_INVALID_ARG, "dis_refine_level: bad pointer, size, pitch or parameter");
    // each factor is bounded before the product, so that it cannot wrap
    if (pitch > (int64_t)hd->rs_floats || h > (int64_t)hd->rs_floats ||
        (unsigned long long)pitch * (unsigned long long)h > (unsigned long long)hd->rs_floats ||
        (size_t)dis::rs_planes(channels) * (size_t)pitch * (size_t)h > hd->rs_floats)
        return fail(hd, DIS_ERR_INVALID_ARG, "dis_refine_level: level larger than the handle's scratch");
    LevelJob J;
    std::memset(&J, 0, sizeof(J));
    J.P0 = I0;
    J.P1 = I1;
    J.w = w;
    J.h = h;
    J.pitch = (int)pitch;
    J.plane = (long long)pitch * h;
    J.C = channels;
    J.U = reinterpret_cast<float2*>(U);
    J.rs = reinterpret_cast<float*>(hd->arena + hd->off_rs);
    long long tiles = 0;
    dis::set_refine_tiles(J, tiles);
    dis::RefineArgs a{outer, inner, delta, gamma, alpha, omega, hd->refine_fused, hd->refine_split_px, channels, dof};
    const long long tp = (long long)w * h, th = (long long)h * ((w + 1) / 2);
    cudaError_t e = dis::launch_refine(dis::single_job(J), tp, th, tiles, a, hd->lc, (cudaStream_t)stream);
    return e == cudaSuccess ? DIS_OK : cuda_fail(hd, e, "dis_refine_level");
}

dis_status dis_refine_level(dis_handle* hd, const float* I0, const float* I1, int w, int h, int64_t pitch,
                            int channels, float* U, int outer, int inner, float delta, float gamma, float alpha,
                            float omega, void* stream)
{
    return dis_refine_level_ex(hd, I0, I1, w, h, pitch, channels, U, outer, inner, delta, gamma, alpha, omega, 2,
                               stream);
}

dis_status dis_upsample_flow(const float* Uin, int wi, int hi, float factor, float* Uout, int wo, int ho, void* stream)
{
    if (!Uin || !Uout || wi < 1 || hi < 1 || wo < 1 || ho < 1 || !(factor > 0.0f) || !finite(factor) ||
        (long long)wo * ho > (1LL << 30) || (long long)wi * hi > (1LL << 30))
        return fail(nullptr, DIS_ERR_INVALID_ARG, "dis_upsample_flow: bad pointer, size or factor");
    UpJob J;
    std::memset(&J, 0, sizeof(J));
    J.in = reinterpret_cast<const float2*>(Uin);
    J.out = reinterpret_cast<float2*>(Uout);
    J.wi = wi;
    J.hi = hi;
    J.wo = wo;
    J.ho = ho;
    J.factor = factor;
    cudaError_t e = dis::launch_upsample(dis::single_job(J), ho, stage_lc(), (cudaStream_t)stream);
    return e == cudaSuccess ? DIS_OK : cuda_fail(nullptr, e, "dis_upsample_flow");
}

}  // extern "C"

namespace dis {

LaunchCfg stage_launch_cfg() { return stage_lc(); }

void set_thread_error(const std::string& msg) { g_err = msg; }

}  // namespace dis

// ---- autotuner ---------------------------------------------------------------------------
extern "C" dis_status dis_autotune(dis_handle* hd, const dis_pair* pairs, int n, const dis_params* p, void* stream,
                                   int* chosen_lanes)
{
    if (!hd) return fail(nullptr, DIS_ERR_INVALID_ARG, "handle is NULL");
    std::string verr;
    dis_status vst = validate(p, verr);
    if (vst != DIS_OK) return fail(hd, vst, verr);
    int opts[8];
    // the stereo and robust-norm searches have their own (grouped) forms
    const bool flow_l2 = p->dof == 2 && p->norm == 0 && p->term_eps == 0.0f;
    const int nopt = flow_l2 ? dis::search_lane_options(p->patch_size, opts)
                             : dis::search_mode_options(p->patch_size, opts);
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return fail(hd, DIS_ERR_CUDA, "dis_autotune: event creation failed");
    }
    // one candidate: a warm-up call (builds its graph), then the sum of 3 timed calls
    auto time_calls = [&](float& tot) -> dis_status {
        dis_status r = dis_compute_flow_batched(hd, pairs, n, p, stream);
        tot = 0.0f;
        for (int k = 0; k < 3 && r == DIS_OK; ++k) {
            cudaEventRecord(e0, s);
            r = dis_compute_flow_batched(hd, pairs, n, p, stream);
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) r = cuda_fail(hd, cudaGetLastError(), "dis_autotune");
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            tot += ms;
        }
        return r;
    };
    const int ps = p->patch_size;
    const int keep = hd->search_lanes[ps], keep_refine = hd->refine_fused;
    float best_ms = 1e30f;
    int best = keep, best_refine = keep_refine;
    dis_status st = DIS_OK;
    // the search form first, with the refinement form as it is
    for (int k = 0; k < nopt && st == DIS_OK; ++k) {
        hd->search_lanes[ps] = opts[k];
        float tot = 0.0f;
        st = time_calls(tot);
        if (st == DIS_OK && tot < best_ms) {
            best_ms = tot;
            best = opts[k];
        }
    }
    // then the refinement launch form: per-sweep launches, or fused passes split into two
    // launches above a threshold, tried at every gap between the pixel counts of the levels
    // (all pairs of a level together) and at "never" / "always" (forms 2 and 3)
    const long long keep_split = hd->refine_split_px;
    long long best_split = keep_split;
    if (st == DIS_OK && p->refine) {
        hd->search_lanes[ps] = best;
        best_ms = 1e30f;
        std::vector<long long> level_px;
        {
            std::vector<PairIn> v;
            int ss_max = 0;
            for (int i = 0; i < n; ++i) {
                int ss = 0, sf = 0;
                std::string e;
                if (resolve_levels(pairs[i].width, pairs[i].height, *p, ss, sf, e) == DIS_OK) ss_max = std::max(ss_max, ss);
            }
            for (int s = 0; s <= ss_max; ++s) {
                long long px = 0;
                for (int i = 0; i < n; ++i) px += (long long)level_dim(pairs[i].width, s) * level_dim(pairs[i].height, s);
                level_px.push_back(px * (p->fb ? 2 : 1));
            }
        }
        std::vector<std::pair<int, long long>> cand = {{0, keep_split}, {2, keep_split}, {3, keep_split}};
        for (long long px : level_px) cand.push_back({1, px});  // split the levels larger than this one
        for (size_t k = 0; k < cand.size() && st == DIS_OK; ++k) {
            hd->refine_fused = cand[k].first;
            hd->refine_split_px = cand[k].second;
            float tot = 0.0f;
            st = time_calls(tot);
            if (st == DIS_OK && tot < best_ms) {
                best_ms = tot;
                best_refine = cand[k].first;
                best_split = cand[k].second;
            }
        }
        // form 1 with a threshold at the largest level is form 2: report it as form 1
        if (best_refine == 2) {
            best_refine = 1;
            best_split = dis::kRefineSplitNever;
        }
    }
    hd->search_lanes[ps] = (st == DIS_OK) ? best : keep;
    hd->refine_fused = (st == DIS_OK) ? best_refine : keep_refine;
    hd->refine_split_px = (st == DIS_OK) ? best_split : keep_split;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (chosen_lanes) *chosen_lanes = hd->search_lanes[ps];
    return st;
}

extern "C" dis_status dis_get_tuning(const dis_handle* hd, int patch_size, int* search_variant, int* refine_fusion)
{
    if (!hd || patch_size < 2 || patch_size > kMaxPatch)
        return fail(const_cast<dis_handle*>(hd), DIS_ERR_INVALID_ARG, "dis_get_tuning: handle NULL or bad patch size");
    if (search_variant) {
        int opts[8];
        dis::search_lane_options(patch_size, opts);
        *search_variant = hd->search_lanes[patch_size] ? hd->search_lanes[patch_size] : opts[0];
    }
    if (refine_fusion) *refine_fusion = hd->refine_fused;
    return DIS_OK;
}

extern "C" dis_status dis_last_call_kernels(const dis_handle* hd, int* count)
{
    if (!hd || !count) return fail(const_cast<dis_handle*>(hd), DIS_ERR_INVALID_ARG, "dis_last_call_kernels: NULL argument");
    *count = hd->last_kernels;
    return DIS_OK;
}

extern "C" int dis_search_variants(int patch_size, int* out, int cap)
{
    if (patch_size < 2 || patch_size > kMaxPatch) return 0;
    int opts[8];
    const int n = dis::search_lane_options(patch_size, opts);
    for (int k = 0; out && k < n && k < cap; ++k) out[k] = opts[k];
    return n;
}

extern "C" int dis_search_mode_variants(int patch_size, int* out, int cap)
{
    if (patch_size < 2 || patch_size > kMaxPatch) return 0;
    int opts[8];
    const int n = dis::search_mode_options(patch_size, opts);
    for (int k = 0; out && k < n && k < cap; ++k) out[k] = opts[k];
    return n;
}

extern "C" dis_status dis_set_search_variant(dis_handle* hd, int patch_size, int lanes)
{
    if (!hd) return fail(nullptr, DIS_ERR_INVALID_ARG, "handle is NULL");
    if (patch_size < 2 || patch_size > kMaxPatch || !(variant_ok(patch_size, lanes, false) || variant_ok(patch_size, lanes, true)))
        return fail(hd, DIS_ERR_INVALID_ARG, "dis_set_search_variant: not a variant of this patch size");
    hd->search_lanes[patch_size] = lanes;
    return DIS_OK;
}

// ---- host helpers shared with the backward pass (dis_backward.cu) ------------------------
namespace dis_host {

int pitch_of_w(int w) { return pitch_of(w); }
int level_dim_of(int d, int s) { return level_dim(d, s); }
int stride_of_params(const dis_params& p) { return stride_of(p); }
int grid_count(int L, int ps, int stride) { return grid_n(L, ps, stride); }
dis_status validate_params(const dis_params* p, std::string& err) { return validate(p, err); }
dis_status levels_of(int W, int H, const dis_params& p, int& ss, int& sf, std::string& err)
{
    return resolve_levels(W, H, p, ss, sf, err);
}
dis_status set_fail(dis_handle* h, dis_status st, const std::string& msg) { return fail(h, st, msg); }
dis_status set_cuda_fail(dis_handle* h, cudaError_t e, const char* what) { return cuda_fail(h, e, what); }

}  // namespace dis_host
