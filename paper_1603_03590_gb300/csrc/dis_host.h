// Private host-side declarations of the DIS library: the handle and helpers shared by the
// forward (dis_api.cu) and backward (dis_backward.cu) translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/dis.h"
#include "dis_internal.cuh"

// The handle: one device arena (max_batch slots of per-level planes, a refinement scratch,
// a job-table region, the search work queue), the job upload state and the CUDA-graph cache.
struct dis_handle {
    int max_w = 0, max_h = 0, max_batch = 0, C = 1, levels = 0, device = 0;
    char* arena = nullptr;
    size_t arena_bytes = 0, slot_bytes = 0;
    std::vector<size_t> off_img, off_U, off_pu, off_pui, off_pst;  // per level, within a slot
    size_t off_rs = 0;
    size_t rs_floats = 0;  // capacity of the refinement scratch (floats)
    // job tables kept on the device: a call whose tables equal a resident one uploads nothing
    // (callers that alternate between buffer sets, such as the host-buffer call's two staging
    // halves, keep one table per set)
    static constexpr int kJobSlots = 4;
    char* jobs_dev = nullptr;     // kJobSlots tables of jobs_bytes each
    size_t jobs_bytes = 0;
    char* jobs_pinned = nullptr;  // kJobSlots pinned staging areas of the uploads
    cudaEvent_t jobs_ev[kJobSlots] = {};       // each slot's latest upload ...
    cudaStream_t jobs_stream[kJobSlots] = {};  // ... and the stream it was issued on
    bool jobs_ok[kJobSlots] = {};
    std::vector<char> jobs_blob[kJobSlots];
    unsigned long long jobs_stamp[kJobSlots] = {};  // last use, for replacement
    unsigned long long jobs_clock = 0;
    int jobs_slot = 0;               // slot of the latest upload_jobs
    const char* jobs_cur = nullptr;  // its device table
    cudaStream_t cap_stream = nullptr;
    struct Graph {
        std::vector<int64_t> key;
        cudaGraphExec_t exec;
        int kernels;  // kernel nodes of the captured graph
    };
    std::vector<Graph> graphs;
    // graphs of the differentiable form's calls (dis_replay_flow, dis_backward), keyed on every
    // pointer, size and parameter of the call: a key is captured the second time it is seen,
    // so calls whose buffers change every time launch directly instead of capturing each time
    std::vector<Graph> bwd_graphs;
    std::vector<std::vector<int64_t>> bwd_seen;
    dis::LaunchCfg lc{};
    bool use_graphs = true;
    int search_lanes[17] = {};  // autotuned lanes per patch by patch size (0 = default)
    int refine_fused = 1;       // refinement launch form (dis_set_refine_fusion)
    long long refine_split_px = dis::kRefineSplitNever;  // form 1's split threshold (dis_set_refine_split)
    int last_kernels = -1;      // kernels of the graph the most recent call replayed (-1: none)
    unsigned int* wq = nullptr;  // the search work queue in the arena (lc.wq while enabled)
    // probe: events recorded around one launch group in every call (also inside graphs)
    int probe_kind = -1, probe_level = 0;
    cudaEvent_t probe_a = nullptr, probe_b = nullptr;
    bool probe_armed = false;  // a call with the probe has been issued since it was set
    // host-buffer batched calls: two halves of device staging (frames in, flows out), a stream
    // for the copies in and one for the copies out, and per half the events "frames copied in",
    // "flows computed", "flows copied out"
    struct HostStage {
        char* buf = nullptr;
        size_t half_bytes = 0;
        cudaStream_t cs_in = nullptr, cs_out = nullptr;
        cudaEvent_t ev_in[2] = {nullptr, nullptr}, ev_out[2] = {nullptr, nullptr}, ev_done[2] = {nullptr, nullptr};
        bool used[2] = {false, false};
        int next = 0, last = -1;
    } hs;
    std::string err = "no error";
};


namespace dis_host {
int pitch_of_w(int w);
int level_dim_of(int d, int s);
int stride_of_params(const dis_params& p);
int grid_count(int L, int ps, int stride);
dis_status validate_params(const dis_params* p, std::string& err);
dis_status levels_of(int W, int H, const dis_params& p, int& ss, int& sf, std::string& err);
dis_status set_fail(dis_handle* h, dis_status st, const std::string& msg);
dis_status set_cuda_fail(dis_handle* h, cudaError_t e, const char* what);
int graph_kernel_nodes(cudaGraph_t graph);
}  // namespace dis_host
