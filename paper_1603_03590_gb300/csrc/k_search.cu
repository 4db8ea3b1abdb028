// Search variants of the flow search: dispatch between the grouped form (k_search_grouped.cuh),
// the lane-per-patch form (k_search_lane.cu) and the warp-cooperative form (k_search_coop.cu).
#include "k_search_grouped.cuh"

namespace dis {

// Search variants: 0 = the default grouped form (8 lanes per patch up to 8x8 patches, 16
// above); 4, 8, 16, 32 = this grouped form with that many lanes per patch (compile-time 8x8
// and 12x12 sizes); 1 = the lane-per-patch form (k_search_lane.cu; `planes`: the jobs carry
// the search planes); 100 + G = the warp-cooperative form with G patches per warp
// (k_search_coop.cu).  Unsupported values fall back to the default.
cudaError_t launch_search(const Jobs<LevelJob>& js, long long total, int ps, int stride, int iters,
                          const LaunchCfg& lc, cudaStream_t s, int lanes, bool planes)
{
    if (total <= 0) return cudaSuccess;
    if (lanes > 100 && search_coop_supported(ps, lanes - 100))
        return launch_search_coop(js, total, ps, stride, iters, lanes - 100, lc, s);
    if (lanes == 1) return launch_search_lane(js, total, ps, stride, iters, lc, s, planes);
    const int n = ps * ps;
    if (ps == 8) {
        switch (lanes) {
            case 4: return launch_lp<4, 16, 8, 5>(js, total, ps, stride, iters, lc, s);
            case 16: return launch_lp<16, 4, 8>(js, total, ps, stride, iters, lc, s);
            default: return launch_lp<8, 8, 8, 8>(js, total, ps, stride, iters, lc, s);
        }
    }
    if (ps == 12) {
        switch (lanes) {
            case 8: return launch_lp<8, 18, 12>(js, total, ps, stride, iters, lc, s);
            case 32: return launch_lp<32, 5, 12>(js, total, ps, stride, iters, lc, s);
            default: return launch_lp<16, 9, 12, 7, true>(js, total, ps, stride, iters, lc, s);
        }
    }
    if (ps < 8) {
        switch ((n + 7) / 8) {
            case 1: return launch_lp<8, 1, 0>(js, total, ps, stride, iters, lc, s);
            case 2: return launch_lp<8, 2, 0>(js, total, ps, stride, iters, lc, s);
            case 4: return launch_lp<8, 4, 0>(js, total, ps, stride, iters, lc, s);
            case 5: return launch_lp<8, 5, 0>(js, total, ps, stride, iters, lc, s);
            default: return launch_lp<8, 7, 0>(js, total, ps, stride, iters, lc, s);
        }
    }
    return launch_lp<16, 16, 0>(js, total, ps, stride, iters, lc, s);
}

int search_lane_options(int ps, int* out)
{
    if (ps == 8) {
        const int v[6] = {8, 4, 1, 102, 104, 108};
        for (int k = 0; k < 6; ++k) out[k] = v[k];
        return 6;
    }
    if (ps == 12) {
        const int v[5] = {16, 8, 1, 102, 104};
        for (int k = 0; k < 5; ++k) out[k] = v[k];
        return 5;
    }
    out[0] = ps < 8 ? 8 : 16;
    out[1] = 1;
    return 2;
}

}  // namespace dis
