// Stereo (one degree of freedom) and robust-norm modes of the patch search, and the search with
// early termination on a small step, in the grouped form of k_search_grouped.cuh (see its
// header for the arithmetic of each mode).
#include "k_search_grouped.cuh"

namespace dis {

template <int DOF, bool ROBUST>
static cudaError_t launch_mode(const Jobs<LevelJob>& js, long long total, int ps, int stride, int iters, int norm,
                               float huber_b, float term2, int lanes, const LaunchCfg& lc, cudaStream_t s)
{
    // resident blocks per SM, measured: the robust form keeps four coefficients per pixel in
    // registers, so fewer blocks (chosen so that nothing spills); the 12x12 16-lane L2 form runs
    // six blocks at the cost of a few spilled registers; wider groups hold fewer pixels per lane
    constexpr int MB8 = ROBUST ? (DOF == 1 ? 3 : 4) : 6, MB12 = ROBUST ? (DOF == 1 ? 2 : 3) : 6;
    constexpr int MBW = ROBUST ? (DOF == 1 ? 4 : 5) : 6, MB32 = ROBUST ? MBW : 5;
    if (ps == 8) {
        if (lanes == 16)
            return launch_lp<16, 4, 8, MBW, true, DOF, ROBUST, true>(js, total, ps, stride, iters, lc, s, norm, huber_b, term2);
        return launch_lp<8, 8, 8, MB8, true, DOF, ROBUST, true>(js, total, ps, stride, iters, lc, s, norm, huber_b, term2);
    }
    if (ps == 12) {
        if (lanes == 32)
            return launch_lp<32, 5, 12, MB32, true, DOF, ROBUST, true>(js, total, ps, stride, iters, lc, s, norm, huber_b, term2);
        return launch_lp<16, 9, 12, MB12, true, DOF, ROBUST, true>(js, total, ps, stride, iters, lc, s, norm, huber_b, term2);
    }
    if (ps < 8) return launch_lp<8, 7, 0, 4, true, DOF, ROBUST, true>(js, total, ps, stride, iters, lc, s, norm, huber_b, term2);
    return launch_lp<16, 16, 0, 2, true, DOF, ROBUST, true>(js, total, ps, stride, iters, lc, s, norm, huber_b, term2);
}

cudaError_t launch_search_mode(const Jobs<LevelJob>& js, long long total, int ps, int stride, int iters, int dof,
                               int norm, float huber_b, float term_eps, int lanes, const LaunchCfg& lc, cudaStream_t s)
{
    if (total <= 0) return cudaSuccess;
    const float term2 = term_eps * term_eps;
    if (norm == 0) {
        if (dof == 1) return launch_mode<1, false>(js, total, ps, stride, iters, 0, 0.0f, term2, lanes, lc, s);
        return launch_mode<2, false>(js, total, ps, stride, iters, 0, 0.0f, term2, lanes, lc, s);
    }
    if (dof == 1) return launch_mode<1, true>(js, total, ps, stride, iters, norm, huber_b, term2, lanes, lc, s);
    return launch_mode<2, true>(js, total, ps, stride, iters, norm, huber_b, term2, lanes, lc, s);
}

int search_mode_options(int ps, int* out)
{
    if (ps == 8 || ps == 12) {
        out[0] = ps == 8 ? 8 : 16;
        out[1] = ps == 8 ? 16 : 32;
        return 2;
    }
    out[0] = ps < 8 ? 8 : 16;
    return 1;
}

}  // namespace dis
