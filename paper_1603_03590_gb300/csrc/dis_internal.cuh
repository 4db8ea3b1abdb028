// Internal declarations of the DIS CUDA path: job descriptors and kernel launchers.
//
// Every kernel works on a flattened list of work items (pixels, patches, same-colour
// pixels) spanning one or many "jobs" (a frame pair at one pyramid level).  A job list is
// either a device array (batched form, built once per plan) or one job passed by value in
// the kernel parameters (single pair, per-stage entry points: no device allocation).
// Kernels are grid-stride loops, so one persistent launch covers all pairs of a phase.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

namespace dis {

// Patch / pyramid / refinement work of one frame pair at one pyramid level.
struct LevelJob {
    const float* S0;      // search image of frame t (channel mean), row pitch `pitch`
    const float* S1;      // search image of frame t+1
    const float* P0;      // channel planes of frame t (C planes, `plane` floats apart)
    const float* P1;      // channel planes of frame t+1
    const float2* Uc;     // flow the patches start from (coarser level or initial flow), or null
    float2* U;            // dense flow of this level, w*h
    float2* pu;           // patch flows, nx*ny
    float2* pui;          // patch initial flows (nullable)
    int* pst;             // patch status (nullable): 0 ok, 1 reset, 2 flat
    const float2* frozen; // replayed increments (nullable)
    float2* record;       // recorded increments (nullable)
    float* rs;            // refinement scratch: (15 C + 8) planes of `plane` floats
    const float4* tpl;    // search planes (nullable; may alias rs, written before the search):
    const float4* tap;    //   (I0, gx, gy, 0) and the four bilinear taps of I1 per pixel
    long long plane;      // pitch * h
    long long patch_base; // first flattened patch of this job
    long long pix_base;   // first flattened pixel
    long long half_base;  // first flattened same-colour pixel (h * ceil(w/2) per colour)
    long long tile_base;  // first flattened refinement tile (kRefineTile^2 pixels each)
    int tiles_x;          // refinement tiles per row
    int w, h, pitch;
    int wc, hc;
    float cscale;
    int nx, ny;
    int C;
    // forward-backward consistency: the job of the other direction of the same pair (same
    // size and grid, frames exchanged) and, in this job's refinement scratch, the lists of the
    // other direction's patches whose moved box meets each of this job's refinement tiles:
    // fb_cnt (counts, then offsets), fb_cur (fill cursors, then list ends), fb_list.
    int partner;
    int* fb_cnt;
    int* fb_cur;
    int* fb_list;
};

// One pyramid step of `nplanes` consecutive planes.
struct PyrJob {
    const float* in;
    float* out;
    long long in_plane, out_plane;
    long long base;  // first flattened work unit of the job (pyr_units: plane, band, column chunk)
    int win, hin, pin, wout, hout, pout, nplanes;
    int band;  // output rows per work unit (pyr_band)
};

// Level-0 preparation: scale the caller's frames, form the channel mean.
struct PrepJob {
    const float* I0;
    const float* I1;
    long long in_plane;
    float* S0;
    float* S1;
    float* P0;  // null when the channel planes are not needed (C == 1 or no refinement)
    float* P1;
    long long out_plane;
    long long base;  // first flattened row of the job
    int w, h, in_pitch, out_pitch, C;
    int vec;  // the input rows start on 16-byte boundaries (float4 loads)
    float scale;
};

// Bilinear up-scaling of a flow field.
struct UpJob {
    const float2* in;
    float2* out;
    long long base;  // first flattened output row of the job
    int wi, hi, wo, ho;
    float factor;
};

// A job list: device array (dev != null, n entries) or a single job by value.
template <class J>
struct Jobs {
    const J* dev;
    J one;
    int n;
};

template <class J>
inline Jobs<J> single_job(const J& j)
{
    Jobs<J> r;
    r.dev = nullptr;
    r.one = j;
    r.n = 1;
    return r;
}

template <class J>
inline Jobs<J> device_jobs(const J* dev, int n)
{
    Jobs<J> r = {};
    r.dev = dev;
    r.n = n;
    return r;
}

// Refinement scratch plane indices (per channel c: intermediate, data; then shared planes).
// Intermediate (6 C): the mean image (I0 + I1w)/2, I_z = I1w - I0, I_x, I_y (the last two in the
// per-sweep form only), two free planes (an increment of the fused form, channel 0).  Data
// (9 C, per-sweep form): sqrt(b0)(Ix, Iy, Iz), sqrt(bx)(Ixx, Ixy, Ixz), sqrt(by)(Ixy, Iyy, Iyz).
// System (6, per-sweep form; the fused form keeps an increment in the first two): A11 A12 A22
// b1 b2 psiS.  Increment (2): du, dv.  (The FP64 differentiable form indexes its own scratch with
// these functions, its six intermediate planes holding I1w, I_x, I_y, I_z, I_xz, I_yz.)
__host__ __device__ inline int rs_mid(int C, int c, int k) { return c * 6 + k; }
__host__ __device__ inline int rs_dat(int C, int c, int k) { return 6 * C + c * 9 + k; }
__host__ __device__ inline int rs_sys(int C, int k) { return 15 * C + k; }
__host__ __device__ inline int rs_du(int C, int k) { return 15 * C + 6 + k; }
__host__ __device__ inline int rs_planes(int C) { return 15 * C + 8; }

struct LaunchCfg {
    int sm_count;
    int max_blocks_256;  // resident 256-thread blocks per SM for the elementwise kernels
    // Work queue of the grouped patch search and the forward-backward densification (two zeroed
    // counters in device memory owned by a handle: the next item to hand out, the groups or
    // blocks that found none left; the last to finish zeroes both again, so consecutive launches
    // on the handle's stream and graph replays each start from zero).  Null: the static
    // grid-stride assignment.
    unsigned int* wq = nullptr;
};

// Launchers (return the launch error).  `total` = number of flattened items.
cudaError_t launch_prep(const Jobs<PrepJob>& js, long long rows, const LaunchCfg& lc, cudaStream_t s);
cudaError_t launch_pyr_down(const Jobs<PyrJob>& js, long long units, const LaunchCfg& lc, cudaStream_t s);
// Work units of a pyramid job: its planes x bands of `band` output rows x chunks of output
// columns; and the band height for a call (8, 2 or 1) from its unit counts at band 8 and 2.
long long pyr_units(int wout, int hout, int nplanes, int band);
int pyr_band(long long units_at_full_band, long long units_at_band2, int sm_count);
cudaError_t launch_sobel(const float* in, int w, int h, int pitch, float* gx, float* gy, int out_pitch,
                         const LaunchCfg& lc, cudaStream_t s);
// lanes: lanes per patch (0 or 1 = the lane-per-patch form; see search_lane_options).  planes:
// the jobs carry tpl / tap (written by launch_search_planes); used by the lane-per-patch form.
cudaError_t launch_search_lane(const Jobs<LevelJob>& js, long long total, int ps, int stride, int iters,
                               const LaunchCfg& lc, cudaStream_t s, bool planes);
cudaError_t launch_search(const Jobs<LevelJob>& js, long long total, int ps, int stride, int iters,
                          const LaunchCfg& lc, cudaStream_t s, int lanes = 0, bool planes = false);
// Warp-cooperative form with g patches per warp (k_search_coop.cu), for patch sizes 8 and 12.
bool search_coop_supported(int ps, int g);
cudaError_t launch_search_coop(const Jobs<LevelJob>& js, long long total, int ps, int stride, int iters, int g,
                               const LaunchCfg& lc, cudaStream_t s);
// Writes the search planes tpl / tap of every job (thread per pixel, flattened by pix_base).
cudaError_t launch_search_planes(const Jobs<LevelJob>& js, long long total_pix, const LaunchCfg& lc, cudaStream_t s);
// Lanes-per-patch variants the search offers for patch size ps (first = default); returns the count.
int search_lane_options(int ps, int* out);
// The stereo (dof 1) and robust-norm (norm 1 L1, 2 Huber with threshold huber_b) searches, and
// any search with early termination (term_eps > 0: stop after a step of length <= term_eps), in
// the grouped form with `lanes` lanes per patch when that is one of search_mode_options(ps), else
// the first of them.  The flow search with the L2 norm and no early termination is launch_search.
cudaError_t launch_search_mode(const Jobs<LevelJob>& js, long long total, int ps, int stride, int iters, int dof,
                               int norm, float huber_b, float term_eps, int lanes, const LaunchCfg& lc,
                               cudaStream_t s);
// Group widths of the stereo and robust-norm searches for patch size ps (the first is the default).
int search_mode_options(int ps, int* out);
// Densification with forward-backward consistency over jobs that come in partner pairs: lists
// the patches of each job by the tiles of its partner that their moved boxes meet (four
// launches), then merges, per tile, the job's own patches with the partner's listed ones.
cudaError_t launch_densify_fb(const Jobs<LevelJob>& js, long long total_patches, long long total_tiles, int njobs,
                              int ps, int stride, const LaunchCfg& lc, cudaStream_t s);
// Ints of refinement scratch the lists of one job take (at most), for a w x h level.
long long fb_scratch_ints(int w, int h, int ps, int stride);
// Plain densification of `total` pixels; `tiles` > 0: the jobs carry their refinement tiles
// (tile_base, tiles_x), `tiles` in all, and the tiled form runs where the stride allows it.
cudaError_t launch_densify(const Jobs<LevelJob>& js, long long total, long long tiles, int ps, int stride,
                           const LaunchCfg& lc, cudaStream_t s);
constexpr long long kRefineSplitNever = 1LL << 62;
struct RefineArgs {
    int outer, inner;
    float delta, gamma, alpha, omega;
    int fused = 1;      // 0: per-sweep launches; 1: each pass in one fused launch up to
                        // split_px pixels per launch, in two above; 2: one fused launch,
                        // 3: two fused launches per pass, whenever inner allows
    long long split_px = kRefineSplitNever;  // form 1's threshold
    int C = 1;          // channels of every job of the launch
    int dof = 2;        // 1: stereo, the vertical increment stays 0
};
// Square tiles of the fused outer-iteration kernel; at most kRefineMaxFusedInner inner sweeps
// (2 half-sweeps each) run in one launch, the halo being as wide as the half-sweeps.
constexpr int kRefineTile = 32;
constexpr int kRefineMaxFusedInner = 5;
inline long long refine_tiles(int w, int h)
{
    return (long long)((w + kRefineTile - 1) / kRefineTile) * ((h + kRefineTile - 1) / kRefineTile);
}
inline void set_refine_tiles(LevelJob& J, long long& tile_base)
{
    J.tiles_x = (J.w + kRefineTile - 1) / kRefineTile;
    J.tile_base = tile_base;
    tile_base += refine_tiles(J.w, J.h);
}
cudaError_t launch_refine(const Jobs<LevelJob>& js, long long total_pix, long long total_half, long long total_tiles,
                          const RefineArgs& a, const LaunchCfg& lc, cudaStream_t s);
cudaError_t launch_upsample(const Jobs<UpJob>& js, long long rows, const LaunchCfg& lc, cudaStream_t s);

LaunchCfg query_launch_cfg();

// ---- differentiable form: FP64 replay and adjoint of one level of one pair ---------------
// Adjoint planes (level pitch x height each): gD[9] gsys[6] gdU[2] gmid[8] tmp[4] gIx gIy gI1w.
enum { ADJ_GD = 0, ADJ_GSYS = 9, ADJ_GDU = 15, ADJ_GM = 17, ADJ_GT = 25, ADJ_GIX = 29, ADJ_GIY = 30,
       ADJ_GI1W = 31, ADJ_PLANES = 32 };

struct Lvl64 {
    const double* S0;         // level images (0..255 scale), row pitch `pitch`
    const double* S1;
    const double2* U;         // refinement input: the densified flow (dense w*h)
    double* rs;               // refinement scratch ((15 + 8) planes, C = 1 layout of rs_*)
    double* ga;               // adjoint planes, ADJ_PLANES x plane
    double* gS0;              // gradient of S0 (accumulated, pitch)
    unsigned long long* gS1;  // gradient of S1 in 2^-48 fixed point (accumulated, pitch)
    double2* gU;              // gradient of the densified flow (accumulated, dense)
    long long plane;
    int w, h, pitch;
    double delta, gamma, alpha, omega;
    int dof;  // 1: stereo, the SOR solves the scalar x equation and dv stays 0
};

struct Dens64 {
    const double2* pu;   // patch flows u_i = u_init,i + Delta_i
    double2* gpu;        // gradient of the patch flows
    const double2* gUd;  // gradient of the densified flow (dense)
    int nx, ny, ps, stride;
};

cudaError_t launch_prep64(const float* I, int w, int h, int in_pitch, double scale, double* S, int pitch,
                          const LaunchCfg& lc, cudaStream_t s);
cudaError_t launch_pyr64(const double* in, int win, int hin, int pin, double* out, int wout, int hout, int pout,
                         const LaunchCfg& lc, cudaStream_t s);
cudaError_t launch_uinit64(const Dens64& A, int w, int h, const double2* Uc, int wc, int hc, double cs,
                           const float2* frozen, double2* pu, const LaunchCfg& lc, cudaStream_t s);
cudaError_t launch_densify64(const double* S0, const double* S1, int w, int h, int pitch, const Dens64& A,
                             const double2* Uc, int wc, int hc, double cs, double2* Ud, const LaunchCfg& lc,
                             cudaStream_t s);
cudaError_t launch_ref64_prepare(const Lvl64& L, const LaunchCfg& lc, cudaStream_t s);
cudaError_t launch_ref64_weights(const Lvl64& L, const LaunchCfg& lc, cudaStream_t s);
cudaError_t launch_ref64_sor(const Lvl64& L, int colour, const LaunchCfg& lc, cudaStream_t s);
cudaError_t launch_ref64_apply(const Lvl64& L, double2* Uout, const LaunchCfg& lc, cudaStream_t s);
cudaError_t launch_loss(const float* I0, const float* I1, int w, int h, int pitch, int C, const float2* flow, float eps,
                        double* partials, int max_partials, double* loss_out, float2* gflow, float* gI0,
                        unsigned long long* gI1acc, const LaunchCfg& lc, cudaStream_t s);
cudaError_t launch_fx_to_float(const unsigned long long* acc, int apitch, float* out, int opitch, int w, int h,
                               double scale, bool accumulate, const LaunchCfg& lc, cudaStream_t s);
cudaError_t launch_fx_to_double(const unsigned long long* acc, int apitch, double* out, int opitch, int w, int h,
                                double scale, bool accumulate, const LaunchCfg& lc, cudaStream_t s);
cudaError_t launch_sor_bwd(const Lvl64& L, const double* st_du, const double* st_dv, int colour, const LaunchCfg& lc,
                           cudaStream_t s);
cudaError_t launch_weights_bwd(const Lvl64& L, const double* st_du, const double* st_dv, const LaunchCfg& lc,
                               cudaStream_t s);
cudaError_t launch_deriv_warp_bwd(const Lvl64& L, const LaunchCfg& lc, cudaStream_t s);
cudaError_t launch_start_flow(const Lvl64& L, const double2* g, const LaunchCfg& lc, cudaStream_t s);
cudaError_t launch_dens_bwd(const Lvl64& L, const Dens64& A, const LaunchCfg& lc, cudaStream_t s);
cudaError_t launch_uinit_bwd(const Dens64& A, int w, int h, unsigned long long* gUc, int wc, int hc, double cs,
                             const LaunchCfg& lc, cudaStream_t s);
// Implicit-function gradient of the converged search at every patch with a nonzero frozen
// increment (see k_adjoint.cu): scatters into L.gS1 and gS0acc (2^-48 fixed point, pitch) and
// zeroes those patches' A.gpu.
cudaError_t launch_search_ift_bwd(const Lvl64& L, const Dens64& A, const float2* frozen, unsigned long long* gS0acc,
                                  int dof, const LaunchCfg& lc, cudaStream_t s);
cudaError_t launch_pyr_bwd(const double* gc, int wc, int hc, int pc, double* gf, int wf, int hf, int pf,
                           const LaunchCfg& lc, cudaStream_t s);
cudaError_t launch_f2_to_d2(const float2* in, double2* out, long long n, const LaunchCfg& lc, cudaStream_t s);
// FP64 final up-scaling (out = factor * in(x / factor), bilinear, clamped) and its transpose,
// accumulated into gin (2^-48 fixed point, dense wi*hi*2).
cudaError_t launch_upsample64(const double2* in, int wi, int hi, double factor, double2* out, int wo, int ho,
                              const LaunchCfg& lc, cudaStream_t s);
cudaError_t launch_upsample_bwd(const double2* gout, int wo, int ho, double factor, unsigned long long* gin, int wi,
                                int hi, const LaunchCfg& lc, cudaStream_t s);
cudaError_t launch_d2_to_f2(const double2* in, float2* out, long long n, const LaunchCfg& lc, cudaStream_t s);
cudaError_t launch_scale_out(const double* in, int ipitch, float* out, int opitch, int w, int h, double scale,
                             const LaunchCfg& lc, cudaStream_t s);

// Launch configuration of the handle-less entry points (cached per host thread).
LaunchCfg stage_launch_cfg();
// Message returned by dis_last_error_string(NULL) for handle-less calls of this thread.
void set_thread_error(const std::string& msg);

}  // namespace dis
