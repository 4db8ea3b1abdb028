/*
 * dis.h - C ABI of the GB300 (sm_103a) implementation of Dense Inverse Search optical flow
 * (Kroeger, Timofte, Dai, Van Gool, "Fast Optical Flow using Dense Inverse Search").
 *
 * The problem (Sec. 2.1, Eq. 1; Alg. 1): given a reference frame I_t (I0) and a query frame
 * I_{t+1} (I1), return a dense displacement field U with I1(x + U(x)) ~ I0(x).  U is in
 * full-resolution pixels, u along x (columns) and v along y (rows), stored interleaved
 * H x W x 2 float.
 *
 * Conventions shared by every entry point:
 *  - Every image, flow and patch pointer is caller-owned DEVICE memory (cudaMalloc'd or a
 *    torch CUDA tensor), FP32, row-major.  Images have a row pitch given in elements
 *    (>= width); colour images are planar C x H x W with planes pitch * H elements apart.
 *    Flow fields are dense (row pitch = width), interleaved (u, v).
 *  - Intensities are expected in [0, 1]; internally they are multiplied by
 *    dis_params.intensity_scale (255) so that the max(1, |d|) rule of Eq. 3 acts on the
 *    paper's 8-bit scale.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  All work is enqueued
 *    asynchronously on it; the call returns as soon as it is enqueued.  Host-detectable
 *    errors (bad arguments, sizes, allocation failure, launch failure) are returned
 *    immediately and leave every output untouched; device-side failures surface as
 *    DIS_ERR_CUDA on a later call.
 *  - Handles are not thread-safe: use one handle per host thread / stream.
 *  - No entry point throws.  Device memory is allocated by dis_create (the arena) and by
 *    dis_compute_flow_batched_host, which grows the handle's own host-copy staging on first
 *    use or when a larger batch arrives; every other entry point allocates nothing.
 */
#ifndef DIS_H
#define DIS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum dis_status {
    DIS_OK = 0,
    DIS_ERR_INVALID_ARG = 1,   /* null pointer, bad size, bad parameter */
    DIS_ERR_OUT_OF_MEMORY = 2, /* device allocation in dis_create failed */
    DIS_ERR_CUDA = 3,          /* a CUDA call or kernel launch failed */
    DIS_ERR_TOO_SMALL = 4,     /* the image is smaller than one patch at the coarsest level */
    DIS_ERR_TIMEOUT = 5,       /* reserved: a bounded device-side wait gave up */
    DIS_ERR_NOT_SUPPORTED = 6  /* valid request outside what the library implements */
} dis_status;

/* Parameters of the method (Table 1, Sec. 3.1).  dis_default_params fills the paper's
 * defaults; `struct_size` must be sizeof(dis_params) (ABI versioning). */
typedef struct dis_params {
    uint32_t struct_size;
    int32_t patch_size;      /* theta_ps, 2..16 */
    float overlap;           /* theta_ov in [0,1); stride = ps - floor(ov * ps) (>= 1) */
    int32_t stride_override; /* > 0: patch stride in pixels, overriding theta_ov */
    int32_t grad_iters;      /* theta_it >= 0: inverse-search iterations per patch */
    int32_t coarsest_scale;  /* theta_ss; -1: ceil(log2(2 W / (8 theta_ps))) (Sec. 3.1) */
    int32_t finest_scale;    /* theta_sf >= 0 */
    int32_t refine;          /* 1: variational refinement on each level (Sec. 2.3) */
    int32_t var_outer;       /* theta_vo; -1: s + 1 at scale s (Sec. 3.1) */
    int32_t var_inner;       /* theta_vi: red-black SOR sweeps per outer iteration */
    float delta, gamma, alpha; /* intensity / gradient / smoothness weights (5, 10, 10) */
    float sor_omega;         /* SOR over-relaxation, (0, 2) (the paper does not state it: 1.6) */
    float intensity_scale;   /* 255 */
    int32_t channels;        /* 1 (grayscale) or 3 (RGB, planar) */
    int32_t dof;             /* 2: optical flow; 1: stereo, horizontal displacements only (supplementary,
                              * depth from stereo: v keeps its initial value, the search takes the scalar
                              * step of the x component, the refinement leaves dv at 0) */
    int32_t norm;            /* search error norm (supplementary, robust error norms): 0 L2, 1 L1
                              * (e <- sign(e) sqrt|e|), 2 Huber (e <- e if |e| < huber_b, else
                              * sign(e) sqrt(2 huber_b |e| - huber_b^2)); e = I1(x + u) - mean - T */
    float huber_b;           /* Huber threshold on the intensity_scale scale, > 0 (5) */
    float term_eps;          /* > 0: a patch's search stops after the first update whose step length
                              * is at most term_eps px (early termination for small residuals,
                              * supplementary Sec. C; runs in the grouped search forms); 0: theta_it
                              * iterations (the search still ends early where that result is already
                              * known exactly) */
    int32_t fb;              /* 1: forward-backward consistency (supplementary Sec. B (ii)): both
                              * directions are searched and refined, each densification merges the
                              * other direction's patches (dis_densify_level_fb); n pairs take 2 n of
                              * the handle's max_batch slots; no initial flow, recorded / frozen
                              * increments or checkpoints (DIS_ERR_NOT_SUPPORTED); 0: off */
    int32_t search_grad;     /* differentiable form (dis_backward): 0 treats the recorded search
                              * increments as constants (stop-gradient through the search); 1 takes
                              * the implicit-function gradient of the converged search at every patch
                              * with a nonzero increment (L2 norm only) */
} dis_params;

/* Presets for dis_default_params.  OP1..OP4 are the paper's operating points
 * (Sec. 3.3: theta_sf/theta_it/theta_ps/theta_ov = 3/16/8/0.30 without refinement,
 * 3/12/8/0.40, 1/16/12/0.75, 0/256/12/0.75).  FAST/MEDIUM/DENSE are the workload presets
 * used by the benchmarks (patch 8 / 30 % / 16 it / finest 2 / no refinement; patch 8 / 50 %
 * / 32 it / refinement; patch 12 / 75 % / 128 it / refinement).  STEREO_OP1..OP4 and
 * STEREO_DENSE are OP1..OP4 and DENSE for depth from stereo (supplementary, depth from stereo):
 * dof = 1 and theta_it halved. */
enum {
    DIS_PRESET_DEFAULT = 0,
    DIS_PRESET_OP1 = 1,
    DIS_PRESET_OP2 = 2,
    DIS_PRESET_OP3 = 3,
    DIS_PRESET_OP4 = 4,
    DIS_PRESET_FAST = 5,
    DIS_PRESET_MEDIUM = 6,
    DIS_PRESET_DENSE = 7,
    DIS_PRESET_STEREO_OP1 = 8,
    DIS_PRESET_STEREO_OP2 = 9,
    DIS_PRESET_STEREO_OP3 = 10,
    DIS_PRESET_STEREO_OP4 = 11,
    DIS_PRESET_STEREO_DENSE = 12
};

typedef struct dis_handle dis_handle;

/* One frame pair of a batched call: device pointers, sizes and pitch as for
 * dis_compute_flow.  Pairs of one call may all differ in size. */
typedef struct dis_pair {
    const float* I0;
    const float* I1;
    int32_t width;
    int32_t height;
    int64_t pitch;   /* row pitch of I0 / I1 in elements */
    float* flow_out; /* height * width * 2 */
} dis_pair;

/* Fill `p` with a preset.  Never fails; p == NULL is ignored. */
void dis_default_params(dis_params* p, int preset);

/* Resolve the pyramid of a W x H frame under `p` (Sec. 3.1 and Alg. 1): coarsest and finest
 * processed scale, and the number of patches over all processed levels.  Returns
 * DIS_ERR_TOO_SMALL when the coarsest level cannot hold one patch. */
dis_status dis_levels(int width, int height, const dis_params* p, int* coarsest, int* finest, int64_t* total_patches);

/* Create a handle owning one device arena (the paper allocates all memory at once,
 * supplementary Sec. C) large enough for `max_batch` pairs of up to max_w x max_h with
 * `channels` channels.  Allocates on the current device.  *out is NULL on error. */
dis_status dis_create(dis_handle** out, int max_w, int max_h, int max_batch, int channels);

/* Release the arena, cached CUDA graphs and the handle.  NULL is ignored.  Synchronises
 * the handle's internal stream first. */
void dis_destroy(dis_handle* h);

/* Message of the last error on `h` (or of the last handle-less call in this thread when
 * h == NULL).  Never NULL; valid until the next call on the same handle / thread. */
const char* dis_last_error_string(const dis_handle* h);

/* Bytes of device memory owned by the handle (the arena). */
int64_t dis_arena_bytes(const dis_handle* h);

/* Whole method (Alg. 1) on one pair: pyramid, then per level s = theta_ss .. theta_sf:
 * patch grid, initialisation, inverse search, densification (Eq. 3), variational
 * refinement; finally bilinear up-scaling to full resolution (Sec. 3.1).
 * I0 / I1: `channels` planes of hgt x w, row pitch `pitch` elements; flow_out: hgt*w*2.
 * Requires w <= max_w, hgt <= max_h of the handle and p->channels == handle channels. */
dis_status dis_compute_flow(dis_handle* h, const float* I0, const float* I1, int w, int hgt, int64_t pitch,
                            const dis_params* p, float* flow_out, void* stream);

/* dis_compute_flow with forward-backward consistency (supplementary Sec. B (ii); p->fb is
 * taken as 1): flow_out receives the forward flow (I0 -> I1), flow_b_out (nullable) the
 * backward flow (I1 -> I0), same layout.  Needs a handle with max_batch >= 2. */
dis_status dis_compute_flow_fb(dis_handle* h, const float* I0, const float* I1, int w, int hgt, int64_t pitch,
                               const dis_params* p, float* flow_out, float* flow_b_out, void* stream);

/* Same as dis_compute_flow, with the differentiable form's extras (not in the paper):
 *  init_flow   (nullable): replaces the zero flow above the coarsest level (Alg. 1 line 1);
 *              given at the resolution of level theta_ss, in that level's pixels.
 *  frozen_in   (nullable): total_patches x 2 per-patch increments u_i - u_init,i, coarsest
 *              level first, replayed instead of searching (stop-gradient search).
 *  record_out  (nullable): receives those increments (0 for reset and flat patches).
 *  checkpoints (nullable): receives the densified flow U_s of every processed level,
 *              coarsest first, each level's w_s*h_s*2 floats back to back (dis_levels
 *              gives the sizes). */
dis_status dis_compute_flow_ex(dis_handle* h, const float* I0, const float* I1, int w, int hgt, int64_t pitch,
                               const dis_params* p, const float* init_flow, const float* frozen_in,
                               float* record_out, float* checkpoints, float* flow_out, void* stream);

/* Batched form (not in the paper): n pairs of arbitrary sizes (each within the handle's
 * max size; n <= max_batch) in one pass.  Every phase (pyramid level, search, densification,
 * refinement sweep) runs as one persistent kernel over a flattened work list of all pairs,
 * and the whole call is replayed from a cached CUDA graph when the sizes and parameters
 * repeat. */
dis_status dis_compute_flow_batched(dis_handle* h, const dis_pair* pairs, int n, const dis_params* p, void* stream);

/* dis_compute_flow_batched on frames and flows in HOST memory (pinned memory gives full copy
 * speed; pageable memory works, slower).  The handle copies the frames of the n pairs into
 * device staging of its own (allocated on first use and grown when a call needs more), computes
 * on `stream`, and copies the flows back into each pair's host flow_out.  The copies run on a
 * stream of the handle, and the staging is double-buffered, so the copies of one call overlap
 * the computation of the previous one.  The call returns once the work is enqueued: host
 * buffers must stay valid and unchanged, and flows must not be read, until
 * dis_host_flows_ready(h, stream) has been issued and `stream` synchronised. */
dis_status dis_compute_flow_batched_host(dis_handle* h, const dis_pair* pairs, int n, const dis_params* p,
                                        void* stream);

/* Makes `stream` wait until the flows of every earlier dis_compute_flow_batched_host call on h
 * are in host memory (synchronise `stream` afterwards to wait on the host). */
dis_status dis_host_flows_ready(dis_handle* h, void* stream);

/* Tracing (not in the paper): runs the batched call once without a CUDA graph, with events on
 * `stream` on both sides of every launch group of the plan, synchronises `stream` and writes one
 * record per group (up to `cap`; *count receives the total): the kind below, the pyramid level
 * (0 = finest) and the group's device time in milliseconds.  A group is one kernel launch,
 * except DIS_LAUNCH_REFINE, which covers all launches of one level's refinement.  Writes the
 * pairs' flow_out like dis_compute_flow_batched. */
enum {
    DIS_LAUNCH_PREP = 0,          /* level-0 scaling / channel mean */
    DIS_LAUNCH_PYRAMID = 1,       /* one pyramid step */
    DIS_LAUNCH_SEARCH_PLANES = 2, /* per-pixel search data of one level */
    DIS_LAUNCH_SEARCH = 3,        /* inverse search of one level */
    DIS_LAUNCH_DENSIFY = 4,       /* densification of one level */
    DIS_LAUNCH_REFINE = 5,        /* variational refinement of one level */
    DIS_LAUNCH_UPSAMPLE = 6       /* final up-scaling */
};
typedef struct dis_launch_record {
    int kind;
    int level;
    float ms;
} dis_launch_record;
dis_status dis_trace_batched(dis_handle* h, const dis_pair* pairs, int n, const dis_params* p, void* stream,
                             dis_launch_record* out, int cap, int* count);

/* Refinement launch form (not in the paper) for handle h.  A fused launch runs lagged-weight
 * passes with their SOR sweeps on shared-memory tiles whose halo is as wide as the half-sweeps
 * it runs (up to 5 sweeps per pass; more always use per-sweep launches).  fused = 1 (the
 * default) runs each pass in one fused launch, except that launches of more pixels than the
 * handle's split threshold (dis_set_refine_split; default: none, which measures fastest on
 * GB300 for the dense 1024x436 workload) run each pass as two fused launches of half the sweeps
 * (half the halo); 2 always uses one launch per pass, 3 always two, 0 one launch per
 * half-sweep plus thread-per-pixel derivative kernels (no halo, no shared memory).  All forms
 * give the same result bit for bit.  Other values: DIS_ERR_INVALID_ARG. */
dis_status dis_set_refine_fusion(dis_handle* h, int fused);

/* Split threshold of refinement form 1 (not in the paper): a level whose pixels over all pairs
 * of the call exceed `pixels` runs each pass in two fused launches; pixels < 0: never split (the
 * default).  dis_autotune sets it.  dis_get_refine_split reports it (-1: never).  Calls with
 * different thresholds use different cached graphs. */
dis_status dis_set_refine_split(dis_handle* h, int64_t pixels);
dis_status dis_get_refine_split(const dis_handle* h, int64_t* pixels);

/* Work scheduling (not in the paper) for handle h.  on = 1 (the default): the grouped search
 * kernels hand out patches, and the forward-backward densification its tiles, from a work queue
 * in the handle's arena (two counters; each group of lanes or block claims its next item with
 * one atomic, so those that drew cheap items take more of them); on = 0: a fixed grid stride.
 * Both give the same result bit for bit; the queue keeps every SM busy to the end of the launch.
 * Calls with and without the queue use different cached graphs.  Other values:
 * DIS_ERR_INVALID_ARG. */
dis_status dis_set_work_queue(dis_handle* h, int on);

/* Probe (not in the paper): from now on every call of handle h records two events of its own
 * around the launch group (kind, level) - inside the CUDA graph when the call replays one - so
 * that the group's device time in a normal call can be read with dis_probe_ms.  kind < 0
 * removes the probe.  Calls with and without a probe use different cached graphs. */
dis_status dis_set_probe(dis_handle* h, int kind, int level);

/* Device time in ms of the probed launch group in the most recent call that ran it (waits for
 * that group to finish).  DIS_ERR_INVALID_ARG when no such call has been issued. */
dis_status dis_probe_ms(dis_handle* h, float* ms);

/* Autotuner (not in the paper): time the inverse-search variants the library offers for this
 * workload on the caller's pairs (the batched call, 4 runs per variant, synchronising
 * `stream`) and keep the fastest in the handle for later calls with the same patch size; then,
 * when p->refine is set, time the refinement launch forms of dis_set_refine_fusion (0, 2, 3, and
 * 1 with a split threshold between every two level sizes of the call) with that search and keep
 * the fastest form and threshold.  The runs write the pairs' flow_out.  *chosen_lanes
 * (nullable) receives the chosen search variant code (dis_get_tuning reports both choices):
 *   4, 8, 16, 32   grouped: that many lanes share one patch (every group runs its own updates
 *                  and rebuilds its cell sums alone);
 *   1              lane per patch: one lane runs a patch's updates, the warp rebuilds the cell
 *                  sums of each patch that needs it together (reads two per-pixel planes);
 *   100 + G        warp-cooperative: G patches per warp, 32/G lanes per patch for the updates,
 *                  the whole warp for every rebuild (templates in shared memory).
 * All variants compute the same method; they differ in rounding order only. */
dis_status dis_autotune(dis_handle* h, const dis_pair* pairs, int n, const dis_params* p, void* stream,
                        int* chosen_lanes);

/* The search variant (the default one when none is pinned) and the refinement launch form
 * (dis_set_refine_fusion) handle h uses for patch size ps; either pointer may be NULL. */
dis_status dis_get_tuning(const dis_handle* h, int patch_size, int* search_variant, int* refine_fusion);

/* Kernels launched by the most recent call on h (not in the paper): the kernel nodes of the CUDA
 * graph that call replayed, counted when the graph was captured.  *count is -1 when that call
 * ran without a graph (checkpoints, or graphs disabled) or no call has run yet. */
dis_status dis_last_call_kernels(const dis_handle* h, int* count);

/* Search variants offered for patch size ps (codes as for dis_autotune, the default first):
 * writes up to `cap` of them to out (nullable when cap is 0) and returns their count, or 0 for
 * a patch size outside [2, 16]. */
int dis_search_variants(int patch_size, int* out, int cap);

/* The variants of the stereo and robust-norm searches (dis_params.dof 1 or norm != 0): group
 * widths of the grouped form (lanes per patch; 8 and 16 at 8x8, 16 and 32 at 12x12, one
 * otherwise), the first being their default.  A handle whose variant for ps is not one of them
 * runs these searches with the default; dis_autotune chooses among them for such params.  Same
 * conventions as dis_search_variants. */
int dis_search_mode_variants(int patch_size, int* out, int cap);

/* Pins the search variant of handle h for patch size ps to `lanes` (one of
 * dis_search_variants(ps) or dis_search_mode_variants(ps)), as dis_autotune would;
 * DIS_ERR_INVALID_ARG otherwise. */
dis_status dis_set_search_variant(dis_handle* h, int patch_size, int lanes);

/* ---- per-stage entry points (one pyramid level; used for per-stage parity tests and by
 * callers that drive the level loop themselves).  No allocation; caller-owned buffers. */

/* Pyramid step (Sec. 3.1, theta_sd = 2): out = even samples of [1 4 6 4 1]/16 separable
 * blur of `in` (replicated border).  out is ceil(w/2) x ceil(h/2) with pitch out_pitch. */
dis_status dis_pyr_down(const float* in, int w, int h, int64_t in_pitch, float* out, int64_t out_pitch,
                        void* stream);

/* Image gradients (Sec. 3.1 "image pyramid including image gradients"): 3x3 Sobel / 8 with
 * replicated border; gx along x, gy along y, both with pitch out_pitch. */
dis_status dis_sobel(const float* in, int w, int h, int64_t pitch, float* gx, float* gy, int64_t out_pitch,
                     void* stream);

/* Steps 1-3 of Alg. 1 on one level (Sec. 2.1, supplementary Sec. A): for every patch of the
 * grid (row-major), u_init = cscale * Uc(c / cscale) at the patch centre c (Uc NULL: zero;
 * cscale = theta_sd = 2 for the coarser level's flow), theta_it inverse-compositional
 * updates with mean-normalised patches, then the outlier reset |u - u_init| > theta_ps.
 * I0, I1: search images of the level, 0..255 scale, row pitch `pitch`; the Sobel gradients
 * of I0 are computed inside.  u_out / uinit_out: nx*ny*2; status_out: nx*ny ints
 * (0 ok, 1 reset, 2 flat).  uinit_out and status_out are nullable. */
dis_status dis_search_level(const float* I0, const float* I1, int w, int h, int64_t pitch, const float* Uc, int wc,
                            int hc, float cscale, int ps, int stride, int iters, float* u_out, float* uinit_out,
                            int* status_out, void* stream);

/* dis_search_level with an explicit search variant (0 = the default, else one of
 * dis_search_variants(ps)); the lane-per-patch variant reads the images here, not the
 * per-pixel planes of the handle path, with the same result bit for bit. */
dis_status dis_search_level_ex(const float* I0, const float* I1, int w, int h, int64_t pitch, const float* Uc, int wc,
                               int hc, float cscale, int ps, int stride, int iters, int variant, float* u_out,
                               float* uinit_out, int* status_out, void* stream);

/* dis_search_level_ex with the search's degrees of freedom, error norm and early termination
 * (dis_params.dof, norm, huber_b and term_eps).  dof 1 leaves the v component of u_out at
 * u_init; status 2 (flat) then means sum S'_x^2 <= 1e-6 tr(H') / 2.  For dof 1, norm != 0 or
 * term_eps > 0 the variant is 0 (the default) or one of dis_search_mode_variants(ps); dof 2 with
 * norm 0 and term_eps 0 is dis_search_level_ex.  DIS_ERR_INVALID_ARG for a dof outside {1, 2}, a
 * norm outside {0, 1, 2}, huber_b <= 0 or term_eps < 0. */
dis_status dis_search_level_ex2(const float* I0, const float* I1, int w, int h, int64_t pitch, const float* Uc,
                                int wc, int hc, float cscale, int ps, int stride, int iters, int variant, int dof,
                                int norm, float huber_b, float term_eps, float* u_out, float* uinit_out,
                                int* status_out, void* stream);

/* Step 4 of Alg. 1 (Eq. 3): U(x) = sum_i w_i(x) u_i / sum_i w_i(x) over the patches covering
 * x, w_i(x) = 1 / max(1, |I1(x + u_i) - I0(x)|).  u: nx*ny*2 patch flows; U_out: w*h*2.
 * Uc / cscale give the fallback for uncovered pixels as in dis_search_level. */
dis_status dis_densify_level(const float* I0, const float* I1, int w, int h, int64_t pitch, const float* u, int ps,
                             int stride, const float* Uc, int wc, int hc, float cscale, float* U_out, void* stream);

/* Step 4 with forward-backward consistency (supplementary Sec. B (ii)): both directions' dense
 * fields at once.  U_out (on I0's grid) merges the forward patches u (grid on I0, displacements
 * into I1; Eq. 3) with the backward patches ub (grid on I1, displacements into I0): backward
 * patch j gives pixel x the weight mu_j(x) / max(1, |I0(x) - I1(x - ub_j)|) (I1 bilinear) and
 * the displacement -ub_j, mu_j(x) being its bilinear footprint moved by ub_j (the sum over its
 * template pixels q of the bilinear weight that q + ub_j gives x: 1 inside the moved box, fading
 * to 0 over one pixel around it).  Ub_out is the same with the roles of (I0, u) and (I1, ub) exchanged.  u, ub: nx*ny*2;
 * U_out, Ub_out: w*h*2.  The per-tile patch lists live in the scratch of the handle's first two
 * pair slots (max_batch >= 2, w x h within its size).  Deterministic: the other direction's
 * contributions are summed in 64-bit fixed point. */
dis_status dis_densify_level_fb(dis_handle* hd, const float* I0, const float* I1, int w, int h, int64_t pitch,
                                const float* u, const float* ub, int ps, int stride, float* U_out, float* Ub_out,
                                void* stream);

/* Step 5 of Alg. 1 (Sec. 2.3): `outer` lagged-nonlinearity iterations of `inner` red-black
 * SOR sweeps on the intensity + gradient + smoothness energy; U (w*h*2) is refined in place.
 * I0 / I1: `channels` planes each, 0..255 scale, row pitch `pitch`, planes pitch*h apart.
 * Uses the handle's arena as scratch (w, h within its max size). */
dis_status dis_refine_level(dis_handle* hd, const float* I0, const float* I1, int w, int h, int64_t pitch,
                            int channels, float* U, int outer, int inner, float delta, float gamma, float alpha,
                            float omega, void* stream);

/* dis_refine_level with the degrees of freedom: dof 1 (stereo) keeps the v component of U and
 * solves, at every SOR step, the scalar equation of the x increment,
 * (A11 + sum_q w_pq) du = b1 + sum_q w_pq (U_q + dU_q - U_p)_x; dof 2 is dis_refine_level. */
dis_status dis_refine_level_ex(dis_handle* hd, const float* I0, const float* I1, int w, int h, int64_t pitch,
                               int channels, float* U, int outer, int inner, float delta, float gamma, float alpha,
                               float omega, int dof, void* stream);

/* Up-scaling (Sec. 3.1, last paragraph): Uout(x) = factor * Uin(x / factor), bilinear with
 * clamping.  Uin: wi*hi*2, Uout: wo*ho*2. */
dis_status dis_upsample_flow(const float* Uin, int wi, int hi, float factor, float* Uout, int wo, int ho,
                             void* stream);

/* ---- differentiable form (not in the paper) -------------------------------------------
 * The differentiable map F(I0, I1, init_flow) is DIS with every patch search replaced by its
 * recorded increment (u_i = u_init,i + Delta_i, Delta_i frozen: a converged argmin does not
 * depend on where it started), so gradients flow through the bilinear sampling of the initial
 * displacement, the densification weights (Eq. 3), the unrolled red-black SOR of the variational
 * refinement (Sec. 2.3) and the pyramid.  Record the increments with dis_compute_flow_ex
 * (record_out); dis_replay_flow evaluates F and dis_backward its gradient.  Both compute in
 * double precision: the refinement's robust weights Psi'(a^2) = 1 / (2 sqrt(a^2 + eps^2))
 * (eps = 0.001) make the gradient depend on flow and residual differences near 1e-6, below the
 * resolution of FP32 flow values.  Grayscale only (DIS_ERR_NOT_SUPPORTED otherwise; no
 * forward-backward consistency); with finest_scale > 0 the final bilinear up-scaling (and its
 * transpose) is part of F, with dof 1 the stereo refinement.  The search norm does not enter F (it only decides the recorded increments).  frozen: dis_levels' total_patches x 2 floats, coarsest level first; init_flow
 * (nullable): level theta_ss resolution, dense, 2 floats per pixel.  Nothing is allocated: the
 * caller passes a device workspace of dis_backward_workspace_bytes bytes.  Each call is a chain
 * of several hundred short launches: a call whose pointers, sizes and parameters all equal those
 * of an earlier call on the handle (the handle remembers the last 16 such keys and keeps graphs
 * of the last 8) is captured once into a CUDA graph and replayed with one launch after that,
 * with the same results bit for bit (environment DIS_NO_GRAPH=1 at dis_create: never). */

/* Photometric loss L = mean over channels and pixels of sqrt((I1(x + U(x)) - I0(x))^2 + eps^2)
 * (Charbonnier, eps = 0.001 by default) on the [0,1] scale, and its gradient with respect to
 * the flow (h*w*2), I0 and I1 (planar, pitch `pitch`).  loss_out: one device double.
 * scratch: device bytes >= dis_photometric_loss_scratch_bytes(...).  Deterministic. */
int64_t dis_photometric_loss_scratch_bytes(int width, int height, int64_t pitch, int channels);
dis_status dis_photometric_loss(const float* I0, const float* I1, int w, int h, int64_t pitch, int channels,
                                const float* flow, float eps, double* loss_out, float* grad_flow, float* grad_I0,
                                float* grad_I1, void* scratch, int64_t scratch_bytes, void* stream);

/* Device workspace for dis_replay_flow / dis_backward on a W x H pair under `p` (-1: invalid). */
int64_t dis_backward_workspace_bytes(int width, int height, const dis_params* p);

/* F(I0, I1, init_flow) with the recorded increments `frozen`, in FP64; flow_out: h*w*2 floats. */
dis_status dis_replay_flow(dis_handle* h, const float* I0, const float* I1, int w, int hgt, int64_t pitch,
                           const dis_params* p, const float* init_flow, const float* frozen, float* flow_out,
                           void* workspace, int64_t workspace_bytes, void* stream);

/* Gradient of a scalar loss through F: given grad_flow = dLoss/dF (h*w*2), writes dLoss/dI0 and
 * dLoss/dI1 (full resolution, [0,1] scale, row pitch grad_pitch) and, when grad_init_flow is
 * not NULL (init_flow must then be given), dLoss/dinit_flow.  Image-gradient scatters accumulate
 * in 64-bit fixed point, so the result is deterministic. */
dis_status dis_backward(dis_handle* h, const float* I0, const float* I1, int w, int hgt, int64_t pitch,
                        const dis_params* p, const float* init_flow, const float* frozen, const float* grad_flow,
                        float* grad_I0, float* grad_I1, int64_t grad_pitch, float* grad_init_flow, void* workspace,
                        int64_t workspace_bytes, void* stream);

/* ---- allocation-free variant (no counterpart in the paper) ----------------------------
 * dis_refine_level needs a handle, i.e. device memory that dis_create obtained with
 * cudaMalloc.  Callers that cannot allocate device memory - a plugin inside a host application
 * that owns the whole memory budget through its own pool, or a latency-critical loop that may
 * not call cudaMalloc / cudaFree because they can synchronise the device - use this variant:
 * same operation, arguments and result as dis_refine_level, but its scratch is a fixed device
 * array of DIS_NOALLOC_SCRATCH_FLOATS floats (16 MiB) built into the library, which every
 * device that loads the library holds until the process exits.  The call allocates nothing;
 * the caller still owns I0, I1 and U.
 *  - Size limit: (15 * channels + 8) * pitch * h must not exceed DIS_NOALLOC_SCRATCH_FLOATS
 *    (e.g. a 512 x 256 grayscale level with pitch 512: 3,014,656 floats); larger levels are
 *    rejected with DIS_ERR_INVALID_ARG before any work is enqueued.
 *  - The first call on a device looks up the array's device address (cudaGetSymbolAddress,
 *    with that device current) and caches it; make that first call before any stream capture.
 *    cudaDeviceReset on a device releases the array with its context, which leaves the cached
 *    address stale: do not call this entry point on a device after resetting it.
 *  - It always uses refinement launch form 1 (dis_set_refine_fusion mode 1) with the default
 *    split threshold: one fused launch per outer pass; all launch forms give the same flow bit
 *    for bit.
 *  - All calls share the one array, which keeps the last call's contents (the call itself
 *    zeroes what must start at zero).  Calls whose GPU work overlaps - on different streams
 *    or host threads - race on it: serialise them (e.g. one stream).
 *  - Errors are reported through dis_last_error_string(NULL). */
#define DIS_NOALLOC_SCRATCH_FLOATS (1u << 22)
dis_status dis_refine_level_noalloc(const float* I0, const float* I1, int w, int h, int64_t pitch, int channels,
                                    float* U, int outer, int inner, float delta, float gamma, float alpha, float omega,
                                    void* stream);

#ifdef __cplusplus
}
#endif

#endif /* DIS_H */
