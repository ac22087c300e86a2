/*
 * fmb.h -- C ABI of the GB300 (sm_103a) renderer for the simplified, two-parameter
 * Fuzzy Metaballs model of "Flexible Techniques for Differentiable Rendering with
 * 3D Gaussians" (Keselman & Hebert, WACV 2024).
 *
 * Model (paper Sec. 3.1-3.2, Sec. 5, Sec. 6):
 *   Gaussian i: mean mu_i, precision Sigma_i^-1 = L_i L_i^T with L_i lower
 *   triangular (Sec. 3.1 parameterises the shape by an inverse square root of the
 *   precision), weight lambda_i > 0.
 *   For the ray v (unit length, world frame) from the camera centre o of a pixel:
 *     t_i     = (mu_i - o)^T Sigma_i^-1 v / (v^T Sigma_i^-1 v)   (max-likelihood
 *               depth along the ray, next to Eq. 2)
 *     d_i     = -1/2 (o + v t_i - mu_i)^T Sigma_i^-1 (o + v t_i - mu_i) + ln lambda_i  (Eq. 2)
 *     delta_i = exp(d_i)                                            (Eq. 4)
 *     w_i     = exp(beta1 d_i - (beta2 / eta) t_i)                  (Eq. 7)
 *     depth   = sum_i w_i t_i / sum_i w_i                           (Eq. 3)
 *     alpha   = 1 - exp(-sum_i delta_i)                             (Eq. 8)
 *     normal  = R n_f, n_f = N/|N|, N = sum_i w_i n_i / sum_i w_i,
 *               n_i = Sigma_i^-1 (o + v t_i - mu_i) / |...|         (Eq. 17 blended by Eq. 3)
 *     flow_j  = pi(R_j p + t_j) - (x + 1/2, y + 1/2), p = o + v depth,
 *               pi(X) = (fx X0/X2 + cx, fy X1/X2 + cy)              (Sec. 5)
 *   The blend is sort-free: outputs do not depend on the order of the Gaussians.
 *
 * Conventions for every entry point:
 *   - All array pointers are DEVICE pointers owned by the caller, fp32 (or int64
 *     where stated), C-contiguous.  Pointers named h_* are HOST pointers, read
 *     before the call returns.
 *   - The library never allocates device memory.  Scratch memory is the caller's
 *     `workspace` (size from fmb_workspace_bytes, base aligned to 256 bytes).
 *   - Work is enqueued on `stream` and the call returns without synchronising.
 *   - Invalid arguments are reported before anything is enqueued.  No C++ exception
 *     crosses the ABI.  On a non-OK status, fmb_last_error() returns a message
 *     (thread-local, valid until the next call on the same thread).
 *   - Every buffer must hold the elements its description states, in terms of G
 *     (the Gaussians, h_obj_offsets[n_objects]), P_total (the plane entries) and
 *     n_poses.  The library sees pointers only and cannot check their sizes: a
 *     short buffer is read or written past its end.  (The Python binding checks
 *     every tensor's size before it calls.)
 *   - Invalid data that is not checked on the host (lambda <= 0, a singular L, a
 *     flow target point at or behind its camera plane, NaN inputs) gives NaN or Inf
 *     in the affected outputs; it never makes a kernel read or write out of bounds.
 *   - Pose: 12 floats, R (3x3 row-major) then t, world -> camera:
 *     x_cam = R x_world + t; OpenCV axes (x right, y down, z forward).
 *   - Pixel (x, y) of a view is ray (x + 1/2 - cx)/fx, (y + 1/2 - cy)/fy, 1,
 *     normalised; pixels are stored row-major, p = y * W + x.
 *   - Depth is the distance along the unit ray (not z-depth).
 */
#ifndef FMB_H
#define FMB_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A CUDA stream (same type as cudaStream_t / CUstream); NULL = legacy default stream. */
typedef struct CUstream_st* fmb_stream_t;

typedef enum {
  FMB_OK = 0,
  FMB_ERR_INVALID_ARG = 1, /* a size, index, pointer or parameter failed host validation */
  FMB_ERR_CUDA = 2,        /* a CUDA runtime call or kernel launch failed */
  FMB_ERR_TIMEOUT = 3,     /* a bounded device-side wait gave up (see fmb_read_device_status) */
  FMB_ERR_WORKSPACE = 4    /* workspace missing, too small or misaligned */
} fmb_status;

/* Renderer parameters.  beta1, beta2: Eq. 7 (Sec. 7 uses beta1 = 21.4, beta2 = 3.14);
 * eta: the shape scale of Sec. 3.1 (> 0; 1 = no rescaling). */
typedef struct {
  float beta1;
  float beta2;
  float eta;
  int variant;       /* 0 = two-parameter model of Sec. 3.2 (Eq. 7 weights);
                        1 = alpha compositing of Sec. 3.3 (Eq. 9-10 weights, hits sorted by
                        depth per ray; at most 256 Gaussians per object; saved[0] then
                        holds W = sum of the weights instead of the log2 normaliser) */
  int want_normals;  /* 1: compute the blended normal plane (Eq. 17) and its adjoint */
  int n_flow;        /* flow slots per view, 0..2 (Sec. 5: forward i+1 and backward i-1) */
  int deterministic; /* backward: 1 = fixed-order two-stage reduction, 0 = fp32 atomics */
  int use_persistent;/* 1: persistent launch (one grid of resident CTAs popping (view, tile)
                        work items, most expensive first, from a counter in the workspace);
                        0: one CTA per work item */
  int fwd_rays_per_thread; /* tile hints; 0 = library default.  rays per forward thread: 1, 2 or 4 */
  int fwd_threads;         /* 128 */
  int bwd_ray_tile;        /* rays per backward CTA, 32..1024 */
  int bwd_threads;         /* backward threads per CTA: a multiple of 32 up to 160 */
  int store_pairs;   /* 1: stored-intermediate adjoint.  The forward also writes every
                        pair's hit depth t, log2 weight and density (Eq. 2, 4, 7) into
                        the workspace -- 12 bytes per (pixel, Gaussian) pair, what a
                        reverse-mode autodiff of the renderer (the paper's JAX code,
                        Sec. 4) keeps -- and the backward reads them instead of
                        recomputing them.  The backward must then be given the
                        workspace of the forward call of the same batch, unchanged.
                        0 (default): recompute from the saved per-pixel normalisers. */
  int colors;        /* 1: every Gaussian carries an RGB colour, blended by Eq. 3 like the
                        depth (Sec. 3.1) into a colour plane, with its adjoint (the
                        colours and color/g_color/grad_colors arguments are then
                        required / used); 0: no colours (those arguments are ignored).
                        Not with store_pairs. */
  int fwd_ksplit;    /* forward Gaussian splitting, for batches with too few rays to fill
                        the GPU (a ray minibatch, one small view): each of n splits renders
                        a share of every object's Gaussians into per-ray partial sums (32
                        bytes per ray and split, in the workspace), which a second kernel
                        merges (the max-shifted sums of Eq. 3 combine exactly) and turns
                        into the planes.  0 = automatic (up to 6 splits when the ray
                        tiles fill less than half a wave of the GPU and an object has
                        at least 128 Gaussians), 1 = never, 2..8 = that many splits.
                        Two-parameter model only; ignored with colors or store_pairs. */
  int keep_order;    /* variant 1 only.  1: the forward also keeps each ray's depth order
                        of the object's Gaussians (the result of its per-ray sort, Eq. 10)
                        in the workspace -- 32 M bytes per plane entry, M = 2, 4 or 8 for
                        a largest object of at most 64, 128 or 256 Gaussians -- and the
                        backward walks it, four threads per ray, instead of sorting again;
                        a ray whose stored order is not strictly increasing in its own
                        recomputed depths (equal depths; bytes another call left), and every
                        ray of an object of fewer than 8 Gaussians, is sorted afresh, so the
                        gradients do not depend on the workspace's content beyond the
                        rounding of the two summation orders.  Give the backward the workspace of the forward call of the same
                        batch, unchanged (as with store_pairs), for the speed.  0 (default):
                        the backward sorts each ray afresh.  Not with
                        fmb_render_forward_noalloc. */
  int bwd_gblocks;   /* two-parameter backward: Gaussian blocks per object (each block is a
                        CTA per ray tile; more blocks spread a small batch over more SMs, at
                        the price of one set of per-ray records per block).  0 = automatic
                        (the fewest blocks of at most min(2 bwd_threads, 256) Gaussians, or
                        up to three more where they fill the threads better), 1..64 = at
                        least that many (at most one per Gaussian).  A tile hint like
                        bwd_ray_tile: the gradients are the same up to the rounding of their
                        sums.  Ignored by alpha compositing and the loss attribution. */
} fmb_params;

/* One camera view of one object.  Planes of the view start at pixel `pix_offset`
 * of the batched output buffers (see fmb_render_forward).
 *
 * Ray batches (the random ray minibatches of Sec. 4, drawn across all frames):
 * with `rays` set, the view renders only the pixels listed there (device array of
 * n_rays row-major pixel indices y * W + x, any order, repeats allowed; indices
 * outside the image give the rays through those pixel coordinates) and its planes
 * hold n_rays entries in list order instead of W * H.  NULL: the whole image. */
typedef struct {
  int W, H;               /* image size in pixels, >= 1 */
  float fx, fy, cx, cy;   /* pinhole intrinsics; fx, fy > 0 (Sec. 5 uses fx = fy, centred) */
  int object;             /* index of the object (Gaussian range) this view renders */
  int pose;               /* index into poses: the camera's pose */
  int flow_target[2];     /* pose indices of the flow targets of slots 0 and 1, or -1 */
  long long pix_offset;   /* first pixel of this view in the batched planes */
  const int* rays;        /* device: pixel indices of a ray batch, or NULL */
  int n_rays;             /* entries of rays (>= 1 when rays is set) */
  int reserved;           /* 0 */
} fmb_view;

/*
 * Forward render of a batch of views (paper Eq. 2, 3, 4, 7, 8, 17 and Sec. 5 flow).
 *
 * Scene: n_objects objects; object k owns Gaussians [h_obj_offsets[k],
 * h_obj_offsets[k+1]) (host int64 array of n_objects + 1 entries, starting at 0,
 * non-decreasing, every object with >= 1 Gaussian).  means: [G][3]; chol: [G][6]
 * packed (L00, L10, L11, L20, L21, L22); weights: [G] (lambda > 0), with
 * G = h_obj_offsets[n_objects].  colors: [G][3] (params->colors; else ignored,
 * may be NULL).  poses: [n_poses][12].
 *
 * Outputs (device, overwritten for every pixel of every view; P_v = W*H):
 *   depth  [P_total]          depth[pix_offset + p]
 *   alpha  [P_total]          alpha[pix_offset + p]
 *   normal [3*P_total]        per view a [3][P_v] block at 3*pix_offset (camera
 *                             frame, unit length); may be NULL if !want_normals
 *   flow   [2*n_flow*P_total] per view a [n_flow][2][P_v] block at
 *                             2*n_flow*pix_offset, in pixels (u then v); a slot
 *                             whose flow_target is -1 is written as 0; NULL if
 *                             n_flow == 0
 *   color  [3*P_total]        per view a [3][P_v] block at 3*pix_offset: Eq. 3
 *                             with the Gaussians' colours (params->colors; else
 *                             ignored, may be NULL)
 *   saved  [3*P_total]        per view a [3][P_v] block at 3*pix_offset:
 *                             0: log2 of sum_i 2^(e_i log2 e), e_i = beta1 d_i - (beta2/eta) t_i
 *                                (variant 1: W = sum_i w_i)
 *                             1: sum_i delta_i;  2: |N| (0 without normals)
 *                             The backward pass needs it.
 * Views may not overlap in the output planes (checked).
 * workspace: >= fmb_workspace_bytes(...) bytes, 256-byte aligned; its contents
 * are scratch and need not be preserved between calls, except with
 * store_pairs = 1, where the forward leaves the per-pair values there for the
 * backward of the same batch (workspace size then grows by 12 bytes per pair,
 * rounded up: 12 x sum over views of P_v x (K_v rounded up to a multiple of 4)),
 * and with keep_order = 1 (variant 1), where it leaves each ray's depth order
 * there (32 M bytes per plane entry).
 * A Gaussian-split forward (fwd_ksplit, fmb_forward_ksplit) also keeps 32 bytes per
 * ray and split of partial sums there between its two kernels.
 */
fmb_status fmb_render_forward(const fmb_params* params, int n_objects, const long long* h_obj_offsets,
                              const float* means, const float* chol, const float* weights, const float* colors,
                              int n_poses, const float* poses, int n_views, const fmb_view* h_views,
                              float* depth, float* alpha, float* normal, float* flow, float* color, float* saved,
                              void* workspace, size_t workspace_bytes, fmb_stream_t stream);

/*
 * Adjoint of fmb_render_forward (the derivative of the renderer defined above;
 * the paper differentiates its JAX renderer automatically, Sec. 4).  By default it
 * recomputes every ray-Gaussian term from the saved per-pixel log-normaliser
 * instead of storing per-pair values; with store_pairs = 1 it reads the forward's
 * stored t, log2 weight and density from the workspace (the forward call of the
 * same batch must have used this workspace and these params).
 *
 * Inputs: the same scene, poses, views and params as the forward call; the
 * forward's depth, normal (NULL if !want_normals), color (colour mode) and saved
 * planes; the upstream gradients g_depth, g_alpha, g_normal, g_flow, g_color in
 * the layouts of the forward outputs (each may be NULL = zero).
 * Outputs (overwritten, never accumulated): grad_means [G][3], grad_chol [G][6],
 * grad_weights [G] (d/d lambda), grad_colors [G][3] (colour mode), grad_poses
 * [n_poses][12] (d/dR as a free 3x3 matrix, row-major, then d/dt; NULL = pose
 * gradients not computed).
 * deterministic = 1 gives bitwise-reproducible results (fixed-order two-stage
 * reduction through the workspace); 0 uses fp32 atomics.
 */
fmb_status fmb_render_backward(const fmb_params* params, int n_objects, const long long* h_obj_offsets,
                               const float* means, const float* chol, const float* weights, const float* colors,
                               int n_poses, const float* poses, int n_views, const fmb_view* h_views,
                               const float* depth, const float* normal, const float* color, const float* saved,
                               const float* g_depth, const float* g_alpha, const float* g_normal,
                               const float* g_flow, const float* g_color, float* grad_means, float* grad_chol,
                               float* grad_weights, float* grad_colors, float* grad_poses, void* workspace,
                               size_t workspace_bytes, fmb_stream_t stream);

/*
 * fmb_render_forward without a workspace argument, for callers that cannot
 * allocate device memory (a plugin whose host application owns all device memory
 * and exposes no allocator, or a real-time path where cudaMalloc's implicit device
 * synchronisation is not acceptable).  The paper has no counterpart: this is a
 * deployment variant of the same forward render, with the same arguments,
 * layouts and results minus `workspace`/`workspace_bytes`.
 *
 * Its scratch is one fixed 1 MiB array in the library (held on every device that
 * loads the library until the process exits): a batch needs 256 + 64 x (sum over
 * views of the view's Gaussian count) bytes (plus 16 more per view and Gaussian
 * with colours, each region rounded up to 256), and a larger batch is rejected with
 * FMB_ERR_WORKSPACE.  Nothing is allocated.  The first call on each device looks up
 * the array's device address (cudaGetSymbolAddress); make that first call before
 * any stream capture.  All calls share the array: calls whose GPU work overlaps
 * (different streams or host threads) race on it.  The device address is cached
 * per device for the life of the process: after a device reset (cudaDeviceReset,
 * or any teardown of the device's primary context) this entry point must not be
 * called again.  Errors are reported as for fmb_render_forward; the device status
 * word (nonzero when a bounded wait gave up and the planes are invalid) lives in
 * the fixed array, cleared by every call, and is read by fmb_read_noalloc_status.
 */
fmb_status fmb_render_forward_noalloc(const fmb_params* params, int n_objects, const long long* h_obj_offsets,
                                      const float* means, const float* chol, const float* weights,
                                      const float* colors, int n_poses, const float* poses, int n_views,
                                      const fmb_view* h_views, float* depth, float* alpha, float* normal,
                                      float* flow, float* color, float* saved, fmb_stream_t stream);

/* Copies the status word of fmb_render_forward_noalloc's fixed scratch to
 * *h_status and synchronises `stream` (the stream of the call being checked):
 * 0 = no device-side error; nonzero = a bounded wait of that call gave up and its
 * outputs are invalid.  Allocates nothing.  The paper has no counterpart (like
 * fmb_read_device_status, this reports on the execution, not on the method).
 * With calls on several streams in flight, the word is that of whichever call
 * wrote it last. */
fmb_status fmb_read_noalloc_status(int* h_status, fmb_stream_t stream);

/*
 * Oriented point export (Sec. 6: the oriented point set a Poisson surface
 * reconstruction takes; the Poisson solve itself is not part of this library).
 * For every pixel of the batch, from the depth and saved planes of a
 * fmb_render_forward call with the same scene, views and params:
 *   points        [3*P_total] per view a [3][P_v] block at 3*pix_offset: the
 *                 rendered point o + v D (world frame)
 *   normal_tf     same layout: Eq. 17's per-Gaussian normal evaluated at the
 *                 rendered depth D instead of the hit depth, blended by Eq. 3 with
 *                 the variant's weights, unit length and turned to face the camera
 *                 (world frame; 0 where the blend vanishes)
 *   normal_screen same layout: Eq. 16, the normalised cross product of the
 *                 differences to the rendered points of the right and lower
 *                 neighbour pixels (left / upper on the last column / row), turned
 *                 to face the camera (world frame; 0 for one-pixel-wide images)
 *   quality       [P_total]: max_i w_i / sum_j w_j, the direct-intersection quality
 *                 that Sec. 6 thresholds (typically at 0.9)
 * Any output may be NULL.  workspace as for fmb_render_forward (it is rewritten).
 */
fmb_status fmb_render_points(const fmb_params* params, int n_objects, const long long* h_obj_offsets,
                             const float* means, const float* chol, const float* weights, int n_poses,
                             const float* poses, int n_views, const fmb_view* h_views, const float* depth,
                             const float* saved, float* points, float* normal_tf, float* normal_screen,
                             float* quality, void* workspace, size_t workspace_bytes, fmb_stream_t stream);

/*
 * Loss attribution of Sec. 8, the input of the splitting criterion (Eq. 19): for
 * every Gaussian i, attribution[i] = sum over the batch's rays j of
 * ray_loss[j] * w_ij / sum_k w_kj, with the weights of params->variant (Eq. 7 or
 * Eq. 9-10).  The paper averages over a random batch of M rays (about 5 % of the
 * data): give the batch as ray batches (fmb_view.rays) and divide by M.
 * ray_loss: [P_total] in the layout of the depth plane (rays with zero loss are
 * skipped); saved: the forward's saved planes for the same batch and params
 * (two-parameter weights are rebuilt from its log2 normaliser; NULL is allowed for
 * variant 1, which re-renders).  attribution: [G] (overwritten; fp32 atomics, so
 * the summation order varies between runs).  workspace as for fmb_render_forward
 * (rewritten).
 */
fmb_status fmb_loss_attribution(const fmb_params* params, int n_objects, const long long* h_obj_offsets,
                                const float* means, const float* chol, const float* weights, int n_poses,
                                const float* poses, int n_views, const fmb_view* h_views, const float* saved,
                                const float* ray_loss, float* attribution, void* workspace, size_t workspace_bytes,
                                fmb_stream_t stream);

/* Workspace bytes needed by fmb_render_forward and fmb_render_backward for this
 * batch (the larger of the two).  Returns 0 on invalid arguments (see
 * fmb_last_error). */
size_t fmb_workspace_bytes(const fmb_params* params, int n_objects, const long long* h_obj_offsets,
                           int n_views, const fmb_view* h_views);

/* Gaussian splits the two-parameter forward uses for this batch (params->fwd_ksplit
 * resolved: 1 = unsplit; a split forward launches one more kernel, the merge of the
 * per-ray partial sums).  Host-only query, like fmb_workspace_bytes; 0 on invalid
 * input (message in fmb_last_error).  The paper has no counterpart: this reports
 * a launch decision of this implementation. */
int fmb_forward_ksplit(const fmb_params* params, int n_objects, const long long* h_obj_offsets, int n_views,
                       const fmb_view* h_views);

/* Kernel launches one call of this batch enqueues: pass 0 = fmb_render_forward,
 * pass 1 = fmb_render_backward (want_pose: grad_poses given).  Host-only query,
 * like fmb_workspace_bytes; -1 on invalid input (message in fmb_last_error).  The
 * paper has no counterpart: this reports a launch decision of this
 * implementation (the batch is split into launches of at most a fixed number of
 * views: 64, or 256 for a two-parameter forward or backward of more than 64
 * views; a Gaussian-split forward adds a merge; deterministic mode adds the
 * second-stage reductions). */
int fmb_launch_count(const fmb_params* params, int n_objects, const long long* h_obj_offsets, int n_views,
                     const fmb_view* h_views, int pass, int want_pose);

/* Copies the device status word of a workspace to *h_status and synchronises
 * `stream`: 0 = no device-side error; nonzero = a bounded wait gave up (the
 * outputs of that call are invalid).  The word is cleared by every render call. */
fmb_status fmb_read_device_status(const void* workspace, int* h_status, fmb_stream_t stream);

/* Adam hyper-parameters (Kingma & Ba): learning rate, moment decays, epsilon. */
typedef struct {
  float lr;
  float beta1;
  float beta2;
  float eps;
} fmb_adam_params;

/*
 * One fused Adam step, in place, over n fp32 parameters param[0..n) with
 * gradients grad and moment buffers m, v (device, zero-initialised by the caller
 * before the first step).  The paper optimises with Adam (Sec. 4).  Entries
 * [positive_begin, n) are positive parameters (the Gaussian weights lambda): their
 * gradient is taken with respect to log(param) and the update is multiplicative,
 * so they stay positive.  step_counter: device int holding the number of steps
 * taken so far; the call uses step+1 for the bias correction and then increments
 * it on the device, so the call can be captured once in a CUDA graph and replayed.
 * Pack the scene as one buffer [means | chol | weights] (3G + 6G + G floats) and
 * pass positive_begin = 9G.  Returns FMB_ERR_INVALID_ARG on bad arguments.
 */
fmb_status fmb_adam_step(const fmb_adam_params* p, float* param, const float* grad, float* m, float* v,
                         long long n, long long positive_begin, int* step_counter, fmb_stream_t stream);

/* ALU throughput probe (a measurement utility, not part of the paper's method):
 * launches `blocks` CTAs of 256 threads that each run 8 independent chains of
 * `iters` operations of one kind -- 0: FP32 FMA, 1: packed FP32x2 FMA (two FMAs per
 * instruction), 2: ex2.approx, 3: rcp.approx, 4: rsqrt.approx -- and store one float
 * per thread into `out` (device, >= blocks * 256 floats).  Time it with events on
 * `stream` to get the GPU's FP32-pipe and SFU rates.  Returns FMB_ERR_INVALID_ARG
 * on bad arguments, FMB_ERR_CUDA if the launch fails. */
fmb_status fmb_probe_alu(int kind, int blocks, int iters, float* out, fmb_stream_t stream);

/* Message for the last non-OK status returned on this thread ("" if none). */
const char* fmb_last_error(void);

/* Library version string. */
const char* fmb_version(void);

/* Fills *p with the default parameters (beta1 21.4, beta2 3.14, eta 1, normals on,
 * one flow slot, atomics, plain launch, default tiles). */
void fmb_default_params(fmb_params* p);

#ifdef __cplusplus
}
#endif

#endif /* FMB_H */
