/*
 * fbp.h - C ABI of the GB300 library for accelerated filtered back projection
 * (IIR ramp filtering + fast Hough transform back projection; Dolmatova, Chukalina and
 * Nikolaev, "Accelerated FBP for computed tomography image reconstruction",
 * arXiv 2007.06289).
 *
 * Data (all float32, row-major, C order):
 *   sinogram  [count][K][M]    angle theta_k = k*pi/K, detector offset r_m = m - (M-1)/2
 *                              pixels; a value is the line integral over
 *                              {(x-c0) cos(theta) + (y-c0) sin(theta) = r}, c0 = (N-1)/2
 *   filtered  [count][K][M]    the ramp-filtered sinogram (Eq. 12)
 *   linogram  [count][4][N][2N] quarters in the order v-, v+, h-, h+ (Sec. 4.1); row i holds
 *                              lines of slope sigma_i = i/(N-1); column c holds intercept
 *                              u = c (v-, h-) or u = N-1-c (v+, h+); rows are pre-weighted
 *   image     [count][N][N]    f[y][x], pixel centres at integer (x, y)
 *
 * Conventions shared by every call:
 *   - N is a power of two with 2 <= N <= 4096; K >= 2 and M >= 2 are free.
 *   - Device pointers are owned by the caller, must be 16-byte aligned (else
 *     FBP_ERR_MISALIGNED) and must not overlap unless a call says so.  Rows need not be
 *     aligned.
 *   - Every call is asynchronous on `stream` (a cudaStream_t; NULL is the legacy default
 *     stream).  Arguments are validated before anything is launched: a call that returns
 *     FBP_ERR_INVALID_ARG, FBP_ERR_MISALIGNED or FBP_ERR_UNSUPPORTED has launched nothing.
 *     A CUDA launch failure returns FBP_ERR_CUDA (earlier launches of the same call may
 *     already be queued).
 *   - A plan is not thread-safe: calls on one plan must be issued from one host thread.
 *     Calls that use the plan's workspace must not overlap on the GPU (issue them on one
 *     stream, or order them with events).
 *   - No call throws.  No call synchronises the device except fbp_plan_destroy,
 *     fbp_last_device_error and the allocations a plan makes on first use (its workspace,
 *     the adjoint workspace, the SIRT tables) or when a larger chunk needs a larger one.
 */
#ifndef FBP_H
#define FBP_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fbp_plan_s* fbp_plan_t;

typedef enum {
    FBP_OK = 0,
    FBP_ERR_INVALID_ARG = 1,   /* null pointer, bad size, bad coefficient set */
    FBP_ERR_UNSUPPORTED = 2,   /* N not a power of two in [2, 4096], filter order > 8 */
    FBP_ERR_MISALIGNED = 3,    /* a pointer is not 16-byte aligned */
    FBP_ERR_OOM = 4,           /* device or host allocation failed */
    FBP_ERR_CUDA = 5,          /* a CUDA runtime call or launch failed */
    FBP_ERR_TIMEOUT = 6,       /* a bounded wait inside a kernel gave up */
    FBP_ERR_INTERNAL = 7       /* a kernel's own consistency check failed */
} fbp_status;

#define FBP_MAX_ORDER 8

/* Coefficients of the causal recursive filter of Eq. 9 / Eq. 13:
 *   y(n) = sum_{k<mb} b[k] p(n-k) - sum_{k=1..q} a[k-1] y(n-k),
 * used unchanged (a+ = a-, b+ = b-, text after Eq. 13) by the anticausal filter.
 * 1 <= mb <= 8, 0 <= q <= 8; entries past mb / q are ignored.  The filter must be stable
 * with distinct poles (roots of z^q + a[0] z^(q-1) + ... + a[q-1] strictly inside the unit
 * circle and pairwise separated); fbp_plan checks both.
 * The plan turns the coefficients (in float64) into the same transfer function in
 * parallel form, sum_j r_j / (1 - p_j z^-1) plus direct taps, and the kernels run that form
 * in float32: rounding the direct-form a[] to float32 can move poles near z = 1 outside
 * the unit circle, while poles and residues round harmlessly. */
typedef struct {
    int mb;
    int q;
    double b[FBP_MAX_ORDER];
    double a[FBP_MAX_ORDER];
} fbp_iir_coeffs;

/* Built-in coefficients fitted for image size N and order q = mb = `order` (2..6) by a
 * simplex search on the weighted response error (Sec. 3, text after Eq. 13).
 * order <= 0 selects the default order 3 (the paper's setting, Sec. 5).
 * Errors: FBP_ERR_INVALID_ARG (out == NULL), FBP_ERR_UNSUPPORTED (no table entry). */
fbp_status fbp_default_coeffs(int N, int order, fbp_iir_coeffs* out);

/* Create a plan for slices of an N x N image from K angles x M bins, `batch` slices per
 * call.  coeffs == NULL selects fbp_default_coeffs(N, 0).  fuse_k is the number of Hough
 * stages done by the first back-projection pass (1..6, at least 2 when it leaves stages to a
 * second pass, which takes at most 6; 0 chooses).  The plan builds its
 * per-row geometry tables (Eq. 14-15) on the host in float64 and uploads them; it
 * allocates no workspace yet.  The current CUDA device at creation is the plan's device.
 * Errors: FBP_ERR_INVALID_ARG, FBP_ERR_UNSUPPORTED, FBP_ERR_OOM, FBP_ERR_CUDA. */
fbp_status fbp_plan(fbp_plan_t* out, int N, int K, int M, int batch,
                    const fbp_iir_coeffs* coeffs, int fuse_k);

/* Synchronise the plan's device, free everything the plan owns.  NULL is accepted. */
fbp_status fbp_plan_destroy(fbp_plan_t plan);

/* Bytes of device workspace that fbp_reconstruct, fbp_fht_backproject,
 * fbp_reconstruct_host and fbp_direct_reconstruct need (0 if plan == NULL). */
size_t fbp_workspace_bytes(fbp_plan_t plan);

/* Slices per kernel sequence (1 .. batch, at most 4096; 0 restores the default: 16 slices,
 * fewer where their first-pass buffers would pass 4 GiB).  Every launch of the fused
 * pipeline then covers `chunk` slices (fbp_reconstruct_host stages at most 2 slices per
 * copy); results do not depend on it, bit for bit.  Changes fbp_workspace_bytes, so it must
 * come before the plan has a workspace.  No counterpart in the paper (an execution knob).
 * Errors: FBP_ERR_INVALID_ARG (NULL plan, chunk out of range, workspace already present). */
fbp_status fbp_set_chunk(fbp_plan_t plan, int chunk);

/* Hand the plan a caller-owned device workspace of at least fbp_workspace_bytes bytes
 * (16-byte aligned).  Without one the plan allocates its own on first use (cudaMalloc),
 * which must then not happen inside a CUDA graph capture.  d_ws == NULL drops a caller
 * workspace (the plan will allocate on next use).
 * Errors: FBP_ERR_INVALID_ARG (too small), FBP_ERR_MISALIGNED. */
fbp_status fbp_set_workspace(fbp_plan_t plan, void* d_ws, size_t bytes);

/* Eq. 12-13: filtered = causal + anticausal recursive filtering of every projection row,
 * zero state outside [0, M).  d_sino [batch][K][M] -> d_filt [batch][K][M]; the two may be
 * the same buffer. */
fbp_status fbp_filter_iir(fbp_plan_t plan, const float* d_sino, float* d_filt, void* stream);

/* Eq. 8 with L0 = M-1: the exact (non-recursive) ramp filter of every projection row,
 * p~(n) = sum_{|k| <= M-1} h(k) p(n-k), h of Eq. 7 -- the filter of the direct FBP
 * comparator, exposed so that the fast back projection can be run on exactly filtered data
 * (which separates the recursive filter's share of the error from the dyadic lines').
 * d_sino [batch][K][M] -> d_filt [batch][K][M] (distinct buffers).  Theta(K M^2). */
fbp_status fbp_filter_fir(fbp_plan_t plan, const float* d_sino, float* d_filt, void* stream);

/* Sec. 4.1-4.2, Eq. 14-15: bilinear resampling of the filtered sinogram into the four
 * weighted linogram quarters.  d_filt [batch][K][M] -> d_lin [batch][4][N][2N]; every
 * entry of d_lin is written. */
fbp_status fbp_resample_st(fbp_plan_t plan, const float* d_filt, float* d_lin, void* stream);

/* Sec. 4.4-4.5, Eq. 16-22: fast Hough transform of every quarter along dyadic patterns and
 * the sum of the four quarter images, (F_v- + F_v+) + (F_h- + F_h+), in float32.
 * d_lin [batch][4][N][2N] (read only) -> d_img [batch][N][N].  Uses the workspace.
 * Only linogram entries with column c <= N-1+i can reach the image. */
fbp_status fbp_fht_backproject(fbp_plan_t plan, const float* d_lin, float* d_img, void* stream);

/* The whole method: fbp_filter_iir, fbp_resample_st and fbp_fht_backproject composed, with
 * the linogram never written to memory.  d_sino [batch][K][M] -> d_img [batch][N][N].
 * The result equals the composition of the three calls bit for bit.  Uses the workspace. */
fbp_status fbp_reconstruct(fbp_plan_t plan, const float* d_sino, float* d_img, void* stream);

/* fbp_reconstruct from and to HOST memory: copies `count` slices (any count >= 1) of
 * h_sino [count][K][M] to the device, reconstructs and copies h_img [count][N][N] back,
 * pipelining copies and compute over chunks of slices on internal streams ordered after
 * `stream`; `stream` is ordered after the last copy.  Host buffers should be pinned
 * (cudaHostAlloc / cudaHostRegister) for the copies to overlap.  Uses the workspace. */
fbp_status fbp_reconstruct_host(fbp_plan_t plan, const float* h_sino, float* h_img, int count,
                                void* stream);

/* ------------------------------------------------------------------ adjoints
 * The fast reconstruction is linear in the sinogram, f = H(L(F p)) (F: Eq. 12-13, L:
 * Eq. 14-15, H: Eq. 16-22); these are its transposes, for gradients with respect to the
 * sinogram.  The filter is symmetric (causal + anticausal with zero state at both ends), so
 * fbp_filter_iir is its own adjoint.  Layouts as in the forward calls; `batch` slices.
 * The first call allocates an adjoint workspace (chunk x (2 linograms + 1 sinogram)). */

/* H^T: image gradient d_img_grad [batch][N][N] -> linogram gradient d_lin_grad
 * [batch][4][N][2N] (every entry written; zero where no pattern reaches).  Float32, the
 * stage recursion transposed: bit-reproducible.  Errors as fbp_fht_backproject. */
fbp_status fbp_fht_backproject_adjoint(fbp_plan_t plan, const float* d_img_grad,
                                       float* d_lin_grad, void* stream);

/* Eq. 17, the forward direction: the fast Hough (discrete Radon) transform of images
 * d_img [batch][N][N] in linogram coordinates, d_lin [batch][4][N][2N]: entry [q][i][c] is
 * the sum of the image's pixels along the dyadic line of quarter q, slope i/(N-1) and
 * intercept c (the '+' quarters stored flipped as in the back projection).  It is the
 * transpose of the back projection (the same kernels as fbp_fht_backproject_adjoint), so
 * <fbp_hough_project(f), L> = <f, fbp_fht_backproject(L)>.  No filtering, no resampling. */
fbp_status fbp_hough_project(fbp_plan_t plan, const float* d_img, float* d_lin, void* stream);

/* L^T: linogram gradient [batch][4][N][2N] -> filtered-sinogram gradient [batch][K][M]
 * (every entry overwritten): each sample's gradient times its four bilinear weights (the
 * forward's float32 weights and fixed-point positions), gathered per detector bin in a fixed
 * order, no atomics: bit-reproducible from run to run. */
fbp_status fbp_resample_st_adjoint(fbp_plan_t plan, const float* d_lin_grad,
                                   float* d_filt_grad, void* stream);

/* (H L F)^T = F L^T H^T: image gradient [batch][N][N] -> sinogram gradient [batch][K][M]
 * (bit-reproducible: all three steps are). */
fbp_status fbp_reconstruct_adjoint(fbp_plan_t plan, const float* d_img_grad,
                                   float* d_sino_grad, void* stream);

/* ------------------------------------------------------------------ algebraic reconstruction
 * The iterative method the paper points to beside its fast FBP (Sec. 4.4: an algebraic
 * reconstruction built on the fast Hough transform), in its simultaneous form (SIRT) on the
 * same operators: A = fbp_hough_project (dyadic line sums of an image), A^T =
 * fbp_fht_backproject (back projection of a linogram).
 *
 * fbp_hough_data: sinograms d_sino [batch][K][M] -> Hough-space data d_lin [batch][4][N][2N]
 * (every entry written): the sinogram sampled bilinearly at the linogram points (Eq. 14-15,
 * the resampling's positions and angle interpolation, zero outside the detector) divided by
 * the path length per row sqrt(1 + sigma^2), since a dyadic line visits one pixel per row;
 * no filter and no row weights.  For an image f, A f approximates fbp_hough_data of its
 * sinogram.
 *
 * fbp_sirt: `iters` steps of f <- f + lambda C^-1 A^T (R^-1 (b - A f)), R = A 1 (pixels on
 * each line), C = A^T 1 (lines through each pixel), entries where R or C vanishes left out,
 * on images d_img [batch][N][N] (in: the starting image, e.g. zeros or the fast FBP; out:
 * the result) for data d_lin_data [batch][4][N][2N].  0 < lambda < 2 (else
 * FBP_ERR_INVALID_ARG); iters >= 0.  Float32.  The first call makes the plan's R^-1 and
 * C^-1 tables (one slice, 40 N^2 bytes) on its stream: a later call on another stream must
 * be ordered after it.  Uses both workspaces.  Errors as fbp_reconstruct. */
fbp_status fbp_hough_data(fbp_plan_t plan, const float* d_sino, float* d_lin, void* stream);

/* Fast (approximate) Radon transform: images d_img [batch][N][N] -> sinograms d_sino
 * [batch][K][M] (every entry written), theta_k = k pi / K, r_m = m - (M-1)/2.  The dyadic
 * line sums of fbp_hough_project (Eq. 17) resampled: for each theta_k its line class and
 * slope sigma, the two linogram rows around sigma (N-1) read at the column of offset r_m
 * (linear in the column), mixed linearly in the slope, times the path length per row
 * sqrt(1 + sigma^2).  Uses the adjoint workspace.  Errors as fbp_reconstruct. */
fbp_status fbp_radon(fbp_plan_t plan, const float* d_img, float* d_sino, void* stream);
fbp_status fbp_sirt(fbp_plan_t plan, const float* d_lin_data, float* d_img, int iters,
                    float lambda, void* stream);

/* ------------------------------------------------------------------ learned corrector
 * A residual CNN applied after the fast reconstruction, y = x + net(x): six 3x3
 * convolutions (1 -> 32 -> 32 -> 32 -> 32 -> 32 -> 1 channels, zero padding, ReLU between),
 * trained to map fast images towards direct-FBP images.  No counterpart in the paper: a
 * learned extension.  Parameters: one fp32 device array of fbp_cnn_param_count() floats,
 * layer after layer, each layer's weights [co][ci][3][3] then its biases [co].  The four
 * 32 -> 32 layers run as bf16 implicit GEMMs on the tcgen05 tensor cores (accumulators in
 * tensor memory, fp32; operands staged by bulk copies), hidden activations and gradients
 * stored as bf16.  The 32 -> 1 layer runs on the tensor cores too, its fp32 weights split
 * exactly into three bf16 parts, and so do the hidden layers' weight gradients (fp32
 * accumulation over all pixels); the first layer and the 1-channel layers' weight
 * gradients run in fp32 on the CUDA cores.  Images:
 * [batch][N][N] fp32, N a power of two in 16..4096.  The caller provides the workspace
 * (16-byte aligned).  Calls that share a workspace must not overlap on the GPU. */
size_t fbp_cnn_param_count(void);

/* Workspace bytes for `batch` images of N x N; train != 0 keeps the activations for
 * fbp_cnn_backward.  0 for unsupported sizes. */
size_t fbp_cnn_workspace_bytes(int N, int batch, int train);

/* d_y = d_x + net(d_x).  With train != 0 the activations stay in the workspace for a
 * following fbp_cnn_backward on the same images.  Errors: FBP_ERR_UNSUPPORTED (N),
 * FBP_ERR_INVALID_ARG (NULL, workspace too small), FBP_ERR_MISALIGNED, FBP_ERR_CUDA. */
fbp_status fbp_cnn_forward(const float* d_params, const float* d_x, float* d_y, void* d_ws,
                           size_t ws_bytes, int N, int batch, int train, void* stream);

/* Gradient of a loss with respect to the parameters, given its gradient d_gy with respect
 * to the output of the preceding fbp_cnn_forward(train = 1) call on the same workspace and
 * images: d_gparams [fbp_cnn_param_count()] is overwritten (float atomics: the last bits
 * depend on the order of the additions). */
fbp_status fbp_cnn_backward(const float* d_params, const float* d_x, const float* d_gy,
                            float* d_gparams, void* d_ws, size_t ws_bytes, int N, int batch,
                            void* stream);

/* Synchronise the current device and read (then clear) the corrector's device status word:
 * FBP_ERR_TIMEOUT if a tensor-core convolution gave up a bounded wait (about a second) for
 * its copies or its matrix products since the last read -- its output is then incomplete --;
 * in the library built with FBP_BOUNDS_CHECK (libfbp_checked.so), FBP_ERR_INTERNAL if a
 * corrector kernel formed an index or a bulk-copy range outside its buffer (the access is
 * skipped); else FBP_OK.  The first code recorded wins.  FBP_ERR_CUDA if the device cannot
 * be read. */
fbp_status fbp_cnn_last_error(void);

/* ------------------------------------------------------------------ ragged volumes
 * A volume whose slices differ in size (N, K, M), each slice in its own buffers.  No
 * counterpart in the paper (which reconstructs one slice at a time); an execution layer
 * over the same pipeline. */
typedef struct {
    int N, K, M;            /* image size (power of two, 2..4096), angles, detector bins */
    const float* d_sino;    /* device [K][M], 16-byte aligned, caller-owned */
    float* d_img;           /* device [N][N], 16-byte aligned, caller-owned */
} fbp_item;

typedef struct fbp_volume_s* fbp_volume_t;

enum { FBP_VOLUME_GRAPH = 1 };  /* capture the whole volume into a CUDA graph, replay it */

/* Executor for `count` items: items are grouped by (N, K, M); each group gets a plan with
 * the built-in coefficients of its N (order `order`, 0 = default), device tables of its
 * items' pointers, a workspace and a stream.  All device memory is allocated here.
 * fbp_volume_run then reconstructs every item (each image bit-identical to reconstructing
 * that slice alone with fbp_reconstruct).  The item array is copied; the buffers it points
 * to must stay valid while the volume is used.
 * Errors: FBP_ERR_INVALID_ARG (NULL, count < 1, K or M < 2, unknown flags),
 * FBP_ERR_MISALIGNED, FBP_ERR_UNSUPPORTED (N), FBP_ERR_OOM, FBP_ERR_CUDA. */
fbp_status fbp_volume_create(fbp_volume_t* out, const fbp_item* items, int count, int order,
                             int flags);

/* Reconstruct every item, asynchronously on `stream` (the groups run on internal streams
 * forked from and joined back into `stream`).  With FBP_VOLUME_GRAPH the first call
 * captures the work into a CUDA graph and every call launches that graph; `stream` must
 * then be a created stream (not the legacy or per-thread default: FBP_ERR_INVALID_ARG). */
fbp_status fbp_volume_run(fbp_volume_t v, void* stream);

/* Autotuner: for every group, times the supported first-pass fusion depths and 1, 2, 4, 8,
 * 16 slices per launch (up to the group's size) on the volume's own items, on `stream`,
 * and keeps the fastest pair.  Synchronous.  Overwrites the items' images (with the same
 * bits every choice gives).  fuse_k_out / chunk_out (optional, [groups]) receive the
 * choices.  A captured graph is dropped and re-captured by the next run. */
fbp_status fbp_volume_tune(fbp_volume_t v, void* stream, int* fuse_k_out, int* chunk_out);

/* Number of groups and the total workspace bytes of their plans. */
fbp_status fbp_volume_info(fbp_volume_t v, int* groups, size_t* workspace_bytes);

/* Shape, item count, fusion depth and slices per launch of group `group` (groups are
 * numbered in order of their first item). */
fbp_status fbp_volume_group(fbp_volume_t v, int group, int* N, int* K, int* M, int* items,
                            int* fuse_k, int* chunk);

/* Free everything the volume owns (waits for the device first).  NULL is a no-op. */
fbp_status fbp_volume_destroy(fbp_volume_t v);

/* Allocation-free variant of fbp_fht_backproject, for callers that cannot allocate device
 * memory (code running inside another framework's memory pool, plugins handed only their
 * input and output buffers, real-time loops where an allocation may stall or fail): it
 * needs no plan and no workspace.  The paper has no counterpart; this is an interface
 * convenience.  d_lin [count][4][N][2N] (read only) -> d_img [count][N][N], same layout
 * and bit-identical results as fbp_fht_backproject.
 * Its scratch is a fixed device array inside the library, sized for one slice of N up to
 * FBP_STATIC_MAX_N (8 MiB), which every GPU that loads the library holds until the process
 * exits; slices are processed one after another through it.  No call allocates or frees
 * memory.  The first call on a device looks up the array's device address and sets the
 * kernels' shared-memory limits for that device, so make it before any stream capture;
 * with lazy module loading the driver may back the array with device memory only at that
 * lookup, so the first call on a device can fail with FBP_ERR_OOM when the device is full
 * (later calls cannot).
 * All calls share the array: calls that overlap on the GPU race (issue them on one stream
 * or order them with events).
 * Errors: FBP_ERR_UNSUPPORTED (N not a power of two in [2, FBP_STATIC_MAX_N]),
 * FBP_ERR_INVALID_ARG (count < 1, null pointer), FBP_ERR_MISALIGNED, FBP_ERR_OOM (first
 * call on a device only), FBP_ERR_CUDA. */
#define FBP_STATIC_MAX_N 512
fbp_status fbp_fht_backproject_static(int N, int count, const float* d_lin, float* d_img,
                                      void* stream);

/* Comparator, not the paper's method: direct Theta(N^3) FBP (Eq. 3-5 with the exact FIR
 * ramp of Eq. 8, L0 = M-1, and pixel-driven linear-interpolation back projection,
 * f = (pi/K) sum_k p~_k((x-c0) cos theta_k + (y-c0) sin theta_k)).
 * d_sino [batch][K][M] -> d_img [batch][N][N].  Uses the workspace. */
fbp_status fbp_direct_reconstruct(fbp_plan_t plan, const float* d_sino, float* d_img,
                                  void* stream);

/* Plan shape: any output pointer may be NULL. */
fbp_status fbp_plan_info(fbp_plan_t plan, int* N, int* K, int* M, int* batch, int* fuse_k,
                         int* chunk);

/* Kernels of the library, for fbp_profile_read.  The paper has no counterpart: these are
 * measurement hooks. */
typedef enum {
    FBP_KERNEL_IIR = 0,            /* recursive ramp filter (Eq. 12-13) */
    FBP_KERNEL_RESAMPLE = 1,       /* stand-alone resampling (fbp_resample_st) */
    FBP_KERNEL_PASS1_RESAMPLE = 2, /* resampling fused with the first Hough pass */
    FBP_KERNEL_PASS1_LINOGRAM = 3, /* first Hough pass reading a stored linogram */
    FBP_KERNEL_PASS2 = 4,          /* second Hough pass, v quarters (stores F_v- + F_v+) */
    FBP_KERNEL_FIR = 5,            /* comparator: exact FIR ramp */
    FBP_KERNEL_DIRECT_BP = 6,      /* comparator: pixel-driven back projection */
    FBP_KERNEL_PASS2_H = 7,        /* second Hough pass, h quarters (adds F_h- + F_h+) */
    FBP_KERNEL_COUNT = 8
} fbp_kernel_id;

/* Measurement hooks (no counterpart in the paper).  The plan always counts the kernels it
 * launches.  With profiling enabled it also records a pair of CUDA events around every
 * launch, on the stream the kernel is launched on (events are created lazily, so enable
 * profiling outside any CUDA graph capture).  fbp_profile_read synchronises on the last
 * recorded event and returns, for one kernel id, the summed event-timed duration in ms and
 * the number of launches since the last reset.  fbp_profile_reset clears both. */
fbp_status fbp_profile_enable(fbp_plan_t plan, int enable);
fbp_status fbp_profile_reset(fbp_plan_t plan);
fbp_status fbp_profile_read(fbp_plan_t plan, int kernel, double* total_ms, long long* launches);

/* Static text for a status code. */
const char* fbp_status_str(fbp_status status);

/* Synchronise the plan's device and read (then clear) the plan's device status word:
 * FBP_ERR_INTERNAL when a kernel rejected a geometry-table row naming an angle row outside
 * the sinogram (checked in every build; the row is resampled as zeros) or, in the library
 * built with FBP_BOUNDS_CHECK (libfbp_checked.so, include/fbp_check.h), an index outside its
 * buffer or Hough tile in a kernel of the reconstruction, its adjoints, the Hough-space
 * data, the fast Radon transform or SIRT (the access is skipped); FBP_ERR_TIMEOUT when a
 * second-pass CTA gave up its bounded wait (about a second) for its bulk row copies (its
 * output tile is then wrong); FBP_OK if none since the last read.  The corrector's kernels
 * report through fbp_cnn_last_error. */
fbp_status fbp_last_device_error(fbp_plan_t plan);

#ifdef __cplusplus
}
#endif

#endif /* FBP_H */
