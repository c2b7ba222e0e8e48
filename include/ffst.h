/*
 * ffst.h - C ABI of the GB300-native Fast Finite Shearlet Transform (FFST).
 *
 * The transform follows Haeuser & Steidl, "Fast Finite Shearlet Transform:
 * a tutorial" (arXiv:1202.1773):
 *   forward  c_i = ifft2( psi_hat_i * fft2(f) ),  i = 0..eta-1     (Sec. 3.1, eq. shearletTransform)
 *   inverse  f   = ifft2( sum_i psi_hat_i * fft2(c_i) / sum_i psi_hat_i^2 )  (Sec. 3.3, eq. inverseShearletTransform)
 *   adjoint  f   = ifft2( sum_i psi_hat_i * fft2(c_i) )                      (Sec. 3.2, U^T of eq. shearlet_transform_as_matrix)
 * with the cone-adapted Meyer shearlets of Sec. 2 on the grid of Sec. 3.5.1,
 * the plane order of Sec. 3.5.2 and the real-coefficient mirroring of
 * Sec. 3.8.1 (always on).  All arithmetic is FP32 on the device; FP64 is
 * used only on the host, once per plan, for twiddle and window tables.
 *
 * Conventions shared by every entry point:
 *  - Images are row-major rows x cols float32 (M x N).  Row index m1 goes
 *    with omega_2, column index m2 with omega_1 (Sec. 3.5.2: "the first both
 *    components refer to the omega_2 and omega_1 coordinates").
 *  - A coefficient or spectra stack is plane-major [eta][rows][cols]: plane i
 *    is one contiguous row-major M x N image, planes in the order of Sec. 3.5.2.
 *  - All pointers named "device" must be device memory of the current CUDA
 *    device, allocated and owned by the caller.  The plan owns its own
 *    workspace and tables and frees them in ffst_destroy.
 *  - Calls that take a stream are asynchronous and stream-ordered: they only
 *    enqueue kernels on `stream` (a cudaStream_t, NULL = legacy default
 *    stream); no host<->device copies and no synchronisation.  Two calls on
 *    the same plan must not run concurrently (they share the workspace).
 *  - Errors are returned as ffst_status codes; nothing is thrown across the
 *    ABI.  ffst_last_error() returns a thread-local message for the last
 *    failing call on the calling thread.  Argument errors are detected on the
 *    host before anything is enqueued; FFST_ERR_CUDA reports a failed CUDA
 *    runtime call (launch or allocation), after which the outputs are
 *    unspecified.
 *  - Supported sizes: 8 <= rows, cols <= 4096, odd and prime sizes included;
 *    scales in 1..8 (or <= 0 for the default j0 of Sec. 3.1).  Columns of a
 *    height that is a power of two or one of 240, 320, 384, 480, 640, 768,
 *    and rows of a width that is twice one of those, run native FFT lines;
 *    any other height or width runs generic lines and never the fused or
 *    persistent launches: a length with no prime factor above 7 (up to 4096)
 *    as mixed-radix passes in shared memory, any other length (up to 2048)
 *    as Bluestein lines (a DFT of length n as a chirp convolution through
 *    power-of-two FFTs, several times slower per line; the environment
 *    variable FFST_BLUESTEIN=1 at plan creation selects them for every
 *    generic length).  Other sizes return FFST_ERR_UNSUPPORTED_SIZE.
 *    ffst_forward_noalloc keeps its own limits (powers of two).
 */
#ifndef FFST_H
#define FFST_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ffst_plan_s* ffst_plan_t;

typedef enum {
  FFST_OK = 0,
  FFST_ERR_INVALID_ARG = 1,      /* null pointer, bad index, bad storage code   */
  FFST_ERR_UNSUPPORTED_SIZE = 2, /* rows/cols/scales outside the supported set  */
  FFST_ERR_OUT_OF_MEMORY = 3,    /* device or host allocation failed            */
  FFST_ERR_CUDA = 4,             /* a CUDA runtime call failed                  */
  FFST_ERR_TIMEOUT = 5,          /* a bounded device-side wait ran out          */
  FFST_ERR_BOUNDS = 6            /* a checked build (FFST_CHECK) caught an index outside its buffer */
} ffst_status;

/* Storage type of a coefficient stack.  Arithmetic is FP32 in every case. */
typedef enum {
  FFST_STORE_F32 = 0,  /* float32 coefficients, plane_scale unused (may be NULL) */
  FFST_STORE_F16 = 1,  /* IEEE half: stores c_i * s_i, s_i a power of two       */
  FFST_STORE_BF16 = 2  /* bfloat16: stores c_i * s_i                             */
} ffst_storage;

/* Plane kinds returned by ffst_plane_index (kappa of Sec. 3.1). */
enum { FFST_CONE_LOWPASS = 0, FFST_CONE_H = 1, FFST_CONE_V = 2, FFST_CONE_SEAM = 3 };

/* Shearlet constructions (ffst_plan_ex). */
enum {
  FFST_VARIANT_CLASSIC = 0, /* Sec. 3.1: radial factor psi1 of one axis per cone, cone low-pass  */
  FFST_VARIANT_SMOOTH = 1   /* Sec. 3.4: 2-D radial factor Psi1 (eq. newPsi1), tensor low-pass */
};

/* Auxiliary function v of every window (ffst_plan_ex); each satisfies
 * v(x) + v(1 - x) = 1, so every choice keeps the Parseval frame. */
enum {
  FFST_V_MEYER = 0,     /* Sec. 2.1 eq. (v): 35x^4 - 84x^5 + 70x^6 - 20x^7 (C^3 shearlets)       */
  FFST_V_QUADRATIC = 1, /* Sec. 2.1: 2x^2 on [0, 1/2], 1 - 2(1-x)^2 on [1/2, 1]                  */
  FFST_V_POLY = 2,      /* Sec. 3.4 remark: v' = c x^k (x-1)^k, v(1) = 1, k = vorder in 1..7 (C^k) */
  FFST_V_CINF = 3       /* Sec. 3.4 remark: s(x-1)/(s(x-1)+s(x)), s(x) = e^{-1/(1+x)^2 - 1/(1-x)^2} */
};

/* Extent of the frequency grid (ffst_plan_ex), the maxScale option of Sec. 3.5.3. */
enum {
  FFST_MAXSCALE_MAX = 0, /* X = 2^{2 j0 - 1} (X_3 of Sec. 3.5.1: the largest finest scale)  */
  FFST_MAXSCALE_MIN = 1  /* X = 2^{2 j0 - 2} (X_2 of Sec. 3.5.1: the smallest finest scale) */
};

/* Grid step of a non-square image (ffst_plan_ex), Sec. 3.5.1.  Both give a
 * Parseval frame and coincide for square images. */
enum {
  FFST_SPACING_COMMON = 0,  /* one step Delta = X / floor(max(M, N)/2) for both axes: the lattice lies
                               in [-Y, Y] x [-X, X] with Y <= X (Sec. 3.5.1's X >= Y, its single Delta
                               with 1/4 < Delta <= 1, and psi(Delta omega) on Omega); what ffst_plan builds */
  FFST_SPACING_PER_AXIS = 1 /* each axis spans [-X, X] with its own step X / floor(L/2) */
};

/*
 * Build a plan for rows x cols images with `scales` scales (j0 of Sec. 3.1;
 * <= 0 selects j0 = floor(1/2 log2 max(rows, cols))).  The number of planes
 * is eta = 2^(j0+2) - 3 (Sec. 3.5.2).  Generates the FP64 window/twiddle
 * tables on the host, uploads them, computes every plane's spectral support
 * on the device (synchronously, on an internal stream) and allocates the
 * workspace.  Uses the current CUDA device.  On success *out owns all of it.
 */
ffst_status ffst_plan(int rows, int cols, int scales, ffst_plan_t* out);

/*
 * As ffst_plan, with the paper's construction options:
 *   variant    FFST_VARIANT_CLASSIC (what ffst_plan builds) or
 *              FFST_VARIANT_SMOOTH, the smooth shearlets of Sec. 3.4 eqs.
 *              (newPsi1), (smoothPsi): every plane's radial factor is
 *              Psi1(4^-j xi) = sqrt(Phi(4^-j xi / 4)^2 - Phi(4^-j xi)^2) with
 *              the tensor scaling function Phi = varphi x varphi of Sec. 2.4
 *              eq. (Phi), which is also the low-pass;
 *   vfun       the auxiliary function v (FFST_V_*), vorder its order k for
 *              FFST_V_POLY (ignored otherwise);
 *   max_scale  FFST_MAXSCALE_MAX (X = 2^{2 j0 - 1}, what ffst_plan builds) or
 *              FFST_MAXSCALE_MIN (X = 2^{2 j0 - 2});
 *   spacing    FFST_SPACING_COMMON (what ffst_plan builds) or
 *              FFST_SPACING_PER_AXIS, the grid step of non-square images.
 * Same planes, order and Parseval property; every transform entry point works
 * on any combination.  FFST_ERR_INVALID_ARG for codes outside these sets or
 * vorder outside 1..7 with FFST_V_POLY.
 */
ffst_status ffst_plan_ex(int rows, int cols, int scales, int variant, int vfun, int vorder, int max_scale,
                         int spacing, ffst_plan_t* out);

/* Query a plan.  Any output pointer may be NULL. */
ffst_status ffst_plan_info(ffst_plan_t plan, int* rows, int* cols, int* scales, int* num_planes);

/*
 * Plane index i -> (kappa, j, k) of Sec. 3.5.2 (the analogue of the paper's
 * shearletScaleShear helper).  cone is one of FFST_CONE_*; for the low-pass
 * j = -1 and k = 0.  Returns FFST_ERR_INVALID_ARG for i outside [0, eta).
 */
ffst_status ffst_plane_index(ffst_plan_t plan, int i, int* cone, int* j, int* k);

/*
 * Write every spectrum psi_hat_i (real, with the Sec. 3.8.1 fix) on the full
 * M x N frequency grid in FFT storage order (index p <-> omega = p for
 * p < ceil(L/2), p - L otherwise) into `psi` (device, [eta][rows][cols]
 * float32).  For tests and inspection; the transforms never read spectra
 * from memory, they generate them in registers.
 */
ffst_status ffst_spectra(ffst_plan_t plan, float* psi, void* stream);

/*
 * Forward transform, Sec. 3.1 eq. (shearletTransform).
 *   img:         device, rows x cols float32, read only.
 *   coeffs:      device, [eta][rows][cols] of the storage type (float, __half
 *                or __nv_bfloat16), fully overwritten.
 *   storage:     an ffst_storage code.
 *   plane_scale: device float[eta]; required (non-NULL) for F16/BF16, where the
 *                forward writes s_i (a power of two chosen from a bound on
 *                max|c_i|) and stores c_i * s_i; ignored for F32.
 */
ffst_status ffst_forward(ffst_plan_t plan, const float* img, void* coeffs, int storage,
                         float* plane_scale, void* stream);

/*
 * Forward transform with fused per-plane statistics and shrinkage (the
 * denoising use named in Sec. 1; the row pass applies them to each
 * coefficient before it is stored, so the unthresholded stack is never
 * written).  Arguments as ffst_forward, plus:
 *   shrink    0: none, 1: soft, c <- sign(c) max(|c| - tau_i, 0),
 *             2: hard, c <- c if |c| > tau_i else 0;
 *   thresh    device [eta] float, tau_i per plane (required when shrink != 0;
 *             in units of the coefficients c, independent of the storage
 *             scale s_i);
 *   mean_abs  device [eta] float or NULL: receives d(i) = 1/(MN) sum |c_i|
 *             (Sec. 3.5.2 eq. shearlet_meanvalue) of the coefficients before
 *             shrinkage, summed in a fixed order (deterministic).
 * Returns FFST_ERR_INVALID_ARG for another shrink code or a missing thresh.
 */
ffst_status ffst_forward_stats(ffst_plan_t plan, const float* img, void* coeffs, int storage, float* plane_scale,
                               int shrink, const float* thresh, float* mean_abs, void* stream);

/*
 * Complex shearlet coefficients from one-sided spectra (Sec. 3.8.2).  For a
 * real image, z_i = sqrt(2) ifft2(psi_hat_i h_i fft2(img)) for i >= 1 and
 * z_0 = the (real) low-pass coefficient, where h_i keeps one side of every
 * pair {omega, -omega}: omega_1 > 0 on C^h and the seam lines, omega_2 > 0
 * on C^v, the other axis deciding on the Nyquist column and row, 1/2 on the
 * self-conjugate grid points.  Re z_i = c_i / sqrt(2) (c of ffst_forward),
 * Im z_i = d_i / sqrt(2) with d_i the real transform for the multiplier
 * -i sign(omega) psi_hat_i; |z_i| and arg z_i are the amplitude and phase.
 *   coeffs  device float [eta][2][rows][cols], planar: Re z_i then Im z_i.
 * ffst_forward_complex runs the real pipeline twice (both parts); FP32 only.
 * ffst_inverse_complex reconstructs the image from the real parts.
 */
ffst_status ffst_forward_complex(ffst_plan_t plan, const float* img, float* coeffs, void* stream);
ffst_status ffst_inverse_complex(ffst_plan_t plan, const float* coeffs, float* img, void* stream);

/*
 * Inverse transform, Sec. 3.3 eq. (inverseShearletTransform), normalised by
 * sum_i psi_hat_i^2 (which the Parseval frame of Sec. 3.2 makes 1).
 *   coeffs:      device [eta][rows][cols] of the storage type, read only.
 *   plane_scale: device float[eta] written by ffst_forward (F16/BF16 only);
 *                stored values are multiplied by 1/s_i on load.
 *   img:         device rows x cols float32, overwritten.
 */
ffst_status ffst_inverse(ffst_plan_t plan, const void* coeffs, int storage,
                         const float* plane_scale, float* img, void* stream);

/*
 * Adjoint T* c = ifft2( sum_i psi_hat_i * fft2(c_i) ) (Sec. 3.2: for a
 * Parseval frame the adjoint U^T is the inverse).  Same arguments as
 * ffst_inverse; omits the normalisation, so it is the exact adjoint of the
 * FP32 forward and the backward pass of the differentiable transform.
 */
ffst_status ffst_adjoint(ffst_plan_t plan, const void* coeffs, int storage,
                         const float* plane_scale, float* img, void* stream);

/*
 * Forward transform for small images that allocates nothing (the paper has
 * no counterpart; it exists for callers that cannot call cudaMalloc, such as
 * processes whose framework has reserved nearly all device memory, plug-ins
 * inside a host application that owns the device's allocator, or hosts that
 * forbid allocation after start-up; ffst_plan allocates, so those callers
 * cannot build a plan).
 *   rows, cols:  powers of two in [8, 256]; scales in 1..4 (<= 0: default j0).
 *                Anything larger returns FFST_ERR_UNSUPPORTED_SIZE before any
 *                work is enqueued.
 *   img:         device, rows x cols float32, read only.
 *   coeffs:      device, [eta][rows][cols] float32, fully overwritten.
 * Same result as ffst_forward with FFST_STORE_F32 (to FP32 rounding; the
 * grid of FFST_SPACING_COMMON).  All tables and intermediates live in one
 * static device array of about 2.5 MB that every GPU loading the library
 * holds until the process exits.  Every call looks up that array's address
 * on the current device (host side, no allocation); the first call on a
 * device also loads the library's device code there, so make it before any
 * stream capture.  Calls share the array and each call rewrites every word
 * it reads: two calls whose work overlaps on the GPU race and corrupt each
 * other.
 */
ffst_status ffst_forward_noalloc(int rows, int cols, int scales, const float* img, float* coeffs, void* stream);

/*
 * Autotune a plan's launch configuration for coefficient storage `storage`,
 * each direction apart, on the plan's own shape (`reps` timed calls per
 * candidate after one warm-up):
 *   1. the plane-group budget: 32, 64, 96, 128 or 192 MB of column-pass
 *      intermediates per launch;
 *   2. at those budgets, the kernel configuration (ffst_plan_set_kernels):
 *      fused plane-pass launches (square powers of two) or separate row and
 *      column launches with each row-FFT variant that exists for the row
 *      length, and for the inverse also 1, 2, 4 or the default number of
 *      plane chunks of its sum.
 * Keeps the fastest of each.  Allocates a temporary image and coefficient
 * stack of the plan's size (eta*rows*cols elements) and synchronises the
 * device.  When the environment variable FFST_AUTOTUNE_CACHE names a file,
 * the choice is appended to it and later ffst_plan calls for the same device
 * and shape start from it.  The budgets and the fusion choice do not change
 * results; the row variants and the plane chunks change only the rounding
 * order.  *fwd_mb and *inv_mb (either may be NULL) receive the budgets.  The
 * choices only matter for grouped launches (schedule mode 0, the default).
 */
ffst_status ffst_plan_autotune(ffst_plan_t plan, int storage, int reps, double* fwd_mb, double* inv_mb);

/*
 * Kernel configuration of a plan (what ffst_plan_autotune chooses):
 *   fuse_fwd, fuse_inv  1: one launch per plane group holds the column pass
 *                       of that group and the row pass of the previous one
 *                       (square power-of-two images only; ignored otherwise);
 *                       0: separate row and column launches;
 *   row_fwd, row_inv    the FFT of the separate row launches: 0 = 16 elements
 *                       per thread (radix 16 x 16 x 4 at 1024-point lines,
 *                       two shared-memory exchanges); 1 = two rows per team
 *                       with packed two-lane FP32 arithmetic (forward only,
 *                       power-of-two widths 512..4096); 2 = 32 elements per
 *                       thread (radix 32 x 32, one exchange; widths 2048 and
 *                       4096); 3 = as 2 with the exchange done by warp
 *                       shuffles instead of shared memory (width 2048 only:
 *                       one warp per 1024-point line; results bitwise those
 *                       of 2).  Fused launches use 0.
 * The same transform in every configuration (the row variants differ in
 * rounding only).  FFST_ERR_INVALID_ARG for flags other than 0/1 or a row
 * variant the plan's width does not have.
 */
ffst_status ffst_plan_set_kernels(ffst_plan_t plan, int fuse_fwd, int fuse_inv, int row_fwd, int row_inv);
ffst_status ffst_plan_get_kernels(ffst_plan_t plan, int* fuse_fwd, int* fuse_inv, int* row_fwd, int* row_inv);

/* The plane-group budgets (MB) of the plan's forward and inverse. */
ffst_status ffst_plan_group_mb(ffst_plan_t plan, double* fwd_mb, double* inv_mb);

/*
 * Schedule of the per-plane passes (implementation choice, no counterpart in
 * the paper; results are bitwise identical in modes 0 and 1).
 *   mode 0 (default): grouped launches, one per plane group and pass pair.
 *   mode 1: persistent schedule, for square images with 256 <= rows <= 4096
 *           (other sizes keep mode 0): each forward or inverse runs all
 *           plane passes in one launch whose blocks take column and row tasks
 *           from a queue built at plan time, with per-plane counters for the
 *           dependencies and the column intermediates in a ring buffer of
 *           FFST_RING_MB megabytes (default 256), allocated when mode 1 or 2
 *           is first selected.  Measured slower than mode 0 at 2048x2048
 *           (3.3 vs 2.5 ms per forward + inverse).
 *   mode 2: test mode: the persistent forward's first task waits on a
 *           counter that nothing increments, so the bounded wait runs out
 *           (about a second), the launch stops early and ffst_plan_check
 *           returns FFST_ERR_TIMEOUT; the stack is then unspecified.
 * ffst_plan_set_schedule returns FFST_ERR_INVALID_ARG for other modes.
 * ffst_plan_get_schedule stores the mode in effect (0 when the plan has no
 * persistent schedule).
 */
ffst_status ffst_plan_set_schedule(ffst_plan_t plan, int mode);
ffst_status ffst_plan_get_schedule(ffst_plan_t plan, int* mode);

/*
 * Plane chunks of the inverse's column pass (implementation choice, no
 * counterpart in the paper).  The sum over planes of the inverse and the
 * adjoint (Sec. 3.3) runs as nsplit partial sums: chunk k takes the planes
 * [eta k / nsplit, eta (k + 1) / nsplit), each added in plane order into its
 * own [rows][cols/2+1] accumulator, and the final column pass adds the
 * partial sums in chunk order.  More chunks give more parallel column
 * blocks where the panels alone do not fill the GPU (small images); the
 * rounding order, and so the last bits of the result, depend on nsplit but
 * not on the schedule mode or the group budgets.  ffst_plan picks the
 * chunks for about four column blocks per SM (1 at 2048x2048 and above, up
 * to 16 for small images; the environment variable FFST_INV_SPLIT at plan
 * creation overrides); nsplit = 0 restores that choice.  Partial
 * accumulators are allocated on demand (nsplit x rows x (cols/2+1) x 8
 * bytes).  FFST_ERR_INVALID_ARG for nsplit outside 0..16.
 */
ffst_status ffst_plan_set_inverse_split(ffst_plan_t plan, int nsplit);

/*
 * Plane-sharded transforms.  The planes of Sec. 3.1 are independent: a
 * forward over a plane range needs only fft2(f), and the inverse of Sec. 3.3
 * is a sum over planes, so ranks holding disjoint ranges combine their
 * partial spectra with one sum-reduce and one rank finishes.
 *
 * ffst_plan_set_planes restricts the plan's plane passes to [p0, p1)
 * (0 <= p0 < p1 <= eta; the default is every plane).  Afterwards
 * ffst_forward, ffst_forward_stats and ffst_forward_complex write only those
 * planes: `coeffs` holds p1 - p0 planes (plane p0 first); plane_scale and
 * the statistics keep eta entries indexed by the global plane (entries
 * outside the range are unspecified).  ffst_inverse, ffst_adjoint and
 * ffst_inverse_partial read a stack of p1 - p0 planes.  Regroups the plan
 * (synchronises the device; allocates).  FFST_ERR_INVALID_ARG for an empty
 * or out-of-range interval, or while the persistent schedule is selected.
 */
ffst_status ffst_plan_set_planes(ffst_plan_t plan, int p0, int p1);
ffst_status ffst_plan_get_planes(ffst_plan_t plan, int* p0, int* p1);

/*
 * Partial inverse: spectrum = sum over the active planes i of
 * psi_hat_i * fft2(c_i), the half spectrum [rows][cols/2+1] of complex64
 * (interleaved re, im; device, caller-owned, fully overwritten), summed in
 * the plan's fixed plane order.  Sec. 3.3 eq. (inverseShearletTransform)
 * before its ifft2; the sum of the partial spectra of disjoint ranges that
 * cover every plane is the full sum.
 */
ffst_status ffst_inverse_partial(ffst_plan_t plan, const void* coeffs, int storage, const float* plane_scale,
                                 float* spectrum, void* stream);

/*
 * Finish an inverse from a (reduced) half spectrum as written by
 * ffst_inverse_partial: img = ifft2(spectrum / sum_i psi_hat_i^2) over all
 * eta planes when normalise != 0 (ffst_inverse), without the division
 * otherwise (ffst_adjoint).  `spectrum` is used as workspace and left
 * unspecified; img is device rows x cols float32, overwritten.
 */
ffst_status ffst_inverse_finish(ffst_plan_t plan, float* spectrum, int normalise, float* img, void* stream);
ffst_status ffst_plan_get_inverse_split(ffst_plan_t plan, int* nsplit);

/* Shape of the persistent schedule (zeros until it is built): resident
 * blocks per launch, tasks in the forward and inverse queues, ring size in
 * MB.  Any output pointer may be NULL. */
ffst_status ffst_plan_schedule_info(ffst_plan_t plan, int* blocks, int* fwd_tasks, int* inv_tasks, double* ring_mb);

/*
 * Synchronise `stream` and report whether a bounded device-side wait of the
 * persistent schedule ran out since the last check (FFST_ERR_TIMEOUT; the
 * flag is then cleared).  Waits only run out in test mode 2 or on an
 * internal error; the CUDA context stays usable either way.
 */
ffst_status ffst_plan_check(ffst_plan_t plan, void* stream);

/*
 * Batches of images of uneven sizes.  ffst_plan_batched builds one plan per
 * (size, lane) for n images (rows[i] x cols[i], scales[i] <= 0 or NULL for
 * the default) and spreads the images over `lanes` (1..16) internal streams,
 * largest transform first onto the least loaded lane, so transforms of
 * different images run concurrently.  The batched calls fork the lanes from
 * `stream` and join them back before returning control of the stream:
 *   imgs[i], coeffs[i], plane_scales[i] are device pointers as in
 *   ffst_forward / ffst_inverse, passed as host arrays of n pointers
 *   (plane_scales may be NULL for F32 storage).
 * Calls on one batch must not overlap (lanes share plan workspaces).
 */
typedef struct ffst_batch_s* ffst_batch_t;
ffst_status ffst_plan_batched(int n, const int* rows, const int* cols, const int* scales, int lanes,
                              ffst_batch_t* out);
/*
 * Autotune a batch: ffst_plan_autotune once per distinct image shape (on one
 * of its plans), then that shape's configuration on every plan of the shape.
 * Synchronises the device and allocates temporaries of the largest shape.
 * storage and reps as for ffst_plan_autotune; stops at the first plan whose
 * tuning fails and returns that status (plans tuned before it keep their
 * new configuration).  Plans take a cached configuration of their shape at
 * creation already; this call times again and appends to the cache.
 */
ffst_status ffst_batch_autotune(ffst_batch_t batch, int storage, int reps);

/* Image i's size, scales, planes and lane.  Any output may be NULL. */
ffst_status ffst_batch_info(ffst_batch_t batch, int i, int* rows, int* cols, int* scales, int* num_planes, int* lane);
ffst_status ffst_forward_batched(ffst_batch_t batch, const float* const* imgs, void* const* coeffs, int storage,
                                 float* const* plane_scales, void* stream);
ffst_status ffst_inverse_batched(ffst_batch_t batch, const void* const* coeffs, int storage,
                                 float* const* plane_scales, float* const* imgs, void* stream);
void ffst_batch_destroy(ffst_batch_t batch);

/*
 * Capture a batched forward (what bit 0) and/or inverse (bit 1, from the
 * same coeffs into out_imgs) into one instantiated CUDA graph.  Runs the
 * work once eagerly first (module loading, kernel attributes), then
 * captures it on an internal stream.  The pointers are baked into the graph;
 * ffst_graph_launch replays it on `stream`, ffst_graph_destroy frees it.
 */
ffst_status ffst_graph_capture_batched(ffst_batch_t batch, int what, const float* const* imgs, void* const* coeffs,
                                       int storage, float* const* plane_scales, float* const* out_imgs,
                                       void** graph_exec);
ffst_status ffst_graph_launch(void* graph_exec, void* stream);
void ffst_graph_destroy(void* graph_exec);

/* Free a plan and everything it owns (synchronises the device first).  NULL is a no-op. */
void ffst_destroy(ffst_plan_t plan);

/* Thread-local message describing the last failing call on this thread ("" if none). */
const char* ffst_last_error(void);

/* Static name of a status code. */
const char* ffst_status_string(int status);

/*
 * Per-kernel timing: while enabled, every kernel the plan launches is
 * bracketed by CUDA events on its launch stream and its duration is added
 * to a per-kind total.  ffst_timing_read synchronises on those events and
 * reports, for kernel kind `kind` (0 .. ffst_timing_kinds()-1), its name,
 * total milliseconds, launch count and the algorithmic HBM bytes of those
 * launches (the bytes a fused kernel must move: see the project's design
 * notes).  ffst_timing_reset clears the totals.
 */
ffst_status ffst_timing_enable(ffst_plan_t plan, int enable);
ffst_status ffst_timing_reset(ffst_plan_t plan);
int ffst_timing_kinds(void);
ffst_status ffst_timing_read(ffst_plan_t plan, int kind, const char** name, double* total_ms,
                             long long* launches, double* algorithmic_bytes);

#ifdef __cplusplus
}
#endif

#endif /* FFST_H */
