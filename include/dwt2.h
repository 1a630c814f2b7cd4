/*
 * dwt2.h -- C ABI of libdwt2: the 2-D discrete wavelet transform computed by
 * the non-separable lifting schemes of Barina, Kula, Matysek and Zemcik,
 * "Accelerating Discrete Wavelet Transforms on Parallel Architectures"
 * (arXiv:1704.08657), on NVIDIA GB300 (sm_103a).
 *
 * Operation (Background and Proposed Schemes sections).  One level splits an
 * image into 2x2 polyphase quads (c1, c2, c3, c4) = (x[2i][2j], x[2i][2j+1],
 * x[2i+1][2j], x[2i+1][2j+1]) and applies, for each lifting pair (P, U) of
 * Eq. 2, the spatial predict T_P then the spatial update S_U (the
 * non-separable lifting "S_U | T_P"), then scaling.  CDF 9/7 has two pairs
 * (alpha, beta), (gamma, delta) with P = a(1 + z), U = b(1 + z^-1) and scaling
 * zeta; the integer-reversible CDF 5/3 has one pair with floor rounding; the
 * interpolating Deslauriers-Dubuc DD 13/7 (Table 1's third wavelet, its
 * constants from the published filter bank) has one pair with the 4-tap
 * P = -(9/16)(1 + z) + (1/16)(z^-1 + z^2), U = (9/32)(1 + z^-1) -
 * (1/32)(z + z^-2) and no scaling step.
 * All schemes compute the same values (Proposed Schemes); the scheme only
 * selects the kernel:
 *   DWT2_NONSEP          spatial predict / update, all terms in one step;
 *   DWT2_NONSEP_REDUCED  the Optimization Approach: the constant parts P0, U0
 *                        applied as separable lifting inside the quad right
 *                        after the non-separable parts P1, U1 (CDF 9/7 and
 *                        DD 13/7, whose P1 and U1 keep three taps each);
 *   DWT2_SEP_LIFTING     the separable lifting T^H, T^V, S^H, S^V per pair;
 *   DWT2_POLYCONV        the polyconvolution N_{P,U} (Proposed Schemes): each
 *                        pair applied as one step on pre-pair values, with
 *                        V = 1 + PU as one 3-tap filter (CDF 9/7 only);
 *   DWT2_CONV            the separable convolution N^V | N^H (Background):
 *                        the 9-tap / 7-tap filter bank, multiplied out from
 *                        the lifting constants, on each row and then on each
 *                        column of the row results (CDF 9/7 only);
 *   DWT2_NONSEP_CONV     the non-separable convolution N = N^V N^H (Proposed
 *                        Schemes): one step of 2-D filters of 9x9, 9x7, 7x9
 *                        and 7x7 pixels, the products of the vertical and
 *                        horizontal taps applied directly (CDF 9/7 only).
 * The kernels stream rows through registers and exchange horizontal
 * neighbours by warp shuffles, so no scheme has barriers between its steps;
 * the schemes differ in arithmetic and in the number of neighbour exchanges
 * (4, 4, 4, 2, 1 and 1 per CDF 9/7 level).
 *
 * Conventions (readings where the paper is silent):
 *   - odd sample x[2n+1] is predicted from x[2n], x[2n+2] (DD 13/7: also
 *     x[2n-2], x[2n+4]); even sample x[2n] is updated from x[2n-1], x[2n+1]
 *     (DD 13/7: also x[2n-3], x[2n+3]);
 *   - boundary: whole-sample symmetric extension (x[-1] = x[1],
 *     x[n] = x[n-2]) in every step;
 *   - CDF 9/7 scaling: low-pass times zeta and high-pass divided by zeta per
 *     axis (LL * zeta^2, HL and LH * 1, HH / zeta^2);
 *   - integer 5/3: d = x_o - floor((x_l + x_r)/2), s = x_e +
 *     floor((d_l + d_r + 2)/4), steps in the order T^H, T^V, S^H, S^V; values
 *     must stay below 2^28 in magnitude (int32 arithmetic);
 *   - layout: Mallat.  Level 1 writes, within the h x w image, LL to
 *     [0, ceil(h/2)) x [0, ceil(w/2)), HL (c2) to the top-right, LH (c3) to the
 *     bottom-left and HH (c4) to the bottom-right; level k+1 transforms the
 *     LL region of level k in place of it.  Every level's input needs both
 *     sides >= 2.
 *
 * Memory and ownership.  The caller owns every device buffer and the stream.
 * A plan owns its device status word, segment counters and persistent-launch
 * tables (device memory allocated when the plan is made) and the launch
 * blocks of several-image plans (host memory, built at the first call for a
 * set of buffers); calls are asynchronous on the given stream and allocate no
 * device memory after the plan is made.  A plan must not be used on two
 * streams at the same time.
 *
 * Errors.  Every function returns DWT2_OK (0) or a negative DWT2_ERR_* code;
 * nothing aborts or traps.  dwt2_strerror() names a code.
 */
#ifndef DWT2_H
#define DWT2_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dwt2_plan_s* dwt2_plan_t;

enum dwt2_wavelet { DWT2_CDF97 = 0, DWT2_CDF53_INT = 1, DWT2_DD137 = 2 };
enum dwt2_dtype { DWT2_F32 = 0, DWT2_F16 = 1, DWT2_BF16 = 2, DWT2_I32 = 3 };
enum dwt2_scheme {
    DWT2_NONSEP = 0,
    DWT2_NONSEP_REDUCED = 1,
    DWT2_SEP_LIFTING = 2,
    DWT2_POLYCONV = 3,
    DWT2_CONV = 4,
    DWT2_NONSEP_CONV = 5
};
enum dwt2_boundary { DWT2_SYMMETRIC = 0 };

#define DWT2_OK 0
#define DWT2_ERR_INVALID_ARG (-1)     /* null pointer, bad enum, bad size      */
#define DWT2_ERR_UNSUPPORTED (-2)     /* wavelet / dtype / scheme combination  */
#define DWT2_ERR_LEVELS_TOO_DEEP (-3) /* some level's input side would be < 2  */
#define DWT2_ERR_MISALIGNED (-4)      /* pointer, offset or pitch alignment    */
#define DWT2_ERR_CUDA (-5)            /* a CUDA runtime call failed            */
#define DWT2_ERR_TIMEOUT (-6)         /* a bounded device wait expired         */
#define DWT2_ERR_DEVICE_CHECK (-7)    /* a device-side bounds check tripped    */
#define DWT2_ERR_TOO_LARGE (-8)       /* beyond dwt2_forward_noalloc's scratch */

/* plan flags */
#define DWT2_FLAG_PERSISTENT 0x1u /* forward: one persistent launch for all images and levels */

/* TEST ONLY -- failure injection on the host side, never for production use:
 * a plan made with this flag has one unit of its forward (the first queued
 * unit of a persistent launch; strip 0 of segment 0 of each level with
 * inter-level overlap) never report completion, so the units that depend on
 * it time out after DWT2_TIMEOUT_MS and dwt2_status returns DWT2_ERR_TIMEOUT
 * while the CUDA context stays usable; the coefficients are then incomplete. */
#define DWT2_TESTONLY_DROP_SIGNAL 0x100u

/* One image of a batch: element offset of its first pixel from the base
 * pointer, its size, and its row pitch in elements (pitch >= w).  The same
 * offset and pitch address its coefficients in the coefficient buffer. */
typedef struct {
    int64_t offset_elems;
    int32_t h, w;
    int64_t pitch_elems;
} dwt2_image_desc;

/*
 * dwt2_plan -- validate a transform and prepare its launches.
 *   out        receives the plan (set to NULL on error).
 *   wavelet    DWT2_CDF97, DWT2_CDF53_INT or DWT2_DD137.
 *   levels     number of pyramid levels, >= 1.
 *   boundary   DWT2_SYMMETRIC.
 *   in_dtype   image element type: DWT2_F32 for CDF 9/7 and DD 13/7,
 *              DWT2_I32 for 5/3.
 *   coef_dtype coefficient element type: F32, F16 or BF16 for CDF 9/7 and
 *              DD 13/7 (the lifting always runs in FP32 and intermediate LL
 *              bands are kept in FP32), I32 for CDF 5/3.
 *   scheme     DWT2_NONSEP, DWT2_NONSEP_REDUCED (CDF 9/7 and DD 13/7; DD 13/7
 *              takes the three lifting schemes, not DWT2_FLAG_PERSISTENT),
 *              DWT2_SEP_LIFTING, DWT2_POLYCONV, DWT2_CONV or DWT2_NONSEP_CONV
 *              (the last three CDF 9/7 only and not with
 *              DWT2_FLAG_PERSISTENT: DWT2_ERR_UNSUPPORTED).  The inverse and
 *              adjoint of a plan run the non-separable lifting kernels for
 *              the last three (the same transform).
 *   n_images   number of images (>= 1); images is a host array of that many
 *              descriptors, copied into the plan.  With several images
 *              dwt2_forward runs each level as launches of up to 76 images
 *              (the inverse and adjoint up to 160), whose parameter blocks are
 *              built at the first call for a set of buffers and reused.
 *   flags      0 or DWT2_FLAG_PERSISTENT: dwt2_forward then runs every level of every
 *              image in one persistent launch whose units take work from a device
 *              queue and wait (bounded by DWT2_TIMEOUT_MS, default 2000) for the
 *              segments of the previous level they read; the plan allocates its
 *              queue tables and a table of TMA tensor maps at creation.  The
 *              first call for a set of input and workspace buffers writes that
 *              table (it synchronises the stream); made during a stream capture
 *              it returns DWT2_ERR_INVALID_ARG.  Later calls on the same buffers
 *              are asynchronous and CUDA-graph capturable.
 * Alignment: the image (input) buffer's base pointer must be 16-byte aligned
 * and offset_elems and pitch_elems multiples of 4 (16 bytes of 4-byte
 * elements), else DWT2_ERR_MISALIGNED; coefficient buffers need only natural
 * element alignment.  The plan allocates its device status word and batch
 * tables on the current device.
 * Environment, read when the plan is made (launch tuning only; results do not
 * depend on it): DWT2_TIMEOUT_MS (bounded device waits, default 2000),
 * DWT2_FWD_CFG and DWT2_SEG_ROWS (forward kernel configuration 0-4 and
 * segment height before any dwt2_autotune), DWT2_PDL (0 launches the forward
 * levels without programmatic dependent launch), DWT2_FUSE_SEG and
 * DWT2_FUSE_PAIRS (run level pairs 0-1, 2-3, ... in one fused launch with that
 * segment height; off by default, slower on GB300), DWT2_PML_SEG_ROWS,
 * DWT2_PML_LAG_PCT and DWT2_PML_CPASYNC (persistent forward),
 * DWT2_INV_EDGE_FIRST (1 / 0: an inverse or adjoint level launches its edge
 * units before / after its inner units; default: before for the adjoint,
 * after for the inverse).
 */
int dwt2_plan(dwt2_plan_t* out, int wavelet, int levels, int boundary, int in_dtype,
              int coef_dtype, int scheme, int n_images, const dwt2_image_desc* images,
              unsigned flags);

/* Bytes of device workspace the caller passes to the transform calls of this
 * plan; 256-byte alignment is required.  It holds the intermediate low-low
 * bands of every level but the last (the forward and the inverse use only
 * these: a one-level plan's forward and inverse may take NULL) and, for CDF
 * 9/7, the adjoint's side buffers: per level 8 * (h + 8) + 8 * w floats for
 * the outputs of the transposed lifting past the image edges, which the
 * adjoint folds back onto their mirrors. */
size_t dwt2_workspace_bytes(dwt2_plan_t plan);

/*
 * dwt2_forward -- coef = W(in), the forward pyramid (Proposed Schemes; the
 * paper's Optimization Approach for DWT2_NONSEP_REDUCED).
 *   in         device pointer to the images (in_dtype), read only.
 *   coef       device pointer to the coefficients (coef_dtype), written; must
 *              not overlap in.
 *   workspace  device pointer to dwt2_workspace_bytes(plan) bytes (may be
 *              NULL for a one-level plan).
 *   stream     a cudaStream_t (NULL for the legacy default stream).
 */
int dwt2_forward(dwt2_plan_t plan, const void* in, void* coef, void* workspace, void* stream);

/* dwt2_inverse -- out = W^-1(coef): every step undone in reverse order
 * (each lifting step is inverted by negating its filter, Eq. 2).
 *   coef (coef_dtype) read only; out (in_dtype) written; no overlap. */
int dwt2_inverse(dwt2_plan_t plan, const void* coef, void* out, void* workspace, void* stream);

/* dwt2_adjoint -- in_grad = W^T(coef_grad), the transpose of the forward
 * operator (not in the paper).  With the symmetric boundary the forward is
 * "extend, lift with no boundary cases, keep the inside", so its transpose is
 * the transposed steps in reverse order on the coefficient gradient extended
 * by zeros, followed by the fold that adds every output past an edge onto its
 * whole-sample mirror.  CDF 9/7 only; both buffers FP32 and laid out like the
 * image / the coefficients; the workspace is required (side buffers). */
int dwt2_adjoint(dwt2_plan_t plan, const void* coef_grad, void* in_grad, void* workspace,
                 void* stream);

/* dwt2_adjoint_l1 -- in_grad = W^T(scale * sign(detail(coef))): the gradient
 * with respect to the image of scale * (sum of |c| over every detail band),
 * the coarsest LL band excluded, where coef = W(image) (not in the paper; a
 * wavelet-domain L1 loss for training and regularised reconstruction).  The
 * sign is taken inside the adjoint's band loads, so no gradient array is
 * written.  scale = 1 / (number of detail coefficients) gives the mean.  CDF
 * 9/7 with FP32 coefficients; coef and in_grad as for dwt2_adjoint. */
int dwt2_adjoint_l1(dwt2_plan_t plan, const void* coef, void* in_grad, float scale, void* workspace,
                    void* stream);

/* dwt2_adjoint_l1_dev -- dwt2_adjoint_l1 with the scale scale * *scale_dev,
 * where scale_dev is a device pointer to one float read by the kernels when
 * they run: the gradient of a loss whose upstream gradient lives on the
 * device (autograd) is formed without a host synchronisation, so the call is
 * asynchronous and can be captured in a CUDA graph.  scale_dev must not be
 * NULL and stays valid until the call has completed on the stream. */
int dwt2_adjoint_l1_dev(dwt2_plan_t plan, const void* coef, void* in_grad, const float* scale_dev,
                        float scale, void* workspace, void* stream);

/* dwt2_autotune -- choose the plan's launch configuration (not in the paper).
 * With *choice < 0: run the forward on the given buffers (same arguments as
 * dwt2_forward) for each candidate configuration (kernel tile shape and
 * segment height; segment height and queue lag for persistent plans), a few calls each on
 * the stream timed per level with the plan's profile events, keep the fastest
 * candidate of every level (of the whole launch for persistent plans) and
 * store the choice in *choice: 6 bits per level for the first five levels,
 * deeper levels sharing the fifth field (persistent plans: one index 0-11,
 * segment height 16/24/32/48 times queue lag 300/500/800 % of a GPU round of
 * units).  With *choice >= 0: apply that choice without timing (e.g. from a
 * cache of an earlier run on the same GPU); DWT2_ERR_INVALID_ARG if it is not
 * a valid choice for this plan.  The coefficient buffer is overwritten and the
 * plan's profile ring is reset.  Synchronises the stream; not for use during
 * graph capture. */
int dwt2_autotune(dwt2_plan_t plan, const void* in, void* coef, void* workspace, void* stream,
                  int* choice);

/* dwt2_status -- synchronise the stream, return and clear the plan's device
 * status word: DWT2_OK, DWT2_ERR_TIMEOUT or DWT2_ERR_DEVICE_CHECK. */
int dwt2_status(dwt2_plan_t plan, void* stream);

/* dwt2_checked -- 1 in the range-checked build of this library
 * (libdwt2_checked.so, compiled with DWT2_CHECKED), 0 otherwise.  In the
 * checked build every global access of the forward, inverse and adjoint
 * kernels (band loads and stores, the image, the workspace's low-low bands
 * and side buffers) is first tested against the rectangle of its buffer from
 * the pointer it is about to use; a violation skips the access (a load reads
 * element 0 instead), sets the plan's status word so that dwt2_status returns
 * DWT2_ERR_DEVICE_CHECK, and stops the kernel at the end of the unit: a
 * stand-in for a memory checker, at a cost in speed.  Results of a checked
 * build without a violation equal the normal build's bit for bit. */
int dwt2_checked(void);

/* dwt2_profile -- when enable != 0, every later transform call of this plan
 * records a CUDA event pair on its stream around the launches of each pyramid
 * level (all images of a batch together), in a ring of the last 256 calls;
 * enabling resets the ring.  The events belong to the plan.  Not in the
 * paper: a measurement hook. */
int dwt2_profile(dwt2_plan_t plan, int enable);

/* dwt2_profile_read -- wait for the recorded calls' events and write, for each
 * of the first n levels (finest first), the mean elapsed milliseconds over the
 * calls in the ring to ms[0 .. n-1]; n <= the plan's levels.
 * DWT2_ERR_INVALID_ARG if nothing was recorded. */
int dwt2_profile_read(dwt2_plan_t plan, float* ms, int n);

/*
 * dwt2_forward_noalloc -- the forward pyramid of one image, allocating no
 * device memory (the paper has no counterpart: this is a service for callers
 * that cannot allocate when they transform, e.g. code running during a CUDA
 * graph capture that forbids cudaMalloc, real-time pipelines that allow no
 * allocation after start-up, or plug-ins whose host owns all device memory).
 *   wavelet, levels, scheme, coef_dtype  as for dwt2_plan, CDF 9/7 or CDF 5/3
 *              only (in_dtype follows the wavelet: F32 for CDF 9/7, I32 for
 *              CDF 5/3); schemes DWT2_NONSEP, DWT2_NONSEP_REDUCED (CDF 9/7)
 *              and DWT2_SEP_LIFTING.
 *   h, w, pitch_elems  the image; pitch a multiple of 4 elements.
 *   in         device pointer to the image, 16-byte aligned, read only.
 *   coef       device pointer to the coefficients (Mallat layout, same pitch).
 *   stream     a cudaStream_t (NULL for the legacy default stream).
 * The intermediate low-low bands live in a static 32 MiB device array inside
 * the library (held by every GPU that loads it until exit), in two
 * alternating buffers: levels 1, 3, 5, ... write their low-low band (FP32 or
 * int32, ceil(h_l / 2) rows of round4(ceil(w_l / 2)) elements for a level
 * input of h_l x w_l) to the first, levels 2, 4, ... to the second, and the
 * request fits when the largest band of each kind, each rounded up to 256
 * bytes, add up to at most 32 MiB; else DWT2_ERR_TOO_LARGE before any GPU
 * work.  A one-level transform uses no scratch; a square n x n image fits
 * for n <= 5176 at any depth (4096 x 4096 takes 20 MiB).  The first call on a
 * device looks up the array's device address; make it before any stream
 * capture.  All calls share the array, so calls that overlap on the GPU race;
 * order them on one stream.  Same results as dwt2_forward.
 */
int dwt2_forward_noalloc(int wavelet, int levels, int scheme, int coef_dtype, int h, int w,
                         int64_t pitch_elems, const void* in, void* coef, void* stream);

/* dwt2_noalloc_status -- synchronise the stream, then return and clear the
 * status word that dwt2_forward_noalloc calls on the current device share
 * (another static word of the library, zero when it is loaded): DWT2_OK, or
 * DWT2_ERR_TIMEOUT when a bounded device wait (DWT2_TIMEOUT_MS, default 2000,
 * read at the first call on the device) ran out in some call since the last
 * read, in which case that call's coefficients are incomplete.  Allocates
 * nothing. */
int dwt2_noalloc_status(void* stream);

/*
 * Row bands of one image (not in the paper, whose Evaluation scales one GPU
 * over image resolution): an image too large for one GPU, or a pyramid to be
 * spread over several GPUs, is cut into n_bands bands of whole rows that
 * transform independently -- no data moves between bands -- and whose owned
 * rows are then copied into the image's Mallat layout.
 *
 * Band b owns input rows [own0, own1): the cuts are the multiples of
 * 2^levels nearest to b*h/n_bands (the last band ends at h), so the band's
 * 2x2 quads are the image's quads at every level.  It transforms rows
 * [in0, in1) = [own0 - H, own1 + H) clipped to [0, h), where H is
 * a*(2^levels - 1) rounded up to a multiple of 2^levels and a is the reach of
 * one level in rows of its input (4 for CDF 9/7, 2 for CDF 5/3, 6 for DD
 * 13/7: the half length of the longer analysis filter).  Every coefficient
 * the band owns then depends on image rows only (the symmetric extension at
 * the band's cut edges reaches only rows other bands own), so a band
 * transform computes exactly the coefficients of the whole-image transform
 * for its owned rows.  The halo rows are transformed twice (by two bands):
 * with n bands, 2*(n-1)*H extra rows in all.
 */

/* dwt2_band_rows -- rows[0..3] = own0, own1, in0, in1 of band `band`
 * (0 <= band < n_bands) of an image of h rows and `levels` levels of
 * `wavelet`.  DWT2_ERR_INVALID_ARG when a band would own fewer than
 * 2^levels rows.  Host only (no CUDA call). */
int dwt2_band_rows(int wavelet, int levels, int h, int n_bands, int band, int32_t rows[4]);

/* dwt2_band_rects -- the copy that dwt2_band_stitch performs, as rectangles
 * of five int32 each: source row (in the band's own coefficients, rows
 * counted from in0), destination row (in the image's coefficients), number
 * of rows, first column and number of columns (the same columns in both).
 * With rects == NULL and max_rects == 0 returns the count; else writes up to
 * max_rects rectangles and returns their count (DWT2_ERR_INVALID_ARG when
 * more are needed).  Host only. */
int dwt2_band_rects(int wavelet, int levels, int h, int w, int n_bands, int band, int32_t* rects,
                    int max_rects);

/* dwt2_band_stitch -- copy the coefficients band `band` owns from its own
 * forward transform into the image's coefficient buffer (one kernel launch,
 * asynchronous on the stream).
 *   band_coef   device pointer: the band's coefficients, (in1 - in0) rows of
 *               w elements in Mallat layout (what dwt2_forward of a plan of
 *               the (in1 - in0) x w image starting at input row in0 writes),
 *               row pitch band_pitch elements.
 *   coef        device pointer: the image's coefficients (h rows, pitch
 *               `pitch`), written only in the band's owned rectangles.
 * Both of coef_dtype, naturally aligned; levels and wavelet as for the band
 * transform, levels <= 24. */
int dwt2_band_stitch(int wavelet, int levels, int coef_dtype, int h, int w, int n_bands, int band,
                     const void* band_coef, int64_t band_pitch, void* coef, int64_t pitch, void* stream);

/* dwt2_destroy -- free the plan (NULL is accepted). */
void dwt2_destroy(dwt2_plan_t plan);

/* dwt2_strerror -- static description of an error code. */
const char* dwt2_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* DWT2_H */
