/*
 * fdas.h -- C ABI of the GB300 (sm_103a) FDAS correlation library.
 *
 * Fourier Domain Acceleration Search by the correlation technique: a
 * normalised complex spectrum is correlated with a bank of acceleration
 * templates, one per trial frequency derivative z, by overlap-save (segment
 * FFT -> pointwise multiply per template -> inverse FFT -> discard the
 * contaminated edges -> power at full and half bins), giving the f-fdot power
 * plane, which is then thresholded for candidates (Sections 2-4).
 *
 * Conventions for every call:
 *  - Pointers marked (device) are CUDA device pointers owned by the caller;
 *    the library allocates no device memory.  Pointers marked (host) are
 *    ordinary host memory.
 *  - Complex values are interleaved float pairs (re, im); a "complex" array
 *    of length n is float[2n], 8-byte aligned (16-byte where stated).
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Every
 *    compute call is asynchronous on that stream and returns before the GPU
 *    work finishes.
 *  - Return value: FDAS_OK (0) or a negative FDAS_E_* code.  Arguments are
 *    validated before anything is launched; on FDAS_E_INVAL nothing was
 *    launched.  FDAS_E_CUDA reports a launch error of this call.
 *  - Conditions found on the device (candidate overflow) are OR-ed as
 *    FDAS_STATUS_* bits into a caller-owned device int32 status word, which
 *    the caller zeroes and reads back after synchronising.
 *  - Calls may run concurrently on different streams if their output
 *    buffers do not overlap.
 */
#ifndef FDAS_H
#define FDAS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FDAS_OK 0
#define FDAS_E_INVAL (-1)       /* bad argument; nothing launched */
#define FDAS_E_CUDA (-2)        /* a CUDA launch or runtime error */
#define FDAS_E_OVERFLOW (-3)    /* candidate buffer too small (see status word) */
#define FDAS_E_TIMEOUT (-4)     /* a bounded device wait gave up (see status word) */
#define FDAS_E_UNSUPPORTED (-5) /* valid but unsupported size or device */

#define FDAS_STATUS_TIMEOUT 1   /* status-word bit: a device wait gave up */
#define FDAS_STATUS_OVERFLOW 2  /* status-word bit: more candidates than `cap` */

#define FDAS_CAND_PEAK 1        /* fdas_cand.flags bit: local maximum (8 neighbours) */

/* Search parameters.
 *  L        overlap-save segment (FFT) length: 1024, 2048 or 4096 (Section 3,
 *           Fig. 1: blocks of L = B + M points).
 *  M        padded template width in taps: a multiple of 4 with
 *           64 <= M <= L/2; each segment yields B = L - M useful bins and
 *           the longest template must fit: h(max|z|) <= M/2 - 1.  M is the
 *           largest overlap used: on a symmetric grid the convolver splits
 *           the templates into up to FDAS_MAX_GROUPS groups of increasing |z|
 *           and gives each group the smallest overlap its longest template
 *           needs (fdas_template_groups); the overlap only moves segment
 *           boundaries, not the correlation values.
 *  zmin, zmax, zstep
 *           template grid z_j = zmin + j*zstep, j = 0..K-1,
 *           K = (zmax - zmin)/zstep + 1; zstep >= 1, (zmax - zmin) % zstep == 0.
 *           If zmin == -zmax the grid is symmetric and the bank stores only
 *           the z >= 0 templates: a z < 0 template is applied as the
 *           complex conjugate of its +|z| partner with reversed frequency
 *           index (Section 4.2).
 *  interbin 1: plane rows hold 2*nb columns, column 2r = |F_r|^2 and
 *           column 2r+1 = (pi/4)^2 |F_r - F_{r+1}|^2 (Eq. f-interp), the last
 *           one 0;  0: rows hold nb columns |F_r|^2;  2: 2-bin Fourier
 *           interpolation (Section 3, after Eq. f-interp): rows hold 2*nb
 *           columns, column m = |F(m/2)|^2 with the correlation evaluated at
 *           every half bin, F(rho) = sum over bins k with |k - rho| <= h of
 *           spec[k] conj(R_z(k - rho)); the convolver works on the spectrum
 *           with zeros interleaved (2*nb positions) and templates sampled
 *           every half bin, so it needs 4h(max|z|) + 2 <= M, and the bank
 *           holds every template (no +-z pairing: R_{-z}(d) = -conj(R_z(d))
 *           at half-integer d).
 * The template half-width is h(z) = ceil(|z|/2) + 8 taps. */
typedef struct {
    int32_t L;
    int32_t M;
    int32_t zmin;
    int32_t zmax;
    int32_t zstep;
    int32_t interbin;
} fdas_params;

/* One threshold crossing: plane row (z index), column (2r or 2r+1 with
 * interbinning, r without), power, FDAS_CAND_* flags. */
typedef struct {
    int32_t z_idx;
    int32_t col;
    float power;
    int32_t flags;
} fdas_cand;

/* Threshold applied inside fdas_correlate's epilogue (flags are 0: no peak
 * test).  `count` (device) is reset to 0 by the call and ends holding the
 * number of crossings found, which may exceed `cap`; only the first `cap`
 * are stored, in no particular order, and FDAS_STATUS_OVERFLOW is set. */
typedef struct {
    float thr;          /* strict: power > thr */
    fdas_cand *out;     /* (device) cap entries */
    int32_t cap;
    int32_t *count;     /* (device) one int32 */
} fdas_fused_threshold;

/* Message for an FDAS_* return code (static string). */
const char *fdas_strerror(int code);

/* Library version as "major.minor.patch" (static string). */
const char *fdas_version(void);

/* Template half-width h(z) = ceil(|z|/2) + 8 taps. */
int32_t fdas_half_width(int32_t z);

/* Number of templates K of the grid (< 0: FDAS_E_INVAL). */
int32_t fdas_num_templates(const fdas_params *p);

/* Number of bank rows K' (K, or (K+1)/2-ish for a symmetric grid; < 0 on
 * error).  Bank row b holds template z = zmin + (b + j0)*zstep, where j0 is
 * the number of negative z in a symmetric grid and 0 otherwise. */
int32_t fdas_bank_rows(const fdas_params *p);

/* Size of the template bank in floats: fdas_bank_rows(p) * R * 2, with R =
 * L + 32 complex values per row for L = 1024 and L + 16 otherwise. */
int64_t fdas_bank_floats(const fdas_params *p);

/* Number of overlap-save segments for nb bins at overlap M: ceil(nb / (L - M)). */
int64_t fdas_num_segments(const fdas_params *p, int64_t nb);

#define FDAS_MAX_GROUPS 4

/* Template groups of the convolver.  Group g covers count[g] plane rows:
 * the bank rows first_row[g] .. first_row[g+1]-1 and, on a symmetric grid,
 * their -z partners (z = 0 once, in group 0); its segments discard
 * overlap[g] points (>= 2 h + 2 for each of its templates, a multiple of 4,
 * at least 64, at most M), so they yield L - overlap[g] bins each.  The
 * groups minimise the convolver's work, sum over groups of
 * (count + 0.5) / (L - overlap) (a segment's forward FFT costs about half
 * a template pass).  overlap, first_row, count: (host) FDAS_MAX_GROUPS
 * entries each, or NULL.  Returns the number of groups (1 on grids that are
 * not symmetric), or FDAS_E_INVAL. */
int32_t fdas_template_groups(const fdas_params *p, int32_t *overlap, int32_t *first_row,
                             int32_t *count);

/* Plane row width in floats for nb bins (2*nb with interbinning, else nb). */
int64_t fdas_plane_width(const fdas_params *p, int64_t nb);

/*
 * fdas_make_templates -- build the frequency-domain template bank
 * (a1: Section 2 Eq. 23; Section 3 Fig. 1 and the zero-filled centring of
 * the L-point filter; Section 4.2 +/-z symmetry).
 *
 * For bank row b with template z, the response is
 *   R_z(d) = int_0^1 exp(i 2 pi (z u^2/2 - (d + z/2) u)) du   (FP64, Fresnel)
 * for d = -h..h, the FIR kernel g[j] = conj(R_z(-j)) is placed circularly
 * (j >= 0 at the start, j < 0 at the end, zeros between) and
 *   H_z[k] = (1/L) sum_j g[j] exp(-i 2 pi j k / L),  k = 0..L-1
 * is stored in FP32 in the order the convolver for L reads it.
 * L = 2048, 4096 (one CTA per segment FFT): digit-reversed; a row is
 * L + 16 complex values:
 *   bank[(b*(L+16) + s)*2 + {0,1}] = H_z[k(s)] (re, im), slot s = 0..L-1,
 *   with Q = L/256, T = L/16, s = 2*(ip*T + t) + e, i = 2*ip + e,
 *   t = a*Q + c1, i = s2*Q + c2  ->  k(s) = a + 16*(c1 + Q*s2) + 256*c2;
 *   slots L..L+15 repeat, for the 16 frequencies of t = 0, the values at
 *   -k mod L: complex L + 2*j + 1 - e holds H_z[-k(s)] of slot
 *   s = 2*(7-j)*T + e (j = 0..7, e = 0..1), which lets conjugated templates
 *   be read with one access pattern for every thread.
 * L = 1024 (one warp per segment FFT, lane l holding k = l + 32 i in
 * register i): a row is 16 x 33 complex pairs (L + 32 complex values); pair
 * j*33 + l (l < 32) holds (H_z[l + 64 j], H_z[l + 64 j + 32]) and pair
 * j*33 + 32 holds (H_z[64 j + 32], H_z[(64 j + 64) mod 1024]), the values
 * lane 0 needs for a conjugated template, so that every lane reads a
 * conjugated row at pair 527 - 33 j - l.
 * bank: (device) fdas_bank_floats(p) floats, 16-byte aligned; written.
 * Errors: FDAS_E_INVAL for bad params or NULL bank.
 */
int fdas_make_templates(const fdas_params *p, float *bank, void *stream);

/* Workspace bytes fdas_normalise needs for n samples (0 if n unsupported):
 * n/2 complex values for a power of two, 3 P for the other even lengths (P
 * the least length >= n - 1 of the form 2^m or 3 * 2^m, 3 * 2^m <= 3 * 2^22). */
size_t fdas_normalise_workspace_bytes(int64_t n);

/*
 * fdas_normalise -- real FFT of the series and running-median
 * normalisation (a2-a3: Section 3 first paragraph on the workflow, Section
 * 4.1 real-to-complex transform, DFT sign of Section 4.2).
 *   X_k = sum_t series[t] exp(-i 2 pi k t / n),  k = 0..n/2-1,  X_0 := 0
 *   (the Nyquist bin is dropped);  for each block of `median_block`
 *   consecutive bins (the last block takes the remainder), m = the lower
 *   median (rank floor((len-1)/2)) of |X_k|^2 in the block, and
 *   spec_k = X_k / sqrt(m / ln 2)  (0 if m == 0), so noise power has mean 1.
 * series: (device) n floats, 8-byte aligned.  n: a power of two with
 *   2^13 <= n <= 2^25, or any even n with 2^13 < n <= 2^24; the N = n/2
 *   point DFT of the packed samples then runs as Bluestein's chirp-z
 *   convolution, Z_k = c_k sum_m (z_m c_m) conj(c_{k-m}), c_m = exp(-i pi
 *   m^2/N), with FFTs of length P >= n - 1 (2^m or 3 * 2^m).  median_block:
 *   32..8192.
 * spec: (device) n/2 complex, written.
 * work: (device) fdas_normalise_workspace_bytes(n) bytes, 16-byte aligned;
 *   scratch, contents undefined afterwards.
 * Errors: FDAS_E_INVAL (NULL pointers, unsupported n or block, work_bytes
 *   too small).
 */
int fdas_normalise(const float *series, int64_t n, int32_t median_block, float *spec,
                   void *work, size_t work_bytes, void *stream);

/* Bytes of the Bluestein kernel spectrum for a series of n samples: P
 * complex values (P as in fdas_normalise_workspace_bytes) for an even n that
 * is not a power of two and that fdas_normalise accepts, else 0. */
size_t fdas_bluestein_bytes(int64_t n);

/*
 * fdas_bluestein_prepare -- the input-independent part of fdas_normalise's
 * Bluestein convolution for n samples (N = n/2): the spectrum
 *   B = FFT_P(b),  b_j = conj(c_j) for 0 <= j < N, b_{P-j} = conj(c_j) for
 *   0 < j < N, zeros between,  c_j = exp(-i pi j^2 / N),
 * the same values fdas_normalise computes on every call.  Like an FFT
 * library's plan: computed once per length and passed to every
 * fdas_normalise_prepared call for that length, it removes one of the
 * three P-point FFTs from each call.
 * chirp_spec: (device) fdas_bluestein_bytes(n) bytes, 16-byte aligned;
 *   written.  work: (device) fdas_normalise_workspace_bytes(n) bytes,
 *   16-byte aligned, scratch.
 * Errors: FDAS_E_INVAL (NULL or misaligned pointers, n a power of two or
 *   unsupported, work_bytes too small).
 */
int fdas_bluestein_prepare(int64_t n, void *chirp_spec, void *work, size_t work_bytes,
                           void *stream);

/*
 * fdas_normalise_prepared -- fdas_normalise with the Bluestein kernel
 * spectrum supplied (from fdas_bluestein_prepare for the same n); the
 * results are bit-identical to fdas_normalise's.  For a power-of-two n
 * chirp_spec is not read (may be NULL) and the call is fdas_normalise.
 * Other arguments, layout and errors as fdas_normalise; FDAS_E_INVAL also
 * for a NULL or misaligned chirp_spec when n is not a power of two.
 */
int fdas_normalise_prepared(const float *series, int64_t n, int32_t median_block, float *spec,
                            void *work, size_t work_bytes, const void *chirp_spec,
                            void *stream);

/* Largest series length fdas_normalise_noalloc accepts (2^20 samples). */
#define FDAS_NOALLOC_MAX_N (1 << 20)

/*
 * fdas_normalise_noalloc -- fdas_normalise without a caller workspace.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory when they call in, e.g. a real-time pipeline
 * that reserves all of its device memory at start-up and must not allocate
 * afterwards (cudaMalloc may synchronise the device, and can fail once memory
 * is fragmented), or code running inside another program's hook with no
 * access to an allocator.  The workspace is a fixed device array inside the
 * library (FDAS_NOALLOC_MAX_N * 4 bytes = 4 MiB per GPU, held by every GPU
 * that loads the library until the process exits); nothing is allocated or
 * freed by the call.
 * The first call on a device looks up that device's copy of the array
 * (cudaGetSymbolAddress) and caches it; make that first call before any
 * stream capture.  All calls on a device share the one array: calls that may
 * overlap on the GPU (different streams, no ordering between them) race and
 * must not be issued.  The array needs no clearing between calls (every
 * value is written before it is read).
 * Arguments, layout and results are those of fdas_normalise.
 * Errors: FDAS_E_UNSUPPORTED if n > FDAS_NOALLOC_MAX_N or n is not a power
 * of two (other lengths need a larger workspace); otherwise as
 * fdas_normalise; FDAS_E_CUDA if the array's address cannot be obtained.
 */
int fdas_normalise_noalloc(const float *series, int64_t n, int32_t median_block, float *spec,
                           void *stream);

/*
 * fdas_correlate -- the fused overlap-save convolver (a4-a7: Section 3
 * Fig. 1 and the text after it; Section 4.1 Fig. 3; Section 4.2 fused
 * on-chip FFT/multiply/inverse-FFT/power; Eq. f-interp).
 * For every template row j (z_j) and bin r = 0..nb-1:
 *   F_j(r) = sum_{d=-h}^{h} spec[r + d] conj(R_{z_j}(d))   (spec = 0 outside [0,nb)),
 * computed by segments s = 0..S-1 of L bins starting at bin s*B - M/2
 * (B = L - M), one forward FFT per segment, one multiply + inverse FFT per
 * (segment, template), keeping positions M/2..M/2+B of each inverse FFT.
 * plane[j*row_stride + c] then holds the power plane (interbin layout in
 * fdas_params); the plane is written once, no other global memory is used.
 * spec: (device) nb complex.  bank: (device) as made by fdas_make_templates
 *   for the same p, 16-byte aligned.  plane: (device) K rows of row_stride
 *   floats, 16-byte aligned, row_stride >= fdas_plane_width and a multiple
 *   of 4.  nb >= 1.
 * fused: NULL, or a threshold applied to every plane value as it is written.
 * status: (device) int32 word for FDAS_STATUS_* bits, or NULL.
 * Errors: FDAS_E_INVAL (bad params, alignment, NULL pointers).
 */
int fdas_correlate(const fdas_params *p, const float *spec, int64_t nb, const float *bank,
                   float *plane, int64_t row_stride, const fdas_fused_threshold *fused,
                   int32_t *status, void *stream);

/*
 * fdas_debug_wait_timeout -- a diagnostic of the convolver's failure path,
 * not a search.  Every wait of the convolver is bounded; this call runs the
 * L = 1024 convolver (interbin 0 or 1) on the same arguments as
 * fdas_correlate but arms the first template row's barrier in every CTA
 * without issuing the row's copy, and lets each wait poll `polls` times
 * (1 .. 2^24).  The first wait of every CTA therefore runs out with nothing
 * in flight: the kernel ORs FDAS_STATUS_TIMEOUT into *status, stops all of
 * its warps, waits (bounded) for the copies it did issue, and returns.  The
 * plane is left with unspecified contents; the device stays usable.
 * status: (device) int32, required.  Errors: FDAS_E_INVAL (as fdas_correlate,
 * NULL status, polls out of range), FDAS_E_UNSUPPORTED (L != 1024 or
 * interbin 2).
 */
int fdas_debug_wait_timeout(const fdas_params *p, const float *spec, int64_t nb, const float *bank,
                            float *plane, int64_t row_stride, uint32_t polls, int32_t *status,
                            void *stream);

/* 16-bit plane element types (fdas_correlate_plane16). */
#define FDAS_PLANE_F16 1        /* IEEE binary16: 11 significant bits, largest finite 65504 */
#define FDAS_PLANE_BF16 2       /* bfloat16: 8 significant bits, FP32 range */

/*
 * fdas_correlate_plane16 -- fdas_correlate writing the plane as 16-bit
 * floats, 2 bytes per point instead of 4 (half the plane's memory and write
 * traffic; e.g. for harmonic summing or for more dispersion trials per plane
 * pool).  Powers are computed in FP32 exactly as in fdas_correlate and
 * rounded to nearest on the store; a power above 65504 becomes +inf in FP16.
 * The fused threshold compares the FP32 values, so its candidates, with their
 * FP32 powers, equal those of fdas_correlate.
 * type: FDAS_PLANE_F16 or FDAS_PLANE_BF16.
 * plane: (device) K rows of row_stride 16-bit elements, 16-byte aligned;
 *   row_stride >= fdas_plane_width and a multiple of 4.
 * Other arguments, layout and errors as fdas_correlate; FDAS_E_INVAL for any
 * other type; FDAS_E_UNSUPPORTED with interbin 2.
 */
int fdas_correlate_plane16(const fdas_params *p, int32_t type, const float *spec, int64_t nb,
                           const float *bank, void *plane, int64_t row_stride,
                           const fdas_fused_threshold *fused, int32_t *status, void *stream);

/*
 * fdas_harmonic_sum -- incremental harmonic sums of the plane with a fused
 * threshold (the search stage after the plane: a periodic signal with
 * fundamental (r, z) has its h-th harmonic at (h r, h z); Sections 3 and 7).
 * For every fundamental (row j, column c) whose harmonics lie on the plane:
 *   S_H(j, c) = sum_{h=1}^{H} plane[(h - 1) zmin/zstep + h j][h c],
 * for H = 2, 4, 8 (levels 1..nlevels), since column h c holds h r and row
 * (h - 1) zmin/zstep + h j holds h z_j.  A fundamental stops at the first
 * level whose harmonics leave the plane.  Every S_H > thr[level - 1] is
 * listed as a fdas_cand (z_idx = j, col = c, power = S_H, flags = H), in no
 * particular order; count (device) is reset by the call and ends holding the
 * number found, which may exceed cap (FDAS_STATUS_OVERFLOW then set).
 * plane_type: 0 (float), FDAS_PLANE_F16 or FDAS_PLANE_BF16.
 * plane: (device) fdas_num_templates(p) rows of row_stride elements; width
 *   columns (fdas_plane_width).  thr: (host) nlevels thresholds, nlevels 1..3.
 * Errors: FDAS_E_INVAL (bad params or pointers, zmin not a multiple of zstep).
 */
int fdas_harmonic_sum(const fdas_params *p, int32_t plane_type, const void *plane, int64_t width,
                      int64_t row_stride, int32_t nlevels, const float *thr, fdas_cand *out,
                      int32_t cap, int32_t *count, int32_t *status, void *stream);

/*
 * fdas_harmonic_plan_bytes, fdas_harmonic_plan, fdas_harmonic_sum_planned --
 * fdas_harmonic_sum with its thread blocks taken in ray order.  With y =
 * z/zstep, a fundamental (y, c) and all its harmonics (h y, h c) share
 * u = c/|y|.  The plan lists the (fundamental row, block of 1024 columns)
 * pairs sorted by u, so the rows that read the same 32-byte sectors of the
 * plane are read close together in time and L2 serves most repeats.  The
 * results equal fdas_harmonic_sum's: the same candidates, in another order.
 * fdas_harmonic_plan_bytes: device bytes of the plan for grid p and plane
 *   width `width` (0 if p is invalid or the plan would pass 2^31 blocks).
 * fdas_harmonic_plan: builds the plan on the host and copies it to `plan`
 *   (device, 16-byte aligned, plan_bytes >= fdas_harmonic_plan_bytes); it
 *   returns when the copy is done.  A plan serves every plane of the same
 *   grid and width.
 * fdas_harmonic_sum_planned: arguments as fdas_harmonic_sum, plus the plan.
 *   A plan made for another grid or width is detected on the device: no
 *   candidate is listed and FDAS_STATUS_BADPLAN is set in the status word.
 * Errors: FDAS_E_INVAL (bad params, pointers or sizes), FDAS_E_CUDA.
 */
#define FDAS_STATUS_BADPLAN 4   /* status-word bit: a harmonic plan does not match the call */
size_t fdas_harmonic_plan_bytes(const fdas_params *p, int64_t width);
int fdas_harmonic_plan(const fdas_params *p, int64_t width, void *plan, size_t plan_bytes);
int fdas_harmonic_sum_planned(const fdas_params *p, int32_t plane_type, const void *plane,
                              int64_t width, int64_t row_stride, int32_t nlevels, const float *thr,
                              fdas_cand *out, int32_t cap, int32_t *count, int32_t *status,
                              const void *plan, size_t plan_bytes, void *stream);

/*
 * fdas_noise_means -- mean power of pure noise in every plane row, for
 * significances (the paper leaves the statistics of single-bin, interbinned
 * and Fourier-interpolated powers open, Section 5.2).  With the normalised
 * spectrum unit-variance complex Gaussian noise, every plane value is
 * exponential: P(power > x) = exp(-x / mean).
 *   means[2j]   : even columns (full bins; integer positions with interbin 2)
 *                 sum_{|d|<=h} |R(d)|^2
 *   means[2j+1] : odd columns: interbin 1 half bins (pi/4)^2 sum_d |Rt(d) -
 *                 Rt(d-1)|^2 (Rt = R on |d| <= h, 0 outside); interbin 2
 *                 half-integer positions sum_{|d|<=h-1/2} |R(d)|^2; interbin 0
 *                 the full-bin mean again.
 * Row j holds z_j = zmin + j*zstep; R in FP64.  means: (device) 2 K floats.
 */
int fdas_noise_means(const fdas_params *p, float *means, void *stream);

/* Arithmetic of the convolver's radix-16 DFT passes (fdas_correlate_split). */
#define FDAS_PREC_FP32 0        /* FP32 on the CUDA cores, as fdas_correlate */
#define FDAS_PREC_FP16_SPLIT 1  /* FP16 hi+lo operands on tensor cores, FP32 accumulation */
#define FDAS_PREC_BF16_SPLIT 2  /* BF16 hi+lo operands on tensor cores, FP32 accumulation */
#define FDAS_PREC_BF16_SPLIT3 3 /* BF16 hi+mid+lo operands on tensor cores, FP32 accumulation */

/*
 * fdas_correlate_split -- fdas_correlate with the two radix-16 passes of
 * every forward and every inverse segment FFT done as matrix products on the
 * tensor cores (a9), for L = 2048 and 4096.  Section 4.2 writes the DFT as a product with the
 * Fourier matrix (Eq. matrixDFT) factorised into sparse stages
 * (Eq. CTfactorization); here one radix-16 stage over 32 segment columns is
 * the real product Y(32x32) = X(32x32) W(32x32) (re/im interleaved), each
 * operand split into a 16-bit part and a 16-bit remainder, x = x_hi + x_lo,
 * W = W_hi + W_lo, with Y = x_hi W_hi + x_hi W_lo + x_lo W_hi accumulated in
 * FP32 (the lo*lo term is dropped).  The radix-(L/256) pass, the twiddles,
 * the template product and the powers stay FP32; `bank` is the FP32 bank of
 * fdas_make_templates.
 * prec: FDAS_PREC_FP32 (identical to fdas_correlate), FDAS_PREC_FP16_SPLIT
 *   (parts of 11 significant bits each, 22 together; each DFT instance is
 *   scaled by a power of two into FP16's range), FDAS_PREC_BF16_SPLIT (8 + 8
 *   bits, FP32 range; its error exceeds 1e-3 of power at L >= 2048) or
 *   FDAS_PREC_BF16_SPLIT3 (three BF16 parts, 8 + 8 + 8 bits, six products:
 *   Xh Wh + Xh Wm + Xm Wh + Xh Wl + Xl Wh + Xm Wm).
 * Other arguments, layout and errors as fdas_correlate; FDAS_E_INVAL for any
 * other prec; FDAS_E_UNSUPPORTED for L = 1024 (its one-warp convolver has no
 * split form) or interbin 2 with a split prec.
 */
int fdas_correlate_split(const fdas_params *p, int32_t prec, const float *spec, int64_t nb,
                         const float *bank, float *plane, int64_t row_stride,
                         const fdas_fused_threshold *fused, int32_t *status, void *stream);

/*
 * Batched search over many series (a10), e.g. the dispersion trials of one
 * observation, each with its own length: one persistent launch walks the
 * (trial, segment, template) work items of all trials with the same static
 * balancing as fdas_correlate, so uneven lengths share the GPU evenly.
 */
typedef struct {
    const float *spec;      /* (device) nb complex, 8-byte aligned */
    int64_t nb;             /* bins of this series (>= 1) */
    float *plane;           /* (device) K rows of row_stride floats, 16-byte aligned */
    int64_t row_stride;     /* >= fdas_plane_width(p, nb), multiple of 4 */
    int64_t item_begin;     /* first work item of this trial (set by fdas_batch_plan) */
} fdas_trial;

/* Launch tuning (NULL or 0 fields = defaults). */
typedef struct {
    int32_t ctas_per_sm;    /* persistent CTAs per SM, 0 = the occupancy maximum */
    int32_t templates_per_block;  /* L = 1024: templates a CTA applies to a segment
                                   * before the next segment (the work order within
                                   * a template group); 0 = the whole group, so one
                                   * forward FFT per segment serves every template.
                                   * Ignored for L = 2048, 4096. */
} fdas_tuning;

/*
 * fdas_batch_plan -- validate a host array of trials for p and fill each
 * item_begin; returns the total number of work items (< 0: FDAS_E_INVAL).
 * Copy the array unchanged to device memory for fdas_correlate_batched.
 */
int64_t fdas_batch_plan(const fdas_params *p, fdas_trial *trials, int32_t ntrials);

/*
 * fdas_correlate_batched -- fdas_correlate for ntrials series in one launch.
 * trials: (device) the array planned by fdas_batch_plan; total_items its
 * return value.  Every plane gets what fdas_correlate would write for its
 * series.  With `fused`, candidates of all trials go to one list, the
 * trial's position in `trials` in bits 8..31 of fdas_cand.flags.  The call
 * only launches kernels (and resets the fused count), so it can be captured
 * into a CUDA graph once it has run once on the device.  Errors: FDAS_E_INVAL for bad params,
 * pointers or counts (the device array itself is not re-validated).
 */
int fdas_correlate_batched(const fdas_params *p, const fdas_trial *trials, int32_t ntrials,
                           int64_t total_items, const float *bank,
                           const fdas_fused_threshold *fused, const fdas_tuning *tuning,
                           int32_t *status, void *stream);

/*
 * fdas_threshold -- candidates of a power plane (a8: Section 3, comparing
 * the Fourier power with a pre-computed threshold).
 * Emits every (row, col) with plane value > thr (strict).  With
 * FDAS_CAND_PEAK in `want_flags`, flags gets FDAS_CAND_PEAK where the value
 * is a local maximum of its 8 neighbours (strictly above neighbours earlier
 * in row-major order, at least equal to later ones).
 * plane: (device) rows x width floats, row stride row_stride >= width.
 * out: (device) cap entries, unordered.  count: (device) reset to 0 by the
 * call, ends holding the total number of crossings (may exceed cap).
 * status: (device) FDAS_STATUS_OVERFLOW is OR-ed in when count > cap; may be
 * NULL.  Errors: FDAS_E_INVAL.
 */
int fdas_threshold(const float *plane, int32_t rows, int64_t width, int64_t row_stride,
                   float thr, int32_t want_flags, fdas_cand *out, int32_t cap,
                   int32_t *count, int32_t *status, void *stream);

/*
 * Candidate refinement over continuous (r, z) (a11).  The paper improves the
 * (r, z) of a detection by fine-binning the f-fdot plane around it (Section
 * 5.2, last paragraph); here the correlation power of Eq. 23 is evaluated
 * off the grid and maximised by gradient ascent:
 *   S(r, z) = sum_{k=[r]-m}^{[r]+m} spec[k] conj(R_z(k - r)),  P = |S|^2,
 *   [r] = floor(r + 1/2), spec[k] = 0 outside [0, nb),
 * with R_z(d) the FP64 template response of fdas_make_templates at real
 * offset d and real z.  m is the fixed tap half-window (h(zmax) covers every
 * template of a search).  All arithmetic is FP64 except the spectrum itself.
 *
 * fdas_refine_fwd: P[c], dP/dr (dPdr, optional), dP/dz (dPdz, optional) and
 *   S (re, im pairs, optional) for candidates c < ncand at (r[c], z[c]).
 * fdas_refine_bwd: accumulates into grad_spec (complex, nb values) the
 *   gradient of sum_c gP[c] P[c] with respect to the spectrum,
 *   grad_spec[k] += gP[c] * 2 S[c] R_z(k - r) (derivative with respect to the
 *   real part plus i times that with respect to the imaginary part); S as
 *   returned by fdas_refine_fwd.  Uses float atomics: the summation order of
 *   overlapping candidates is not fixed.
 * fdas_refine: `steps` steps of gradient ascent on log P per candidate,
 *   r += clamp(lr_r (dP/dr)/P, -0.5, 0.5), z += clamp(lr_z (dP/dz)/P, -2, 2),
 *   then r_out, z_out and the final P_out.
 * Pointers are device pointers; r, z, P, S, gP, r_out, z_out, P_out are
 * double arrays of ncand (S: 2*ncand).  Errors: FDAS_E_INVAL.
 */
int fdas_refine_fwd(const float *spec, int64_t nb, const double *r, const double *z,
                    int32_t ncand, int32_t m, double *P, double *dPdr, double *dPdz, double *S,
                    void *stream);
int fdas_refine_bwd(const float *spec, int64_t nb, const double *r, const double *z,
                    int32_t ncand, int32_t m, const double *S, const double *gP, float *grad_spec,
                    void *stream);
int fdas_refine(const float *spec, int64_t nb, const double *r_in, const double *z_in,
                int32_t ncand, int32_t m, int32_t steps, double lr_r, double lr_z, double *r_out,
                double *z_out, double *P_out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* FDAS_H */
