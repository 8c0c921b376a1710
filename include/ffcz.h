/*
 * ffcz.h -- C ABI of the FFCz alternating-projection library for B300 (sm_103a).
 *
 * The library edits a lossy compressor's spatial error vector e = x_hat - x
 * until it lies in both the s-cube |e_n| <= eps_s and the f-cube
 * |Re delta_k| <= eps_f, |Im delta_k| <= eps_f, where delta = DFT(e) is the
 * unnormalised DFT of Eq. 1 and its nD analogue (Sec. III, Sec. IV-A,
 * constraints_v1).  The loop is Alg. 1 (Sec. IV-B): forward FFT, feasibility
 * check, f-cube clip, inverse FFT, s-cube clip.
 *
 * Conventions shared by every call
 *  - Device pointers are CUDA global-memory addresses on the device that was
 *    current when the plan was made.  The caller owns them; the library never
 *    frees or retains them after a call returns.
 *  - The plan owns all of its workspace (spectrum buffers, loop state).
 *  - All work is ordered on the plan's stream.  Each call blocks the calling
 *    host thread until its stream work is done and its stats are written.
 *  - Errors never cross the ABI as exceptions: every call returns an
 *    ffcz_status; ffcz_last_error() gives a detail string for the calling
 *    thread's most recent failure.
 *  - A field is row-major with the LAST axis contiguous.  Supported items:
 *    2D and 3D with every axis a power of two, each axis length in [8, 1024]
 *    and the last axis in [16, 2048]; 1D of ANY length N in [32, 524288]
 *    (the DFT is then computed by Bluestein's chirp-z identity on a
 *    power-of-two length P >= 2N - 1).  Other shapes return
 *    FFCZ_ERR_UNSUPPORTED.
 *  - Batches: `batch` items of one rank `ndim`; item i has the shape
 *    shapes[i*ndim .. i*ndim+ndim-1]; items are packed back to back in the
 *    float32 buffer, item i starting after the elements of items 0..i-1.
 *    Every item runs its own loop and stops on its own (Alg. 1 per item).
 */
#ifndef FFCZ_H_
#define FFCZ_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ffcz_plan_s* ffcz_plan_t;

typedef enum {
  FFCZ_OK = 0,
  FFCZ_ERR_INVALID = 1,        /* bad argument (null pointer, bad bound, ...) */
  FFCZ_ERR_UNSUPPORTED = 2,    /* shape or option the library does not handle */
  FFCZ_ERR_CUDA = 3,           /* a CUDA runtime call failed */
  FFCZ_ERR_NOT_CONVERGED = 4,  /* max_iters reached; the last iterate is in e */
  FFCZ_ERR_CERT_FAILED = 5,    /* FP64 certification failed after all repairs */
  FFCZ_ERR_NONFINITE = 6,      /* NaN or Inf met in e or in its spectrum */
  FFCZ_ERR_TIMEOUT = 7,        /* a bounded device wait gave up */
  FFCZ_ERR_OOM = 8             /* workspace allocation failed */
} ffcz_status;

/* Options.  Fill with ffcz_default_opts() and change what you need. */
typedef struct {
  int32_t max_iters;   /* iteration cap (the paper loops without one); default 10000 */
  int32_t min_iters;   /* do not stop before this many iterations (forced runs); 0 */
  double shrink;       /* eta: clip to E(1-eta), Delta(1-eta), stop when the
                          violation <= Delta(1-eta/2) (bound shrink of Sec. IV-B,
                          m = 16); default 2^-16 */
  int32_t precision;   /* 32: FP32 loop (default); 64: FP64 loop */
  int32_t certify;     /* 1 (default): FP64 certification after the loop */
  int32_t max_repairs; /* FP64 repair rounds when certification fails; default 2 */
  int32_t K;           /* backward: number of forced forward iterations; 50 */
  int32_t ckpt_every;  /* backward: checkpoint interval m; 10 */
  int32_t chunk;       /* max iterations launched between host checks; 16 */
  int32_t use_graph;   /* 0: direct launches, host checks between chunks;
                          1: chunks replayed as CUDA graphs, host checks between;
                          2 (default): the whole loop on the device, one graph
                          with a conditional WHILE node (no host round trip) */
  int32_t count_active;/* 1 (default): count active clips for ffcz_stats */
  int32_t edits;       /* 1: record the spatial and frequency edits of Alg. 1
                          (ffcz_edits_dense / ffcz_edits_compact read them);
                          default 0 */
  int32_t pointwise;   /* 1: pointwise bounds E_n, Delta_k (ffcz_correct_pw);
                          default 0 */
  int32_t method;      /* projection of the loop (the alternatives Sec. III
                          names to POCS); every method checks its candidate
                          point with the rule of Alg. 1 and returns it:
                          0 (default) POCS, Alg. 1;
                          1 Dykstra: y = P_F'(x + p), p += x - y,
                            x = P_S'(y + q), q += y - x; converges to the
                            point of the intersection nearest to e0; checks x;
                          2 Douglas-Rachford on (F', S'): y = P_F'(z),
                            x = P_S'(2y - z), z += x - y; checks x;
                          3 ADMM, a = P_F'(b - u), b = P_S'(a + u),
                            u += a - b; checks a against the s-cube
                            (max|a| <= E(1 - eta/2)).
                          Methods 1-3 need precision 32 and no edits or
                          pointwise bounds (else UNSUPPORTED); they use one
                          more spectrum buffer (1, 2; 1D items: N complex
                          values each) and two float32 fields (1, 3); a
                          failed certification is repaired with FP64
                          iterations of Alg. 1 */
  int32_t keep_masks;  /* 1: ffcz_correct_ckpt also keeps the clips' masks of
                          all K steps in the plan (about 1 bit per point for
                          the spatial and 2 per packed value for the frequency
                          masks, per step), and ffcz_correct_backward_ckpt
                          then runs the adjoint steps without replaying the
                          segments (1D items: one byte per point and per bin
                          per step); default 0: replay from the checkpoints */
} ffcz_opts;

/* Per-item results. */
typedef struct {
  int32_t status;      /* ffcz_status of this item */
  int32_t iters;       /* (f-clip, s-clip) pairs executed */
  int32_t repairs;     /* FP64 repair rounds run */
  int32_t certified;   /* 1 if the FP64 check passed against the true bounds */
  int32_t preclipped;  /* 1 if e0 was outside the s-cube and was clipped first */
  int32_t host_copies; /* ffcz_correct_host: copies of the field back to
                          e_host (0 when the field came out unchanged, the
                          host buffer already holding the result); else 0 */
  double f_ratio;      /* last loop violation / eps_f (working precision);
                          method 3 after >= 1 iteration: max|a_t| / eps_s,
                          its stopping measure */
  double s_ratio;      /* max|e| / eps_s after the call (FP64 check) */
  double f_margin64;   /* 1 - (FP64 violation + FP64 FFT error bound) / eps_f */
  double s_margin64;   /* 1 - max|e| / eps_s (exact) */
  int64_t active_s;    /* points moved by the last s-clip */
  int64_t active_f;    /* full-spectrum bins moved by the last f-clip */
  float ms_total;      /* device time of the whole call, milliseconds */
  float ms_cert;       /* device time of certification, milliseconds */
} ffcz_stats;

/* Fill *opts with the defaults listed above. */
void ffcz_default_opts(ffcz_opts* opts);

/*
 * ffcz_plan -- validate the shapes, size and allocate the workspace, upload
 * the FP64-derived twiddle tables and bind the plan to `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).
 *   out     : receives the plan handle (owned by the caller; ffcz_destroy)
 *   ndim    : 1, 2 or 3 (every item of a plan has this rank)
 *   shapes  : host array of batch*ndim extents (see the batch convention)
 *   batch   : number of items, >= 1
 *   opts    : NULL for defaults; copied into the plan
 * Errors: INVALID (null out, ndim/batch out of range), UNSUPPORTED (shape),
 * OOM, CUDA.
 * Workspace: two float32 spectrum buffers (4 bytes per point each; 8 bytes
 * per Bluestein point P for 1D items), one FP64 spectrum buffer for
 * certification (twice that) and, when precision 64 or a repair needs them,
 * two FP64 loop buffers (allocated on first use).  1D plans also hold the
 * FFT of each item's wrapped chirp (built here in float32, in float64 on
 * first use).
 */
ffcz_status ffcz_plan(ffcz_plan_t* out, int ndim, const int64_t* shapes,
                      int64_t batch, const ffcz_opts* opts, void* cuda_stream);

/* Rebind the plan to another stream (e.g. torch's current stream). */
ffcz_status ffcz_set_stream(ffcz_plan_t plan, void* cuda_stream);

/* Bytes of device workspace the plan holds now. */
size_t ffcz_workspace_bytes(ffcz_plan_t plan);

/*
 * Edits (Alg. 1 "spat_edits"/"freq_edits", Sec. IV-B), recorded by
 * ffcz_correct when the plan was created with opts.edits = 1 (1D, 2D and
 * 3D items).  Spatial edits: the sum of the s-clip displacements eps' - eps
 * (the pre-loop clip of an input outside the s-cube included), float32,
 * laid out like e.  Frequency edits: the sum of the f-clip displacements
 * delta' - delta of every check that did not stop the loop, stored as the
 * half spectrum of a real-input FFT: complex64 (Re, Im float pairs)
 * [Nz][Ny][Nx/2+1] per item (2D: [Ny][Nx/2+1]; 1D: [N/2+1]), items back to
 * back.  In exact arithmetic e_out - e_in = spatial edits + IFFT(frequency
 * edits).
 * The edits describe the last ffcz_correct call on the plan.
 *
 * ffcz_edit_layout -- (any plan; 1D items: N points and N/2 + 1 bins, the
 * layout of their pointwise frequency bounds) sizes and offsets for item `item`
 * (0-based), or the totals for item = -1, into out[6] (host): points, half-spectrum bins,
 * offset of the item's spatial flags (bytes), spatial codes (int32), frequency
 * flags (bytes), frequency codes (int32; two per bin).  For item = -1 the
 * last four are the array sizes ffcz_edits_compact needs.
 *
 * ffcz_edits_dense -- copy the dense edits to device memory: s_dev (float32,
 * total points) and f_dev (float32 pairs, total bins x 2); either may be NULL.
 *
 * ffcz_edits_compact -- CompactEdits and QuantizeEdits (Alg. 1) of every
 * item into device arrays at the offsets of ffcz_edit_layout: flags = 1 for
 * each nonzero component (a frequency bin is nonzero if Re or Im is), packed
 * 8 per byte with the first component in the least significant bit; codes =
 * rint(edit / q) for the nonzero components in order, q = 2 eps / 2^m_bits
 * (eps = eps_s or eps_f of the last call, m_bits in [2, 30]; the paper uses
 * 16), the division and rounding in float32, ties to even, Re and Im coded
 * separately.  counts (host, 2 per item, may be NULL) receives the number of
 * nonzero spatial and frequency components of each item.  Synchronises the
 * plan's stream.  All three return FFCZ_ERR_INVALID for a plan created without
 * opts.edits.
 */
ffcz_status ffcz_edit_layout(ffcz_plan_t plan, int64_t item, int64_t* out);
ffcz_status ffcz_edits_dense(ffcz_plan_t plan, float* s_dev, float* f_dev);
ffcz_status ffcz_edits_compact(ffcz_plan_t plan, int m_bits, uint8_t* s_flags, int32_t* s_codes,
                               uint8_t* f_flags, int32_t* f_codes, int64_t* counts);

/*
 * ffcz_apply_edits -- the decompression side (Sec. IV-B, "Applying edits to
 * the decompressed data"): x_hat += S~ + IFFT(F~), where S~ and F~ are the
 * dequantized edits (code * q, q = 2 eps / 2^m_bits, eps = eps_s / eps_f per
 * item) given in the stored form of ffcz_edits_compact (flags and codes at
 * the offsets of ffcz_edit_layout; device memory, read only).  xhat_dev:
 * device float32, the packed items of the base reconstruction, updated in
 * place.  Any plan (opts.edits not needed); uses the plan's spectrum
 * buffers, so it must not overlap a ffcz_correct call on the same plan.
 * Synchronises the plan's stream.
 */
ffcz_status ffcz_apply_edits(ffcz_plan_t plan, float* xhat_dev, const double* eps_s, const double* eps_f,
                             int m_bits, const uint8_t* s_flags, const int32_t* s_codes,
                             const uint8_t* f_flags, const int32_t* f_codes);

/*
 * ffcz_edits_compact16 -- ffcz_edits_compact with the codes stored in 16
 * bits (Sec. IV-B: m-bit codes, m = 16 in the paper), for m_bits in [2, 16].
 * The codes are those of ffcz_edits_compact, in the same order; a code in
 * [-32767, 32767] is stored as itself (int16), any other (the end point
 * 2^15 of m = 16, where an edit equals the bound, or an edit larger than the
 * bound) as the escape -32768, its value going to the item's int32 list
 * (*_wide) in order of appearance.  Regions: flags as in ffcz_edit_layout;
 * codes and lists at the same element offsets as ffcz_edit_layout's code
 * offsets (int16 and int32 elements; a list never holds more entries than
 * its region has codes).  counts (host, 4 per item, may be NULL): nonzero
 * spatial components, nonzero frequency bins, spatial escapes, frequency
 * escapes -- what a reader needs with the flags, codes and lists.
 * Synchronises the plan's stream; FFCZ_ERR_INVALID for a plan created
 * without opts.edits or m_bits outside [2, 16].
 *
 * ffcz_apply_edits16 -- ffcz_apply_edits from the 16-bit form: the arrays
 * of ffcz_edits_compact16 (device, read only) and its counts (host, 4 per
 * item).  FFCZ_ERR_INVALID when a count is out of range or the number of
 * escapes in an item's codes differs from its count (nothing applied).
 */
ffcz_status ffcz_edits_compact16(ffcz_plan_t plan, int m_bits, uint8_t* s_flags, int16_t* s_codes,
                                 int32_t* s_wide, uint8_t* f_flags, int16_t* f_codes, int32_t* f_wide,
                                 int64_t* counts);
ffcz_status ffcz_apply_edits16(ffcz_plan_t plan, float* xhat_dev, const double* eps_s, const double* eps_f,
                               int m_bits, const uint8_t* s_flags, const int16_t* s_codes, const int32_t* s_wide,
                               const uint8_t* f_flags, const int16_t* f_codes, const int32_t* f_wide,
                               const int64_t* counts);

/*
 * ffcz_correct_pw -- ffcz_correct with pointwise bounds (the generalisation
 * E_n, Delta_k^Re, Delta_k^Im named in Sec. IV-A), for a plan created with
 * opts.pointwise = 1.
 *   eb_dev : device float32, E_n > 0 (normal) for every point, laid out like e.
 *   db_dev : device float32 pairs (Delta^Re, Delta^Im) > 0 on each item's
 *            half spectrum of a real-input FFT, [Nz][Ny][Nx/2+1] (2D:
 *            [Ny][Nx/2+1]; 1D: [N/2+1], bin N - k taking the bounds of bin
 *            k), items back to back (the offsets of ffcz_edit_layout).
 *            Bounds in the kx = 0 and kx = Nx/2 planes must be even in
 *            (ky, kz), as the spectrum of a real field is.
 * The point n is clipped to E_n (1 - eta), Re/Im of bin k to
 * Delta_k^Re/Im (1 - eta); the loop stops when max_k max(|Re|/Delta^Re,
 * |Im|/Delta^Im) <= 1 - eta/2.  Stats carry the normalised ratios (f_ratio,
 * s_ratio; margins 1 - ratio), and certification requires max|e_n|/E_n <= 1
 * and (FP64 normalised violation) + (FP64 rounding bound) / min_k Delta_k <= 1.
 * The bounds are copied into the plan (the call may reuse its inputs at
 * once).  Bounds must be normal float32 values (FLT_MIN <= b <= FLT_MAX):
 * zero, subnormal, negative or non-finite bounds give FFCZ_ERR_INVALID.  On a
 * pointwise plan ffcz_correct, ffcz_correct_host, ffcz_check, the backward and
 * the edit compaction/application (whose codes are relative to scalar bounds)
 * return FFCZ_ERR_INVALID.
 */
ffcz_status ffcz_correct_pw(ffcz_plan_t plan, float* e_dev, const float* eb_dev, const float* db_dev,
                            ffcz_stats* stats);

/*
 * ffcz_power_spectrum_bounds -- pointwise frequency bounds that keep every
 * shell of the power spectrum (Sec. III: P(k) = sum of |X|^2 over the bins
 * at rounded distance k from the zero frequency, after the normalisation
 * (x - mean)/mean) within a relative error rho (Sec. V, power-spectrum
 * preservation).  Reading of the unspecified mapping: per shell s, with
 * A_s = sum |X_k| and P_s = sum |X_k|^2 over the shell's n_s bins, any error
 * with |Re|, |Im| <= d_s changes P_s by at most 2 sqrt2 d_s A_s + 2 n_s d_s^2,
 * so d_s is the positive root of that expression = rho P_s; the
 * zero-frequency shell takes the smallest d of the other shells.  The mean
 * normalisation cancels out of d (a relative bound is scale-free).
 *   x_dev  : device float32, the ORIGINAL fields (packed items).
 *   rho    : host, one relative bound > 0 per item.
 *   db_dev : device float32 pairs, output in the layout ffcz_correct_pw reads
 *            (Delta^Re = Delta^Im = d of the bin's shell; 1D items: the
 *            shell of bin k <= N/2 is k, the pair of bins k and N - k).
 * The transform runs in float32 on the plan's first spectrum buffer (not
 * concurrently with a ffcz_correct on the same plan); synchronises.
 */
ffcz_status ffcz_power_spectrum_bounds(ffcz_plan_t plan, const float* x_dev, const double* rho, float* db_dev);

/*
 * ffcz_plan_describe -- one line per item group: the group's shape, member
 * count and the pass variants the tuner chose for it (tile width, or "tma"
 * for the persistent copy-engine-fed kernels).  Writes at most `len` bytes
 * including the terminating NUL into `buf` (host memory, caller-owned);
 * returns the length the full text needs (excluding the NUL), or -1 for a
 * null plan.
 */
int ffcz_plan_describe(ffcz_plan_t plan, char* buf, int len);

/*
 * ffcz_correct -- Alg. 1 on every item, in place.
 *   e_dev  : device float32, the packed items; in: e0 = x_hat - x (Alg. 1,
 *            first step); out: the corrected error e*.  x_hat' = x + e*.
 *   eps_s  : host array[batch], spatial bounds E > 0 (constraints_v1)
 *   eps_f  : host array[batch], frequency bounds Delta > 0 in unnormalised DFT
 *            units (constraints_v1; Eq. 1 scaling)
 *   stats  : host array[batch] or NULL
 * Before the loop, an item with some |e0_n| > E is clipped to E(1-eta)
 * (the paper assumes e0 starts in the s-cube).  An item that is already
 * feasible returns after 0 iterations with e bit-identical.  On
 * NOT_CONVERGED the last iterate is left in e.  With certify = 1 the result
 * is checked in FP64 (see ffcz_check) and, on failure, refined by FP64
 * iterations (at most max_repairs rounds).
 * Returns the worst item status (OK < NOT_CONVERGED < CERT_FAILED <
 * NONFINITE) or a call-level error.
 */
ffcz_status ffcz_correct(ffcz_plan_t plan, float* e_dev, const double* eps_s,
                         const double* eps_f, ffcz_stats* stats);

/*
 * ffcz_correct_host -- ffcz_correct on host memory: copies e_host to the
 * plan's device staging buffer, corrects, copies the result back.
 * e_host may be pageable or pinned; it is read and written in place.  For
 * single-item 2D/3D plans the upload runs in row chunks while the FP64
 * certification's x pass processes the chunks already on the device; when
 * the loop stops at 0 iterations without a pre-clip (the field unchanged)
 * the certification continues from that pass, else it runs in full (3D
 * items: the y pass of the certification runs on each chunk of whole
 * z-planes too).  A field that comes out of the loop unchanged (0 iterations,
 * no pre-clip) is not copied back: e_host already holds it.  Otherwise the
 * copy back starts on a second stream as soon as the loop is done, while the
 * FP64 certification (which only reads the field) runs; if a repair round
 * changes the field, it waits for that copy and copies the field again.
 * stats.host_copies counts the copies back.
 */
ffcz_status ffcz_correct_host(ffcz_plan_t plan, float* e_host, const double* eps_s,
                              const double* eps_f, ffcz_stats* stats);

/*
 * ffcz_check -- FP64 certification of e against the TRUE bounds
 * (constraints_v1 with <=): max|e_n| <= E and, for every DFT bin,
 * max(|Re|, |Im|) + b <= Delta, where b is a rigorous bound on the FP64 FFT's
 * rounding error (error analysis of Cooley-Tukey FFTs: log2(N) stages of
 * radix-2/4/8 butterflies with correctly rounded twiddles):
 * b = 10 (log2 N + 2) u sqrt(N) ||e||_2, u = 2^-53, with ||e||_2 bounded by
 * the smaller of the float32 sum of squares (inflated for its rounding and
 * for squares below the float32 normal range) and sqrt(N) max|e|; for 1D
 * Bluestein items b = 10 (2 log2 P + 6) u 2N ||e||_2.
 * Does not modify e.  stats[i].certified, s_ratio, f_margin64, s_margin64 are
 * filled.  Returns OK if every item passes, CERT_FAILED otherwise.
 */
ffcz_status ffcz_check(ffcz_plan_t plan, const float* e_dev, const double* eps_s,
                       const double* eps_f, ffcz_stats* stats);

/*
 * ffcz_correct_backward -- vector-Jacobian product of e0 -> e_K, where e_K
 * is the result of exactly K forced iterations (opts.K; min_iters = max_iters
 * = K; no certification).  One step e <- P_s(IDFT(P_f(DFT(e)))) has the
 * Jacobian M_s IDFT M_f DFT; IDFT M_f DFT is symmetric in the real frequency
 * basis of Sec. IV-A, so the transposed step is g <- IDFT(M_f DFT(M_s g)).
 * M_s, M_f are the clips' active-set masks (1 where |value| <= bound).  The
 * masks are regenerated by replaying the forward from float32 checkpoints of
 * e taken every opts.ckpt_every iterations.
 *   e0_dev       : device float32 input of the forward (not modified)
 *   grad_out_dev : device float32 dL/de_K
 *   grad_in_dev  : device float32 output dL/de0 (may not alias the others)
 * All three packed like e (items back to back); eps_s / eps_f per item.  Plans
 * of any batch and any mix of shapes: every item runs exactly K steps, and
 * each item's product is that of its own single-item plan.  1D items run the
 * transposed step on the Bluestein passes: g <- Re(IDFT(M_f DFT(M_s g))), M_f
 * per bin k < N (the forward takes the real part after its inverse).
 */
ffcz_status ffcz_correct_backward(ffcz_plan_t plan, const float* e0_dev,
                                  const float* grad_out_dev, float* grad_in_dev,
                                  const double* eps_s, const double* eps_f);

/*
 * Differentiable form without the second forward: ffcz_correct_ckpt is
 * ffcz_correct for the plan of ffcz_correct_backward (min_iters = max_iters
 * = opts.K, precision 32, certify 0; else FFCZ_ERR_INVALID: a repair would
 * change e_K after the recorded steps) whose loop also writes the backward's float32
 * checkpoints -- e_t at t = 0 (e0 after the pre-clip), m, 2m, ... below K,
 * m = opts.ckpt_every -- to ckpt_dev; ffcz_correct_backward_ckpt then
 * replays each segment from them instead of running the K-step forward
 * again (same vector-Jacobian product as ffcz_correct_backward, bit for bit).
 *   ckpt_dev : device float32 of ffcz_ckpt_floats(plan) values
 *              (ceil(K / m) x N), owned by the caller; the pair of calls
 *              must use the same e0, bounds and buffer.
 *   e_dev    : (forward) e0 in, e_K out; e0_dev (backward): the forward's
 *              input, unmodified.
 * The forward's loop runs its x pass in the form with checkpoint writes.
 * ffcz_ckpt_floats returns 0 for a NULL plan.
 */
int64_t ffcz_ckpt_floats(ffcz_plan_t plan);
ffcz_status ffcz_correct_ckpt(ffcz_plan_t plan, float* e_dev, const double* eps_s, const double* eps_f,
                              float* ckpt_dev, ffcz_stats* stats);
ffcz_status ffcz_correct_backward_ckpt(ffcz_plan_t plan, const float* e0_dev, const float* ckpt_dev,
                                       const float* grad_out_dev, float* grad_in_dev,
                                       const double* eps_s, const double* eps_f);

/* Release the plan and its workspace.  NULL is ignored. */
void ffcz_destroy(ffcz_plan_t plan);

/* Static description of a status code. */
const char* ffcz_strerror(ffcz_status status);

/* Detail of the calling thread's most recent failure ("" if none). */
const char* ffcz_last_error(void);

/* Number of kernel launches issued by this process so far (all plans). */
int64_t ffcz_launch_count(void);

/*
 * ffcz_fp64_peak -- measurement support, not part of the method: the FP64
 * rate of the current device, measured with a kernel of independent FP64
 * dependency chains (kind 0: fused multiply-adds, counted as 2 flops each;
 * kind 1: adds, 1 flop each) on eight 256-thread blocks per SM, timed with
 * CUDA events on `cuda_stream` (best of three after a warm-up).  Writes
 * flops per second to *flops_per_s (host).  Allocates and frees 8 bytes of
 * device memory; synchronises the stream.
 */
ffcz_status ffcz_fp64_peak(int kind, void* cuda_stream, double* flops_per_s);

/*
 * Per-kernel device-time profile of a plan (measurement support, not part of
 * the method).  ffcz_profile_enable(plan, 1) clears the table and makes every
 * later call record a CUDA event pair around each of its launches (loop
 * chunks are then launched directly instead of as graphs); 0 turns it off.
 * Entries are keyed by kernel kind, precision and pencil length, e.g.
 * "chk<f32,512>"; ffcz_profile_entry copies entry i's key into name
 * (truncated to name_len), its summed milliseconds and its launch count.
 */
ffcz_status ffcz_profile_enable(ffcz_plan_t plan, int on);
int ffcz_profile_count(ffcz_plan_t plan);
ffcz_status ffcz_profile_entry(ffcz_plan_t plan, int i, char* name, int name_len, double* ms,
                               int64_t* launches);

/*
 * ffcz_check_static -- ffcz_check for one 2D or 3D field WITHOUT a plan and
 * WITHOUT allocating device memory.  The paper has no counterpart: this is an
 * entry point for callers that cannot allocate when they need the check --
 * hosts whose memory manager (a framework's caching allocator, a pool sized
 * at start-up) owns the whole device so that no other allocation may happen,
 * callback-driven pipelines that must not reach the allocator, and
 * validation steps that must not fail for lack of memory mid-run.
 *   e_dev       : device float32 field (row-major, last axis contiguous);
 *                 read only
 *   ndim, shape : 2 or 3 extents, same rules as ffcz_plan
 *   eps_s, eps_f: the true bounds E, Delta (> 0)
 *   cuda_stream : cudaStream_t the work is ordered on (NULL = legacy stream);
 *                 the call waits for this stream before returning (the
 *                 stats are read back to the host)
 *   stats       : host pointer or NULL; certified, s_ratio, f_margin64 and
 *                 s_margin64 are filled, the rest is zero
 * Scratch: a fixed file-scope device array (about 32 MiB plus 260 KiB of
 * tables and state) that every device loading the library holds until the
 * process exits.  Fields of more than FFCZ_STATIC_MAX_POINTS points are
 * rejected with FFCZ_ERR_INVALID (detail in ffcz_last_error()) before any
 * GPU work.  The FIRST call on each device sets that device up (takes the
 * array's address with cudaGetSymbolAddress, uploads the twiddle tables with
 * blocking copies and loads every kernel the call launches): make it before
 * any stream capture.  All calls on a device share the array (each call
 * re-initialises what must start at zero); calls whose GPU work overlaps --
 * other streams, other host threads -- race and may return wrong results.
 * No cudaMalloc, cudaFree or allocating library routine is called.
 * Returns OK (certified), CERT_FAILED, INVALID, UNSUPPORTED or CUDA.
 */
#define FFCZ_STATIC_MAX_POINTS (1 << 22)
ffcz_status ffcz_check_static(const float* e_dev, int ndim, const int64_t* shape,
                              double eps_s, double eps_f, void* cuda_stream,
                              ffcz_stats* stats);

#ifdef __cplusplus
}
#endif

#endif /* FFCZ_H_ */
