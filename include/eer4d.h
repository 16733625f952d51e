/*
 * eer4d.h -- C ABI of libeer4d.so: linear-index electron-event (EER) data to
 * COM-DPC and single-sideband (SSB) phase-contrast images on one GB300 GPU.
 *
 * Paper: Pelz et al., "Real-time interactive 4D-STEM phase-contrast imaging
 * from electron event representation data" (arXiv 2104.06336).
 *
 * Conventions for every entry point
 * ---------------------------------
 * - d_* arguments are device pointers; h_* arguments are host pointers.  The
 *   caller allocates and owns every buffer.  The library allocates device
 *   memory only in eer4d_plan_create (small tables) and frees it in
 *   eer4d_plan_destroy.  No entry point synchronises the device.
 * - All work is enqueued on `stream` (a cudaStream_t; NULL is the legacy
 *   default stream) and runs asynchronously.
 * - Argument errors found on the host return a negative EER4D_E* code at once
 *   and enqueue nothing.  Data errors found on the device (bad index, bad
 *   offsets, count overflow, timeout) never trap: the offending events are
 *   dropped, a bit is OR-ed into d_status[0] and counters are bumped.
 *   d_status points to 4 uint32 words that the caller zeroes before use:
 *     [0] EER4D_ST_* bits   [1] dropped events (idx >= W*H)
 *     [2] pixel counts above 2048 in one frame   [3] reserved
 *   eer4d_status_code() maps a copied-back status block to an EER4D_E* code.
 * - A CUDA launch failure returns EER4D_ECUDA.
 *
 * Event data (Sec. II, Fig. 1b): frame f (scan position f = y*scan_nx + x,
 * raster order) holds the events d_idx[d_off[f] .. d_off[f+1]) of the
 * uint32 raw linear detector indices idx = y*det_w + x.  d_off is uint64
 * with n_frames+1 entries indexing into d_idx, which has n_idx entries.
 */
#ifndef EER4D_H
#define EER4D_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ------------------------------------------------------ */
#define EER4D_OK         0
#define EER4D_EINVAL    -1  /* bad argument (host check) */
#define EER4D_ERANGE    -2  /* event index >= det_w*det_h (device) */
#define EER4D_EOFFSETS  -3  /* offsets decreasing or beyond n_idx (device) */
#define EER4D_EOVERFLOW -4  /* a binned pixel got more than 2048 events in one frame (device) */
#define EER4D_ETIMEOUT  -5  /* a bounded device wait gave up (device) */
#define EER4D_ECUDA     -6  /* a CUDA call failed */
#define EER4D_ENOMEM    -7  /* plan tables could not be allocated */
#define EER4D_EORDER    -8  /* ssb_accumulate chunks not delivered in frame order */
#define EER4D_ESCRATCH  -9  /* plan needs more than the static scratch of ssb_reconstruct_static */
#define EER4D_EBOUNDS  -10  /* a bounds check of the EER4D_CHECKS debug build failed (device) */

/* ---- device status bits (d_status[0]) ---------------------------------- */
#define EER4D_ST_RANGE    0x01u
#define EER4D_ST_OFFSETS  0x02u
#define EER4D_ST_OVERFLOW 0x04u
#define EER4D_ST_TIMEOUT  0x08u
#define EER4D_ST_ROTATION 0x10u  /* candidates of one call differ in rotation */
#define EER4D_ST_BOUNDS   0x20u  /* debug build (-DEER4D_CHECKS): an index derived from data or
                                    tables fell outside its buffer; the access was skipped */

/* ---- plan options ------------------------------------------------------- */
#define EER4D_FP32_FFT   0  /* scan transform: FP32 radix FFT */
#define EER4D_SPLIT_FP16 1  /* scan transform: split hi+lo FP16 DFT on tensor cores */
#define EER4D_FP32_FFT_2PASS 2  /* FP32 radix FFT, always as two launches (x per chunk,
                                   y at the end) through a full-size intermediate; the
                                   same arithmetic as EER4D_FP32_FFT */
#define EER4D_FP32_STOCKHAM 3   /* the plain form: FP32 shared-memory Stockham FFT
                                   (radix 8/4/2 and odd primes) for both axes, two
                                   launches plus a transpose */
#define EER4D_NORM_NONE  0  /* Eq. 3 as printed: S(K) = sum over K(K) */
#define EER4D_NORM_AREA  1  /* S(K) / |K(K)| (0 when the set is empty) */

/* Detector, crop and scan geometry.  k = (u - dc_u, v - dc_v) is a binned
 * detector pixel measured from the optical axis.  Binned pixel
 * u = floor((x - crop_x0) / bin), v = floor((y - crop_y0) / bin),
 * 0 <= u < pw, 0 <= v < ph.  Pixels with |k| < crop_px are kept (numbered
 * row-major, v outer); those with |k|^2 < k0_px^2 (float32) are bright-field.
 * Scan frequency index m (numpy fftfreq order) maps to K' = m * kpm binned
 * pixels on each axis. */
typedef struct eer4d_geom {
  uint32_t det_w, det_h;      /* raw detector pixels */
  uint32_t bin;               /* binning factor (>= 1) */
  int32_t  crop_x0, crop_y0;  /* raw pixel where binned pixel 0 starts */
  uint32_t pw, ph;            /* binned window */
  uint32_t dc_u, dc_v;        /* binned pixel of the optical axis */
  double   k0_px;             /* aperture radius alpha/dalpha (binned px) */
  double   crop_px;           /* crop radius (binned px), >= k0_px */
  uint32_t scan_ny, scan_nx;  /* scan positions (both even, 2..4096) */
  double   kpm_y, kpm_x;      /* K' per scan frequency index (binned px) */
  double   lambda_A;          /* electron wavelength (Angstrom) */
  double   dalpha_rad;        /* binned pixel angle (rad) */
  double   step_A;            /* scan step (Angstrom), for DPC frequencies */
  double   dalpha_raw_rad;    /* raw pixel angle (rad), for COM units */
} eer4d_geom;

typedef struct eer4d_info {
  int32_t P;        /* kept (cropped) pixels */
  int32_t P_pad;    /* P rounded up to a multiple of 16: pixel stride of G */
  int32_t P_bf;     /* bright-field pixels */
  int32_t n_rows;   /* detector rows holding bright-field pixels */
  int32_t nkx;      /* scan_nx/2 + 1 stored K_x columns of G */
  int32_t trotter_list_max;  /* upper bound of |K(K)| + |K(-K)| */
  int32_t p_begin, p_end;    /* kept pixels [p_begin, p_end) of the full plan's numbering
                                this plan owns (0, P for a plan of eer4d_plan_create) */
} eer4d_info;

typedef struct eer4d_plan eer4d_plan;

/* Aberrations are passed as double[5] per candidate, in this order:
 *   C1 (defocus, A), C12a, C12b (two-fold astigmatism, A), C3 (spherical, A),
 *   rot (scan rotation, rad; K' = R(rot) K'_0 counter-clockwise).
 * chi(k) = 2 pi / lambda [C1 w^2/2 + (C12a (wx^2-wy^2) + C12b 2 wx wy)/2
 *          + C3 w^4/4], w = k * dalpha_rad (Krivanek notation; the paper
 * gives no formula), and the probe is A(k) = exp(-i chi(k)) inside |k| < k0. */

/* ---- plan ---------------------------------------------------------------- */
/* Validates the geometry, builds the pixel, row and FFT tables on the current
 * device.  precision: EER4D_FP32_FFT, EER4D_SPLIT_FP16, EER4D_FP32_FFT_2PASS or
 * EER4D_FP32_STOCKHAM; norm:
 * EER4D_NORM_NONE or EER4D_NORM_AREA.  Returns EINVAL for an invalid
 * geometry (zero sizes, odd scan, crop_px < k0_px, more than 32767 kept
 * pixels, scan side > 4096), ENOMEM/ECUDA when the tables cannot be made. */
int eer4d_plan_create(const eer4d_geom* h_geom, int precision, int norm, eer4d_plan** out);
void eer4d_plan_destroy(eer4d_plan* plan);
int eer4d_plan_info(const eer4d_plan* plan, eer4d_info* h_info);

/* Bytes the caller allocates: counts (the accumulation workspace of
 * ssb_accumulate), G (the resident spectrum) and scratch (the largest need of
 * com_dpc, ssb_reconstruct with n_cand candidates, ssb_grad and
 * ssb_variance_grad). */
int eer4d_workspace_bytes(const eer4d_plan* plan, int n_cand, size_t* counts_bytes,
                          size_t* G_bytes, size_t* scratch_bytes);

int eer4d_status_code(const uint32_t* h_status4);
const char* eer4d_strerror(int code);
/* Text of the last CUDA error seen by an entry point of the calling thread. */
const char* eer4d_last_error(void);

/* ---- a1: ingest and validate (Sec. II; Table 1 "sum all frames") ---------
 * Checks the CSR (monotone offsets inside [0, n_idx], indices < W*H) and
 * accumulates (adds to what the buffers hold) the PACBED histogram
 * d_pacbed[H*W] (int64, nullable) and the integer totals d_totals[3] =
 * (sum x, sum y, count) over all valid events (int64, nullable), whose ratio
 * is the PACBED centre of mass used to centre the pattern (Sec. IV). */
int eer_load_csr(const eer4d_plan* plan, const uint32_t* d_idx, uint64_t n_idx,
                 const uint64_t* d_off, uint64_t n_frames, int64_t* d_pacbed,
                 int64_t* d_totals, uint32_t* d_status, void* stream);

/* ---- run-length-encoded EER (Sec. II, Fig. 1c; Table 1) ---------------------
 * Re-codes run-length-encoded frames to linear-index encoding in O(C).  Within
 * frame f (runs d_runs[d_off[f] .. d_off[f+1])) the hits are in ascending
 * linear index and run j is the distance from the previous hit of the frame
 * (run 0: the linear index of the first hit), so
 *   d_idx[j] = run_0 + ... + run_j   (sums restart at every frame).
 * d_idx (uint32 [n]) may be d_runs itself.  A sum above 2^32 - 1 is written as
 * 0xFFFFFFFF (dropped as out of range by the other calls) and sets
 * EER4D_ST_RANGE; offsets that decrease or pass n set EER4D_ST_OFFSETS (the
 * frame's range is clipped).  Needs no plan. */
int eer_decode_rle(const uint32_t* d_runs, uint64_t n, const uint64_t* d_off, uint64_t n_frames,
                   uint32_t* d_idx, uint32_t* d_status, void* stream);

/* ---- a2 + a3: centre of mass and DPC (Eq. 4; Sec. V) -----------------------
 * For the whole scan (n_frames = scan_ny*scan_nx): d_sums[3][F] (int64
 * Sx, Sy, N per frame, exact), d_com[2][F] (float, COM - centre in raw px; 0
 * for an empty frame) and, when d_phase is not NULL, the regularised Fourier
 * integration phi = IFFT[-i (Kx Cx^ + Ky Cy^)/(lam1 + K^2 + lam2 K^4)]
 * (DC = 0, C in 1/A = COM * dalpha_raw/lambda, K = fftfreq(N, step_A)).
 * The centre is d_totals[0..1]/d_totals[2] when d_totals is not NULL, else
 * (cx, cy).  d_scratch needs 8*F bytes when d_phase is not NULL. */
int com_dpc(const eer4d_plan* plan, const uint32_t* d_idx, uint64_t n_idx, const uint64_t* d_off,
            int64_t* d_sums, float* d_com, float* d_phase, const int64_t* d_totals, double cx,
            double cy, double lam1, double lam2, void* d_scratch, uint32_t* d_status, void* stream);

/* com_dpc from per-frame sums already formed (d_sums int64 [3][F], e.g. by
 * ssb_accumulate_com): the same centre, COM maps and DPC phase, without a
 * pass over the events.  Same outputs, scratch and errors as com_dpc. */
int com_dpc_sums(const eer4d_plan* plan, const int64_t* d_sums, float* d_com, float* d_phase,
                 const int64_t* d_totals, double cx, double cy, double lam1, double lam2,
                 void* d_scratch, uint32_t* d_status, void* stream);

/* ---- virtual detectors (Table 1: operations in O(C) on linear-index EER) ----
 * For every frame f the number of events in each of n_rings (1..EER4D_MAX_RINGS)
 * annuli about the pattern centre: ring j holds the raw pixels (x, y) with
 *   h_radii[j]^2 <= (x - cx)^2 + (y - cy)^2 < h_radii[j+1]^2
 * (h_radii: host, n_rings + 1 ascending radii in raw px; squares and sums in
 * double, round to nearest, no fused multiply-add).  One ring from 0 to the
 * bright-field radius is a bright-field detector, an annulus outside it an
 * annular dark-field one, many thin rings a radial sum.  The centre is
 * d_totals[0..1]/d_totals[2] (the PACBED centre of mass from eer_load_csr)
 * when d_totals is not NULL, else (cx, cy).  Output d_out int32
 * [n_rings][n_frames] (ring-major, each ring an image in scan order).
 * d_scratch needs det_w*det_h bytes (within eer4d_workspace_bytes' scratch).
 * Events with idx >= det_w*det_h are dropped (EER4D_ST_RANGE), bad offsets
 * set EER4D_ST_OFFSETS. */
#define EER4D_MAX_RINGS 64
int virtual_detectors(const eer4d_plan* plan, const uint32_t* d_idx, uint64_t n_idx,
                      const uint64_t* d_off, uint64_t n_frames, const double* h_radii, int n_rings,
                      const int64_t* d_totals, double cx, double cy, void* d_scratch,
                      int32_t* d_out, uint32_t* d_status, void* stream);

/* ---- iterative regularised DPC (Sec. V) --------------------------------------
 * The gradient-descent form of the DPC integration: with C = d_com (float
 * [2][F], COM - centre in raw px as com_dpc writes it) times dalpha_raw/lambda,
 *   R = M (C - grad phi^l / 2 pi),
 *   phi^{l+1} = phi^l + mu IFFT[-i (Kx R^x + Ky R^y) / (lam1 + K^2 + lam2 K^4)],
 * phi^0 = 0, n_iter steps (the update as printed has no residual; this is its
 * reading), on a periodic grid of pad x pad times the scan (pad 1 or 2; with
 * 2 the scan is the top-left quarter, M its indicator, so nothing wraps
 * around).  Derivatives are spectral (iK); DC and Nyquist bins of the update
 * are zero.  Output d_phase float [F] = phi^{n_iter} on the scan.  d_scratch
 * needs 24 * pad^2 * F bytes (scratch_bytes is checked).  With pad = 1,
 * lam1 = lam2 = 0 the result is (1 - (1 - mu)^n_iter) times com_dpc's
 * one-shot integration on bins other than Nyquist. */
int dpc_iterative(const eer4d_plan* plan, const float* d_com, double lam1, double lam2, double mu,
                  int n_iter, int pad, void* d_scratch, size_t scratch_bytes, float* d_phase,
                  void* stream);

/* ---- a4 + a5: bin/crop/densify and the G function (Table 1; Sec. IV) -------
 * Scatters frames [first_frame, first_frame + n_frames) into the counts at
 * the start of the workspace d_counts (fp16 [P_pad][scan_ny*scan_nx], exact
 * integers up to 2048; eer4d_workspace_bytes gives the workspace size).  The
 * rest of the workspace (from the next 256-byte boundary) holds the
 * intermediate of the scan DFT:
 *  - FP32_FFT plans of square scans with side 128, 256, 512 or 1024: nothing
 *    until is_last; then one persistent launch does both axes through a ring
 *    of four pixel-group slabs (the two in use kept in L2) and its task counters;
 *  - otherwise: the DFT along x of every scan row completed by this chunk,
 *    complex64 [scan_nx/2+1][scan_ny][P_pad]; with is_last the DFT along y.
 * Chunks must arrive in frame order starting at frame 0 (else EORDER).  With
 * is_last (the chunk ends at the last frame) d_G receives
 * G(k, K) = F_{R->K} counts: complex64 [scan_nx/2+1][P_pad][scan_ny]
 * (K_x >= 0 half, K_y innermost; G(k,-K) = conj G(k,K)).  The fused launch's
 * bounded waits set EER4D_ST_TIMEOUT if they give up. */
int ssb_accumulate(eer4d_plan* plan, const uint32_t* d_idx, uint64_t n_idx, const uint64_t* d_off,
                   uint64_t first_frame, uint64_t n_frames, void* d_counts, void* d_G,
                   int is_last, uint32_t* d_status, void* stream);

/* ---- a1 + a2 + a4 + a5 in one pass over the events ------------------------
 * ssb_accumulate whose scatter pass also forms, for the frames
 * [first_frame, first_frame + n_frames), the per-frame COM sums of com_dpc
 * (Eq. 4): d_sums int64 [3][F] (Sx, Sy, N of the frame's in-range events,
 * exact) and adds them to d_totals int64 [3] (the PACBED totals of
 * eer_load_csr, for the centre; zero it before the first chunk).  Offsets and
 * indices are checked as in eer_load_csr (EER4D_ST_OFFSETS, EER4D_ST_RANGE).
 * A frame with more than 65535 events sets EER4D_ST_OVERFLOW (as in
 * ssb_accumulate) and its sums then cover its first 65535 events.  Follow
 * with com_dpc_sums for the COM maps and the DPC phase.  Same arguments,
 * workspace and errors as ssb_accumulate otherwise; d_sums and d_totals must
 * not be NULL. */
int ssb_accumulate_com(eer4d_plan* plan, const uint32_t* d_idx, uint64_t n_idx,
                       const uint64_t* d_off, uint64_t first_frame, uint64_t n_frames,
                       void* d_counts, void* d_G, int is_last, int64_t* d_sums, int64_t* d_totals,
                       uint32_t* d_status, void* stream);

/* ---- a6 + a7: SSB trotter integration and phase image (Eq. 3) --------------
 * For each candidate c (d_aberr: double[n_cand][5] on the device, so a CUDA
 * graph can replay with new values): S(K) = sum_{k in K(K)} G(k,K)
 * exp(-i (chi(k) - chi(k - K'))) [/|K(K)|], and
 * phi_c = (N_R/Gbar0) Im(IFFT2(S)), Gbar0 = mean of G(k,0) over bright-field
 * pixels.  d_phase: float [n_cand][F] (nullable); d_var: double [n_cand]
 * population variance of phi_c (nullable).  All candidates must share the
 * rotation of candidate 0 (else EER4D_ST_ROTATION; the mask of candidate 0
 * is used).  1 <= n_cand <= 1024. */
int ssb_reconstruct(const eer4d_plan* plan, const void* d_G, const double* d_aberr, int n_cand,
                    void* d_scratch, float* d_phase, double* d_var, uint32_t* d_status, void* stream);

/* ---- a8: adjoint with respect to the aberrations ----------------------------
 * d_grad[5] (double) = sum_R g(R) d phi(R)/d theta for theta = (C1, C12a,
 * C12b, C3, rot) and the upstream gradient g = d_grad_phase (float [F]); the
 * trotter mask is held fixed (it is piecewise constant in rot). */
int ssb_grad(const eer4d_plan* plan, const void* d_G, const double* d_aberr,
             const float* d_grad_phase, double* d_grad, void* d_scratch, uint32_t* d_status,
             void* stream);

/* Fused refocus objective: V = variance of phi and dV/dtheta (double[5]) in
 * one pass over G (Parseval: V = sum_K |Phi^(K)|^2 / N_R^2), plus phi
 * (float [F], nullable). */
int ssb_variance_grad(const eer4d_plan* plan, const void* d_G, const double* d_aberr,
                      void* d_scratch, float* d_phase, double* d_var, double* d_grad,
                      uint32_t* d_status, void* stream);

/* Diagnostic: d_count[F] (int32, [scan_ny][scan_nx] bins) = |K(K)| for the
 * rotation d_aberr[4], from the same mask code the trotter kernel runs
 * (set K of Sec. IV).  d_scratch as for ssb_reconstruct with one candidate. */
int ssb_trotter_counts(const eer4d_plan* plan, const double* d_aberr, int32_t* d_count,
                       void* d_scratch, void* stream);

/* Refocus step (gradient ascent on the image variance, the interactive
 * virtual-focus loop of Sec. IV / Fig. 2 driven by the adjoint): computes V,
 * dV/dtheta and phi at d_aberr (as ssb_variance_grad), then updates in place
 * d_aberr[j] += d_step[j] * dV/dtheta_j on the device.  Every operand lives
 * on the device, so a CUDA graph of this call replays with the updated
 * aberrations. */
int ssb_refocus_step(const eer4d_plan* plan, const void* d_G, double* d_aberr, const double* d_step,
                     void* d_scratch, float* d_phase, double* d_var, double* d_grad,
                     uint32_t* d_status, void* stream);

/* The same refocus step with an Adam update instead of a fixed step, so a
 * captured graph of it converges from any start (for example all
 * aberrations 0) without tuning a step per parameter.  In scaled parameters
 * x_j = theta_j / scale_j: m1 = 0.9 m1 + 0.1 g, m2 = 0.999 m2 + 0.001 g^2
 * (g = dV/dtheta_j scale_j), theta_j += scale_j lr_j m1^ / (sqrt(m2^) + 1e-12)
 * with the bias-corrected moments m^ of step t.  d_rate double[10] = lr[5]
 * (lr_j = 0 holds theta_j), scale[5]; d_state double[11] = m1[5], m2[5], t,
 * zeroed by the caller before the first step and carried from step to
 * step. */
int ssb_refocus_step_adam(const eer4d_plan* plan, const void* d_G, double* d_aberr,
                          const double* d_rate, double* d_state, void* d_scratch, float* d_phase,
                          double* d_var, double* d_grad, uint32_t* d_status, void* stream);

/* ---- G-function viewer (Fig. 2, middle panel) -------------------------------
 * G(k, K) at n (1..EER4D_MAX_SLICES) scan frequencies, for judging residual
 * aberrations: h_bins (host) holds n pairs (m_y, m_x) of DFT bin indices
 * (0 <= m_y < scan_ny, 0 <= m_x < scan_nx; bins with m_x > scan_nx/2 are read
 * as conj G(k, -K)).  d_out complex64 [n][ph][pw] on the binned detector
 * window: kept pixel k at (v, u) = (k_y + dc_v, k_x + dc_u), zero elsewhere.
 * EINVAL for a bin out of range. */
#define EER4D_MAX_SLICES 64
int ssb_g_slices(const eer4d_plan* plan, const void* d_G, const int32_t* h_bins, int n,
                 void* d_out, void* stream);

/* ---- several datasets in one launch (Sec. IV, S(K) of Eq. 3 per dataset) -----
 * Uneven batches: n_sets (1..EER4D_MAX_SETS) datasets recorded with one
 * detector geometry (identical det_w, det_h, bin, crop, aperture, wavelength
 * and pixel angle; the scans and doses may differ) are reconstructed by one
 * persistent trotter launch over the bins of all of them, then one variance
 * reduction over all and each dataset's inverse transform.  h_plans[i] (host
 * array) is dataset i's plan and h_G[i] (host array of device pointers) its G
 * from ssb_accumulate; d_aberr is double [n_sets][5], row i the aberrations
 * (and scan rotation) of dataset i.  Outputs: h_phase[i] (host array of device
 * pointers, the array or any entry NULL to skip) float [scan_ny_i][scan_nx_i];
 * d_var double [n_sets] (nullable).  d_scratch needs the bytes
 * eer4d_batched_scratch_bytes returns.  EINVAL when n_sets is out of range, a
 * pointer is NULL or the detector geometries differ.  Stage events, if any,
 * are those of h_plans[0]. */
#define EER4D_MAX_SETS 32
int eer4d_batched_scratch_bytes(const eer4d_plan* const* h_plans, int n_sets, size_t* h_bytes);
int ssb_reconstruct_batched(const eer4d_plan* const* h_plans, const void* const* h_G, int n_sets,
                            const double* d_aberr, void* d_scratch, float* const* h_phase,
                            double* d_var, uint32_t* d_status, void* stream);

/* ---- pixel shards: one dataset over several GPUs (Sec. IV) --------------------
 * G(k, K) is a transform of each detector pixel's image on its own, and the
 * trotter sum of Eq. 3 is a sum over pixels k, so the pixels of one dataset
 * can be split between GPUs that then exchange only the partial spectra
 * ("no inter-device transfers" of the data itself, Sec. IV).
 *
 * eer4d_shard_range (host only, needs no GPU): shard `shard` of `n_shards`
 * (1..EER4D_MAX_SHARDS) of P kept pixels is [*h_begin, *h_end) =
 * [floor(P shard / n), floor(P (shard + 1) / n)).
 *
 * eer4d_plan_create_shard: the plan eer4d_plan_create would make, restricted
 * to that shard of its kept pixels (numbered row-major, v outer), renumbered
 * from 0.  Its ssb_accumulate reads every event and keeps only its own pixels
 * (other pixels' events are dropped like events outside the crop, with no
 * status bit); its counts, G and trotter lists cover its pixels only.
 * EINVAL when the shard holds no bright-field pixel (with the default
 * bright-field crop every kept pixel is bright-field).  COM and DPC do not
 * depend on the pixels: any plan computes them for the whole frame.
 *
 * ssb_spectrum_partial: this shard's share of the spectrum of ssb_reconstruct
 * for n_cand candidates (as there, all of one rotation): d_H complex64
 * [n_cand][scan_ny][scan_nx/2+1] = N_R (S_g(b) - conj S_g(-b)) / (2 i) for
 * the stored bins b = (m_y, m_x <= scan_nx/2), S_g the sum of Eq. 3 over this
 * plan's bright-field pixels, and d_g0 double[2] = (sum of G(k, 0) over them,
 * their number).  Shares of all shards add up (element-wise sums of d_H and
 * of d_g0, e.g. one all-reduce) to those of the whole pixel set.  Plans with
 * EER4D_NORM_AREA return EINVAL (the per-bin set sizes would need their own
 * exchange).  d_scratch as for ssb_reconstruct with n_cand candidates.
 *
 * ssb_image_from_spectrum: from summed shares (d_H, d_g0 as above, every
 * shard's added), phi_c = Im(IFFT2(S)) N_R / Gbar0 with Gbar0 = d_g0[0] /
 * d_g0[1] (phi = 0 when d_g0[0] is 0), written to d_phase float [n_cand][F]
 * (nullable), and the variance to d_var double [n_cand] (nullable); equal to
 * ssb_reconstruct on an unsharded plan up to rounding.  Any plan of the
 * dataset may be passed; d_H is read only.  d_scratch as for ssb_reconstruct
 * with n_cand candidates. */
#define EER4D_MAX_SHARDS 64
int eer4d_shard_range(int P, int shard, int n_shards, int* h_begin, int* h_end);
int eer4d_plan_create_shard(const eer4d_geom* h_geom, int precision, int norm, int shard,
                            int n_shards, eer4d_plan** out);
int ssb_spectrum_partial(const eer4d_plan* plan, const void* d_G, const double* d_aberr,
                         int n_cand, void* d_scratch, void* d_H, double* d_g0, uint32_t* d_status,
                         void* stream);
int ssb_image_from_spectrum(const eer4d_plan* plan, const void* d_H, const double* d_g0,
                            int n_cand, void* d_scratch, float* d_phase, double* d_var,
                            void* stream);

/* ---- reconstruction without scratch allocation --------------------------------
 * The paper has no counterpart to this entry point; it exists for callers that
 * cannot allocate device memory where they want an image (a host application
 * that owns every device buffer, or a real-time acquisition loop that must
 * not call cudaMalloc because it can synchronise the device).
 * ssb_reconstruct_static computes what ssb_reconstruct computes for ONE
 * candidate (d_aberr: double[5]; d_phase: float [F], nullable; d_var: double
 * [1], nullable) but takes no scratch argument and allocates nothing: its
 * working memory is a static device array of EER4D_STATIC_SCRATCH_BYTES
 * (8 MiB) inside the library, held by every GPU that loads the library until
 * the process exits.  A plan needing more (scans beyond about 1024x1024)
 * returns EER4D_ESCRATCH with nothing enqueued.  All calls on a device share
 * the array, which keeps the last call's contents (nothing in it needs to
 * start at zero); calls that overlap on the GPU race on it, so order them on
 * one stream.  The first call on each device looks up the array's device
 * address; make that first call before any stream capture.  The address is
 * kept for the life of the process, so it assumes the device is not reset
 * (cudaDeviceReset) while the library is in use. */
#define EER4D_STATIC_SCRATCH_BYTES (8u << 20)
int ssb_reconstruct_static(const eer4d_plan* plan, const void* d_G, const double* d_aberr,
                           float* d_phase, double* d_var, uint32_t* d_status, void* stream);

/* ---- split DFT factors of the tensor-core scan transform (Sec. IV) ------------
 * Host only (needs no GPU): the factors the EER4D_SPLIT_FP16 scan DFT builds
 * its tables from.  For k in [0, n_k), x in [0, n) and c in {0, 1}:
 * w = cos(2 pi e / n) (c = 0) or -sin(2 pi e / n) (c = 1) with the exact
 * integer phase index e = (k x) mod n, evaluated in double;
 * h_hi[(k n + x) 2 + c] = bits of fp16(w) and h_lo[...] = bits of
 * fp16(w - hi), so hi + lo carries about 22 significant bits of w.  h_hi and
 * h_lo (caller-owned) hold 2 n n_k uint16 each.  EINVAL for n outside
 * [1, 65536], n_k outside [1, n] or a NULL buffer. */
int eer4d_dft_split_factors(int n, int n_k, uint16_t* h_hi, uint16_t* h_lo);

/* ---- launch-shape autotuner (not part of the method) --------------------------
 * Tile and grid shapes of the three main kernels.  Zero means the built-in
 * choice.  scatter_tf: frames per scatter tile (a power of two, 4..128);
 * *_ctas_per_sm: resident CTAs per SM of the persistent grids of the scatter,
 * the fused scan DFT and the trotter kernel (capped by occupancy).  ms: the
 * times (ms) the autotuner measured for its choices (scatter, DFT, trotter). */
typedef struct eer4d_tuning {
  int32_t scatter_tf;
  int32_t scatter_ctas_per_sm;
  int32_t dft_ctas_per_sm;
  int32_t trotter_ctas_per_sm;
  float   ms[3];
} eer4d_tuning;
/* Times the candidate shapes on the caller's data and keeps the fastest in the
 * plan: scatter (16..128 frames per tile x 1..3 CTAs/SM) over
 * the whole CSR (d_idx, d_off for all scan_ny*scan_nx frames), the fused scan
 * DFT (1..4 CTAs/SM; plans without it keep 0) and the trotter kernel with the
 * aberrations d_aberr (double[5]) (1..3 CTAs/SM).  d_work, d_G and d_scratch
 * are the buffers of eer4d_workspace_bytes (n_cand >= 1); they are
 * overwritten.  Synchronises `stream` (a set-up call: not for stream
 * capture).  The choice is written to *h_out (nullable).  Results of every
 * call are unchanged by the choice except the summation order of the adjoint's
 * per-block partial sums. */
int eer4d_autotune(eer4d_plan* plan, const uint32_t* d_idx, uint64_t n_idx, const uint64_t* d_off,
                   void* d_work, void* d_G, void* d_scratch, const double* d_aberr,
                   uint32_t* d_status, void* stream, eer4d_tuning* h_out);
/* Applies a stored choice (for example from a cache of earlier eer4d_autotune
 * results) without timing; EINVAL for values out of range. */
int eer4d_set_tuning(eer4d_plan* plan, const eer4d_tuning* h_tuning);
int eer4d_get_tuning(const eer4d_plan* plan, eer4d_tuning* h_tuning);

/* ---- measurement hooks (not part of the method) ------------------------------
 * Stage ids for eer4d_set_stage_events. */
#define EER4D_STAGE_VALIDATE 0  /* eer_load_csr */
#define EER4D_STAGE_COM      1  /* per-frame COM sums (com_dpc) */
#define EER4D_STAGE_DPC      2  /* Fourier integration (com_dpc) */
#define EER4D_STAGE_SCATTER  3  /* bin/crop/densify (ssb_accumulate) */
#define EER4D_STAGE_DFT_X    4  /* scan DFT along x (ssb_accumulate) */
#define EER4D_STAGE_DFT_Y    5  /* scan DFT along y (ssb_accumulate, last chunk) */
#define EER4D_STAGE_TROTTER  6  /* trotter integration / adjoint */
#define EER4D_STAGE_IMAGE    7  /* variance and inverse transform to phi */
#define EER4D_STAGE_DFT_XY   8  /* fused scan DFT along x and y (ssb_accumulate, last chunk) */
#define EER4D_N_STAGES       9
/* When set, each stage records ev_start[s] before and ev_stop[s] after its
 * kernels on the launching stream.  The arrays hold EER4D_N_STAGES
 * cudaEvent_t owned by the caller (NULL entries are skipped); passing NULL
 * arrays clears the hook. */
int eer4d_set_stage_events(eer4d_plan* plan, void* const* ev_start, void* const* ev_stop);
/* Failure-path self test: runs the bounded device wait of the fused scan DFT
 * (the wait for a producer that has not arrived) on a counter that nothing
 * increments.  After its limit (1 s) the wait gives up, sets
 * EER4D_ST_TIMEOUT in d_status and the kernel returns; the context stays
 * usable.  d_scratch: 8 bytes of device memory.  Enqueues one small kernel. */
int eer4d_selftest_wait(void* d_scratch, uint32_t* d_status, void* stream);
/* Number of kernels the library has launched in this process. */
uint64_t eer4d_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* EER4D_H */
