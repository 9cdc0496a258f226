/*
 * lma.h -- C-ABI of the GB300 Lattice Multislice Algorithm (LMA) library.
 *
 * The library computes STEM images with the Lattice Multislice Algorithm of
 * arXiv:2310.16829 (Fig. lma_pseudocode): multislice propagation of the
 * lattice translates u_i of a localized input wave (Sec. 4.2.1, step 1),
 * synthesis of every probe's exit wave as a linear combination of the
 * propagated translates (Sec. 4.2.2, step 2), the annular detector of the 2D
 * STEM reading (Sec. 3.1) and the frozen-phonon average (Sec. 3.1, last
 * paragraph). Local recompute after a change of one atomic column follows
 * Sec. 4.2.6.
 *
 * Conventions (all functions):
 *   - Arrays are row-major [y][x]; pixel j sits at j*dx; boundaries are
 *     periodic. Complex values are interleaved (re, im) float pairs.
 *   - Every function returns an lma_status; no exception crosses the ABI. On
 *     error, lma_last_error(ctx) returns a message for that context.
 *   - Input arrays are owned by the caller and are copied during the call;
 *     the caller may free them on return. Opaque handles are owned by the
 *     library until the matching lma_free_* / lma_destroy. Output buffers are
 *     allocated by the caller.
 *   - "stream" is a cudaStream_t passed as void* (NULL = default stream).
 *     Device work is queued on it; a call that writes a HOST output buffer
 *     synchronizes that stream before returning. An output pointer may be
 *     host or device memory: the library asks the CUDA runtime which.
 *   - One context per host thread. Contexts created with device = -1 are
 *     host-only: the host-side functions (geometry, coefficients) work, every
 *     device call returns LMA_ERR_UNSUPPORTED.
 *   - Sizes: the propagation window W and the detection window D are 128
 *     pixels in this version (LMA_ERR_UNSUPPORTED otherwise); the grid must be
 *     at least W pixels in each direction.
 */
#ifndef LMA_H
#define LMA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t lma_status;
#define LMA_OK 0
#define LMA_ERR_INVALID 1      /* bad argument, incompatible lattices, off-grid position */
#define LMA_ERR_OOM 2          /* device or host allocation failed */
#define LMA_ERR_CUDA 3         /* CUDA runtime error (message in lma_last_error) */
#define LMA_ERR_TIMEOUT 4      /* a bounded device wait gave up */
#define LMA_ERR_UNSUPPORTED 5  /* valid request outside what the library implements */

#define LMA_BASIS_GAUSS 0      /* u = g_sigma (Sec. 4.2.3, Gaussians) */
#define LMA_BASIS_PROBE 1      /* u = psi_0^init (Sec. 4.2.3, first paragraph) */
#define LMA_BASIS_TRIG 2       /* u = phi_n(2 pi x / l_x) phi_n(2 pi y / l_y), trigonometric polynomials (Sec. 4.2.3) */
#define LMA_BASIS_TRIG_RADIAL 3 /* u = phi_n(2 pi |v| / l_x), the circularly symmetric option (Sec. 4.2.3) */

/* Coefficients of the input waves for each probe (lma_basis_desc.coef_mode). */
#define LMA_COEF_LSQ 0          /* least squares over the L nearest input waves (eqs. lma_approximation_exit1_0 /
                                   exit2_0), for every kind of input wave */
#define LMA_COEF_TRIG_CLOSED 1  /* LMA_BASIS_TRIG only: the closed form of Sec. 2 and Sec. 4.2.3 (no least
                                   squares). The probe's DFT coefficients P(k) with |k_x|, |k_y| <= n give
                                   a(d) = sum_k P(k) / (N_x N_y w_kx w_ky m_x m_y) e^{2 pi i (k_x d_x / N_x + k_y d_y / N_y)}
                                   for the input wave at offset d from the probe, w_k = cos(k pi / (2n + 2)),
                                   m_x x m_y input waves of I_f. With m = 2n + 1 per axis this is the M^-1 of
                                   Sec. 2 (derived from its definition M = diag(w) W, W_{k,j} = e^{-2 pi i jk/(2n+1)});
                                   with m > 2n + 1 (power-of-two grids, which 2n + 1 never divides) it is the
                                   exact minimum-norm representation. The probe uses the values at its L
                                   nearest input waves; needs m_x, m_y >= 2n + 1. */

#define LMA_PREC_C64 0         /* complex64 everywhere on the device */
#define LMA_PREC_FP16_STORE 1  /* FP32 propagation; exit waves stored as FP16 pairs with a per-wave
                                  power-of-two scale: half the store; bright-field readings within
                                  1e-3, weak annular (HAADF) readings are not (FP16 rounding noise) */
#define LMA_PREC_MIXED 2       /* the 32-point DFT stages of the slice step (Sec. 3.2 multislice step)
                                  as split-FP16 (hi + lo) tensor-core products accumulated in FP32;
                                  the other stages in FP32, exit waves stored in complex64 */

#define LMA_EDIT_REMOVE 0      /* remove the atoms of a column */
#define LMA_EDIT_SET_SPECIES 1 /* give the atoms of a column another species */

#define LMA_IMAGE_RECOMPUTE 1u /* treat every stored exit wave as stale (full path) */
#define LMA_MAX_RINGS 256      /* rings of one 3D STEM image */
#define LMA_IMAGE_GRAPH 2u     /* lma_image_many: replay the device work as one CUDA graph */
#define LMA_IMAGE_AUTOTUNE 4u  /* time every slice launch mode, and every synthesis form (gather
                                  strip width and grid, grouped shapes), on this call's first
                                  launch of each shape and keep the fastest for that shape
                                  (lma_tuning_read, lma_synth_tuning_read) */

/* Partition strategies of a probe region (Sec. 4.2.4). */
#define LMA_PART_ROWS 0                    /* row by row */
#define LMA_PART_RECTANGLES 1              /* equal rectangles, row-major order */
#define LMA_PART_RECTANGLES_COLUMN_MAJOR 2 /* equal rectangles, column-major order */
#define LMA_PART_GREEDY 3                  /* greedy growth from a start probe */

/* How the CTAs of a slice launch (step a3) take their translates. */
#define LMA_SLICE_AUTO -1          /* the tuned mode of the launch shape, else the default */
#define LMA_SLICE_ONE_PER_ITEM 0   /* one CTA per translate, scheduled by the hardware */
#define LMA_SLICE_PERSISTENT 1     /* one CTA per SM, translates taken with a fixed stride */
#define LMA_SLICE_DYNAMIC 2        /* one CTA per SM, translates taken from an atomic counter */

typedef struct lma_ctx lma_ctx;
typedef struct lma_specimen lma_specimen;
typedef struct lma_basis lma_basis;

/* Simulation grid (Sec. 3.2, complexity paragraph: X x Y pixels over l_x x l_y). */
typedef struct {
  int32_t nx, ny;          /* pixels */
  double lx, ly;           /* Angstrom */
  double slice_dz;         /* slice thickness epsilon, Angstrom */
  int32_t n_slices;        /* N */
  double lambda;           /* electron wavelength, Angstrom */
  double sigma;            /* interaction constant, rad/(V*Angstrom) (eq. schroedinger_equation) */
  double bandlimit_frac;   /* propagator mask radius as a fraction of Nyquist (2/3 typical) */
} lma_grid;

/* Projected potential per atom and slice: peak[species] * sum_t frac_t exp(-r^2 / 2 w_t^2)
 * for r < r_cut, in V*Angstrom; the slice integral v_eps of Sec. 3.2. */
typedef struct {
  int32_t n_species;
  const double* peak;        /* [n_species] */
  int32_t n_terms;           /* 1..4 */
  const double* term_frac;   /* [n_terms] */
  const double* term_width;  /* [n_terms], Angstrom */
  double r_cut;              /* Angstrom, hard cutoff, < min(lx, ly) / 2 */
} lma_potential;

/* One frozen-phonon configuration (structure of arrays). */
typedef struct {
  int64_t n_atoms;
  const double* x;           /* [n_atoms] Angstrom */
  const double* y;           /* [n_atoms] Angstrom */
  const int32_t* slice;      /* [n_atoms] 0..n_slices-1 */
  const int16_t* species;    /* [n_atoms] 0..n_species-1 */
} lma_atoms;

/* Probe (eqs. probe_wave_function, aberration_function, aperture_function). */
typedef struct {
  double alpha_max;          /* rad */
  double cs;                 /* third-order spherical aberration C_s, Angstrom */
  double defocus;            /* focus Z, Angstrom */
} lma_probe;

/* Input-wave lattice and approximation parameters (Sec. 4.2.1 options (i)-(iii)). */
typedef struct {
  int32_t kind;              /* LMA_BASIS_* */
  double gauss_sigma;        /* Angstrom; 0 selects lambda / (2 alpha_max) */
  int32_t in_spacing_px[2];  /* input lattice spacing r_x, r_y in pixels; must divide nx, ny */
  int32_t in_offset_px[2];   /* I_offset in pixels, 0 <= offset < spacing */
  int32_t f;                 /* keep every f-th input wave (I_f) */
  int32_t L;                 /* input waves per probe (I_{f,p,L}) */
  int32_t window;            /* W: propagation window X' = Y' (128) */
  int32_t det_window;        /* D: synthesis / detection window (128) */
  int32_t precision;         /* LMA_PREC_C64, LMA_PREC_FP16_STORE or LMA_PREC_MIXED */
  int32_t phonon_batch;      /* configurations propagated per launch and held at once;
                                0 = as many as fit in 40 % of the free device memory */
  int32_t trig_degree;       /* LMA_BASIS_TRIG*: degree n of phi_n(t) = sum_{|k|<=n} e^{ikt} cos(k pi/(2n+2));
                                0 = round(alpha_max l_x / lambda) (maximum probe frequency / Fourier pixel) */
  int32_t coef_mode;         /* LMA_COEF_LSQ or LMA_COEF_TRIG_CLOSED */
} lma_basis_desc;

/* Annular detector r1 <= lambda |k| < r2 (rad), intersected with the bandlimit (Sec. 3.1, 2D STEM). */
typedef struct { double r1, r2; } lma_detector;

/* A rectangle of the probe lattice: p(a, b) = (px0 + a*sx, py0 + b*sy) mod grid, pixels. */
typedef struct {
  int32_t px0, py0;
  int32_t npx, npy;
  int32_t spacing_px[2];
} lma_region;

/* A memory bound for the exit-wave store (Sec. 4.2.4): the probe region is split into
 * parts P_1..P_l whose translates I_{f,P_j,L} number at most max_resident each; parts are
 * computed in order and the exit waves shared by consecutive parts are kept. */
typedef struct {
  int32_t strategy;          /* LMA_PART_* */
  int32_t start;             /* LMA_PART_GREEDY: first probe, region index b * npx + a */
  int64_t max_resident;      /* M: exit waves of one configuration held at once, >= L */
} lma_partition_desc;

/* Summary of a basis (host-side numbers). */
typedef struct {
  int64_t n_translates;      /* |I_f| */
  int32_t nax, nay;          /* I_f lattice points along x, y */
  int32_t n_sets;            /* coefficient sets computed so far (Case 1: 1, Case 2: c*d) */
  int32_t L, window, det_window;
  double gauss_sigma;        /* Angstrom, resolved */
  int64_t exit_wave_bytes;   /* device bytes of one configuration's exit-wave store */
  int32_t phonon_batch;      /* resolved phonon batch (0 before the first device use) */
} lma_basis_info;

/* ---- context ------------------------------------------------------------------------- */

/* Create a context on CUDA device `device` (or a host-only context with device = -1).
 * A context and the specimens and bases made in it serve one host thread: its calls
 * must not overlap in time, also not on different streams (the slice work counter, the
 * item-list cache, the pinned staging buffer of host copies and the grouped synthesis's
 * probe-wave buffer belong to the context).
 * Use one context per thread for concurrent work.
 * Errors: LMA_ERR_CUDA if the device cannot be selected, LMA_ERR_OOM. */
lma_status lma_create(int32_t device, lma_ctx** out);
/* Release the context with its graphs, caches and staging buffers; free its specimens and
 * bases first. NULL is ignored. */
void lma_destroy(lma_ctx* ctx);
/* Last error message of the context ("" if none). The pointer stays valid until the next call. */
const char* lma_last_error(const lma_ctx* ctx);

/* ---- specimen (step a1: projected potential and transmission, Sec. 3.2) -------------- */

/* Copy grid, potential model and n_phonons atom lists into a new specimen.
 * Atoms are ordered by slice with a stable sort; that order fixes the
 * summation order of the potential. No device work happens here.
 * Errors: LMA_ERR_INVALID (non-positive sizes, slice or species out of range,
 * r_cut >= half the cell, n_terms outside 1..4). */
lma_status lma_create_specimen(lma_ctx* ctx, const lma_grid* grid, const lma_potential* pot,
                               const lma_atoms* phonons, int32_t n_phonons, lma_specimen** out);
/* Release the specimen and its device memory (atoms, transmissions); free its bases first.
 * Errors: LMA_ERR_INVALID for NULL. */
lma_status lma_free_specimen(lma_specimen* spec);

/* Build t_s = exp(i sigma v_s) for all slices of configuration `phonon` on the
 * device (Sec. 3.2, transmission function) and copy it to `out`
 * ([n_slices][ny][nx] complex64, host or device). For parity tests. */
lma_status lma_transmission(lma_ctx* ctx, lma_specimen* spec, int32_t phonon, float* out,
                            void* stream);

/* Replace the atoms of all configurations (same count as at creation; same
 * validation as lma_create_specimen). Every transmission and exit wave built
 * from the old atoms becomes stale. Host-side copy; the device upload happens
 * at the next device call that needs the atoms. */
lma_status lma_specimen_set_atoms(lma_ctx* ctx, lma_specimen* spec, const lma_atoms* phonons,
                                  int32_t n_phonons);

/* ---- basis (steps a2 and a3) ----------------------------------------------------------- */

/* Create the input-wave basis: the lattice I_f (Sec. 4.2.1), the input wave u
 * on its W x W window (Sec. 4.2.3), and the per-slice propagator
 * exp(-i pi lambda eps |k|^2) with the bandlimit mask (Sec. 3.2). Least-squares
 * coefficients (Sec. 4.2.2) are computed on the host in FP64 when a probe
 * class is first needed. Device memory is allocated on first device use.
 * Errors: LMA_ERR_INVALID when the lattice does not cover the grid, f does not
 * divide R, offset >= spacing, L > |I_f| or L > 64; LMA_ERR_UNSUPPORTED for
 * W or D != 128 or a grid smaller than W. */
lma_status lma_create_basis(lma_ctx* ctx, const lma_specimen* spec, const lma_probe* probe,
                            const lma_basis_desc* desc, lma_basis** out);
/* Release the basis and its device memory (exit-wave store, tables). The handle is
 * invalid afterwards. Errors: LMA_ERR_INVALID for NULL. */
lma_status lma_free_basis(lma_basis* basis);
/* Fill *out with the basis summary (lma_basis_info). Host-only; no device work.
 * Errors: LMA_ERR_INVALID for a NULL argument. */
lma_status lma_basis_get_info(const lma_basis* basis, lma_basis_info* out);

/* Coefficients of the probe at pixel (px, py) (eqs. lma_approximation_exit1_0 /
 * exit2_0): alpha[2L] (re, im) FP64, offsets[2L] (dx, dy) of the L nearest
 * translates relative to the probe (pixels, minimum image), translates[L] their
 * indices in I_f (raster order, x fastest), err[2] = relative L2 and sup error
 * of the probe approximation. Host-only; works on host-only contexts. Any of
 * the output pointers may be NULL. */
lma_status lma_basis_coefficients(lma_ctx* ctx, lma_basis* basis, int32_t px, int32_t py,
                                  double* alpha, int32_t* offsets, int64_t* translates,
                                  double* err);

/* Step 1 of Fig. lma_pseudocode for configuration `phonon`: build t (step a1)
 * and propagate every translate of I_f through all slices on its W x W window
 * (step a3), keeping the exit waves U_i resident in HBM.
 * Errors: LMA_ERR_INVALID (phonon out of range), LMA_ERR_OOM, LMA_ERR_CUDA. */
lma_status lma_propagate_basis(lma_ctx* ctx, lma_specimen* spec, lma_basis* basis,
                               int32_t phonon, void* stream);

/* Copy the stored exit wave U_i of translate `translate` ([W][W] complex64, window
 * origin at its position - W/2) to `out` (host or device). Fails with
 * LMA_ERR_INVALID if that exit wave is not current. */
lma_status lma_exit_wave(lma_ctx* ctx, lma_basis* basis, int64_t translate, float* out,
                         void* stream);

/* ---- image (steps a4-a6) ---------------------------------------------------------------- */

/* STEM image of a probe-lattice region: for every phonon configuration, the
 * exit waves the region needs are made current (steps a1, a3; only stale ones
 * unless LMA_IMAGE_RECOMPUTE), each probe's exit wave is synthesized on its
 * D x D window (step a4, Sec. 4.2.2), the detectors are read from its DFT
 * (step a5, Sec. 3.1) and the readings are averaged over configurations in
 * FP64 (step a6). out[n_det][npy][npx] (double, host or device).
 * Errors: LMA_ERR_INVALID (empty detectors, probe off the grid, n_det > 4). */
lma_status lma_image(lma_ctx* ctx, lma_specimen* spec, lma_basis* basis,
                     const lma_detector* det, int32_t n_det, const lma_region* region,
                     uint32_t flags, double* out, void* stream);

/* 3D STEM image (Sec. 3.1, eq. for 3D STEM): ring a = 0..n_rings-1 collects the
 * synthesized exit wave's (1/D^2) |DFT|^2 over a*ring_width <= lambda |k| < (a+1)*ring_width
 * (rad), intersected with the bandlimit, on the D x D window; averaged over the
 * configurations in FP64. Ring sums run in a fixed order (bitwise reproducible).
 * out[n_rings][npy][npx] (double, host or device). Exit waves are made current as for
 * lma_image (flags: LMA_IMAGE_RECOMPUTE, LMA_IMAGE_AUTOTUNE).
 * Errors: LMA_ERR_INVALID (ring_width <= 0, n_rings outside 1..LMA_MAX_RINGS, bad region). */
lma_status lma_image_rings(lma_ctx* ctx, lma_specimen* spec, lma_basis* basis, double ring_width,
                           int32_t n_rings, const lma_region* region, uint32_t flags, double* out,
                           void* stream);

/* 4D STEM image (Sec. 3.1, eq. for 4D STEM): for every probe the diffraction pattern
 * (1/D^2) |DFT(Psi_p)|^2 of its synthesized exit wave on the D x D window, sampled at the
 * frequencies (a, b) * (1/(D dx), 1/(D dy)) for |a| <= half_x, |b| <= half_y, zero outside
 * the bandlimit, averaged over configurations (FP64 sum, stored as float).
 * out[npy][npx][2 half_y + 1][2 half_x + 1] (float, host or device), entry [b + half_y]
 * [a + half_x]. Errors: LMA_ERR_INVALID (half widths outside 0..D/2-1, bad region). */
lma_status lma_image_4d(lma_ctx* ctx, lma_specimen* spec, lma_basis* basis, int32_t half_x,
                        int32_t half_y, const lma_region* region, uint32_t flags, float* out,
                        void* stream);

/* ---- real-space propagation (Sec. 3.2) --------------------------------------------------- */

/* 2D STEM image with the propagation step of every slice computed as a periodic convolution
 * on the W x W window with q discretized to K1 x K2 pixels (Sec. 3.2 costs it as N(XY +
 * XY K1 K2) against N(2XY + 2XY log XY) for the Fourier step). q is the inverse DFT of the
 * window propagator exp(-i pi lambda eps |k|^2) times the bandlimit (FP64, rounded once to
 * complex64) at offsets -(K/2) .. K/2; with K1 = K2 = W it would reproduce the Fourier step.
 * Always recomputes; afterwards the basis's stored exit waves are marked stale for
 * lma_image. out as for lma_image. Errors: LMA_ERR_INVALID (K1 not odd in 3..25, K2 not odd
 * in 1..25, bad detectors or region), LMA_ERR_UNSUPPORTED (mixed store). */
lma_status lma_image_realspace(lma_ctx* ctx, lma_specimen* spec, lma_basis* basis, int32_t K1, int32_t K2,
                               const lma_detector* det, int32_t n_det, const lma_region* region,
                               uint32_t flags, double* out, void* stream);

/* Self-test of the bounded device waits. The tensor-core slice kernel (LMA_PREC_MIXED) and
 * the W = 256 slice kernel wait on shared-memory mbarriers for the MMAs and bulk copies they
 * issue, each wait one polling lane per warp with at most 2000 suspended tries of up to 1 ms;
 * a wait that gives up sets the launch's status word, the kernel returns, and the next call
 * that reads results returns LMA_ERR_TIMEOUT. This call runs that wait on an mbarrier phase
 * that nothing completes, in one warp (which = 0, as in the tensor-core kernel's per-tile
 * waits) or in the 16 warps of a CTA (which = 1, as in the W = 256 kernel's panel waits), on
 * `stream`, synchronizes it and returns what a real give-up returns: LMA_ERR_TIMEOUT with its
 * message; the status word is cleared and the context stays usable. LMA_ERR_INVALID for
 * another `which`, LMA_ERR_UNSUPPORTED without a device. Takes a few seconds. */
lma_status lma_selftest_wait(lma_ctx* ctx, int32_t which, void* stream);

/* Per-slice amplification of the real-space propagation step (Sec. 3.2, complexity
 * paragraph): with q the K1 x K2 kernel that lma_image_realspace uses (the inverse DFT of
 * the window's propagator and bandlimit, truncated to odd K1, K2 <= W pixels), the
 * convolution multiplies spectral component k of the W x W window by Q(k) = sum over the
 * kernel offsets d of q(d) exp(-2 pi i k.d / W). *gain_all receives max_k |Q(k)| over the
 * window and *gain_band the maximum over the bandlimit's disc. The Fourier step has
 * |P(k)| <= 1; a gain above 1 grows those components slice by slice. Host-only (FP64),
 * any context. LMA_ERR_INVALID for even or out-of-range K. */
lma_status lma_realspace_gain(lma_ctx* ctx, const lma_basis* basis, int32_t K1, int32_t K2, double* gain_all,
                              double* gain_band);

/* ---- partial coherence and the choice of L ---------------------------------------------- */

#define LMA_MAX_VARIANTS 32

/* Partially coherent 2D STEM image: the simulation repeated over probe variants and
 * averaged (Sec. 1), computed from one set of exit waves. The input waves, and so the
 * exit waves, do not depend on the probe: each variant's coefficients are fitted to its
 * own probe (least squares on the basis's input waves, as in Sec. 4.2.2, or the closed
 * form of LMA_COEF_TRIG_CLOSED when the basis uses it), its image is
 * synthesized and read out from the shared exit waves, and the images are averaged with
 * weights w_v / sum w. Variants may differ in defocus and C_s; alpha_max must equal the
 * basis probe's. out[n_det][npy][npx] (double, host or device); flags as for lma_image.
 * Errors: LMA_ERR_INVALID (n_variants outside 1..LMA_MAX_VARIANTS, negative or all-zero
 * weights, another aperture), and as for lma_image. */
lma_status lma_image_coherent(lma_ctx* ctx, lma_specimen* spec, lma_basis* basis, const lma_probe* variants,
                              const double* weights, int32_t n_variants, const lma_detector* det,
                              int32_t n_det, const lma_region* region, uint32_t flags, double* out,
                              void* stream);

/* The smallest L in 1..L_max whose probe approximation error in the supremum norm,
 * relative to the probe's maximum, is at most eps_sup for every coefficient class of the
 * region (Sec. 4.2.6 fixes L by such a target). desc gives the input waves, the lattice
 * and the coefficient mode (its L is ignored). *L_out = 0 when no L reaches the target; *err_out = the error at
 * the returned L (or at L_max). Host-only work. Errors: LMA_ERR_INVALID (L_max outside
 * 1..64 or above |I_f|, eps_sup <= 0, bad region or basis description). */
lma_status lma_select_L(lma_ctx* ctx, const lma_specimen* spec, const lma_probe* probe,
                        const lma_basis_desc* desc, const lma_region* region, int32_t L_max,
                        double eps_sup, int32_t* L_out, double* err_out);

/* ---- memory-bounded partition (Sec. 4.2.4) ------------------------------------------------ */

/* Partition of a probe region under a memory bound. Strategies:
 *  - rows: probes in raster order join the current part while its translates stay within M;
 *  - rectangles: one tile shape w x h from probe (0, 0), clipped at the edges, of largest
 *    area such that a tile anchored at every phase of the probe/lattice period needs at
 *    most M translates (for each width the height grows while that holds; ties: squarer,
 *    then wider);
 *  - greedy: from `start`, add the unassigned 8-neighbour of the last added probe that
 *    adds the fewest translates (ties by (b, a)); a part closes when that neighbour would
 *    exceed M and the next part starts with it; with no unassigned neighbour, continue at
 *    the first unassigned probe in raster order.
 * Outputs (each may be NULL): part[npy * npx] = part index of each probe (parts in
 * processing order), n_parts = l, runs = T_{P_1..P_l} (Multislice runs per configuration:
 * sum of |I(P_j)| minus the translates shared by consecutive parts), peak = max |I(P_j)|.
 * Host-only work (valid in a host-only context). Errors: LMA_ERR_INVALID (bad region,
 * strategy, start, or max_resident < L). */
lma_status lma_partition(lma_ctx* ctx, lma_basis* basis, const lma_region* region,
                         const lma_partition_desc* desc, int32_t* part, int32_t* n_parts,
                         int64_t* runs, int64_t* peak);

/* 2D STEM image (as lma_image, always recomputing) with an exit-wave store of
 * max_resident waves per configuration instead of |I_f|: for each configuration the parts
 * are propagated and read out in order, keeping the waves shared by consecutive parts.
 * Every exit wave and reading is computed as in lma_image, so the image is bitwise equal
 * to lma_image's. The device store is max_resident * W^2 * 8 bytes (complex64) or half
 * that (LMA_PREC_FP16_STORE); the plan's tables are kept in the basis for the next call.
 * Errors as for lma_image and lma_partition. */
lma_status lma_image_partitioned(lma_ctx* ctx, lma_specimen* spec, lma_basis* basis,
                                 const lma_detector* det, int32_t n_det, const lma_region* region,
                                 const lma_partition_desc* desc, uint32_t flags, double* out,
                                 void* stream);

/* Images of several specimens (of any sizes) in one call on one stream (the
 * batching form of steps a1-a6): for each specimen its configurations go through
 * the slice and synthesis kernels in phonon batches (see lma_basis_desc). With
 * LMA_IMAGE_GRAPH (which requires LMA_IMAGE_RECOMPUTE, device outputs and a
 * non-default stream) the whole sequence of launches of all specimens is
 * captured once into a CUDA graph and replayed by later calls with the same
 * arguments; the host only uploads changed atoms before the replay. A call whose
 * buffers moved (new region, new sizes) captures a new graph.
 * outs[k] is device memory, [n_det][npy_k][npx_k] doubles.
 * Errors as for lma_image; LMA_ERR_INVALID for a host output or the default
 * stream with LMA_IMAGE_GRAPH. */
lma_status lma_image_many(lma_ctx* ctx, int32_t n, lma_specimen* const* specs,
                          lma_basis* const* bases, const lma_detector* det, int32_t n_det,
                          const lma_region* regions, uint32_t flags, double* const* outs,
                          void* stream);

/* ---- local recompute (step a7, Sec. 4.2.6) --------------------------------------------- */

/* Edit one atomic column in every configuration: atoms whose lateral
 * minimum-image distance to (cx, cy) is below r_site are removed
 * (LMA_EDIT_REMOVE) or set to new_species (LMA_EDIT_SET_SPECIES). Marks stale
 * the transmission pixels within r_cut of the touched atoms and the exit waves
 * whose W x W window meets those pixels; the next lma_image rebuilds and
 * re-propagates only those. Outputs (may be NULL): number of atoms changed,
 * number of exit waves marked stale. Host-only bookkeeping; no device work. */
lma_status lma_edit_column(lma_ctx* ctx, lma_specimen* spec, lma_basis* basis, double cx,
                           double cy, double r_site, int32_t op, int16_t new_species,
                           int64_t* n_atoms_changed, int64_t* n_stale);

/* For each probe of `region`, 1 if any of its L translates is stale, else 0
 * (out_mask[npy][npx], host). Returns the count in *n_affected. Host-only. */
lma_status lma_affected_probes(lma_ctx* ctx, lma_basis* basis, const lma_region* region,
                               uint8_t* out_mask, int64_t* n_affected);

/* ---- readout without device allocation -------------------------------------------------- */

/* The readout of steps a4-a5 for callers that cannot allocate device memory:
 * an application whose device memory is already taken by its own allocator or
 * by a framework's caching allocator, or a process that must not grow its
 * device footprint while it runs. The paper has no counterpart; this is a
 * service of the library.
 *
 * The caller passes the exit waves ([n_translates][W][W] complex64, device
 * memory, e.g. filled with lma_exit_wave) and the output
 * (out[n_det][npy][npx] double, device memory); the readings are those of one
 * configuration, as lma_image gives for a specimen with one configuration. The
 * per-call tables and the FP64 accumulator live in one file-scope device array
 * of 8 MiB that every device loading this library holds until the process
 * exits; no cudaMalloc, cudaFree or other allocating call is made. A region
 * whose tables do not fit (about 6000 probes at L = 64, 12000 at L = 32) is
 * rejected with LMA_ERR_INVALID and a message giving the limit.
 *
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture
 * begins. (That rule is about this set-up step alone; it says nothing either
 * way about capturing the readout itself.) With CUDA's default lazy module
 * loading, the array -- 8 MiB plus the library's kernels -- comes into being
 * on the device at the library's first kernel launch or first no-allocation
 * call there: a caller whose footprint must not grow later makes one call
 * (or sets CUDA_MODULE_LOADING=EAGER) before that phase starts.
 * Every call shares the array and the accumulator is cleared at the start of
 * each call, so calls that overlap on the GPU (several streams or host
 * threads) race: serialize them. The small host tables are copied from
 * pageable memory, on purpose: a pinned staging buffer would be an
 * allocation. Pageable copies pass through the driver's staging buffer, which
 * the whole process shares, so they can hold up other threads' pageable
 * copies (for instance the uploads of other contexts) for their duration. The
 * call synchronizes `stream` before it returns. Errors as for lma_image;
 * LMA_ERR_INVALID also when exit_waves or out is not device memory. */
lma_status lma_readout_noalloc(lma_ctx* ctx, lma_basis* basis, const float* exit_waves,
                               const lma_detector* det, int32_t n_det, const lma_region* region,
                               double* out, void* stream);

/* ---- measurement ------------------------------------------------------------------------ */

/* Launch counters and CUDA-event durations per kernel. `units` counts the work
 * each launch did: pixel-slices (potential), translate-slices (slice),
 * probes (synthesis), outputs (finalize). */
typedef struct {
  int64_t launches;
  double total_ms;           /* sum of event-timed durations; 0 unless timing is on */
  int64_t units;
} lma_kernel_stat;

typedef struct {
  lma_kernel_stat potential;   /* step a1 */
  lma_kernel_stat slice;       /* step a3 */
  lma_kernel_stat synth;       /* steps a4-a5 (and the FP64 accumulation of a6) */
  lma_kernel_stat finalize;    /* step a6 */
  int64_t allocations;         /* device and pinned host allocations the library made since the
                                  last lma_profile_enable (in any context of the process) */
} lma_profile;

/* One autotuned slice launch shape: the jobs (specimens) of the launch, its
 * translates, store precision and window-origin parity, the chosen
 * LMA_SLICE_* mode and the measured duration of each mode (ms; CUDA events on
 * the caller's stream, one launch each, the launch's own results kept). */
typedef struct {
  int32_t n_jobs;
  int32_t half;              /* 1: FP16 exit-wave store */
  int32_t even;              /* 1: even window origins (16-byte staging) */
  int64_t n_items;           /* translates in the launch */
  int64_t translate_slices;  /* sum over translates of the slice count */
  int32_t mode;              /* LMA_SLICE_* chosen */
  double ms[3];              /* duration per mode, indexed by LMA_SLICE_* */
} lma_tuning;

/* Reset the counters; with on != 0 also record a CUDA event pair around every
 * kernel launch, on the stream the kernel is launched on. */
lma_status lma_profile_enable(lma_ctx* ctx, int32_t on);
/* Wait for the recorded events and return the totals since the last reset. */
lma_status lma_profile_read(lma_ctx* ctx, lma_profile* out);

/* ---- launch modes and autotuning (batching) -------------------------------------------- */

/* Force the slice launch mode of this context (LMA_SLICE_*); LMA_SLICE_AUTO
 * restores the tuned mode of each launch shape, else the default (one CTA per
 * translate for one specimen, dynamic for several). Every mode computes
 * bitwise the same exit waves. LMA_ERR_INVALID for an unknown mode. */
lma_status lma_set_slice_mode(lma_ctx* ctx, int32_t mode);
/* Copy up to cap tuned launch shapes (LMA_IMAGE_AUTOTUNE) to out, oldest
 * first (out may be NULL when cap is 0); *n receives how many the context holds. */
lma_status lma_tuning_read(lma_ctx* ctx, lma_tuning* out, int32_t cap, int32_t* n);

/* One autotuned synthesis launch shape (steps a4-a6 under LMA_IMAGE_AUTOTUNE): the readout,
 * store precision, probe region or list, configurations, L and window W of the launch; the
 * form chosen, and the duration of each variant (ms; CUDA events on the caller's stream, one
 * launch each, or for the grouped form the group and detection launches of every
 * configuration). Variants 0..5 are the per-probe gather, v = 2 s + g: strip width 16, 32, 64
 * for s = 0, 1, 2 (probes are walked in vertical strips of that many columns, which sets how
 * many exit waves the CTAs in flight share in L2) and grid g = 0 one CTA per probe, g = 1
 * persistent (one CTA per SM walking the probes in order). Variants 6 and 7 are the grouped
 * form (LMA_SYNTH_GROUPED) with the group shapes group_shape[0] and group_shape[1] (ms 0 where
 * the launch does not admit it). Every variant gives the same readings bit for bit, so the
 * timed launches' results are kept. Launches over a probe list (edits, partitions) walk the
 * list in order and time the grids of the gather only (ms of the other variants: 0). */
typedef struct {
  int32_t readout;           /* 0: annular detectors, 1: labelled rings (3D), 2: patterns (4D) */
  int32_t half;              /* 1: FP16 exit-wave store */
  int64_t n_items;           /* probes x configurations of the launch */
  int32_t L;                 /* input waves per probe */
  int32_t window;            /* exit-wave window W */
  int32_t strip;             /* chosen strip width (gather) */
  int32_t persistent;        /* chosen grid (gather): 1 persistent, 0 one CTA per probe */
  int32_t grouped;           /* 1: the grouped form was chosen, with group_x x group_y probes */
  int32_t group_x, group_y;
  int32_t group_shape[2][2]; /* the two timed group shapes (x, y) of variants 6 and 7 */
  double ms[8];              /* duration per variant */
} lma_synth_tuning;

/* How the synthesis (step a4) forms each probe's wave Psi_p = sum_j alpha_j U_{i_j}.
 * Both forms sum each probe's terms in ascending translate index and give the same readings
 * bit for bit. */
#define LMA_SYNTH_AUTO -1     /* the tuned form of the launch shape, else the gather */
#define LMA_SYNTH_GATHER 0    /* one CTA per probe gathers its L windows and detects */
#define LMA_SYNTH_GROUPED 1   /* one CTA per group of up to 4 neighbouring probes loads each
                                 exit-wave element once for all of them and writes their waves
                                 to a device buffer (probes x 128 KiB, allocated by the
                                 context); a second pass detects; falls back to the gather
                                 where the launch does not admit it */

/* Force the synthesis form of this context (LMA_SYNTH_*). LMA_ERR_INVALID for an unknown form. */
lma_status lma_set_synth_mode(lma_ctx* ctx, int32_t mode);
/* Largest probe-wave buffer of the grouped synthesis (bytes; 0: the default, 2 GiB). A region
 * whose waves (probes x 128 KiB) exceed it is synthesized in chunks of whole group rows; a
 * limit below one group row's waves leaves the gather. The buffer is allocated on first use
 * (when it has to grow, only if it is at most half the free device memory) and kept by the
 * context; under graph capture a missing or short buffer leaves the gather.
 * LMA_ERR_INVALID for a negative limit. */
lma_status lma_set_synth_buffer_limit(lma_ctx* ctx, int64_t bytes);

/* Copy up to cap tuned synthesis launch shapes to out, oldest first (out may be NULL when cap
 * is 0); *n receives how many the context holds. */
lma_status lma_synth_tuning_read(lma_ctx* ctx, lma_synth_tuning* out, int32_t cap, int32_t* n);

#ifdef __cplusplus
}
#endif

#endif /* LMA_H */
