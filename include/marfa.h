/*
 * marfa.h — C-ABI of the GB300 line-by-line absorption library (libmarfa).
 *
 * The library computes, for every pressure–temperature level of a request, the
 * absorption coefficient k(nu) (or the cross-section sigma(nu)) of a line list on the
 * 2^-11 cm^-1 output grid, following arXiv 2411.03418:
 *   Sec. 2.1, Eqs. (2)-(3)  k(nu; p, T) = n(p, T) sum_j S_j(T) f_j(nu - nu~0_j)
 *   Sec. 2.2, Eqs. (4)-(8)  Lorentz, Gauss and Voigt line shapes, Voigt K(x, y)
 *   Sec. 2.3, Eqs. (9)-(10) Tonkov chi-factor of the line wings
 *   Sec. 2.4                the eleven-grid scheme: line centres on the finest grid,
 *                           wings on grids of steps 2^(1-g) cm^-1 (g = 1..10),
 *                           quadratic 3-point interpolation back onto the finest grid
 *   Appendix A              PT-table files, Appendix B  36-byte line records.
 *
 * Conventions for every call:
 *   - return 0 (MARFA_OK) on success or a negative MARFA_E_* code; nothing is thrown or
 *     aborted across the ABI; marfa_last_error() gives a message (thread-local);
 *   - inputs are copied by the library; outputs are owned by the caller;
 *   - all device work runs on the current CUDA device;
 *   - pointers documented as "host or device" are classified with
 *     cudaPointerGetAttributes; host outputs are filled before the call returns.
 */
#ifndef MARFA_H
#define MARFA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MARFA_OK 0
#define MARFA_E_INVAL (-1)    /* an argument is out of range or inconsistent          */
#define MARFA_E_NOMEM (-2)    /* a device or host allocation failed                    */
#define MARFA_E_CUDA (-3)     /* a CUDA runtime call or a kernel launch failed          */
#define MARFA_E_IO (-4)       /* a PT-table file could not be written                  */
#define MARFA_E_INTERNAL (-5) /* a device-side consistency check failed (bug)           */

/* line shapes (Sec. 2.2); the TEST shapes exist to pin the grid bookkeeping:
 * TEST_CONST adds exactly 1 per line within the cut-off (k counts lines),
 * TEST_QUAD adds S(T)[n](1 + d/4 + d^2/16), d = nu - nu~0 in cm^-1, which the 3-point
 * interpolation reproduces exactly; TEST_QUART adds S(T)[n] sum_{j<=4} (d/4)^j, which the
 * 5-point interpolation reproduces exactly. None applies the chi-factor. */
enum {
  MARFA_SHAPE_LORENTZ = 0,    /* Eq. (4)                                      */
  MARFA_SHAPE_VOIGT = 1,      /* Eqs. (7)-(8), the default of the paper        */
  MARFA_SHAPE_DOPPLER = 2,    /* Eq. (5)                                      */
  MARFA_SHAPE_USER = 4,       /* the user's shape of marfa_shape_user_set (Sec. 2.2: the
                                 shape is whatever function the user points it to) */
  MARFA_SHAPE_VOIGT_PAPER = 3, /* Eqs. (7)-(8) with K as Appendix C computes it:
                                  the Lorentz wing for |x| > 15, the region-4
                                  asymptote for y < 0.02, 1 < |x| < 5.5,
                                  Humlicek's rational approximations elsewhere */
  MARFA_SHAPE_TEST_CONST = 100,
  MARFA_SHAPE_TEST_QUAD = 101,
  MARFA_SHAPE_TEST_QUART = 102
};
enum { MARFA_CHI_NONE = 0, MARFA_CHI_TONKOV = 1 };          /* Eq. (10)          */
enum { MARFA_UNITS_SIGMA = 0,   /* cm^2/molecule, Eq. (3)                      */
       MARFA_UNITS_K_CM1 = 1,   /* cm^-1, Eq. (2) with n in molecules/cm^3      */
       MARFA_UNITS_K_KM1 = 2 }; /* km^-1                                        */

/* Appendix B database record: 36 bytes, no padding, little-endian. */
#pragma pack(push, 1)
typedef struct {
  double nu0;          /* transition wavenumber, cm^-1 (vacuum)                    */
  float S296;          /* intensity at 296 K, cm/molecule                           */
  float gamma_air;     /* air-broadened HWHM at 296 K, cm^-1/atm                     */
  float gamma_self;    /* self-broadened HWHM at 296 K, cm^-1/atm                    */
  float E_lower;       /* lower-state energy E'', cm^-1                              */
  float n_air;         /* temperature exponent of the widths                          */
  int32_t mol_iso;     /* jointMolIso: selects an entry of the species table         */
  float delta_air;     /* pressure shift at 296 K, cm^-1/atm                          */
} marfa_line_t;
#pragma pack(pop)

/* One per jointMolIso code. Q(T)/Q(296) = (T/296)^q_exp stands in for the TIPS table
 * (Sec. 4.2.2); chi_enabled marks molecules the chi-factor applies to (Sec. 2.3). */
typedef struct {
  int32_t mol_iso;
  int32_t chi_enabled;
  double mass_amu;     /* molar mass, g/mol (Sec. 4.2.3)                            */
  double q_exp;
} marfa_species_t;

typedef struct {
  double T_K;          /* temperature, K (> 0)                                      */
  double p_atm;        /* pressure, atm (> 0)                                        */
} marfa_level_t;

typedef struct {
  double nu_lo, nu_hi; /* window, cm^-1: outputs at k 2^-11 with nu_lo <= k 2^-11 <= nu_hi */
  double cutoff;       /* lines contribute where |nu - nu~0| <= cutoff, cm^-1 (0 < cutoff <= 1000) */
  int32_t shape;       /* MARFA_SHAPE_*                                              */
  int32_t chi;         /* MARFA_CHI_*                                                */
  int32_t units;       /* MARFA_UNITS_*                                              */
  int32_t surrogate;   /* 0: plain FP32 Voigt; 1: the learned surrogate (loaded with
                          marfa_surrogate_load on the current device) under its guard;
                          Voigt shape only. Not part of the paper.                    */
  int32_t R_w;         /* wing distance, in steps of a grid, below which that grid
                          refines (1..64; 8 is the default preset)                    */
  int32_t R_c;         /* a grid resolves a core when its step <= W / R_c (1..64)      */
  int32_t stencil;     /* interpolation points per coarse-grid panel: 3 (Sec. 2.4: panels
                          of two steps, quadratic; 0 means 3) or 5 (panels of four steps,
                          quartic; the same partition rules on the wider panels).
                          Not in the paper (its Sec. 2.4 mentions the option).      */
} marfa_request_t;

/* Opaque prepared line list, resident on the device it was prepared on. */
typedef struct marfa_lines marfa_lines_t;

/*
 * Copy n_lines Appendix-B records (host pointer) to the current device, sorted by nu0
 * (stable: ties keep input order), split into per-field arrays, together with the
 * species table (n_species entries, host pointer; every mol_iso of a line must appear
 * exactly once). *out receives a handle owned by the library; free it with
 * marfa_free_lines. Errors: MARFA_E_INVAL (n_lines < 1, non-finite or negative nu0,
 * unknown species, duplicate species), MARFA_E_NOMEM, MARFA_E_CUDA.
 */
int marfa_prepare_lines(const marfa_line_t* lines, int64_t n_lines,
                        const marfa_species_t* species, int32_t n_species,
                        marfa_lines_t** out);

/*
 * The line lists of n_req requests at once (the preparation step of a batch, App. B
 * records per request): lines[q] (n[q] records), species[q] (n_species[q] entries), all
 * host pointers; out[q] receives request q's handle, the same list marfa_prepare_lines
 * would make. The host work of the requests runs in parallel on the library's host
 * threads, the copies to the current device follow in one stream-ordered sequence. On
 * any error no handle is returned (every out[q] NULL, nothing held) and the message
 * names the first failing request. Errors: those of marfa_prepare_lines; MARFA_E_INVAL
 * for n_req < 1 or a NULL array. Not in the paper (it prepares one list at a time).
 */
int marfa_prepare_lines_batch(int32_t n_req, const marfa_line_t* const* lines, const int64_t* n_lines,
                              const marfa_species_t* const* species, const int32_t* n_species,
                              marfa_lines_t** out);

/* Release a handle from marfa_prepare_lines or marfa_prepare_lines_batch (NULL is
 * ignored). Waits until the device has finished every use of the list. */
void marfa_free_lines(marfa_lines_t* lines);

/* Number of output points of a window: #{k : nu_lo <= k 2^-11 <= nu_hi}; 0 if empty,
 * negative (MARFA_E_INVAL) for non-finite or negative bounds. */
int64_t marfa_num_points(double nu_lo, double nu_hi);

/*
 * Absorption of one request at n_levels levels (Sec. 2.1-2.4).
 *   levels : host, [n_levels] T and p;
 *   vmr    : host, [n_levels][n_species] volume mixing ratios in species-table order
 *            (partial pressure vmr*p, number density vmr*p/(k_B T));
 *   k_out  : host or device, [n_levels][npts] float32 row-major, npts =
 *            marfa_num_points(nu_lo, nu_hi); caller-owned;
 *   stream : cudaStream_t to run on (NULL = legacy default stream). With a device
 *            k_out the call is asynchronous on that stream; with a host k_out it
 *            returns when the result is there: page-locked host memory
 *            (cudaHostAlloc / cudaHostRegister) is written by the kernels directly,
 *            pageable memory through a device buffer and a copy back.
 * The line list must cover [nu_lo - cutoff, nu_hi + cutoff] for the sum to be complete;
 * lines outside cannot contribute. The value at a given nu does not depend on the
 * window or on other requests. Errors: MARFA_E_INVAL (window, cut-off, R_w/R_c, enum
 * values, T/p/vmr not finite and positive/non-negative, surrogate not 0/1, surrogate
 * with a shape other than Voigt or with no surrogate loaded on the current device, more
 * than 2^31 points), MARFA_E_NOMEM, MARFA_E_CUDA.
 */
int marfa_absorption(const marfa_lines_t* lines, const marfa_level_t* levels,
                     const double* vmr, int32_t n_levels, const marfa_request_t* rq,
                     float* k_out, void* stream);

/*
 * n_req independent requests in one pass: request r uses lines[r], levels[r],
 * vmr[r], n_levels[r], rq[r] and writes k_out[r] (host or device), with the same
 * meaning as marfa_absorption. All work of all requests goes into the same kernel
 * launches. Results are identical to n_req separate marfa_absorption calls.
 */
int marfa_absorption_batch(int32_t n_req, const marfa_lines_t* const* lines,
                           const marfa_level_t* const* levels, const double* const* vmr,
                           const int32_t* n_levels, const marfa_request_t* rq,
                           float* const* k_out, void* stream);

/*
 * A batch of requests captured once as a CUDA graph and replayed on demand. Creation
 * does everything marfa_absorption_batch does before its first kernel (validation,
 * per-level tables, work lists, device buffers), runs the batch once (so k_out holds the
 * result on return) and captures one graph: level preparation of every request, grid 1,
 * grids 2..10 and the finest grid with the cascade, over all requests together.
 *   k_out    : device, [n_req] pointers to [n_levels[r]][npts_r] float32, owned by the
 *              caller and kept by the plan: every execution rewrites them;
 *   lines    : must stay alive until marfa_plan_destroy; levels, vmr and rq are copied,
 *              and so is the loaded surrogate for requests with surrogate = 1;
 *   flags    : MARFA_PLAN_AUTOTUNE: for each size class of the batch (marfa_plan_classes):
 *              the grid-1 split (1, 2, 3 or 6 CTAs per tile), and for each of grids
 *              2..10 the six summation
 *              kernels (line-major: a thread per candidate line over 32 or over 16 node
 *              pairs; two-phase: warps of 32 node pairs that stage 32 lines at a time;
 *              flattened: the two-phase tiles with the evaluations spread evenly over
 *              the lanes and grouped by Voigt branch; by mechanism: the two-phase tiles
 *              with candidates taken per centre, cut-off edge and chi breakpoint, each
 *              with closed-form ownership, where those lie far enough apart, in a
 *              pass per mechanism or one merged pass), and for the finest grid its four
 *              kernels (8-lane groups per G10 panel; flattened (line, panel) jobs, with
 *              general or closed-form ownership, the latter in a pass per mechanism or
 *              a centre pass and one merged edge/breakpoint pass), on
 *              this batch's own work and keep the fastest (otherwise the defaults of
 *              marfa_diag_variants); MARFA_PLAN_SERIAL: capture
 *              grids 1..10 one after the
 *              other (otherwise they are parallel branches of the graph, which the GPU
 *              runs concurrently, and per-kernel times overlap);
 *   stream   : used for creation (synchronised before return).
 * Results equal marfa_absorption_batch's bit for bit when the kernel choice is the
 * default; the other variants sum in another order (same tolerance to the oracle). With
 * surrogate requests, creation also makes one counted run and gives the grids where the
 * surrogate's guard never holds for this batch the plain kernels (same results).
 * Errors: those of marfa_absorption_batch, host k_out (MARFA_E_INVAL), capture errors
 * (MARFA_E_CUDA). The paper has no counterpart (it runs one level at a time on CPUs).
 */
typedef struct marfa_plan marfa_plan_t;
#define MARFA_PLAN_AUTOTUNE 1
#define MARFA_PLAN_SERIAL 2
int marfa_plan_create(int32_t n_req, const marfa_lines_t* const* lines,
                      const marfa_level_t* const* levels, const double* const* vmr,
                      const int32_t* n_levels, const marfa_request_t* rq, float* const* k_out,
                      int32_t flags, void* stream, marfa_plan_t** out);

/* Replay the plan's graph on stream (asynchronous; NULL = legacy default stream). The
 * current device must be the plan's. */
int marfa_plan_execute(marfa_plan_t* plan, void* stream);

/* Kernel choice and timings (host arrays, each may be NULL): variant[MARFA_PLAN_KINDS]
 * for grids 1..10 and the finest grid (grid 1: -1, its one kernel; grids 2..10: 0
 * line-major over 32 pairs, 1 two-phase, 2 line-major over 16 pairs, 3 flattened, 4 by
 * mechanism (closed-form ownership, a pass per mechanism; the launch takes 1 where it
 * does not apply), 5 by mechanism in one merged pass; finest
 * grid: 0 groups per panel, 1 flattened jobs, 2 flattened jobs by mechanism (1 where it
 * does not apply), 3 the same with a centre pass and one merged pass over the cut-off
 * edges and breakpoints (2 where a line's edge and a breakpoint can share a warp's
 * nodes)); tune_ms[MARFA_PLAN_KINDS][MARFA_PLAN_VARIANTS]
 * the autotuner's time per launch of each variant (-1 when not tuned or not a variant of
 * that kind); kernel_ms[12] device time of the last
 * execution per kernel kind (0 level preparation, 1..10 grids, 11 finest grid; waits for
 * that execution; MARFA_E_CUDA before the first execution). */
#define MARFA_PLAN_KINDS 11
#define MARFA_PLAN_VARIANTS 6
/* These report the kernel choice of request 0's size class (marfa_plan_classes). */
int marfa_plan_info(const marfa_plan_t* plan, int32_t* variant, float* tune_ms, double* kernel_ms);

/*
 * A user-defined line shape (Sec. 2.2: the code calls the shape through a pointer the
 * user may redirect to any function; here a table the library interpolates). g holds n
 * samples (2..4096, finite, >= 0, host array) of a symmetric g(x) at x = k x_max /
 * (n - 1), k = 0..n-1; the shape is g linear between samples and g(x_max) (x_max/|x|)^2
 * beyond x_max, on the Lorentz scaling: x = (nu - nu~0) / gamma_L and
 * f = S / (pi gamma_L) g(x), so that g = 1/(1 + x^2) gives Eq. (4); its half width for
 * the grid choice (g*) is gamma_L. Requests with shape MARFA_SHAPE_USER take it (on the
 * current device; every device needs its own call; a later call replaces the table for
 * later calls and plans). The chi-factor and the cut-off apply as for every shape.
 * Errors: MARFA_E_INVAL (sizes, x_max outside (0, 1e6], bad samples), MARFA_E_CUDA.
 */
int marfa_shape_user_set(const float* g, int32_t n, double x_max);

/* Size classes of a plan: the autotuner treats narrow requests (windows of at most
 * 16 cm^-1, 32769 points) and wider ones apart, since their tiles and candidate counts
 * differ. Host arrays, each may be NULL: req_class[n_req] receives each request's class
 * (0 narrow, 1 wide); choice[2][MARFA_PLAN_KINDS] the choice per class (entry 0: the
 * grid-1 split, the number of CTAs that share a grid-1 tile's candidate lines, 1, 2, 3 or
 * 6; entries 1..10: the variants of marfa_plan_info's layout), -1 for a class with no
 * request; tune_ms[2][MARFA_PLAN_KINDS][MARFA_PLAN_VARIANTS] the autotuner's time per
 * launch of each choice (entry 0: of the splits 1, 2, 3, 6), -1 where not timed. Without
 * MARFA_PLAN_AUTOTUNE the narrow class takes split 2, the wide class split 6, and both
 * the marfa_diag_variants defaults (as marfa_absorption and marfa_absorption_batch do).
 * Errors: MARFA_E_INVAL for a NULL plan. */
#define MARFA_PLAN_CLASSES 2
int marfa_plan_classes(const marfa_plan_t* plan, int32_t* req_class, int32_t* choice, float* tune_ms);

/* Test and tuning hook: the process-wide kernel variants that calls without autotuning
 * use (marfa_absorption, marfa_absorption_batch, marfa_absorption_noalloc and plans
 * created without MARFA_PLAN_AUTOTUNE), in the layout of marfa_plan_info's variant
 * array (entry 0, grid 1, is ignored on set and -1 on get). set (may be NULL): the new
 * defaults, each checked against its kind's range (MARFA_E_INVAL, nothing changed);
 * get (may be NULL): receives the defaults after the call. Every variant computes the
 * same partition; they differ only in the order of the sums (the same tolerance to the
 * oracle). Calls already running keep the variants they started with. */
int marfa_diag_variants(const int32_t* set, int32_t* get);

/* Free the plan's graph and device buffers (waits for the device). */
void marfa_plan_destroy(marfa_plan_t* plan);

/*
 * Appendix A PT-table: write k (host, npts float32 values at k 2^-11 over
 * [nu_lo, nu_hi]) into <dir>/<level_number padded with '_' to 3 chars>.ptbin as
 * direct-access records of 20481 float32 (little-endian) each; record r (1-based,
 * r = int(nu/10)) covers [10 r, 10 r + 10] and sits at byte offset
 * (r - 1) * 20481 * 4. nu_lo and nu_hi must be multiples of 10 with nu_lo < nu_hi and
 * npts must equal marfa_num_points(nu_lo, nu_hi). Records outside the window are left
 * as they are in an existing file (zero in a new one). Errors: MARFA_E_INVAL, MARFA_E_IO.
 */
int marfa_write_pt_table(const char* dir, int32_t level_number, double nu_lo,
                         double nu_hi, const float* k, int64_t npts);

/*
 * Appendix B: line records from the text of a HITRAN .par file (the conversion the
 * paper's utility performs before a run). Records are the 160-column fixed-width lines
 * of the HITRAN 2004+ format; the fields used are molecule (columns 1-2), isotopologue
 * (3: '1'..'9', '0' for 10, 'A', 'B', ... for 11, 12, ...), nu (4-15), S (16-25),
 * gamma_air (36-40), gamma_self (41-45), E'' (46-55), n_air (56-59) and delta_air
 * (60-67); the rest of a record is not read. jointMolIso, whose layout the paper leaves
 * to its documentation, is 100 * molecule + isotopologue.
 *   text, len : host, the file contents; records end with '\n' (a '\r' before it is
 *               dropped); blank lines are skipped; each record needs its first 67 columns;
 *   out, cap  : host, room for cap records (out may be NULL when cap is 0: count only);
 *   n_out     : receives the number of records in text (also when cap is too small).
 * Records keep the file's order. Errors: MARFA_E_INVAL for a malformed or short record
 * (marfa_last_error names its line) and when cap is smaller than the record count
 * (nothing is written then).
 */
int marfa_read_par(const char* text, int64_t len, marfa_line_t* out, int64_t cap, int64_t* n_out);

/*
 * marfa_absorption without any device allocation, for callers that cannot allocate
 * device memory: a host model that has given all free device memory to its own pool
 * (so cudaMalloc would fail or fragment it), or a pipeline that must not let an
 * allocation or a free synchronise the device while its other streams run. The paper
 * has no counterpart of this call; it computes the same k(nu) as marfa_absorption.
 *   - Scratch: a file-scope __device__ array of 32 MiB (MARFA_NOALLOC_SCRATCH_BYTES).
 *     A device commits it when marfa_prepare_lines first runs there: that call looks
 *     up the array's device address (cudaGetSymbolAddress, with the device current),
 *     which loads the part of the library holding it, and fails with MARFA_E_NOMEM if
 *     the 32 MiB cannot be had. From then on the device holds the array until the
 *     process exits, and marfa_absorption_noalloc itself allocates nothing. The set-up
 *     call (marfa_prepare_lines) must come before any stream capture, like any call
 *     that allocates. A request whose per-level line data, grid slots and work lists
 *     exceed the array is rejected with MARFA_E_INVAL (for example: one level of
 *     200,000 lines on a 1000 cm^-1 window fits; sixty such levels do not).
 *   - k_out must be device memory ([n_levels][npts] float32); host outputs are
 *     rejected with MARFA_E_INVAL. lines comes from marfa_prepare_lines.
 *   - Every call reuses the same scratch and leaves its contents there; the kernels
 *     write every value they read, so nothing needs clearing between calls. Calls
 *     whose work overlaps on the GPU (other streams, other host threads) race on the
 *     scratch: serialise them.
 *   - Asynchronous on stream (NULL = legacy default stream); the level tables and work
 *     lists are copied into the scratch from the call's own pageable host memory. A
 *     stream in capture is refused with MARFA_E_INVAL, since those copies would be
 *     recorded from host memory freed when the call returns.
 */
#define MARFA_NOALLOC_SCRATCH_BYTES (32u << 20)
int marfa_absorption_noalloc(const marfa_lines_t* lines, const marfa_level_t* levels,
                             const double* vmr, int32_t n_levels, const marfa_request_t* rq,
                             float* k_out, void* stream);

/* ---------------------------------------------------------------- learned Voigt surrogate
 * Not part of the paper. A 2-64-64-64-1 SiLU network predicts t = ln(K / K0) from
 * u1 = ln y and u2 = ln(1 + |x| / (1 + y)), where
 *   K0(x, y) = exp(-x^2) / (1 + 2y/sqrt(pi)) + y / (sqrt(pi) (x^2 + y^2 + 1)),
 * so that K = K0 exp(t). Parameters: MARFA_MLP_PARAMS float32 packed as W1[64][2], b1[64],
 * W2[64][64], b2[64], W3[64][64], b3[64], W4[64], b4[1] (W row-major [out][in]).
 * Training runs on the current device in FP32 (mean squared error of t, Adam); inference
 * runs on the tensor cores with BF16 W2, W3 and activations and FP32 accumulation.
 */
#define MARFA_MLP_PARAMS 8577
#define MARFA_MLP_MAX_BATCH 65536
/* Guard cells: |x| in [0, 12) in steps of 1/8 (index ix); y by binary exponent
 * e in [-14, 3] and the two leading mantissa bits k, y in [2^e (1 + k/4), 2^e (1 + (k+1)/4))
 * (index iy = 4 (e + 14) + k); cell = iy * MARFA_GUARD_NX + ix. */
#define MARFA_GUARD_NX 96
#define MARFA_GUARD_NY 72

typedef struct {
  int32_t steps;       /* optimiser steps (>= 1)                                     */
  int32_t batch;       /* samples per step (1..MARFA_MLP_MAX_BATCH); step k takes the
                          next batch of consecutive samples, wrapping at the end      */
  int32_t qat;         /* 1: forward pass rounds W2, W3 and the hidden activations of
                          layers 1-2 to BF16 as inference does (straight-through)     */
  int32_t reserved;
  float lr0, lr1;      /* Adam step size, cosine schedule from lr0 (step 0) to lr1    */
} marfa_mlp_train_t;

/* Mean squared error of the network's t over n samples and its gradient (host arrays:
 * params [MARFA_MLP_PARAMS], x, y, t [n] with y > 0, grad [MARFA_MLP_PARAMS] out,
 * loss out; n <= MARFA_MLP_MAX_BATCH). Runs the training kernels once (FP32; qat as
 * in marfa_mlp_train_t). Errors: MARFA_E_INVAL, MARFA_E_NOMEM, MARFA_E_CUDA. */
int marfa_mlp_loss_grad(const float* params, const float* x, const float* y, const float* t,
                        int64_t n, int32_t qat, double* loss, float* grad);

/* Train params (host, in/out) on the n samples (host x, y, t) with Adam; the
 * mean-squared-error of each step goes to loss_curve[steps] (host, may be NULL).
 * Synchronous. Errors: MARFA_E_INVAL, MARFA_E_NOMEM, MARFA_E_CUDA. */
int marfa_mlp_train(float* params, const float* x, const float* y, const float* t, int64_t n,
                    const marfa_mlp_train_t* cfg, float* loss_curve);

/* Make params (host) the surrogate of the current device: convert them to the
 * inference layout and build the guard. A guard cell is switched on when it lies in
 * 1e-4 <= y <= 10, in the region where the plain FP32 Voigt takes its costly branches
 * (y < 1, or x^2 + y^2 < 64), and the surrogate agrees with the plain FP32 Voigt within
 * the relative budget at all samples x samples lattice points spanning the cell
 * (2 <= samples <= 64). cells_on (may be NULL) receives the number of cells switched on
 * and cell_err (host [MARFA_GUARD_NY * MARFA_GUARD_NX], may be NULL) the largest
 * relative difference per cell (-1 outside the eligible region). Replaces a surrogate
 * loaded before; not to be called while absorption calls run. Synchronous. */
int marfa_surrogate_load(const float* params, float budget, int32_t samples, int32_t* cells_on,
                         float* cell_err);

/* Release the loaded surrogate (no-op if none). */
int marfa_surrogate_unload(void);

/* K(x, y) of the loaded surrogate at n points (host arrays; y > 0): guarded = 0 the
 * network alone, guarded = 1 the evaluation the profile kernels use (the network where
 * the guard holds, the plain FP32 Voigt elsewhere). */
int marfa_surrogate_eval(const float* x, const float* y, float* out, int64_t n, int32_t guarded);

/* Message of the last failing call on this thread ("" if none). */
const char* marfa_last_error(void);

/* ---------------------------------------------------------------- diagnostics
 * Entry points used by the parity tests; same conventions as above.
 */

/* FP32 Voigt function K(x, y) of Eq. (8) as the kernels evaluate it, at n points
 * (x, y host arrays, out host array; y > 0). */
int marfa_diag_voigt(const float* x, const float* y, float* out, int64_t n);

/* Per-level line data the kernels use: centre c = rint((nu0 + delta p) 2^43) (int64)
 * and g* (the coarsest grid 1..10 resolving the core, 11 = finest), per level and per
 * line in prepared (sorted) order; outputs host arrays [n_levels][n_lines]. The
 * prepared order of input line i is perm[i] (host, [n_lines], may be NULL). */
int marfa_diag_level_lines(const marfa_lines_t* lines, const marfa_level_t* levels,
                           const double* vmr, int32_t n_levels, const marfa_request_t* rq,
                           int64_t* c_out, int8_t* gstar_out, int64_t* perm);

/* Ownership as the kernels decide it, for one level and one grid g (1..10: panels
 * [first, first + count) of width 2^(2-g) cm^-1; 11: finest nodes [first, first + count)),
 * for every line in prepared order: out[line * count + i] = 1 if that grid sums the line
 * there, else 0 (host array [n_lines][count]). */
int marfa_diag_owned(const marfa_lines_t* lines, const marfa_level_t* levels,
                     const double* vmr, int32_t n_levels, const marfa_request_t* rq,
                     int32_t level, int32_t grid, int64_t first, int32_t count,
                     uint8_t* out);

/* marfa_absorption that also counts the distinct (line, node) profile evaluations per
 * level and grid: counts host array [n_levels][11] (grids 1..10, then the finest). */
int marfa_diag_absorption_counted(const marfa_lines_t* lines, const marfa_level_t* levels,
                                  const double* vmr, int32_t n_levels,
                                  const marfa_request_t* rq, float* k_out, int64_t* counts);

/* marfa_absorption with every evaluation counted: counts host array [n_levels][11][5]
 * (grids 1..10, then the finest), per grid: all (line, node) profile evaluations, those
 * the surrogate took, and the plain Voigt evaluations in the 9 x 9 polynomial cells
 * (1/4 <= y < 1 and |x| < 12, or |z| < 4.5 with y >= 1), in the 6- or 15-term
 * asymptotic series (|z| < 100) and in the small-y cells (y < 1/4, |x| < 12); the rest
 * are far-wing two-term evaluations (or other shapes). */
int marfa_diag_absorption_counts(const marfa_lines_t* lines, const marfa_level_t* levels,
                                 const double* vmr, int32_t n_levels, const marfa_request_t* rq,
                                 float* k_out, int64_t* counts);

/* marfa_diag_absorption_counted that also returns, in surrogate_counts (host
 * [n_levels][11]), how many of those evaluations the surrogate took. */
int marfa_diag_absorption_counted_surrogate(const marfa_lines_t* lines,
                                            const marfa_level_t* levels, const double* vmr,
                                            int32_t n_levels, const marfa_request_t* rq,
                                            float* k_out, int64_t* counts,
                                            int64_t* surrogate_counts);

/* The line shape K(x, y) (or f(x) for the non-Voigt shapes, y ignored) as the kernels
 * evaluate it, for shape = MARFA_SHAPE_* at n points (host arrays x, y, out). */
int marfa_diag_shape(int32_t shape, const float* x, const float* y, float* out, int64_t n);

/* The order marfa_prepare_lines gives the lines (host only, no device call): order[j] =
 * the input index of the j-th line of a stable sort by nu0 (host array [n]; the identity
 * when the input is already ordered). Errors: MARFA_E_INVAL (nu0 outside [0, 1e5]),
 * MARFA_E_NOMEM. */
int marfa_diag_line_order(const marfa_line_t* lines, int64_t n, int64_t* order);

/* Issue rate of one instruction kind on this device, for the roofline denominators:
 * pipe 0 FP32 FMA, 1 MUFU ex2.approx, 2 MUFU rcp.approx, 3 MUFU cos.approx. Eight
 * 256-thread CTAs per SM run eight independent dependency chains a thread; five timed
 * launches after one warm-up, CUDA events on the default stream. Writes instructions per
 * second (an FMA counts once) to *ops_per_s. */
int marfa_diag_pipe_rate(int32_t pipe, double* ops_per_s);

/* Per-kernel device time: enable = 1 clears the totals and starts recording CUDA events
 * around every kernel launch of this library (on the launch stream); enable = 0 stops,
 * waits for the recorded events and writes, for the twelve kernel launches of a call
 * (0 level preparation, g = 1..10 the sums on grid g, 11 finest grid + cascade), the
 * summed milliseconds to ms[12] and the launch counts to launches[12] (host arrays,
 * may be NULL). */
int marfa_diag_kernel_timing(int32_t enable, double* ms, int64_t* launches);

/* Error-path testing (no counterpart in the paper): make the nth allocation from now on
 * fail as if memory were exhausted (nth >= 1; 0 disarms). Counted allocations: the
 * stream-ordered device buffers of calls and plans, the line list's device block, host
 * staging buffer and object, plan objects and the surrogate's device buffers. The entry
 * point that meets the failure returns MARFA_E_NOMEM after freeing what it had
 * allocated; the injector then disarms itself. The environment variable
 * MARFA_FAIL_ALLOC=n arms it when the library loads. left (may be NULL) receives the
 * allocations the previous arming still had to let through plus one (0: not armed).
 * Errors: MARFA_E_INVAL for nth < 0. */
int marfa_diag_fail_alloc(int64_t nth, int64_t* left);

/* Device memory in use, for leak checks: after synchronising the current device,
 * pool_used receives the bytes allocated from its default memory pool (the library's
 * stream-ordered buffers) and device_free the free device memory (cudaMemGetInfo); each
 * may be NULL. Errors: MARFA_E_CUDA. */
int marfa_diag_device_memory(int64_t* pool_used, int64_t* device_free);

/* Device-side checks (no counterpart in the paper). A library built with MARFA_DEBUG
 * guards its kernels' indexed shared and global accesses with range checks that, when
 * one fails, skip the access and record a code in a device status word instead of
 * trapping; every call (and plan execution) then waits for the device and returns
 * MARFA_E_INTERNAL naming the first failed check (the word is cleared). An ordinary
 * build has no checks. This entry point runs a probe kernel that makes a store at
 * index of a 32-entry array only when the index is in range: in a MARFA_DEBUG build an
 * index outside 0..31 records check 901 and the call returns MARFA_E_INTERNAL; an
 * ordinary build returns MARFA_OK. debug_build (may be NULL) receives 1 for a
 * MARFA_DEBUG build. */
int marfa_diag_check(int32_t index, int32_t* debug_build);

#ifdef __cplusplus
}
#endif
#endif /* MARFA_H */
