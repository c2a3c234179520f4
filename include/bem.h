/*
 * bem.h - C ABI of the GB300 FFT-BEM library (libbem.so).
 *
 * Contact of a rigid indenter with an elastic layer (thickness h, modulus E1,
 * Poisson ratio nu1) bonded to an elastic half-space (E2, nu2), after
 * Li, Pohrt, Lyashenko and Popov, "Boundary Element Method for non-adhesive and
 * adhesive contacts of a coated elastic half-space" (arXiv:1807.01885).
 *
 * Discretisation (Sec. 2, Fig. 2): a square window of N x N cells of side delta,
 * pressure uniform per cell, stored row-major (cell (r, c) at index r*N + c).
 * The surface operator u = K p (Eq. 1) is evaluated as in Eq. (11):
 *     u = crop( IFFT[ K^(|k|) . FFT(pad(p)) ] )
 * on a 2N x 2N period (zero pressure outside the window), with the compliance
 * K^(k) of Eq. (9)/(10) sampled at k = 2 pi (i, j) / (2N delta).  The k = 0 term,
 * which Eq. (11) leaves undefined ("no DC component", Sec. 2), is the finite part
 * lim_{k->0} [K^(k) - 2/(E2* k)] (dc_mode 0; equal to h/E~1 of Eq. 15 for a
 * rigid base and to 0 for a homogeneous body) or 0 (dc_mode 1).
 *
 * Sign conventions (Sec. 2, condition (c)): p > 0 is compressive; u > 0 points
 * into the body; the indenter height f >= 0 is measured up from its lowest
 * point; d is the indentation depth; the gap is g = u + f - d.
 *
 * Memory: every array argument is a plain pointer to N*N elements of the kernel's
 * precision (double for BEM_FP64, float for BEM_FP32), row-major, owned by the
 * caller.  A pointer may be device memory or host memory (pageable or pinned);
 * host arrays are staged through the library's own device workspace.  The library
 * owns kernel handles and their workspaces.  No call throws; every call returns a
 * bem_status and bem_last_error() gives a message for the calling thread.
 * Calls on one handle must not overlap (the handle's workspace is shared).
 */
#ifndef BEM_H
#define BEM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  BEM_OK = 0,
  BEM_EINVAL = 1,        /* invalid argument (null pointer, nu >= 0.5, h < 0, N not supported...) */
  BEM_ENOMEM = 2,        /* device allocation failed */
  BEM_ECUDA = 3,         /* a CUDA runtime call failed */
  BEM_ENOCONV = 4,       /* iteration limit reached before the tolerance */
  BEM_ETIMEOUT = 5,      /* a bounded device-side wait gave up */
  BEM_ENAN = 6,          /* non-finite value met in a reduction */
  BEM_ECYCLE = 7,        /* adhesive contact set revisited an earlier state */
  BEM_EUNSUPPORTED = 8,  /* a valid request outside what this operator kind supports */
  BEM_EDETACHED = 9      /* adhesive force control: the contact area vanished (the force is
                            below what the contact can carry; under load control the
                            indenter jumps off) */
} bem_status;

enum { BEM_FP64 = 0, BEM_FP32 = 1 };                   /* bem_kernel_desc.precision */
enum { BEM_CTRL_DEPTH = 0, BEM_CTRL_FORCE = 1 };       /* bem_problem.control */
enum { BEM_DC_FINITE_PART = 0, BEM_DC_ZERO = 1 };      /* bem_kernel_desc.dc_mode */
enum { BEM_OP_PERIODIC = 0, BEM_OP_OPEN = 1 };        /* bem_kernel_desc.op_kind */

/* Parameters of the discretised operator (Sec. 2): grid, cell size, layer and
 * substrate.  N is a power of two, 4 <= N <= 2048.  h may be INFINITY (homogeneous
 * E1, nu1), E2 may be INFINITY (rigid base; the paper's E2 = e^100).  0 <= nu < 0.5.
 *
 * op_kind BEM_OP_PERIODIC (0): the paper's periodic product, Eq. (11), with the k = 0
 * rule of dc_mode.  BEM_OP_OPEN (1): the non-periodic operator of a homogeneous
 * half-space (h = INFINITY: E1, nu1; h = 0, or equal materials: E2, nu2): the
 * surface displacement of a uniformly loaded square cell (the real-space form of
 * Eq. 4 integrated over the cell, in closed form) convolved over the open plane, so
 * that no periodic image and no k = 0 convention enter (dc_mode is ignored).  It is
 * evaluated by the same FFT passes: the 2N-periodic wrap-around array of the cell
 * coefficients (offsets up to N - 1, which is all a window of N cells uses) is
 * transformed once, in double, into the compliance table.  A coating of a different
 * material gives BEM_EUNSUPPORTED.  Building the table costs two double matrix
 * products of order N + 1 (about 50 ms at N = 2048). */
typedef struct {
  int32_t N;
  int32_t precision;    /* BEM_FP64: everything in double.  BEM_FP32: FFTs and vectors
                           in float; reductions, CG scalars and the detachment
                           test in double. */
  int32_t dc_mode;
  int32_t op_kind;      /* BEM_OP_PERIODIC or BEM_OP_OPEN (earlier versions: reserved, 0) */
  double delta, h, E1, nu1, E2, nu2;
} bem_kernel_desc;

typedef struct bem_kernel_s* bem_kernel;

/* One contact problem on a kernel's grid.
 *  height        indenter height map f (N*N), host or device.
 *  control       BEM_CTRL_DEPTH: target is the depth d.  BEM_CTRL_FORCE: target is
 *                the total force F = delta^2 sum p and d is found: non-adhesive,
 *                F > 0; adhesive (dgamma > 0), any finite F, starting from the
 *                non-empty contact_mask: every fixed-area solve of the procedure
 *                carries F (d is the multiplier of that constraint), and the
 *                result is BEM_EDETACHED if the area vanishes on the way.
 *  dgamma        work of adhesion; 0 selects non-adhesive contact (p >= 0).  > 0
 *                runs ONE displacement-controlled step of the adhesive procedure of
 *                Sec. 2 at depth target, with the detachment stress of Eq. (12).
 *  tol           relative gap residual ||g||_C / ||u||_C at which CG stops.
 *  max_iter      CG iteration limit (per inner solve in adhesive mode).
 *  p_init        optional warm start (N*N), may be NULL.
 *  contact_mask  adhesive mode: N*N bytes, 1 = in contact; read as the starting
 *                contact area and overwritten with the final one (host or device).
 *                May be NULL (start from no contact).  Ignored when dgamma == 0. */
typedef struct {
  const void* height;
  const void* p_init;
  uint8_t* contact_mask;
  int32_t control;
  int32_t max_iter;
  double target;
  double dgamma;
  double tol;
} bem_problem;

/* Scalars of a solve, all in double. */
typedef struct {
  double force;       /* delta^2 sum p */
  double depth;       /* d (given, or found under force control) */
  double area;        /* delta^2 * number of cells in contact */
  double a_eq;        /* sqrt(area / pi) */
  double residual;    /* CG's convergence measure at exit (recursively updated gap) */
  double err_est;     /* the same measure recomputed from a fresh u = K p */
  int32_t iters;      /* CG iterations (summed over inner solves in adhesive mode) */
  int32_t outer_iters;/* adhesive contact-area updates (1 for non-adhesive) */
  int32_t n_contact;
  int32_t status;     /* bem_status of this solve */
  int32_t matvecs;    /* operator products performed */
  int32_t reserved;
} bem_result;

/* Builds the operator: evaluates Eq. (9)/(10) in double on the device for every
 * |k| of the 2N x 2N grid (folded by symmetry to (N+1)^2 values) and stores it in
 * the kernel's precision.  stream may be NULL (legacy default stream). */
bem_status bem_make_kernel(const bem_kernel_desc* desc, void* cuda_stream, bem_kernel* out);
bem_status bem_destroy_kernel(bem_kernel k);

/* One layer of a coating stack: thickness, Young's modulus, Poisson ratio. */
#define BEM_MAX_LAYERS 8
typedef struct {
  double h, E, nu;
} bem_layer;

/* Builds the operator of a stack of n_layers (1..BEM_MAX_LAYERS) bonded layers,
 * listed from the surface down, on the substrate (desc->E2, desc->nu2; E2 = INFINITY
 * is a rigid base): the multi-layer generalisation of Eqs. (9)/(10), which the paper
 * gives for one layer.  The compliance follows from Eq. (5) with boundary conditions
 * (a)-(d) of Sec. 2 at the surface and at every interface, evaluated in double for
 * every |k| of the grid; the k = 0 entry is the finite part lim_{k->0}[K(k) - 2/(E2* k)]
 * (dc_mode 0; for a rigid base the stack's uniaxial compliance sum h/E~) or 0
 * (dc_mode 1).  desc->N, precision, dc_mode, delta, E2 and nu2 are used as in
 * bem_make_kernel; desc->h, E1 and nu1 are ignored and replaced, in the handle, by the
 * stack's total thickness and the top layer's E and nu (the top layer sets the
 * detachment stress of Eq. 12).  Each layer needs 0 <= h < INFINITY, 0 < E < INFINITY,
 * 0 <= nu < 0.5, and the stack a positive total thickness; else BEM_EINVAL.  One
 * layer gives the table of bem_make_kernel with the same h, E1, nu1 (to rounding). */
bem_status bem_make_kernel_layers(const bem_kernel_desc* desc, int32_t n_layers, const bem_layer* layers,
                                  void* cuda_stream, bem_kernel* out);

/* Rebuilds an existing handle's operator for new parameters in place: desc->N and
 * desc->precision must equal the handle's (BEM_EINVAL otherwise); delta, h, E1, nu1,
 * E2, nu2, dc_mode and op_kind may change (a coating stack made by
 * bem_make_kernel_layers becomes the single coating of desc).  Allocates nothing and
 * keeps the handle's captured iteration graphs valid (they read the table in place),
 * so a pool of handles can serve a stream of instances of one grid size, as the
 * learned warm start's training-set generation does.  Synchronises the stream. */
bem_status bem_rebuild_kernel(bem_kernel k, const bem_kernel_desc* desc, void* cuda_stream);

/* Copies the double-precision compliance table K^(k_ij), i, j in [0, N], row-major
 * (N+1)*(N+1) doubles, in m/Pa-consistent units (no FFT normalisation), to out
 * (host or device).  Entry (0,0) is the DC value chosen by dc_mode. */
bem_status bem_kernel_table(bem_kernel k, void* out, void* cuda_stream);

/* Workspace guard check (a debugging aid, not part of the method): every large array
 * of the handle's workspace (spectrum, tables, twiddles, solver vectors, masks,
 * partial sums, staging) sits between two 256-byte zones of a fixed byte pattern;
 * *bad_bytes receives the number of zone bytes that no longer hold it (0 unless a
 * kernel wrote outside an array).  Synchronises the stream.
 * bem_debug_poke_guard overwrites one byte of the zone after array i (0 <= i < the
 * number of guarded arrays; BEM_EINVAL otherwise) with a host-side memset: fault
 * injection for testing the check, no kernel runs. */
bem_status bem_check_guards(bem_kernel k, int64_t* bad_bytes, void* cuda_stream);
bem_status bem_debug_poke_guard(bem_kernel k, int32_t i);

/* u = K p (Eq. 1 evaluated by Eq. 11).  p and u: N*N, host or device.  Device
 * arguments: asynchronous on the stream.  Host arguments: returns after u is written. */
bem_status bem_matvec(bem_kernel k, const void* p, void* u, void* cuda_stream);

/* Solves one contact problem; writes the pressure to p_out (N*N, host or device)
 * and the scalars to *res (host).  Synchronises the stream before returning.
 * Non-adhesive: Polonsky-Keer constrained conjugate gradients (the method the
 * paper cites for the inverse problem, Sec. 2).  Adhesive: Sec. 2's procedure at
 * one depth: CG on the fixed contact area, penetrating cells join, boundary cells
 * with tension above sigma_c (Eq. 12, compared in double) detach, repeat.
 * Diagnostics: with the environment variable BEM_TRACE set (any value) when the
 * process makes its first non-adhesive solve, every 8-iteration chunk prints the
 * iteration count, the residual and the contact-set counts to stderr. */
bem_status bem_solve_contact(bem_kernel k, const bem_problem* prob, void* p_out,
                             bem_result* res, void* cuda_stream);

/* Solves n independent problems (each with its own kernel and grid size).
 * res is a host array of n results; the return value is BEM_OK if every
 * instance converged, else the first failing status. */
bem_status bem_solve_batch(int32_t n, const bem_kernel* kernels, const bem_problem* probs,
                           void* const* p_out, bem_result* res, void* cuda_stream);

/* Profiling aid (not part of the paper's method): runs `reps` products u = K p
 * (p, u device arrays) with CUDA events recorded on `cuda_stream` around each of
 * the three passes, and writes the mean duration of each pass in milliseconds to
 * ms_out[0] (row forward FFT), ms_out[1] (column FFT x K^ x inverse FFT) and
 * ms_out[2] (row inverse FFT).  Synchronises the stream. */
bem_status bem_profile_passes(bem_kernel k, const void* p, void* u, int32_t reps, float* ms_out,
                              void* cuda_stream);

/* FFT radix of the register passes (N >= 16; an implementation choice, no
 * counterpart in the paper).  Each row and column transform runs as stages of
 * radix 2^row_log2_radix / 2^col_log2_radix (3: radix 8, 4: radix 16) with one
 * shared-memory exchange between stages; results agree to rounding either way.
 * bem_set_radix rebuilds the stage twiddle tables on cuda_stream and drops the
 * handle's captured CG-iteration graph (the next solve on a capturable stream
 * captures it again).  The float path accepts 3 or 4 for each; the double path only
 * 3.  Other values give BEM_EINVAL; N < 16 ignores the call.  Synchronises the
 * stream. */
bem_status bem_set_radix(bem_kernel k, int32_t row_log2_radix, int32_t col_log2_radix, void* cuda_stream);

/* Autotuner of those choices: times every allowed radix of the row passes (forward
 * and inverse together) and of the column pass, `reps` launches each (CUDA events on
 * cuda_stream, minimum over the launches), on the handle's own workspace, keeps the
 * fastest of each and writes it to choice_out[0] (rows) and choice_out[1] (columns),
 * as log2 of the radix (choice_out may be NULL).  Costs about 4 reps products;
 * leaves the handle as bem_set_radix with the chosen values does.  Synchronises the
 * stream. */
bem_status bem_autotune(bem_kernel k, int32_t reps, int32_t* choice_out, void* cuda_stream);

/* u = K p for callers that cannot allocate device memory (no counterpart in the
 * paper; an integration aid).  Some callers may not call cudaMalloc at all: code
 * running under a host framework's memory pool that must not be bypassed, real-time
 * loops where an allocation could stall or fail, plug-ins handed buffers but no
 * allocation rights.  This entry point allocates nothing: it takes the operator
 * parameters (desc->precision must be BEM_FP32, N a power of two with
 * 4 <= N <= BEM_STATIC_MAX_N) and device arrays p and u (N*N floats, 16-byte
 * aligned, caller-owned), and keeps every intermediate (compliance tables, twiddles,
 * half spectrum) in one fixed device array of about 1.4 MB that each GPU loading the
 * library holds until the process exits.  Larger N or host arrays are rejected with
 * BEM_EINVAL.  The first call on a device looks up that array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call before
 * any stream capture.  Every call rewrites the parts of the array it reads, so no
 * clearing is needed, but all calls share the one array: calls that overlap on the
 * GPU (other streams, other threads) race and must be serialised by the caller.
 * Asynchronous on cuda_stream; results equal bem_matvec on a handle made from the
 * same desc. */
#define BEM_STATIC_MAX_N 256
bem_status bem_matvec_static(const bem_kernel_desc* desc, const float* p, float* u, void* cuda_stream);

/* Live per-pass timing (a measurement aid, not part of the method): while on, every
 * product records CUDA events on its stream around each of its three passes; the
 * durations are collected at the library's synchronisation points.
 * bem_pass_timing synchronises the device and returns, per pass (rows forward,
 * columns, rows inverse), the summed milliseconds and the number of timed launches;
 * reset != 0 zeroes the totals. */
bem_status bem_set_pass_timing(bem_kernel k, int32_t on);
bem_status bem_pass_timing(bem_kernel k, double* ms_total, int64_t* launches, int32_t reset);

/* ---- Learned warm start (no counterpart in the paper) --------------------------
 * A Fourier neural operator that predicts a dimensionless pressure field q = p/pbar
 * (pbar = F / L^2) from 7 per-cell features, used as the starting pressure of the
 * contact solve.  Layers: pointwise lift 7 -> width; `layers` blocks
 * z = S(v) + W v + b, v' = gelu(z) (no gelu after the last); projection
 * h = gelu(Q1 v + q1) (width -> hidden), out = Q2 h + q2 (hidden -> 1).  S keeps the
 * Fourier modes kx in {0..m-1, N-m..N-1}, ky in {0..m-1} (m = modes) of each channel,
 * mixes channels with a complex width x width matrix per mode and transforms back
 * (half-spectrum weights 1 for ky = 0, 2 otherwise, factor 1/N^2).  Weights are
 * float masters with a bfloat16 copy used by every kernel; all accumulation is
 * float.  Arrays are device arrays, channels-first: features [B][7][N][N],
 * outputs [B][N][N].  Parameter vector order: P [width][7], p [width],
 * R_re [layers][width][width][2m][m], R_im (same), W [layers][width][width],
 * b [layers][width], Q1 [hidden][width], q1 [hidden], Q2 [hidden], q2 [1].
 * width and hidden must be one of 1, 7, 8, 16, 32, 64; N even and N >= 2 modes. */
typedef struct {
  int32_t width, modes, layers, hidden;
} bem_fno_desc;
typedef struct bem_fno_s* bem_fno;
/* Creates a network on the current device with every parameter zero (load them
 * with bem_fno_set_params); the handle owns its parameter, optimiser and activation
 * buffers (activations grow with B and N on demand).  BEM_EINVAL for a NULL
 * argument, a width or hidden size outside the list above, modes < 1 or layers
 * outside [1, 16]; BEM_ENOMEM (or BEM_ECUDA) if an allocation fails; *out is NULL on
 * failure. */
bem_status bem_fno_create(const bem_fno_desc* desc, bem_fno* out);
/* Synchronises the device and frees everything the handle owns; NULL is a no-op. */
bem_status bem_fno_destroy(bem_fno f);
/* Length of the parameter vector (floats), -1 for a NULL handle. */
int64_t bem_fno_param_count(bem_fno f);
/* copy in float parameters (host or device); resets the optimiser state */
bem_status bem_fno_set_params(bem_fno f, const float* params, int64_t count, void* cuda_stream);
/* copy out the float masters (rounded = 0) or the bfloat16 values in use (rounded = 1) */
bem_status bem_fno_get_params(bem_fno f, float* params, int64_t count, int32_t rounded, void* cuda_stream);
/* Adam's state for checkpoints: the first and second moment vectors (count floats
 * each, host or device) and the number of steps taken.  Restore a checkpoint with
 * bem_fno_set_params (which clears the state) followed by bem_fno_set_state; the
 * next training step then equals the one the saved network would have taken.
 * BEM_EINVAL for a NULL argument, a wrong count or step < 0. */
bem_status bem_fno_get_state(bem_fno f, float* m1, float* m2, int64_t count, int32_t* step, void* cuda_stream);
bem_status bem_fno_set_state(bem_fno f, const float* m1, const float* m2, int64_t count, int32_t step,
                             void* cuda_stream);
/* features of B samples: heights [B][N][N]; params [B][4] doubles (h/delta, E1/E2, nu1,
 * nu2) -> x [B][7][N][N]: height standardised per sample, log(h/delta)/log 200,
 * log(E1/E2)/log 20, nu1, nu2, (column + 1/2)/N, (row + 1/2)/N.  B <= 4096. */
bem_status bem_fno_features(bem_fno f, int32_t B, int32_t N, const float* heights, const double* params, float* x,
                            void* cuda_stream);
/* out = network(x) for B samples (device arrays x [B][7][N][N], out [B][N][N]);
 * asynchronous on cuda_stream.  BEM_EINVAL for host arrays, B < 1, odd N or N < 2
 * modes (the transforms read pairs of floats, 8-byte aligned for even N only). */
bem_status bem_fno_forward(bem_fno f, int32_t B, int32_t N, const float* x, float* out, void* cuda_stream);
/* forward + backward of the loss mean((out - target)^2); writes the gradient (host or
 * device, may be NULL) and the loss; synchronises the stream.  N as for forward. */
bem_status bem_fno_gradients(bem_fno f, int32_t B, int32_t N, const float* x, const float* target, float* grad,
                             double* loss, void* cuda_stream);
/* one Adam step (beta 0.9/0.999, eps 1e-8) on the loss above */
bem_status bem_fno_train_step(bem_fno f, int32_t B, int32_t N, const float* x, const float* target, float lr,
                              double* loss, void* cuda_stream);
/* training target q = p / pbar[b] (pbar: B doubles, device) */
bem_status bem_fno_target(bem_fno f, int32_t B, int32_t N, const float* p, const double* pbar, float* q,
                          void* cuda_stream);
/* warm-start pressure p = pbar[b] * out where out > q_min, 0 elsewhere (pbar: B
 * doubles, device; q_min >= 0).  q_min = 0 keeps every cell the network puts in
 * contact; a larger cut keeps only its confident cells (q_min = 1: above the mean
 * pressure), which starts the solve from a sparser contact set. */
bem_status bem_fno_pressure(bem_fno f, int32_t B, int32_t N, const float* out, const double* pbar, float q_min,
                            float* p, void* cuda_stream);

/* Number of kernel launches the library has issued since it was loaded. */
int64_t bem_launch_count(void);

/* Message for the last failing call on this thread ("" if none). */
const char* bem_last_error(void);

/* ABI version (major * 100 + minor). */
int32_t bem_version(void);

#ifdef __cplusplus
}
#endif

#endif /* BEM_H */
