/*
 * pstd.h -- C ABI of the GB300 DTT-based PSTD library.
 *
 * The library time-steps the linear acoustic equations (Eq. wave_eq)
 *     du/dt = -(1/rho0) dp/dx,   dp/dt = -rho0 c0^2 du/dx
 * in a 1-, 2- or 3-D box whose walls are each Neumann (sound-hard) or
 * Dirichlet (sound-soft), with the sine/cosine pseudospectral scheme of
 * Wise, Jaros, Cox & Treeby (Section 4, Eq. dtt_pstd_solution and its n-D
 * form in Section 4.3):
 *     u_i^{n+1/2} = u_i^{n-1/2} - (dt/rho0)       T_{i,2}^{-1}{ a_{i,1} T_{i,1}{ p^n } }
 *     p^{n+1}     = p^n - dt rho0 c0^2 sum_i      T_{i,1}^{-1}{ a_{i,2} T_{i,2}{ u_i^{n+1/2} } }
 * with the transform pair (T1, T2) and k-space coefficients (a1, a2) of each
 * axis chosen from its wall pair by Table 2.
 *
 * Grid and memory layout (all fields FP32, C order, axis 0 slowest):
 *   - N_i cells of width dx_i per axis; walls at x = 0 and x = N_i dx_i.
 *   - Pressure p lives on the nodes x_j = j dx.  Nodes on a Dirichlet wall
 *     (where p = 0 identically) are not stored, so along axis i p has
 *     N_i+1 (NN), N_i (ND, DN) or N_i-1 (DD) entries, starting at node 0 for
 *     a Neumann left wall and at node 1 for a Dirichlet one.
 *   - Velocity u_i lives on the N_i half-nodes (m + 1/2) dx_i along axis i and
 *     on the stored pressure nodes along every other axis.
 *   - An axis whose right wall is at mid-cell (PSTD_NEUMANN_MID,
 *     PSTD_DIRICHLET_MID below) stores the pressure nodes up to N_i - 1 and
 *     N_i - 1 (Neumann) or N_i (Dirichlet) velocity half-nodes.
 *   pstd_field_shape() returns these shapes.
 *
 * Ownership: the caller allocates and owns every field buffer (device
 * memory, contiguous, FP32, 256-byte aligned as cudaMalloc / torch return it).
 * The plan owns its tables and its scratch accumulator and frees them in
 * pstd_free().
 *
 * Streams and errors: every call that touches device memory enqueues work on
 * the plan's stream and returns without synchronising.  Return value 0 is
 * success; negative values are the PSTD_E* codes below.  No C++ exception
 * crosses this interface.  A CUDA launch error is reported by the call that
 * launched; errors raised while the device runs surface at pstd_sync().
 * A plan is not thread-safe: do not call into one plan from two host
 * threads at once.
 */
#ifndef PSTD_H
#define PSTD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Wall type.  Table 2: Neumann <-> whole-sample symmetric pressure,
 * Dirichlet <-> whole-sample antisymmetric pressure.  PSTD_PERIODIC (both
 * walls of an axis) is Table 2's periodic row, the Fourier PSTD method of
 * Section 2 (Eq. fourier_pstd_solution): the axis stores the N nodes
 * j = 0..N-1 and its derivatives are i k e^{+-i k dx/2} with the DFT
 * wavenumbers of Section 2.
 * PSTD_NEUMANN_MID / PSTD_DIRICHLET_MID (right wall only, N >= 2): the wall
 * lies half a cell past the last node, at x = (N - 1/2) dx, so the axis
 * stores the nodes up to N - 1 and its symmetric-periodic extension has odd
 * period M = 2N - 1: groups III and IV of Table 1 (types V-VIII; pressure
 * WSHS / WSHA / WAHS / WAHA, velocity HAWA / HAWS / HSWA / HSWS).  The
 * velocity half-node on the wall is stored only next to a Dirichlet wall
 * (u is symmetric there), so u_axis has N - 1 (Neumann) or N entries along
 * its axis.  These axes run on the generic FFT route (3- and 5-smooth M),
 * the convolution route or the dense route; plans with a split form
 * (pstd_plan_opts.form 1, 2, 3) reject them with PSTD_EUNSUPPORTED. */
typedef enum {
    PSTD_NEUMANN = 0,
    PSTD_DIRICHLET = 1,
    PSTD_PERIODIC = 2,
    PSTD_NEUMANN_MID = 3,
    PSTD_DIRICHLET_MID = 4
} pstd_bc;

/* How pstd_init_velocity derives u^{-1/2} from the given u(0).
 * PSTD_U_HALFSTEP: u^{-1/2} = u0 + (dt / (2 rho0)) D_p p^0, so that the
 *   time-centred velocity equals u0 at t = 0 (the staggered-grid reading of
 *   "initial particle velocity set to zero" in Section 4.2).
 * PSTD_U_AS_GIVEN: u^{-1/2} = u0. */
typedef enum { PSTD_U_HALFSTEP = 0, PSTD_U_AS_GIVEN = 1 } pstd_uinit;

enum {
    PSTD_OK = 0,
    PSTD_EINVAL = -1,       /* bad descriptor, pointer, axis or field index */
    PSTD_EUNSTABLE = -2,    /* c0 dt |k|_max / 2 > 1: beyond the leapfrog limit */
    PSTD_ENOMEM = -3,       /* device or host allocation failed */
    PSTD_ECUDA = -4,        /* a CUDA runtime call failed (see pstd_last_cuda_error) */
    PSTD_ETIMEOUT = -5,     /* a bounded device-side wait gave up */
    PSTD_EUNSUPPORTED = -6  /* size with no transform schedule (see pstd_plan) */
};

/* Problem statement (Section 4.1 / 4.3; the time step dt = CFL dx / c0 of
 * Section 4.2 is given explicitly, see pstd_dt_from_cfl). */
typedef struct {
    int ndim;              /* 1, 2 or 3 */
    int64_t ncells[3];     /* N_i >= 1 cells per axis (M_i = 2 N_i) */
    double dx[3];          /* grid spacing per axis [m] */
    int bc[3][2];          /* pstd_bc of the [axis][left, right] walls */
    double c0;             /* sound speed [m/s] */
    double rho0;           /* density [kg/m^3] */
    double dt;             /* time step [s] */
    int uinit;             /* pstd_uinit */
} pstd_desc;

typedef struct pstd_plan_s pstd_plan_t;

/* Validate a descriptor and build a plan on the current CUDA device.
 * Builds the FP64 tables (twiddles, wavenumbers, folded k-space
 * coefficients -(dt/rho0) i k e^{+ik dx/2} / M and -(dt rho0 c0^2) i k
 * e^{-ik dx/2} / M of the symmetric-periodic extension of each axis, Table 1)
 * and rounds them once to FP32; allocates them and one scratch accumulator of
 * the pressure shape (ndim >= 2) on the device.  Routes per axis, by the
 * period M of its extension: the register-FFT passes for M in {2..1024
 * powers of two, 96, 192, 384, 768}; shared-memory Stockham FFT passes for
 * other M with prime factors 2, 3 and 5 only; for any other M, a dense
 * operator matrix when N_i <= 64, else a (skew-)circular convolution of
 * length M evaluated as a linear convolution through a circular FFT of
 * length M2 >= 2M - 1: of the 2^a 3^b 5^c lengths up to the next power of
 * two, the one with the least Stockham traffic (M2 x passes).  M2 is at most
 * 8192, i.e. M up to 4096; longer such axes return PSTD_EUNSUPPORTED.
 * `stream` is a cudaStream_t (NULL = legacy default stream).
 * Errors: PSTD_EINVAL (ndim, N_i, dx, c0, rho0, dt, bc or uinit out of
 * range; N_i = 1 with DD walls has no pressure node), PSTD_EUNSTABLE,
 * PSTD_EUNSUPPORTED, PSTD_ENOMEM, PSTD_ECUDA.  *out is NULL on error. */
int pstd_plan(const pstd_desc* desc, void* stream, pstd_plan_t** out);

/* Launch schedule of each axis pass, for tuning; -1 leaves a choice to the
 * plan.  variant 0 keeps many elements per lane and few FFT passes (for axes
 * with many lines), variant 1 spreads each FFT over up to 128 lanes (FFT
 * lengths 256, 512, 768, 1024), variant 2 (length 1024) uses 64 lanes of 16
 * elements, variant 3 (lengths 512, 1024) 128 / 256 lanes of 4 elements (the
 * default for those lengths on axes with too few lines to fill the GPU),
 * variant 4 (lengths 256, 512, 768) variant 1's FFT with its coefficient
 * and twiddle tables read from shared memory instead of registers (fewer
 * registers per thread, more resident CTAs; the default for length 768 on
 * axes with many lines), variant 5 (lengths 256, 512) the same with the
 * tables read from global memory through L1 (neither registers nor shared
 * memory hold them; the default for lengths 256 and 512 on axes with many
 * lines, the 3-D sizes); variants 3, 4 and 5 serve walled (non-periodic)
 * axes only and fix N = L / 2 at compile time.  An unavailable variant gives
 * PSTD_EINVAL.
 * seqs_per_cta: line pairs per CTA (a power of two). */
typedef struct {
    int variant[3];
    int seqs_per_cta[3];
    /* 0: spectral derivatives through FFTs of the symmetric extension (default);
     * 1: split-precision dense form -- each derivative as a GEMM with the
     *    FP64-built operator matrix, FP16 hi/lo split products on the tensor
     *    cores with FP32 accumulation (axes with N <= 1024); affects
     *    pstd_step / pstd_run only;
     * 2: tensor-core split form -- the same dense operators as GEMMs on the
     *    5th-generation tensor cores (tcgen05, kind::tf32): operator and field
     *    each split into TF32 hi + lo parts, Ah Bh + Ah Bl + Al Bh accumulated
     *    in FP32 in tensor memory (axes with N <= 1024); a bounded wait that
     *    gives up is reported by pstd_sync as PSTD_ETIMEOUT;
     * 3: BF16 split form on the 5th-generation tensor cores (tcgen05,
 *    kind::f16): the same dense operators, operator and field cut into three
 *    BF16 slices each on per-(row, 32-wide k block) and per-(line, block)
 *    power-of-two grids, so that each block's main product sums exactly in
 *    tensor memory; FP32 accumulation; operator slices fed by TMA (axes with
 *    N <= 1024); a bounded wait that gives up is reported by pstd_sync as
 *    PSTD_ETIMEOUT. */
    int form;
    /* 1: pstd_run is one cooperative kernel for all its steps, the CTAs
     * meeting at a bounded-wait grid barrier between axis passes (when every
     * axis runs the same register-FFT schedule; otherwise ignored).  A wait
     * that exceeds spin_limit polls (0: about a second) ends the kernel and
     * pstd_sync returns PSTD_ETIMEOUT. */
    int persistent;
    int64_t spin_limit;
    /* Testing aid: the barrier waits for this many arrivals beyond the CTAs
     * launched, so that it cannot complete and the bounded wait must give up
     * (exercises the PSTD_ETIMEOUT path without faulting the GPU). */
    int withhold_arrivals;
} pstd_plan_opts;

/* pstd_plan with explicit schedule options (NULL = all automatic).
 * Errors: those of pstd_plan; PSTD_EINVAL for an option the axis cannot use. */
int pstd_plan_ex(const pstd_desc* desc, void* stream, const pstd_plan_opts* opts,
                 pstd_plan_t** out);

/* pstd_plan_ex with the axis-pass schedules chosen by measurement on the
 * current device: for the FFT form (form 0, not persistent), each axis in
 * turn tries every register-FFT schedule (variant x line pairs per CTA, with
 * 32 to 256 threads per CTA) of its FFT length, timed with CUDA events on
 * `stream` around graph-replayed runs (96 minus 32 steps) on zero-filled
 * scratch fields the call allocates and frees; a candidate replaces the
 * current choice when it is at least 2% faster.  `base` (may be NULL) gives
 * the starting options; the winner is cached per (device, grid, walls, form)
 * for the life of the process, so a second call for the same shape returns at
 * once.  Other forms are built as by pstd_plan_ex.  times_us (may be NULL):
 * [0] the tuned step time, [1] the default schedule's, in microseconds (-1 if
 * not tuned).  The tuning is a property of the implementation; the paper has
 * no counterpart.  Errors: as pstd_plan_ex, PSTD_ENOMEM (scratch). */
int pstd_plan_autotune(const pstd_desc* desc, void* stream, const pstd_plan_opts* base, pstd_plan_t** out,
                       double times_us[2]);

/* The schedule a plan chose for `axis`: variant, lanes per sequence,
 * sequences per CTA, CTAs per launch (-1 for an axis on the generic
 * shared-memory FFT or dense path).  Errors: PSTD_EINVAL. */
int pstd_plan_schedule(const pstd_plan_t* plan, int axis, int out[4]);

/* Whether pstd_run of this plan is one cooperative kernel: out[0] = 1 / 0,
 * out[1] = CTAs, out[2] = threads per CTA.  Errors: PSTD_EINVAL. */
int pstd_plan_persistent(const pstd_plan_t* plan, int out[3]);

/* Shape of field 0 (p) or field i+1 (u_i) as three extents (unused axes 1).
 * Errors: PSTD_EINVAL. */
int pstd_field_shape(const pstd_plan_t* plan, int field, int64_t shape[3]);

/* Elements of field `field` (0 = p, i+1 = u_i); 0 on a bad index. */
int64_t pstd_field_numel(const pstd_plan_t* plan, int field);

/* Staggered spectral derivative along `axis` of one field, without time
 * stepping (Section 3.4, Tables A3 / A6):
 *   dir 0: out = T2^{-1}{ a1 T1{ in } }  (in: pressure-shaped, out: u_axis-shaped)
 *   dir 1: out = T1^{-1}{ a2 T2{ in } }  (in: u_axis-shaped,   out: pressure-shaped)
 * `in` and `out` are device pointers that must not overlap.
 * Errors: PSTD_EINVAL, PSTD_ECUDA. */
int pstd_grad(pstd_plan_t* plan, int axis, int dir, const float* in, float* out);

/* Derive u^{-1/2} in place from p^0 and the velocities already in u[0..ndim-1]
 * according to desc->uinit (PSTD_U_AS_GIVEN leaves u untouched).
 * Errors: PSTD_EINVAL, PSTD_ECUDA. */
int pstd_init_velocity(pstd_plan_t* plan, const float* p0, float* const* u);

/* One leapfrog step in place: (p^n, u^{n-1/2}) -> (p^{n+1}, u^{n+1/2}).
 * `u` is a host array of ndim device pointers.  Errors: PSTD_EINVAL, PSTD_ECUDA. */
int pstd_step(pstd_plan_t* plan, float* p, float* const* u);

/* `nsteps` >= 0 leapfrog steps in place.  The plan records one block of
 * steps in a CUDA graph per (p, u) pointer set on first use and replays it;
 * a tail shorter than the block is launched directly.
 * Errors: PSTD_EINVAL, PSTD_ECUDA. */
int pstd_run(pstd_plan_t* plan, float* p, float* const* u, int64_t nsteps);

/* Discrete energy of the leapfrog state in FP64, computed on the GPU:
 *     E^n = sum_j w_j (p_j^n)^2 / (2 rho0 c0^2)
 *         + (rho0 / 2) sum_i sum_j w_ij u_{i,j}^{n-1/2} u_{i,j}^{n+1/2},
 * the quantity the staggered leapfrog of Eq. (dtt_pstd_solution) conserves
 * (Section 4.1's scheme; a reading, the paper states no energy).  Weights are
 * tensor products over axes: 1/2 on a stored pressure node on a Neumann
 * wall, 1/2 on the velocity half-node a Dirichlet mid-cell wall passes
 * through, 1 elsewhere.  `p` holds p^n, `u_prev` / `u_next` host arrays of
 * ndim device pointers to u^{n-1/2} and u^{n+1/2} (physical velocity, as
 * pstd_step / pstd_run leave it; layout of pstd_field_shape).  Each product is
 * formed in FP64 and summed in FP64 in a fixed order.  Enqueued on the plan's
 * stream after its earlier work; waits for the result and writes it to the
 * host double *energy.  The plan allocates a small FP64 scratch on first use.
 * Errors: PSTD_EINVAL (NULL argument), PSTD_ENOMEM, PSTD_ECUDA. */
int pstd_energy(pstd_plan_t* plan, const float* p, float* const* u_prev, float* const* u_next, double* energy);

/* Synchronise the plan's stream; reports device-side errors, and
 * PSTD_ETIMEOUT once (then clears it) if a bounded wait of a persistent run
 * gave up.  Errors: PSTD_ECUDA, PSTD_ETIMEOUT. */
int pstd_sync(pstd_plan_t* plan);

/* Release the plan (synchronises its stream first).  NULL is a no-op. */
int pstd_free(pstd_plan_t* plan);

/* Static description of an error code. */
const char* pstd_strerror(int code);

/* Text of the last CUDA error seen by any call on this thread ("" if none). */
const char* pstd_last_cuda_error(void);

/* dt = CFL dx / c0 (Section 4.2). */
double pstd_dt_from_cfl(double cfl, double dx, double c0);

/* Number of kernels the last pstd_step / pstd_run / pstd_grad /
 * pstd_init_velocity / pstd_apply / pstd_init_prev / pstd_run2 call on this
 * plan launched (graph replays count their kernel nodes). */
int64_t pstd_last_launch_count(const pstd_plan_t* plan);

/* Library version string. */
const char* pstd_version(void);

/* ---- Plain differentiation and staggered interpolation (Section 3.3) ------- */
/* Field kinds along one axis of a plan: the grid (nodes x_j = j dx or
 * half-nodes (m + 1/2) dx) and the parity class at the walls.  Pressure-like
 * fields are symmetric about a Neumann wall and antisymmetric about a
 * Dirichlet wall, velocity-like fields the reverse; a node where a field is
 * antisymmetric about a wall is zero and not stored.  PSTD_NODES_P is the
 * layout of p and PSTD_HALF_U that of u_axis; PSTD_NODES_U holds e.g. dp/dx on
 * the nodes (N+1 minus one per Neumann wall entries) and PSTD_HALF_P e.g. p
 * interpolated to the half-nodes (N entries).  On a periodic axis every kind
 * has N entries. */
enum { PSTD_NODES_P = 0, PSTD_HALF_U = 1, PSTD_NODES_U = 2, PSTD_HALF_P = 3 };
/* PSTD_OP_DIFF: spectral derivative on the same grid (Tables A1, A4); the
 *   parity class swaps: NODES_P <-> NODES_U, HALF_U <-> HALF_P.
 * PSTD_OP_INTERP: spectral interpolation to the other grid, half a cell
 *   away (Tables A2, A5); the parity class stays: NODES_P <-> HALF_P,
 *   NODES_U <-> HALF_U.
 * (The staggered derivative of Tables A3 / A6 is pstd_grad.) */
enum { PSTD_OP_DIFF = 0, PSTD_OP_INTERP = 1 };

/* Shape of a field of `kind` along `axis` (the other axes as p).
 * Errors: PSTD_EINVAL (bad axis or kind, or a kind with no stored node). */
int pstd_apply_shape(const pstd_plan_t* plan, int axis, int kind, int64_t shape[3]);

/* out = op(in) along `axis`, for a field `in` of `kind` (device pointers,
 * layouts from pstd_apply_shape for `kind` and for the output kind above).
 * The multiplier on the symmetric-periodic extension is i k (differentiation)
 * or e^{+-i k dx/2} (interpolation), with only its real part kept at an even
 * period's Nyquist bin; in exact arithmetic this is the paper's DTT pair of
 * the field's symmetry with its drop / pad bookkeeping.  Tables are built in
 * FP64 on first use of (axis, op, kind) and kept by the plan.
 * Errors: PSTD_EINVAL, PSTD_ENOMEM, PSTD_ECUDA, PSTD_EUNSUPPORTED. */
int pstd_apply(pstd_plan_t* plan, int axis, int op, int kind, const float* in, float* out);

/* ---- Second-order pressure-only form ---------------------------------------- */
/* Writing the pressure update of Eq. (dtt_pstd_solution) (n-D form of
 * Section 4.3) at two consecutive steps and subtracting removes the velocity:
 *   p^{n+1} = 2 p^n - p^{n-1} + (c0 dt)^2 sum_i D_{u,i} D_{p,i} p^n,
 * with D_{p,i} = T_{i,2}^{-1} a_{i,1} T_{i,1} and D_{u,i} = T_{i,1}^{-1} a_{i,2}
 * T_{i,2} of Table 2.  It needs two pressure-shaped fields instead of ndim + 1
 * and equals the coupled leapfrog's pressure when p^{-1} is the pressure that
 * run had one step before p^0 (pstd_init_prev).  The composed operator is the
 * real multiplier -k^2 on each axis's symmetric-periodic extension, evaluated
 * on the same routes as the staggered derivatives; its tables are built in
 * FP64 on first use and kept by the plan.  Plans of any form accept these
 * calls (the split forms' dense operators are not used). */

/* p^{-1} of a run from p^0 with zero initial velocity, into `p_prev`
 * (pressure-shaped device buffers that must not overlap):
 *   desc->uinit == PSTD_U_AS_GIVEN (u^{-1/2} = 0):  p^{-1} = p^0
 *   desc->uinit == PSTD_U_HALFSTEP (Section 4.2's half-step start):
 *     p^{-1} = p^0 + (c0 dt)^2 / 2 sum_i D_{u,i} D_{p,i} p^0.
 * Errors: PSTD_EINVAL, PSTD_ENOMEM, PSTD_ECUDA. */
int pstd_init_prev(pstd_plan_t* plan, const float* p0, float* p_prev);

/* `nsteps` >= 0 steps of the second-order form in place: on entry p holds p^n
 * and p_prev p^{n-1}; on return p holds p^{n+nsteps} and p_prev
 * p^{n+nsteps-1} (pressure-shaped device buffers that must not overlap).
 * During the run the p_prev buffer carries q = p^n - p^{n-1} (converted on
 * entry and back on return): the recurrence becomes q += (c0 dt)^2 sum_i
 * D_{u,i} D_{p,i} p, p += q, which keeps FP32 rounding in the low modes from
 * being amplified by 1 / (omega dt) as the 2 p^n - p^{n-1} form would.  One
 * pass per axis and step, last axis first (the pass of axis 0 also updates
 * p); blocks of steps are graph-replayed per (p, p_prev) pair as in pstd_run.
 * Errors: PSTD_EINVAL, PSTD_ENOMEM, PSTD_ECUDA. */
int pstd_run2(pstd_plan_t* plan, float* p, float* p_prev, int64_t nsteps);

/* ---- Batched runs and reflection coefficients (Section 5) ------------------ */

typedef struct pstd_batch_s pstd_batch_t;

/* Plan `n` >= 1 independent simulations ("members"), member m described by
 * descs[m] (sizes and walls may differ).  Each member gets a plan on its own
 * stream; pstd_batch_run records one CUDA graph per block of steps in which
 * every member is a parallel branch of `stream` (NULL: no graph, direct
 * launches).  Errors: those of pstd_plan for any member. */
int pstd_batch_plan(const pstd_desc* descs, int n, void* stream, pstd_batch_t** out);

/* The plan of member i (for pstd_field_shape); owned by the batch. */
int pstd_batch_member(const pstd_batch_t* batch, int i, pstd_plan_t** plan);

/* pstd_init_velocity of every member.  p[m] is member m's pressure, and
 * u[3 m + a] its velocity along axis a (device pointers).  Errors: PSTD_EINVAL. */
int pstd_batch_init_velocity(pstd_batch_t* batch, float* const* p, float* const* u);

/* `nsteps` leapfrog steps of every member, in place (pointers as above).
 * Errors: PSTD_EINVAL, PSTD_ECUDA. */
int pstd_batch_run(pstd_batch_t* batch, float* const* p, float* const* u, int64_t nsteps);

/* out = sum_m w[m] p_m on the full node lattice x_j = j dx, j = 0..N_i per
 * axis (shape (N_0+1, ..., N_{d-1}+1), C order), the weighted sum of
 * Section 5.  All members must share ndim and ncells; a node a member does not
 * store (a Dirichlet wall) contributes zero.  Sums in FP64, stores FP32.
 * Valid as a reflection-coefficient field for t < 2 L / c0 (3 L / c0 when
 * both walls of every axis are non-reflecting).  Errors: PSTD_EINVAL, PSTD_ECUDA. */
int pstd_batch_combine(pstd_batch_t* batch, const double* w, float* const* p, float* out);

/* Release the batch and its member plans (synchronises first). */
int pstd_batch_free(pstd_batch_t* batch);

/* Kernels launched by the last batch call (graph replays count their nodes). */
int64_t pstd_batch_last_launch_count(const pstd_batch_t* batch);

/* Run every later pstd_batch_run (enable != 0) as ONE cooperative kernel over
 * all members (Section 5's independent runs computed together): each step's
 * axis passes, last axis first, are split into work items (line groups or
 * tiles) over all members, which the resident CTAs take in turn, meeting at a
 * software grid barrier between passes.  When every axis of every member has
 * the same register-FFT schedule (e.g. the 4^d wall combinations of one
 * grid) the kernel runs those passes, with each member's velocity conversion
 * before and after it; otherwise every axis runs the generic shared-memory
 * program (its own FFT, convolution or dense route).  Each barrier wait is
 * bounded by spin_limit polls (0: a default of about a second); on giving up
 * the kernel ends and pstd_batch_sync reports PSTD_ETIMEOUT.
 * withhold_arrivals > 0 makes every barrier wait for that many arrivals that
 * never come (to test the bounded wait).  Results equal the graph path's bit
 * for bit on the register-FFT kernel and on members whose axes all take the
 * generic program there too; a register-FFT axis run by the generic program
 * agrees to rounding.  Errors: PSTD_EINVAL; PSTD_EUNSUPPORTED for a
 * dense-operator form (pstd_plan_opts.form != 0 is not set by pstd_batch_plan,
 * so this does not arise for its members). */
int pstd_batch_set_persistent(pstd_batch_t* batch, int enable, long long spin_limit, int withhold_arrivals);

/* The cooperative kernel pstd_batch_set_persistent would use: 1 register-FFT
 * passes, 2 the generic program.  Errors: PSTD_EINVAL. */
int pstd_batch_persistent_kind(const pstd_batch_t* batch);

/* Wait for the batch's stream.  PSTD_ETIMEOUT (reported once) if a barrier
 * wait of the last cooperative run gave up.  Errors: PSTD_ECUDA. */
int pstd_batch_sync(pstd_batch_t* batch);

/* Section 5 on the host: for per-axis reflection coefficients
 * refl[2 i] = R_L, refl[2 i + 1] = R_R, write the 4^ndim wall combinations as
 * copies of *tmpl with bc replaced (axis 0 slowest; per axis in the order
 * NN, ND, DN, DD) into descs[], and their weights, the product over axes of
 * w = (1/4) M^T r with r = [R_L, 1, R_R, R_L R_R] and M the image-source
 * polarity matrix, into w[].  Errors: PSTD_EINVAL. */
int pstd_reflection_combos(const pstd_desc* tmpl, const double* refl, pstd_desc* descs, double* w);

/* Capacity of pstd_step_noalloc: pressure points, and FFT length 2 N_i per axis. */
#define PSTD_NOALLOC_MAX_POINTS (1 << 22)
#define PSTD_NOALLOC_MAX_FFT 4096

/* `nsteps` >= 0 leapfrog steps in place, like pstd_plan + pstd_run + pstd_free,
 * but without allocating anything: no cudaMalloc, cudaFree or allocating
 * library call, host or device.  The paper has no counterpart; this exists for
 * callers that must not allocate device memory when they call us -- a host
 * application whose device memory belongs to a memory manager (a framework's
 * caching allocator, or a budget fixed at start-up) that forbids allocations
 * it does not make, or a latency-critical loop that cannot pay for cudaMalloc
 * and cudaFree, which may synchronise the device.
 * The caller passes the descriptor, p and the ndim velocity fields (device
 * pointers, the layout of pstd_field_shape) and a cudaStream_t (NULL = legacy
 * default stream).  The scratch accumulator and the coefficient tables live in
 * fixed file-scope device arrays (16 MiB + 384 KiB, held on every GPU that
 * loads the library until the process exits); each call recomputes the tables
 * in FP64 on the device, and looks the arrays' device addresses up on the
 * current device (a host-side query).  Under CUDA's lazy module loading the
 * arrays are committed when the first call on a device loads the module: that
 * first call is the one that takes device memory, so make it once at start-up
 * (and before any stream capture); later calls take none.  All calls share
 * the arrays: calls whose work overlaps on the GPU race, so serialise them
 * (one stream, one host thread).
 * Only Neumann and Dirichlet walls at the grid nodes are supported (periodic
 * axes and mid-cell walls return PSTD_EUNSUPPORTED), on axes whose 2 N_i
 * factors into 2, 3 and 5, with 2 N_i <= PSTD_NOALLOC_MAX_FFT and at most
 * PSTD_NOALLOC_MAX_POINTS pressure points; larger or other sizes return
 * PSTD_EUNSUPPORTED before any device work.  u^{-1/2} must already be in u
 * (see pstd_init_velocity).
 * Errors: PSTD_EINVAL, PSTD_EUNSTABLE, PSTD_EUNSUPPORTED, PSTD_ECUDA. */
int pstd_step_noalloc(const pstd_desc* desc, float* p, float* const* u, int64_t nsteps,
                      void* stream);

/* ---- Learned spectral operator (not in the paper) ------------------------- */
/* Kernels of a spectral neural operator that maps an initial pressure on a
 * box to the pressure a fixed number of leapfrog steps later.  Its spectral
 * layers work in the truncated T1 basis of each axis (Table 2), so they keep
 * the walls.  Every call below enqueues on `stream` (a cudaStream_t, NULL =
 * legacy default stream), takes device pointers to FP32 buffers the caller
 * owns, and returns PSTD_OK, PSTD_EINVAL (bad pointer or size; nothing is
 * launched) or PSTD_ECUDA (launch failed). */

/* C[b] = alpha A[b] B[b] + beta C[b] for b < batch, A[b] M x K, B[b] K x N,
 * element (m, k) of A[b] at A + b sAb + m sAm + k sAk (strides in elements,
 * non-negative, any layout; B and C alike).  beta == 0 ignores C's old
 * contents.  A second batch level (batch2 > 1; 0 or 1 = none) adds
 * b2 sAb2 / sBb2 / sCb2 for b2 < batch2, and its last index uses K_last
 * (0 <= K_last <= K) instead of K: a split of a long reduction into batch2
 * chunks whose partial products the caller sums.  batch * batch2 <= 65535,
 * ceil(M / 256) <= 65535; A and B may be NULL when K == 0. */
typedef struct {
    int64_t batch;
    int M, N, K;
    const float* A;
    int64_t sAb, sAm, sAk;
    const float* B;
    int64_t sBb, sBk, sBn;
    float* C;
    int64_t sCb, sCm, sCn;
    float alpha, beta;
    int64_t batch2;
    int64_t sAb2, sBb2, sCb2;
    int K_last;
} pstd_gemm_desc;
int pstd_nn_gemm(const pstd_gemm_desc* d, void* stream);

/* pstd_nn_gemm on the tensor cores (tcgen05, kind::tf32): A and B are rounded
 * to TF32 (10-bit mantissa, round to nearest) as they are staged, products
 * accumulate in FP32 in tensor memory.  Same descriptor and limits as
 * pstd_nn_gemm except ceil(M / 128) <= 65535.  `status` (device int, may be
 * NULL) is set to 1 if a bounded wait for the tensor cores gave up; that
 * tile is then left unwritten.  Errors: PSTD_EINVAL, PSTD_ECUDA. */
int pstd_nn_gemm_tf32(const pstd_gemm_desc* d, int* status, void* stream);

/* Tensors below are [B][C][P] (B samples, C channels, P points) or [B][P];
 * bias_act, lift and proj_bwd need B C <= 65535, proj B <= 65535.
 * y = act(x + bias[c]) with act 0 = identity, 1 = relu; bias may be NULL. */
int pstd_nn_bias_act(const float* x, const float* bias, float* y, int64_t B, int C, int64_t P, int act,
                     void* stream);
/* dx = dy where act is identity or pre > 0, else 0 (n elements; dx may alias dy). */
int pstd_nn_act_bwd(const float* dy, const float* pre, float* dx, int64_t n, int act, void* stream);
/* v[b][c][i] = w[c] p[b][i] + bias[c]  (lifting 1 -> C channels). */
int pstd_nn_lift(const float* p, const float* w, const float* bias, float* v, int64_t B, int C, int64_t P,
                 void* stream);
/* out[b][i] = sum_c w[c] v[b][c][i] + bias[0]  (projection C -> 1). */
int pstd_nn_proj(const float* v, const float* w, const float* bias, float* out, int64_t B, int C, int64_t P,
                 void* stream);
/* dv[b][c][i] = w[c] dout[b][i]  (adjoint of the projection). */
int pstd_nn_proj_bwd(const float* dout, const float* w, float* dv, int64_t B, int C, int64_t P, void* stream);
/* g[c] = sum_{b,i} x[b][c][i] y[.]: y indexed [b][c][i] when y_has_channels,
 * [b][i] otherwise, and taken as 1 when NULL.  Sums in FP64. */
int pstd_nn_chan_dot(const float* x, const float* y, int y_has_channels, float* g, int64_t B, int C, int64_t P,
                     void* stream);
/* out[j] = sum_b x[b][j], j < n, summed in FP64. */
int pstd_nn_sum_lead(const float* x, float* out, int64_t B, int64_t n, void* stream);
/* Adam with bias correction (Kingma & Ba 2015) on n parameters, step >= 1. */
int pstd_nn_adam(float* w, const float* g, float* m, float* v, int64_t n, float lr, float beta1, float beta2,
                 float eps, int64_t step, void* stream);
/* loss[0] = mean (out - target)^2 over n values; dout = (2/n)(out - target)
 * unless dout is NULL. */
int pstd_nn_mse(const float* out, const float* target, float* dout, float* loss, int64_t n, void* stream);
/* err[b] = ||a_b - ref_b||_2 / ||ref_b||_2 per sample of P values (FP64 sums;
 * the plain norm of the difference where ref_b is zero). */
int pstd_nn_rel_err(const float* a, const float* ref, float* err, int64_t B, int64_t P, void* stream);
/* rms[b] = sqrt(mean_i x[b][i]^2) over P values per sample (FP64 sum). */
int pstd_nn_row_rms(const float* x, float* rms, int64_t B, int64_t P, void* stream);
/* y[b][i] = x[b][i] / s[b] (mode 0; 0 where s[b] == 0) or x[b][i] s[b]
 * (mode 1); y may alias x.  B <= 65535. */
int pstd_nn_row_scale(const float* x, const float* s, float* y, int64_t B, int64_t P, int mode, void* stream);
/* dst = src rounded to the nearest bfloat16, ties to even, stored as FP32. */
int pstd_nn_round_bf16(const float* src, float* dst, int64_t n, void* stream);

/* Host only.  The first K modes of the T1 transform of an axis of `ncells`
 * cells with walls (bc_left, bc_right) in {PSTD_NEUMANN, PSTD_DIRICHLET}, on
 * its lp stored pressure nodes (lp = N+1, N, N, N-1 for NN, ND, DN, DD):
 * T (K x lp, row-major) the unnormalised forward transform's first K rows and
 * I (lp x K) the first K columns of its inverse (Eq. inverse_transforms).
 * Host buffers owned by the caller.  Errors: PSTD_EINVAL (K > lp, bad wall). */
int pstd_sno_basis(int ncells, int bc_left, int bc_right, int K, float* T, float* I);

#ifdef __cplusplus
}
#endif

#endif /* PSTD_H */
