/*
 * mpdata.h -- C ABI of the GB300 MPDATA step library.
 *
 * One MPDATA time step for the generalised transport equation
 *     d_t(G psi) + div(G u psi) = G R                         (paper Sect. 1, Eq. 1)
 * solved in the homogeneous form d_t psi + (1/G) div(G u psi) = 0 (Sect. 3.1, Eq. 3)
 * with the source term applied by the euler_a / euler_b schemes of Sect. 4.1, on a
 * periodic Arakawa-C grid (Sect. 2.3): psi and G at cell centres, the advector
 * GC = G u dt/dx (Sect. 3.1.1, text after Eq. 5) on cell faces.  A step is a
 * donor-cell pass (Eqs. 4-5) followed by n_iters-1 corrective passes with the
 * antidiffusive advector (Eq. 6), optionally with the third-order terms
 * (Sect. 3.1.2), the infinite-gauge variant (Sect. 3.1.5) and the
 * non-oscillatory (FCT) limiter (Sect. 3.1.4).  Everything runs in hand-written
 * CUDA kernels for sm_103a; there is no CPU fallback.
 *
 * Layout (Sect. 3.2.5): row-major, last dimension fastest.  A field of shape
 * (n_0, ..., n_{D-1}) holds N = prod n_d values.  Advector component d is a
 * separate array of N values; its element i sits on the face between cell i and
 * cell i + e_d, wrapping periodically (so each dimension has n_d faces, not the
 * n_d - 1 of the paper's open boundaries).  Batched handles (n_fields > 1) hold
 * fields of possibly different shapes; every per-field array is the
 * concatenation of the fields in order, field f starting at the sum of the cell
 * counts of fields 0..f-1.
 *
 * Ownership: every pointer argument that names a field is a DEVICE pointer
 * (cudaMalloc'd or a tensor's storage on the handle's device), owned by the
 * caller, never freed or retained by the library.  FP32 handles take float
 * arrays, FP64 handles double arrays, aligned to their element size (16 bytes
 * for the vectorised 2D path; misaligned pointers give MPDATA_EINVAL).  The
 * handle owns only its device scratch.  Host pointers are marked "host".
 *
 * Errors: every call returns MPDATA_OK or an MPDATA_E* code; no call aborts the
 * process or throws (the C analogue of the library's std::runtime_error,
 * Sect. 2.4).  All device work is enqueued on the handle's stream and is
 * asynchronous; a device-side failure is reported by the next call on the
 * handle that synchronises (mpdata_reduce, mpdata_sync).  No kernel of this
 * library waits on another block of its grid (block barriers only); the reverse
 * step's kernels, launched as programmatic dependents, wait only for the
 * completion of the kernel before them on the stream.  No call can hang on a
 * device-side wait.
 */
#ifndef MPDATA_GB300_H
#define MPDATA_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mpdata_s* mpdata_t;

/* element types */
enum { MPDATA_F32 = 0, MPDATA_F64 = 1 };

/* option bits (Sect. 3.1.2-3.1.5, 4.1; compile-time opts of the paper become run-time bits) */
enum {
  MPDATA_FCT = 1u,          /* non-oscillatory limiter (Sect. 3.1.4) */
  MPDATA_TOT = 2u,          /* third-order terms (Sect. 3.1.2) */
  MPDATA_IGA = 4u,          /* infinite gauge (Sect. 3.1.5); requires n_iters == 2 */
  MPDATA_NUG = 8u,          /* non-unit G: a G field is passed to every step */
  MPDATA_KAHAN = 16u,       /* compensated summation in the donor-cell passes (Sect. 3.1.1) */
  MPDATA_RHS_EULER_A = 32u, /* psi^{n+1} = ADV(psi^n) + dt R (Sect. 4.1) */
  MPDATA_RHS_EULER_B = 64u, /* psi^{n+1} = ADV(psi^n + dt R) (Sect. 4.1) */
  MPDATA_STAGED = 128u,     /* run the one-kernel-per-sub-step path even where a fused
                               kernel covers the case (comparison and testing) */
  MPDATA_ABS = 256u,        /* variable-sign fields: |psi| in every psi-fraction of the
                               pseudo-velocity (Sect. 3.1.5); excludes MPDATA_IGA.  Runs on
                               the one-kernel-per-sub-step path; no reverse step */
  MPDATA_DFL = 512u,        /* divergent flow (Sect. 3.1.3): the pseudo-velocity gains
                               -1/4 V (div_i + div_{i+e_d}) / Gb, div_j the advector's
                               difference summed over the dimensions across cell j; excludes
                               MPDATA_IGA.  One-kernel-per-sub-step path; no reverse step */
  /* Open edges (Sect. 2.4, bcond::open: a zero-divergence condition on the domain edges)
     along dimension d, bit MPDATA_OPEN0 << d; both ends of that dimension, the others stay
     periodic.  The halo cells beyond an open edge hold the edge cell's value; the n-1 faces
     between cells are interior (advector entries 0 .. n-2 along d, the paper's advector being
     one shorter than the field along its own dimension, Sect. 3.2.5: entry n-1 is not read),
     and each of the two boundary faces carries, for the advector and every pass's
     pseudo-velocity, the value of the adjacent interior face.  An open dimension needs n >= 2.
     One-kernel-per-sub-step path; no reverse step (MPDATA_EUNSUPPORTED) */
  MPDATA_OPEN0 = 1024u,
  MPDATA_OPEN1 = 2048u,
  MPDATA_OPEN2 = 4096u,
  /* Trapezoidal (Crank-Nicolson) source scheme (Sect. 4.1):
     psi^{n+1} = ADV(psi^n + dt/2 R^n) + dt/2 R^{n+1}, for a system whose equations are the
     handle's fields (all of one shape) with sources affine in the state,
     R_e = sum_f A_ef psi_f + b_e (mpdata_set_rhs_linear).  R^{n+1} depends on psi^{n+1}, so
     each cell solves (I - dt/2 A) psi^{n+1} = ADV(psi^n + dt/2 R^n) + dt/2 b.  Excludes the two
     Euler bits; mpdata_step / mpdata_advance then take r = NULL and use dt */
  MPDATA_RHS_TRAPEZ = 65536u,
  /* Shallow-water system with prognosed velocity (Sect. 5): the handle's ndims + 1 fields (one
     shape, G = 1) are the depth h and the momenta q_d = u_d h; advanced by mpdata_sw_advance */
  MPDATA_SW = 131072u
};

/* status codes */
enum {
  MPDATA_OK = 0,
  MPDATA_EINVAL = 1,       /* invalid argument */
  MPDATA_EUNSUPPORTED = 2, /* valid but not supported by this build */
  MPDATA_ECUDA = 3,        /* a CUDA runtime call failed */
  MPDATA_ECOURANT = 4,     /* Courant check failed (sum of outflow advectors / G > 1) */
  MPDATA_ETIMEOUT = 5,     /* reserved for bounded device waits (no kernel of this build waits) */
  MPDATA_ESTOPPED = 6,     /* stopped after a step by mpdata_request_stop */
  MPDATA_ENOMEM = 7        /* device or host allocation failed */
};

/*
 * Creates a handle for n_fields independent fields of ndims dimensions.
 * shapes (host): n_fields * ndims int64 extents, field after field.
 * dtype: MPDATA_F32 or MPDATA_F64.  n_iters >= 1 passes per step (Sect. 3.1.1).
 * opts: OR of MPDATA_* option bits.  cuda_stream: a cudaStream_t (NULL = legacy
 * default stream) on the current device; all work of the handle goes there.
 * Errors: EINVAL for ndims not in 1..3, n_fields < 1, a non-positive extent,
 * n_iters < 1, IGA with n_iters != 2, IGA with ABS or DFL, both RHS bits; ENOMEM; ECUDA.
 */
int mpdata_create(mpdata_t* out, int ndims, int n_fields, const int64_t* shapes, int dtype,
                  int n_iters, uint32_t opts, void* cuda_stream);

/*
 * Sources of the MPDATA_RHS_TRAPEZ scheme (Sect. 4.1): R_e = sum_f A[e * n_fields + f] psi_f + b_e
 * for e, f = 0 .. n_fields - 1, the handle's fields being the system's equations (all of one
 * shape, at most 8).  A (host, n_fields^2 doubles, row-major) is copied; b (device, the
 * handle's total element count in its dtype, field after field, or NULL for b = 0) is kept by
 * pointer and read at every step, so the caller keeps it alive and may change its contents
 * between calls.  The translating oscillator of Sect. 4.2 is A = {0, omega, -omega, 0},
 * b = NULL.  Errors: EINVAL for a handle without MPDATA_RHS_TRAPEZ, fields of different
 * shapes, more than 8 fields, a null A, a misaligned b.  A step whose I - dt/2 A is
 * singular returns EINVAL.
 */
int mpdata_set_rhs_linear(mpdata_t h, const double* A, const void* b);

/*
 * Shallow-water system with prognosed velocity (Sect. 5, the drop of Sect. 5.3-5.4): advances
 * state = [h, q_0, .., q_{ndims-1}] (device, n cells each, the handle's field order) in place by
 * n_steps steps of
 *   h_t + div(u h) = 0,   (q_d)_t + div(u q_d) = -h dh/dx_d   (dimensionless, g = 1),
 * each step: the advector at n+1/2 from the velocities u_d = q_d / h (0 where h <= eps) at n and
 * n-1, extrapolated linearly (1.5 u^n - 0.5 u^{n-1}; u^{n-1} = u^n at the first step after
 * creation or mpdata_sw_reset) and interpolated to the cell walls, times dt/dx; then the
 * trapezoidal scheme (Sect. 4.1) for the momentum sources, centred differences of h, its second
 * half explicit because h has no source; the MPDATA step of each field with the handle's
 * options (FCT, ABS, DFL, IGA, OPEN...).  The handle keeps u^{n-1} between calls (allocated on
 * first use: ENOMEM).  Requires a handle created with MPDATA_SW, n_fields = ndims + 1 of one
 * shape, without NUG and the source bits (EINVAL otherwise, or for dt, dx <= 0).
 */
int mpdata_sw_advance(mpdata_t h, void* state, double dt, double dx, double eps, int n_steps);
/* Forgets u^{n-1}: the next mpdata_sw_advance step starts a run. */
int mpdata_sw_reset(mpdata_t h);

/*
 * Advances psi in place by n_steps >= 1 steps (the paper's advance(), Sect. 3.2.5).
 * 2D steps with n_iters = 2 run fused kernels (one launch per step), 1D fields of up
 * to 2235 (FP64) / 4470 (FP32) cells run the whole call in one launch, the rest run
 * one kernel per sub-step.
 * gc (host array of ndims device pointers): advector components, constant over
 * the call.  g: G field (required iff MPDATA_NUG, else NULL).  r: source term R
 * (required iff an RHS bit is set, else NULL), dt its time step.
 * Errors: EINVAL (null or misaligned pointers, n_steps < 1), ESTOPPED when a stop
 * was requested (the steps already enqueued complete), ECUDA.
 */
int mpdata_step(mpdata_t h, void* psi, const void* const* gc, const void* g, const void* r,
                double dt, int n_steps);

/*
 * Out-of-place variant: reads psi_in, writes psi_out (distinct buffers, or the
 * same buffer for in-place).  gc_scale (host, nullable): n_steps factors; step s
 * uses the advector gc * gc_scale[s] (a time-dependent flow evaluated at the
 * half step, Sect. 3.1.1 text after Eq. 5).  Errors as mpdata_step.
 */
int mpdata_advance(mpdata_t h, const void* psi_in, void* psi_out, const void* const* gc,
                   const void* g, const void* r, double dt, int n_steps, const double* gc_scale);

/*
 * mpdata_advance on a compensated FP32 state.  The paper computes in one precision
 * throughout; this entry point has no counterpart there.  It keeps each cell's value as
 * the pair psi = hi + lo of FP32 numbers (hi in psi_in / psi_out, the small remainder lo
 * in lo_in / lo_out, same layout).  Every quantity of the step (donor-cell fluxes,
 * pseudo-advectors of Eq. 6, FCT bounds and factors) is computed in FP32 from hi, as by
 * mpdata_advance; both donor-cell passes (Eq. 4) add their flux divergence to hi with an
 * error-free two-sum whose rounding error goes to lo (the rounding at the scale of psi, the
 * one that accumulates over long runs), the first pass also moves the low parts with their own
 * donor-cell fluxes, and the pair is renormalised.  sum(hi + lo) is conserved up to the
 * rounding of the flux divergences and of the lo additions (relative drift 3.6e-13 over the
 * 6434 steps of one revolution of the 1024^2 rotation), and the state carries about twice the
 * FP32 precision across steps.  Start from lo = 0 for an FP32 initial field (or
 * lo = x - (float)x for an FP64 one).
 * Requirements: an FP32 handle with one 2D field, n_iters = 2, without MPDATA_TOT,
 * MPDATA_ABS, MPDATA_DFL or MPDATA_STAGED (MPDATA_EUNSUPPORTED otherwise); lo_in / lo_out aliased exactly when
 * psi_in / psi_out are (EINVAL otherwise).  The warp-march kernel runs it (the handle's
 * MPDATA_TUNE_TILE_ROWS applies unless MPDATA_TUNE_KERNEL selects the band march).  The
 * first call allocates a second ping-pong buffer (ENOMEM).  Other errors as mpdata_advance.
 */
int mpdata_advance_compensated(mpdata_t h, const void* psi_in, const void* lo_in, void* psi_out,
                               void* lo_out, const void* const* gc, const void* g, const void* r,
                               double dt, int n_steps, const double* gc_scale);

/*
 * Reverse of ONE step from state psi_n (the derivative of the donor-cell passes,
 * Eqs. 4-5, the antidiffusive advector, Eq. 6 with its multi-D cross terms, the
 * third-order terms of Sect. 3.1.2, the divergent-flow term of Sect. 3.1.3 and |psi| in
 * its psi-fractions, Sect. 3.1.5, and the FCT limiter, Sect. 3.1.4): on entry
 * psi_bar = dL/dpsi^{n+1}, on exit
 * dL/dpsi^n (in place).  gc_bar (host array of ndims device pointers, or NULL):
 * dL/dgc_d is ADDED to gc_bar[d].  Branches (signs, FCT min/max) follow the
 * forward step's choices; [x]+ and [x]- have derivative 1/2 at 0 (|x| 0 at 0); a min/max
 * passes the derivative of its first extremal candidate.  The step is
 * recomputed internally, as mpdata_adjoint_record records it; the adjoint scratch
 * is allocated on first use and kept with the handle.  Errors: EINVAL;
 * EUNSUPPORTED for batched handles, for source terms, open edges, for n_iters > 4 and for 2D
 * fields of 2^31 cells or more; ENOMEM; ECUDA.
 */
int mpdata_adjoint_step(mpdata_t h, const void* psi_n, const void* const* gc, const void* g,
                        void* psi_bar, void* const* gc_bar);

/*
 * mpdata_adjoint_step for a handle with an Euler source term (MPDATA_RHS_EULER_A or _B, Sect.
 * 4.1: psi^{n+1} = ADV(psi^n) + dt R, or ADV(psi^n + dt R)), given the forward step's source r
 * (device, N elements of the handle's dtype, read-only) and dt.  R is an input of the step, not
 * a function of psi, so the reverse passes psi_bar through the source's addition unchanged;
 * under euler_b the step is reversed about psi^n + dt R.  r_bar (device, N elements, or NULL):
 * dL/dR is ADDED to it, dt dL/dpsi^{n+1} (euler_a) or dt dL/dpsi^n (euler_b).  Other arguments
 * and errors as mpdata_adjoint_step; EINVAL also for a NULL r or a misaligned r_bar;
 * EUNSUPPORTED for a handle without either source bit.  (mpdata_adjoint_step,
 * mpdata_adjoint_record and mpdata_adjoint_replay, which take no source, return EUNSUPPORTED
 * for such handles.)
 */
int mpdata_adjoint_step_rhs(mpdata_t h, const void* psi_n, const void* const* gc, const void* g, const void* r,
                            double dt, void* psi_bar, void* const* gc_bar, void* r_bar);

/*
 * mpdata_adjoint_step split in two, so that a caller holding the forward states of several
 * steps (a checkpointed rollout) records each step's tape while it recomputes the states and
 * then runs only the reverse sweeps:
 *
 * mpdata_adjoint_tape_bytes: *bytes = size of one step's tape (device memory the caller
 *   allocates; element-aligned, 16-byte aligned for vector stores; its layout is private to
 *   the library).  It holds psi^(1..K-1) of the donor-cell passes (Eqs. 4-5), the
 *   pseudo-advectors of Eq. 6 and, with MPDATA_FCT, the limited advectors, the bounds and the
 *   factors of Sect. 3.1.4: (K-1)(1+d) arrays of N elements, plus d(K-1) + 2 + 2(K-1) with
 *   FCT (K = n_iters, d = ndims, N = cells).
 * mpdata_adjoint_record: the forward step from psi_n, writing its tape into `tape` and, when
 *   psi_next is not NULL, psi^{n+1} into psi_next (which must not be psi_n).  2D steps with
 *   n_iters = 2 (FP32 and FP64; without Kahan summation, G, infinite gauge, the third-order,
 *   |psi| or divergent-flow terms) and psi_next run the fused step kernel of mpdata_advance
 *   that also writes the tape (one launch); the rest run the staged kernels.  The tape refers to psi_n and gc, which must hold the same values at
 *   replay.
 * mpdata_adjoint_replay: the reverse sweep of the step recorded in `tape`, with the arguments
 *   and result of mpdata_adjoint_step (psi_bar in place, gc_bar accumulated).  Record + replay
 *   gives the result of mpdata_adjoint_step up to the order of the atomic additions of
 *   its scatter kernels.
 * Errors as mpdata_adjoint_step; EINVAL also for a NULL or misaligned tape.
 */
int mpdata_adjoint_tape_bytes(mpdata_t h, size_t* bytes);
int mpdata_adjoint_record(mpdata_t h, const void* psi_n, const void* const* gc, const void* g,
                          void* tape, void* psi_next);
int mpdata_adjoint_replay(mpdata_t h, const void* psi_n, const void* const* gc, const void* g,
                          const void* tape, void* psi_bar, void* const* gc_bar);

/*
 * FP64 reductions over each field (host outputs, n_fields entries each):
 * mass_out[f] = sum G psi (G = 1 when g is NULL).  Synchronises the stream.
 */
int mpdata_reduce(mpdata_t h, const void* psi, const void* g, double* mass_out);

/*
 * FP64 difference norms per field (host outputs, nullable): l2sq_out[f] =
 * sum (a - b)^2, linf_out[f] = max |a - b|.  Synchronises the stream.
 */
int mpdata_diff_norms(mpdata_t h, const void* a, const void* b, double* l2sq_out, double* linf_out);

/*
 * Courant check (Sect. 3.1.1 stability of the donor-cell pass): returns
 * MPDATA_ECOURANT if at some cell sum_d ([gc_d(i)]+ - [gc_d(i - e_d)]-) / G_i > 1,
 * writing that maximum to *max_out (host, nullable).  Synchronises the stream.
 */
int mpdata_check_courant(mpdata_t h, const void* const* gc, const void* g, double* max_out);

/*
 * Asks the handle to stop: later mpdata_step / mpdata_advance calls return
 * MPDATA_ESTOPPED without enqueuing work, and a multi-step call stops after the
 * step in progress (the paper's panic flag, Sect. 3.2.5).  A 1D field small
 * enough for shared memory runs every step of a call in one launch; for it the
 * request takes effect at the next call.  Thread-safe.  mpdata_clear_stop
 * re-arms the handle.
 */
int mpdata_request_stop(mpdata_t h);
int mpdata_clear_stop(mpdata_t h);

/*
 * Tuning knobs of the handle's kernels (set by the autotuner; no counterpart in
 * the paper, whose tiling is the thread decomposition over dimension 0).
 * MPDATA_TUNE_TILE_ROWS: rows of one tile of the fused 2D kernels: the rows each
 *   warp walks down (warp march) or the rows of one block's band (band march);
 *   0 = automatic, otherwise 4..65536.
 * MPDATA_TUNE_KERNEL: fused 2D kernel family for single-field 2D steps:
 *   0 = automatic (band march where the warp march cannot fill the GPU: FP32
 *   fields with fewer than ~600 warp tiles of 8 rows, FP64 fields whose warp
 *   tiles would be 16 rows or less; warp march otherwise), 1 = warp march,
 *   2 = band march, 3 = warp march with lanes of 2 columns instead of 4 (FP32; twice
 *   the warps on a small field; for the FP64 fields, whose lanes already own 2, the warp
 *   march).  Batched handles always use the warp march's persistent kernel, with lanes of 2
 *   columns for FP32 when this knob is 3 (4 otherwise).
 * MPDATA_TUNE_STEPS_PER_LAUNCH: fusion depth S (temporal blocking): 0 or 1 = one step per
 *   launch; 2..4 = mpdata_advance runs its steps in groups of S per launch (the last group
 *   the remainder), each block loading its tile with a 3S-cell halo into shared memory once and
 *   taking it through the S steps there (Eqs. 4-6 with the cross term, FCT, infinite gauge;
 *   same arithmetic as the warp march).  Covers single 2D fields with n_iters = 2, G = 1, no
 *   sources, periodic edges, no third-order, |psi| or divergent-flow terms, no Kahan
 *   summation; other handles and steps ignore it.  FP64: S <= 4 as for FP32.
 * Returns EINVAL for an unknown knob or value.
 */
enum { MPDATA_TUNE_TILE_ROWS = 1, MPDATA_TUNE_KERNEL = 2, MPDATA_TUNE_STEPS_PER_LAUNCH = 3 };
int mpdata_tune(mpdata_t h, int knob, int value);

/* Sends the handle's later work to cuda_stream (a cudaStream_t on the handle's
 * device; NULL = legacy default stream), e.g. a stream that is capturing a CUDA
 * graph of a step loop.  Work already enqueued is not moved. */
int mpdata_set_stream(mpdata_t h, void* cuda_stream);

/* Waits for the handle's stream and returns the first pending device error, if any. */
int mpdata_sync(mpdata_t h);

/* Destroys the handle and frees its scratch (after synchronising its stream). */
int mpdata_destroy(mpdata_t h);

/*
 * Allocation-free step.  The paper has no counterpart: this entry point exists
 * for callers that may not allocate device memory when they advance a field --
 * hosts that give the library a fixed memory budget and forbid allocations after
 * start-up (another allocator owns the device memory), or latency-critical loops
 * that cannot afford cudaMalloc / cudaFree, which may synchronise the device.
 * Such callers cannot create a handle, because mpdata_create allocates scratch.
 *
 * Advances one field (shape (host): ndims extents) by ONE step on the staged
 * kernels, reading psi_in and writing psi_out (the same buffer is allowed),
 * with the same option bits, pointers and alignment rules as mpdata_advance
 * (gc: host array of ndims device pointers; g iff MPDATA_NUG; r iff an RHS bit);
 * cuda_stream is a cudaStream_t or NULL.  It calls no allocating routine: the
 * scratch of the sub-steps lives in one static device array of
 * MPDATA_NOALLOC_SCRATCH_BYTES (16 MiB), which every GPU that loads the library
 * holds until the process exits.  A field needs 16 arrays of its size there, so
 * at most 262144 cells in FP32 and 131072 cells in FP64; larger fields (or any
 * other invalid argument) return MPDATA_EINVAL without launching anything.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, once per device, with that device current); make that
 * first call before any stream capture.  All calls share the array and it keeps
 * the last call's contents (nothing in it needs to start at zero); calls whose
 * work overlaps on the GPU race on it, so serialise them.  Returns MPDATA_OK,
 * MPDATA_EINVAL, MPDATA_EUNSUPPORTED (device index >= 64) or MPDATA_ECUDA.
 */
#define MPDATA_NOALLOC_SCRATCH_BYTES (16u << 20)
int mpdata_step_noalloc(int ndims, const int64_t* shape, int dtype, int n_iters, uint32_t opts,
                        const void* psi_in, void* psi_out, const void* const* gc, const void* g,
                        const void* r, double dt, void* cuda_stream);

/*
 * Diagnostic (no counterpart in the paper): q[i] = n[i] / d[i] for count device doubles,
 * computed with the FP64 division the kernels use (Newton-Raphson reciprocal iteration from
 * the approximate FP64 reciprocal, two iterations, remainder-corrected quotient: within one
 * unit in the last place for normal operands; a zero, infinite or NaN divisor gives NaN).
 * Asynchronous on cuda_stream.  EINVAL for a negative count or null pointers.
 */
int mpdata_selftest_division(const double* n, const double* d, double* q, int64_t count,
                             void* cuda_stream);

/*
 * Diagnostic (no counterpart in the paper): the GPU's fused multiply-add issue rate, the
 * denominator of the FP32 and FP64 arithmetic rooflines.  Launches one kernel on cuda_stream
 * (8 blocks of 256 threads per SM, each thread `iters` rounds of 8 independent FMA chains in
 * the element type dtype, MPDATA_F32 or MPDATA_F64) and stores the number of FMA lane
 * operations it issues in *fma_count; the caller times the launch (CUDA events on the same
 * stream).  sink: device buffer of one element of dtype, written only in a case that never
 * happens.  EINVAL for iters < 1, a null pointer or another dtype.
 */
int mpdata_selftest_fma_rate(int dtype, int64_t iters, void* sink, int64_t* fma_count, void* cuda_stream);

/* Static description of a status code. */
const char* mpdata_strerror(int code);

/* Library version string. */
const char* mpdata_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MPDATA_GB300_H */
