/*
 * mm.h - C ABI of libmm: effective-field evaluation and Landau-Lifshitz time
 * stepping of a finite-difference micromagnetic grid on one GB300 GPU.
 *
 * Method: A. Vansteenkiste and B. Van de Wiele, "MuMax: a new high-performance
 * micromagnetic simulation tool", arXiv:1102.3069 (2011).
 *
 * General conventions (apply to every call below)
 *  - Magnetisation arrays are reduced m = M/Ms, float32, structure-of-arrays
 *    [3][nz][ny][nx] (component, z, y, x; x fastest), contiguous, 3*nx*ny*nz
 *    floats, in DEVICE memory owned by the caller.  Only mm_*_host calls take
 *    host pointers.
 *  - All device work is issued on the stream given to mm_init_geometry and is
 *    asynchronous, except calls that return host scalars (they synchronise that
 *    stream before returning).
 *  - The library never allocates device memory.  The caller allocates one
 *    workspace of mm_workspace_bytes() bytes and hands it over with
 *    mm_set_workspace(); it must stay valid until mm_destroy().
 *  - SI units at the boundary (m, s, A/m, J/m, J/m^3, T, K).  Internally the
 *    library works in units with field unit Ms and time unit 1/(gamma0 Ms)
 *    (the paper's Sec. 3.3 keeps mu0 = gamma0 = Ms = 1 for single precision).
 *  - Return value: MM_OK (0) or a negative mm_status; a message describing the
 *    last failure is available from mm_last_error().  Nothing is thrown across
 *    the ABI.  A failed call leaves the context usable unless it returns
 *    MM_ECUDA.
 */
#ifndef MM_H
#define MM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mm_ctx mm_ctx;   /* opaque; created by mm_init_geometry, freed by mm_destroy */

typedef enum {
    MM_OK = 0,
    MM_EINVAL = -1,          /* bad argument or call order                          */
    MM_ENOMEM = -2,          /* workspace too small / not set                       */
    MM_ECUDA = -3,           /* a CUDA runtime call failed                          */
    MM_ENOTCONVERGED = -4,   /* step size underflow or step budget exhausted        */
    MM_ENONFINITE = -5,      /* NaN/Inf met in m, H or the step error               */
    MM_ETIMEOUT = -6,        /* a bounded wait ran out                              */
    MM_ESTATE = -7           /* operation needs state that is not there yet         */
} mm_status;

/* Time integrators of Sec. 2.2: RK1 Euler, RK2 Heun, RK3 Kutta, RK4 classical
 * (fixed dt); RK12 Heun-Euler, RK23 Bogacki-Shampine, RKCK Cash-Karp and RKDP
 * Dormand-Prince (adaptive step, error bound tol per step). */
enum { MM_EULER = 1, MM_HEUN = 2, MM_RK3 = 3, MM_RK4 = 4, MM_RKDP = 5, MM_RKCK = 6, MM_RK12 = 12, MM_RK23 = 23 };

typedef struct mm_stats {
    long long evals;        /* H_eff evaluations issued since the last mm_load      */
    long long accepted;     /* accepted steps                                       */
    long long rejected;     /* rejected (adaptive) steps                            */
    long long step_index;   /* thermal-noise step counter                           */
    double t;               /* simulated time, s                                    */
    double dt;              /* next proposed step (RKDP) or last fixed step, s      */
    double last_err;        /* last step-error estimate (dimensionless, |dm|)       */
    double max_torque;      /* max_i |m_i x H_i|/Ms at the last state judged by the */
                            /* torque bound (see mm_advance)                        */
    double energy;          /* last energy computed by mm_eval_heff, J              */
    int status;             /* device-side status: 0 or a negative mm_status        */
    int done;               /* 1 when t_end / torque target reached or on failure   */
    double dissipation;     /* W, from the last mm_eval_heff with energy: the rate   */
                            /* -mu0 Ms V gamma0 alpha/(1+alpha^2) sum |m x H|^2 at   */
                            /* which damping removes energy (Eq. 1); it is dE/dt     */
                            /* without spin-transfer torque and thermal field; the   */
                            /* sum is accumulated in FP64                            */
} mm_stats;

/*
 * Create a context for an nx x ny x nz grid of dx x dy x dz cuboid cells
 * (Sec. 2.1.1: regular finite-difference grid of identical cuboids).
 * pbc_x/y/z != 0 makes that axis periodic (Sec. 2.1.1, periodic boundary
 * conditions: periodic images added to the kernel, no zero padding);
 * pbc_images = number of images on each side of a periodic axis (>= 0).
 * Open axes are zero padded to the smallest FFT length >= 2n-1 of the
 * form 2^k or r * 2^l with r = 3, 5, 7 (Sec. 3.3: sizes 2^n {1,3,5,7};
 * the odd factors are compiled for 3 * 2^6 .. 3 * 2^10, 5 * 2^6 .. 5 * 2^9
 * and 7 * 2^6 .. 7 * 2^9).  A periodic axis needs n to be one of those
 * lengths.  nx, ny, nz in [1, 2048] for open axes (padded length <= 4096)
 * and [1, 4096] for periodic ones.  Grids with an odd factor in any padded
 * length run single contexts only: mm_batch_create refuses them (see
 * mm_set_fft_lengths).
 * cuda_stream: a cudaStream_t (NULL = legacy default stream).
 * On success *out owns host memory only; free it with mm_destroy.
 */
int mm_init_geometry(mm_ctx** out, int nx, int ny, int nz, double dx, double dy, double dz,
                     int pbc_x, int pbc_y, int pbc_z, int pbc_images, void* cuda_stream);

/*
 * Which FFT lengths the open axes pad to (an implementation choice within
 * Sec. 3.3's rule): MM_FFT_2357 (default) - the smallest 2^k or r * 2^l
 * (r = 3, 5, 7) >= 2n-1; MM_FFT_POW2 - the smallest power of two >= 2n-1,
 * which batches (mm_batch_create) need for every sample.  Call before
 * mm_set_workspace (the workspace size follows); MM_ESTATE after it,
 * MM_EINVAL for MM_FFT_POW2 with a periodic axis of r * 2^l cells.
 */
enum { MM_FFT_2357 = 0, MM_FFT_POW2 = 1 };
int mm_set_fft_lengths(mm_ctx* ctx, int mode);

/* Device workspace size in bytes for this geometry (kernel, spectra, RK stages). */
size_t mm_workspace_bytes(const mm_ctx* ctx);

/* Hand over the caller-owned device workspace (256-byte aligned, >= mm_workspace_bytes).
 * Uploads the twiddle table and clears the device state; synchronises the stream. */
int mm_set_workspace(mm_ctx* ctx, void* dev_ptr, size_t bytes);

/*
 * Material parameters (Sec. 2, Eq. 1 and Sec. 2.1): saturation magnetisation
 * Ms (A/m, > 0), exchange stiffness Aex (J/m, >= 0; Eq. 3), uniaxial constant
 * Ku (J/m^3; Eq. 4) with easy axis easy_axis[3] (normalised here; may be
 * NULL when Ku == 0), damping alpha (>= 0), gyromagnetic ratio gamma0
 * (m/(A s), > 0; pass 0 for 2.211e5), temperature (K, >= 0; Eq. 6) with the
 * Philox seed of the thermal noise, applied flux density B_applied_T[3] (T).
 * The applied field enters as H = B/mu0.
 */
int mm_set_material(mm_ctx* ctx, double Ms, double Aex, double Ku, const double easy_axis[3],
                    double alpha, double gamma0, double temperature, uint64_t seed,
                    const double B_applied_T[3]);

/*
 * Cubic magnetocrystalline anisotropy (Sec. 2.1.3, Eq. 5):
 *   phi = K1 (a1^2 a2^2 + a2^2 a3^2 + a1^2 a3^2) + K2 a1^2 a2^2 a3^2  (J/m^3)
 * with direction cosines a_i = m . c_i to the cubic axes c1, c2 and
 * c3 = c1 x c2 (c1 is normalised and c2 made orthogonal to it here).  Adds
 * H = -(1/(mu0 Ms)) dphi/dm to H_eff and phi to the energy.  K1 = K2 = 0
 * (the default) switches it off; the axes may then be NULL.
 * MM_EINVAL for non-finite constants or degenerate axes.
 */
int mm_set_cubic_anisotropy(mm_ctx* ctx, double K1, double K2, const double c1[3], const double c2[3]);

/*
 * Per-cell uniaxial easy axes (Sec. 2.1.3, Eq. 4 with an axis u_i in every
 * cell, e.g. a polycrystal's random grain axes): u = device array, float32
 * SoA [3][nz][ny][nx] of unit vectors, caller-owned, read by every later
 * evaluation (not normalised by the library; keep it valid and unchanged
 * while in use).  H_an,i = 2Ku/(mu0 Ms) (m_i . u_i) u_i with the Ku of
 * mm_set_material.  u = NULL returns to the single axis of mm_set_material.
 * MM_EINVAL for a misaligned pointer.
 */
int mm_set_anisotropy_axes(mm_ctx* ctx, const float* u);

/*
 * Fixed maximum variation of m per step (Sec. 2.2: the methods without an
 * error estimate take a fixed time step or a fixed maximum variation of m per
 * step).  With max_dm > 0, mm_advance with MM_EULER, MM_HEUN, MM_RK3 or MM_RK4
 * chooses every step's size on the device as h = max_dm / max_i |dm/dt(m_n)|_i
 * (the size that moves the fastest cell by max_dm to first order), capped at
 * the dt_s argument when that is > 0 (dt_s = 0: no cap), then takes the
 * method's step with it.  Each step evaluates k1 first and forms the stage-2
 * input after h is known.  The thermal field is refused in this mode (its
 * variance depends on the step).  max_dm = 0 (default) returns to fixed dt.
 * MM_EINVAL unless 0 <= max_dm <= 1.
 */
int mm_set_max_dm(mm_ctx* ctx, double max_dm);

/*
 * Layout of the passes (an implementation choice with no counterpart in the
 * paper).  For padded x lengths 64 to 2048 an evaluation inside a step can
 * either run the inverse x transform, the cell-local terms with the stage
 * update, and the forward x transform of the next stage's input as one kernel
 * (MM_LAYOUT_FUSED), or as three kernels with H_demag passing through device
 * memory (MM_LAYOUT_SPLIT).  MM_LAYOUT_CLUSTER runs every evaluation (time
 * steps and mm_eval_heff) as ONE launch of a thread-block cluster of 1 to 16
 * CTAs that keeps the half spectrum in the CTAs' shared memory: 2-D grids
 * only (nz = 1, open z), power-of-two FFT lengths along x and y, and a half
 * spectrum that fits the cluster (up to about 256 x 256 cells); MM_EINVAL for
 * other grids.  A run of steps (mm_advance) is one launch of that cluster
 * for all its standard steps.  MM_LAYOUT_AUTO (default) takes the fused
 * kernel: the cluster launch measured slower on GB300 at every size it
 * applies to.  Results of all layouts agree to float32 rounding.  Batches
 * (mm_batch_*) always use the split passes.
 */
enum { MM_LAYOUT_AUTO = 0, MM_LAYOUT_FUSED = 1, MM_LAYOUT_SPLIT = 2, MM_LAYOUT_CLUSTER = 3 };
int mm_set_pass_layout(mm_ctx* ctx, int layout);

/*
 * Precision of the z transforms of 3-D grids (Sec. 3.3 computes the whole
 * convolution in single precision; this is a variant with no counterpart in
 * the paper).  MM_DFT_FP32 (default): the FP32 column pass.  MM_DFT_SPLIT_BF16:
 * the z transforms (stages i and iii of Sec. 3.2 along z) run as dense DFT
 * matrix products on the tensor cores with bf16 operands split as
 * hi + lo (three products per transform, fp32 accumulation) and the kernel
 * product in fp32 between them.  Its H_eff error against the FP64 oracle,
 * measured on a 32^3 periodic crop, is 1.1e-7 relative (the FP32 pass: 6.2e-8);
 * it is ~17x slower than the FP32 pass on the 256 x 256 x 64 cube and serves
 * precision studies.
 * Only single-context evaluations and steps use it (mm_eval_heff_static and
 * batches keep the FP32 pass).  Call before mm_set_workspace (the variant
 * needs workspace of its own: mm_workspace_bytes grows); MM_ESTATE after it,
 * MM_EINVAL for 2-D grids or a padded z length below 4.
 */
enum { MM_DFT_FP32 = 0, MM_DFT_SPLIT_BF16 = 1 };
int mm_set_dft_precision(mm_ctx* ctx, int mode);

/*
 * Spin-transfer torque of Zhang and Li (Sec. 2.1.4, Eq. 7), a torque added to
 * dm/dt (not a field):
 *   dm/dt += -b_j/(1+alpha^2) [ m x (m x (j.grad)m) + (xi - alpha) m x (j.grad)m ],
 *   b_j = P mu_B / (e Ms (1 + xi^2)),
 * with polarisation P, non-adiabaticity xi and the uniform current density
 * j_A_per_m2[3] (A/m^2; NULL = no current).  (j.grad)m uses central
 * differences; at a free boundary the missing neighbour is the cell itself.
 * P = 0 or j = 0 (the default) switches it off.  MM_EINVAL for non-finite input.
 */
int mm_set_stt(mm_ctx* ctx, double P, double xi, const double j_A_per_m2[3]);

/*
 * Enable (1) or disable (0) the magnetostatic term.  Enabled by default; when
 * enabled, mm_demag_kernel must have run before any evaluation.  Disabling it
 * leaves exchange, anisotropy, Zeeman and thermal terms (used for uncoupled
 * macrospin ensembles and for testing the local terms alone).
 */
int mm_set_demag(mm_ctx* ctx, int enabled);

/*
 * Build the demagnetising kernel (Sec. 2.1.1 Eq. 2; Sec. 3.2: symmetric
 * kernel whose transform is real): the cell-averaged tensor N_ab of every
 * source-target offset is computed in FP64 on the GPU (closed form near the
 * origin, tent-weighted Gauss-Legendre quadrature of the dipole kernel far
 * away; periodic images summed), wrapped into the padded grid, transformed
 * with an FP64 FFT, and its real part times -1/(Px Py Pz) stored in float32
 * on the non-negative-frequency octant.  Uses the workspace's stage buffers as
 * scratch (so it invalidates any loaded state).  Synchronises the stream.
 * out_tensor_host: optional (may be NULL) host buffer of
 *   6 * Oz * Oy * Ox doubles receiving the real-space tensor on the
 *   non-negative offsets, components in the order xx, yy, zz, xy, xz, yz,
 *   layout [comp][oz][oy][ox]; O = n for an open axis, n/2+1 for a periodic
 *   one (periodic entries hold the image sums).
 */
int mm_demag_kernel(mm_ctx* ctx, double* out_tensor_host);

/* Number of doubles mm_demag_kernel writes to out_tensor_host. */
size_t mm_demag_tensor_len(const mm_ctx* ctx);

/*
 * One effective-field evaluation (Sec. 2.1: H_eff = H_ms + H_exch + H_anis +
 * H_applied + H_thermal) at the given m (not renormalised).
 *   m          device, [3][nz][ny][nx] float32 (read only)
 *   h_out      device, same layout, H_eff in A/m (may be NULL)
 *   torque_out device, same layout, dm/dt of Eq. 1 divided by Ms in 1/s (may be NULL)
 *   energy_J_host  host double receiving the total energy in J (thermal field
 *              excluded); may be NULL.  Non-NULL synchronises the stream.
 * The thermal term uses the clock set by mm_set_thermal_clock.
 */
int mm_eval_heff(mm_ctx* ctx, const float* m, float* h_out, float* torque_out, double* energy_J_host);

/* Thermal-noise clock used by mm_eval_heff: step index and the step dt (s) of Eq. 6. */
int mm_set_thermal_clock(mm_ctx* ctx, uint64_t step_index, double dt_s);

/*
 * Load m (device, float32 SoA) as the integrator state, normalised to |m| = 1,
 * set the simulated time to t0_s and the step counter to step_index.  The
 * derivative reused by the first-same-as-last property is invalidated.
 */
int mm_load(mm_ctx* ctx, const float* m, double t0_s, uint64_t step_index);

/* Copy the current state m (device) out.  Asynchronous. */
int mm_store(mm_ctx* ctx, float* m);

/*
 * Enqueue nsteps time steps on the stream without waiting (device-side step
 * control, Sec. 2.2).  Fixed-step methods (MM_EULER, MM_HEUN, MM_RK3, MM_RK4)
 * take dt_s > 0 (or, after mm_set_max_dm, choose each step themselves with
 * dt_s as an optional cap).  Adaptive methods (MM_RK12, MM_RK23, MM_RKCK, MM_RKDP) take
 * the per-step error bound tol (max over cells of |dm|) and the proposed step
 * dt_s (> 0 sets it; <= 0 keeps the current one, 100 fs after mm_load); the
 * step factor is 0.9 (tol/err)^(1/q), q = 2, 3, 5, 5 respectively, clamped to
 * [0.2, 5].  tol < 0 selects fixed steps of dt_s for an adaptive method (the
 * error estimate is still computed and reported).  The thermal field (T > 0)
 * needs a fixed-step method with a fixed dt (MM_EULER, MM_HEUN, MM_RK3 or
 * MM_RK4; one noise draw per step shared by its stages).  t_end_s > 0 stops
 * the run at t_end_s: the Runge-Kutta tableaus (MM_RK3 and above) shorten their
 * last step to end exactly there (with the noise amplitude of the full dt);
 * MM_EULER and MM_HEUN keep their dt and stop at the first step that reaches
 * or passes t_end_s (they may overshoot it by less than one dt).
 * torque_tol > 0 stops the run at the first state where
 * max |m x H|/Ms < torque_tol (relaxation), judged where the method evaluates
 * the field at an accepted state: the last stage of MM_RKDP and MM_RK23 (first
 * same as last) judges the new state; MM_EULER, MM_HEUN and the other
 * tableaus judge the state a step starts from, and then keep that state
 * without taking the step.  mm_stats.max_torque is the torque of the state so
 * judged last (for the latter methods: the state the last step started from).
 * Once stopped, queued steps do no work.
 */
int mm_advance(mm_ctx* ctx, int method, long nsteps, double dt_s, double tol,
               double t_end_s, double torque_tol);

/* Synchronise the stream and read the device-side counters (stats may be NULL). */
int mm_get_stats(mm_ctx* ctx, mm_stats* stats);

/*
 * Checkpoint and resume.  mm_get_state copies the current state m (device
 * SoA, may be NULL) and fills the integrator scalars: simulated time, the
 * step size the next adaptive step will try, the thermal step counter, the
 * step and evaluation counters and whether the last attempt was rejected
 * (synchronises).  mm_set_state loads m exactly as given (no renormalisation)
 * with those scalars, so that mm_advance(..., dt_s = 0, ...) afterwards
 * continues the run as if it had not stopped (the first-same-as-last k1 is
 * evaluated again from m, which gives the same values).  MM_ESTATE without a
 * loaded state, MM_EINVAL for a checkpoint with negative or non-finite fields.
 */
typedef struct mm_checkpoint {
    double t;               /* simulated time, s                                  */
    double dt;              /* next adaptive step size, s                         */
    long long step_index;   /* thermal-noise step counter                         */
    long long accepted, rejected, evals;
    int after_reject;       /* the last attempt was rejected (caps the next growth) */
    int reserved_;
    double t_internal;      /* t and dt in the library's internal time unit         */
    double dt_internal;     /* (1/(gamma0 Ms)); used on restore when they agree with  */
                            /* t and dt, so that the step size is restored exactly    */
} mm_checkpoint;
int mm_get_state(mm_ctx* ctx, float* m, mm_checkpoint* out);
int mm_set_state(mm_ctx* ctx, const float* m, const mm_checkpoint* in);

/*
 * One step (Sec. 2.2) from m (device, in/out): loads m at time *t_s, takes
 * one step of `method` with the proposed/fixed step *dt_s (and error bound
 * tol for the adaptive methods), stores the result back into m and synchronises.
 * On return *accepted = 1/0, *t_s is the new time and *dt_s the next step.
 */
int mm_step(mm_ctx* ctx, float* m, int method, double* t_s, double* dt_s, double tol, int* accepted);

/*
 * Relax m (device, in/out) with adaptive Dormand-Prince until
 * max_i |m_i x H_i|/Ms < torque_tol or max_steps attempted steps; err_tol is
 * the per-step error bound.  The host polls the device every 64 steps.
 * Returns MM_ENOTCONVERGED if the torque bound was not reached.
 */
int mm_relax(mm_ctx* ctx, float* m, double torque_tol, double err_tol, long max_steps,
             long* steps_out, double* torque_out);

/*
 * Host-buffer variant for callers without device memory: copies m_host
 * (pinned or pageable host, [3][nz][ny][nx] float32) to the device, runs
 * nsteps as mm_advance would, and copies the result back into m_host.
 * Synchronises the stream.
 */
int mm_run_host(mm_ctx* ctx, float* m_host, int method, long nsteps, double dt_s, double tol);

/*
 * Per-pass timing (a diagnostic with no counterpart in the paper).  While
 * enabled, every kernel launch of mm_eval_heff / mm_advance is bracketed by
 * CUDA events on the context's stream.  mm_pass_times synchronises and returns,
 * per pass, the summed event time in ms and the number of launches since
 * mm_profile(ctx, 1); arrays of MM_NPASS entries in the order
 * x forward, y conv (2-D), y forward, z conv, y inverse (3-D), x inverse +
 * local terms, stage-2 combine, local terms without demag, x inverse + local
 * terms + forward x transform of the next stage's input, x inverse alone
 * (demag field to a buffer), cell pass reading that buffer, forward x
 * transform of the next stage's input, the one-launch cluster evaluation, the
 * y forward + z column + y inverse pass of 3-D grids with nz <= 8.
 * Time steps use the fused passes; the split passes run under MM_LAYOUT_SPLIT
 * (mm_set_pass_layout) and in batches; small 2-D grids run the cluster launch
 * (MM_LAYOUT_AUTO, MM_LAYOUT_CLUSTER).
 */
enum { MM_NPASS = 14 };
int mm_profile(mm_ctx* ctx, int enable);
int mm_pass_times(mm_ctx* ctx, double* ms_out, long long* count_out);

/*
 * Allocation-free variant of mm_eval_heff (the paper has no counterpart).
 *
 * For callers that cannot allocate device memory at the point where they need
 * a field evaluation: code running inside a host application or plugin that
 * owns the whole device-memory budget and hands out only the buffers it
 * created, and time-critical loops that forbid cudaMalloc after start-up
 * because an allocation can block or synchronise the device.
 *
 * Same inputs and outputs as mm_eval_heff (m read-only; h_out in A/m and
 * torque_out in 1/s, each may be NULL; no energy), but the scratch it needs -
 * the FFT spectra, the twiddle table and the reduction counters - lives in
 * one static device array of MM_STATIC_SCRATCH_BYTES per GPU, which every
 * GPU that loads the library holds until the process exits.  The call
 * allocates nothing (no cudaMalloc, cudaFree or allocating library routine).
 *  - The context needs its material; with the magnetostatic term enabled it
 *    also needs its kernel (mm_demag_kernel, which lives in the caller's
 *    workspace); with mm_set_demag(ctx, 0) no workspace is needed at all.
 *  - Grids whose spectra do not fit in the static scratch (roughly up to
 *    1024 x 512 x 1 cells) are rejected with MM_ENOMEM and a message.
 *  - The first call on a device looks up the array's device address and
 *    fills its twiddle table (with that device current); make that first call
 *    before any stream capture.
 *  - All calls on a device share the one array and it keeps the last call's
 *    contents (the counters are cleared on every call): calls whose work
 *    overlaps on the GPU - on different streams, or from several contexts -
 *    race with each other.  Serialise them.
 * Asynchronous on the context's stream.
 */
#define MM_STATIC_SCRATCH_BYTES (16u << 20)
int mm_eval_heff_static(mm_ctx* ctx, const float* m, float* h_out, float* torque_out);

/* Message describing the last failure of a call on this context (never NULL). */
const char* mm_last_error(const mm_ctx* ctx);

/* Free the context (not the caller's workspace).  NULL is accepted. */
void mm_destroy(mm_ctx* ctx);

/*
 * Batched ensembles (Sec. 3.1 taken to many problems: independent samples stay
 * on the GPU and are stepped together).  The paper runs one problem at a time;
 * the batch runs many independent ones, each with its own context, through
 * the same passes.
 *
 * mm_batch_create takes n ready contexts (workspace set, material set, demag
 * kernel built with mm_demag_kernel, demag enabled; padded FFT lengths 64 to
 * 1024 along x and y, i.e. 32 <= n <= 512 on an open axis and n a power of
 * two from 64 to 1024 on a periodic one; padded length at most 1024 along z)
 * and the CUDA stream all their work then goes on (each context's stream
 * is replaced by it).  The contexts stay owned by the caller and must outlive
 * the batch; while in a batch they should not be stepped on their own.
 * MM_EINVAL if a context does not qualify.
 *
 * Every pass of an evaluation is launched once per FFT length over all
 * samples of that length, with the block bodies of the single-context
 * kernels on the same block decomposition (the batched kernels read each
 * sample's parameters from device memory, so results agree with stepping the
 * sample alone up to float32 rounding).  A standard step is replayed from a
 * CUDA graph.
 *
 * mm_batch_workspace_bytes / mm_batch_set_workspace: a small device buffer
 * (sample descriptors, work lists, a state gather area) the caller allocates;
 * 256-byte aligned; valid until mm_batch_destroy.
 * mm_batch_load(m): m[i] = device SoA magnetisation of sample i (as mm_load,
 * normalised on load).  mm_batch_store(m): copies each sample's state out.
 * mm_batch_advance: nsteps steps of a Runge-Kutta method (MM_RK3 ... MM_RKDP)
 * for every sample; dt_s > 0 sets every sample's step (s); tol as in
 * mm_advance.  Asynchronous after its set-up.  The thermal field is refused.
 * mm_batch_get_stats: out[i] = sample i's statistics (synchronises).
 * mm_batch_relax: loads m, runs Dormand-Prince steps until every sample's
 * max |m x H|/Ms < torque_tol (polled every 64 steps; finished samples leave
 * the launches) or max_steps, stores m back.  steps_out[i], torque_out[i]
 * (may be NULL): per-sample steps taken and final torque; n_converged (may
 * be NULL): how many samples reached the bound.  MM_ENOTCONVERGED if some did
 * not; a sample's device failure is returned as its status.
 */
typedef struct mm_batch mm_batch;
int mm_batch_create(mm_batch** out, mm_ctx* const* ctxs, int n, void* cuda_stream);
size_t mm_batch_workspace_bytes(const mm_batch* b);
int mm_batch_set_workspace(mm_batch* b, void* dev_ptr, size_t bytes);
int mm_batch_load(mm_batch* b, const float* const* m);
int mm_batch_store(mm_batch* b, float* const* m);
int mm_batch_advance(mm_batch* b, int method, long nsteps, double dt_s, double tol);
int mm_batch_get_stats(mm_batch* b, mm_stats* out);
int mm_batch_relax(mm_batch* b, float* const* m, double torque_tol, double err_tol, long max_steps,
                   long* steps_out, double* torque_out, int* n_converged);
/*
 * Batch autotuner.  Every batched FFT pass is compiled with two register
 * budgets (an occupancy-first one and one of at least 80 registers per
 * thread, fewer resident blocks), and the register x passes also with a
 * second tile shape (half the row pairs per block, twice the blocks).  Where
 * a pass has alternatives, the batch times each on its samples when it
 * builds its launch lists (first advance, and after finished samples leave a
 * relaxation) and keeps the fastest; a tile choice rebuilds that pass's work
 * list.  Choices are cached for the process, keyed by pass, FFT length and
 * block count (power of two).  mode 1 (default) tunes, 0 always launches the
 * default kernels, 2 the other register budget wherever there is one, 3 the
 * other tile shape wherever there is one (2 and 3 for tests; results are the
 * same).  MM_EINVAL for other modes.  mm_batch_tuning reports the current launch
 * groups, how many of them had alternatives, and how many run one.
 */
int mm_batch_set_tuning(mm_batch* b, int mode);
int mm_batch_tuning(const mm_batch* b, int* n_groups, int* n_tunable, int* n_alternative);
const char* mm_batch_last_error(const mm_batch* b);
void mm_batch_destroy(mm_batch* b);

#ifdef __cplusplus
}
#endif
#endif /* MM_H */
