/*
 * mrsim.h -- C-ABI of the GB300 spin-based MR simulator (libmrsim.so).
 *
 * The library computes the hot path of a spin-based MR-tomography simulation
 * (Kürsch, "Konzeption und Realisierung eines skalierbaren Simulators für die
 * Magnetresonanz-Tomographie", §5.1.1): every isochromat of a phantom is
 * propagated independently through a pulse sequence of elementary sequences
 * (§4.1, Eq. 4.1: hard RF pulse Eq. 3.19, gradient/off-resonance precession
 * Eqs. 3.5/3.11/3.14, T1/T2 relaxation Eq. 3.5), and at every ADC sample the
 * rotating-frame transverse magnetisation is summed over all spins into the
 * complex signal (Eqs. 3.30-3.32).
 *
 * Conventions (all SI units, angles in rad):
 *   - rotating frame, on resonance; γ is a parameter given as γ/2π in Hz/T;
 *   - an event applies, in this order: the RF pulse at its start, precession
 *     by θ = (γ G·x + Δω)·Δt with Mxy <- Mxy·exp(-jθ) and T2 decay, T1
 *     recovery of Mz towards M0, then (if adc != 0) one sample of
 *     Σ_spins (Mx + jMy)·exp(-j·adc_phase) at the end of the event;
 *   - signals are complex float64, interleaved (re, im), one value per ADC
 *     event, in event order.
 *
 * Errors: every entry point returns an mrsim_status and never aborts the
 * process.  The message of the last failure on a context is available from
 * mrsim_last_error().  Device waits are bounded; a wait that runs out makes the
 * kernel record MRSIM_ETIMEOUT in a device status word, which the next
 * host-visible call (mrsim_stream_status, or any call with host output
 * buffers) reports.
 *
 * Ownership: create functions copy their inputs; the caller keeps ownership of
 * every buffer it passes.  Handles are owned by the caller and released with
 * the matching destroy function (NULL is accepted).  A context must outlive the
 * handles created on it.  Calls on one context are not thread-safe; mrsim_compile
 * uses no context and may run on any thread at any time.
 *
 * Pointers marked "host or device" may be either: the library asks the CUDA
 * runtime what a pointer is and copies host data itself.
 */
#ifndef MRSIM_H
#define MRSIM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MRSIM_OK = 0,
    MRSIM_EINVAL = 1,      /* invalid argument: NaN/Inf, T <= 0, Δt < 0, size mismatch, NULL */
    MRSIM_ENOMEM = 2,      /* host or device allocation failed */
    MRSIM_ECUDA = 3,       /* a CUDA runtime call failed */
    MRSIM_ETIMEOUT = 4,    /* a bounded device wait ran out */
    MRSIM_EUNSUPPORTED = 5 /* valid request this library binary cannot serve (e.g. no sm_103 device) */
} mrsim_status;

typedef enum {
    MRSIM_FP64 = 0,      /* every step in float64 */
    MRSIM_FP32 = 1,      /* rotations/relaxation in float32 with float64 sequence precompute and
                            float-float phase arguments; each sample's sum is a float32 pairwise tree
                            within a warp, a float32 add across the warps of a thread block and a
                            float64 sum across thread blocks */
    MRSIM_FP32_KAHAN = 2 /* the float32 bulk arithmetic with the per-sample spin sum kept in higher
                            precision than float32 across the whole phantom: the same path as
                            MRSIM_FP32, whose cross-block sums are float64 (a stronger form of a
                            compensated float32 sum; the in-block float32 chains are at most
                            128-term pairwise trees plus 16 adds, ~1e-7 relative).  Accepted by
                            every call that takes a precision; results equal MRSIM_FP32's. */
} mrsim_precision;

/* One elementary sequence (§4.1; Eq. 4.1).  64 bytes, no padding. */
typedef struct mrsim_event {
    double dt;        /* duration Δt >= 0 [s] */
    double gx, gy, gz;/* constant gradient during Δt [T/m] */
    double rf_flip;   /* flip angle α of the hard pulse at the start [rad]; 0 = no pulse; sign allowed */
    double rf_phase;  /* phase φ of the pulse axis in the x'y' plane [rad] (Eq. 3.19) */
    double adc_phase; /* receiver demodulation phase [rad] of this event's sample */
    int32_t adc;      /* 1 = take one sample at the end of the event, 0 = none */
    int32_t reserved; /* must be 0 */
} mrsim_event;

typedef struct mrsim_ctx mrsim_ctx;
typedef struct mrsim_phantom mrsim_phantom;
typedef struct mrsim_sequence mrsim_sequence;

/* Optional launch and state controls of mrsim_simulate_ex. Zero-initialise for defaults. */
typedef struct mrsim_options {
    int32_t spins_per_thread;  /* 0 = library choice (tuned table); else 1, 2, 4 or 8 (FP64: 1 or 2) */
    int32_t threads_per_block; /* 0 = library choice; else a multiple of 32 in [32, 1024] */
    uint32_t flags;            /* MRSIM_ACCUMULATE: add into signal_out instead of overwriting it;
                                  MRSIM_TUNE: run mrsim_autotune first if this shape is not tuned yet */
    int32_t reserved;
    const double *state_in;    /* NULL = thermal equilibrium (0,0,M0); else 3*n_spins (Mx,My,Mz), host or device */
    double *state_out;         /* NULL, or 3*n_spins receiving (Mx,My,Mz) after the last event, host or device */
    double *snapshots;         /* NULL, or n_snapshots x n_spins x 3 receiving (Mx,My,Mz) after each snapshot
                                  event of a sequence loaded with mrsim_sequence_load_snapshots; host or device */
} mrsim_options;

#define MRSIM_ACCUMULATE 1u
#define MRSIM_TUNE 2u /* autotune the launch shape on first use with this (precision, spin count) */

/* ---- context ------------------------------------------------------------------------- */

/* Bind a context to CUDA device `device` (must be a compute capability 10.3 GPU). */
mrsim_status mrsim_context_create(int device, mrsim_ctx **out);
void mrsim_context_destroy(mrsim_ctx *ctx);
const char *mrsim_status_string(mrsim_status s);
/* Message of the last failed call on ctx ("" if none).  Owned by ctx, valid until the next call. */
const char *mrsim_last_error(const mrsim_ctx *ctx);
/* Failure log: fn(status, message, user) is called, on the calling thread, for every failed call
 * of any context and for every failed mrsim_compile; NULL removes it.  With the environment
 * variable MRSIM_LOG set (to anything but "0") the same messages also go to stderr. */
typedef void (*mrsim_log_fn)(mrsim_status status, const char *message, void *user);
void mrsim_set_log_callback(mrsim_log_fn fn, void *user);
/* Test hook: the device allocation that follows `after` further successful ones on this context
 * fails once with MRSIM_ENOMEM, as a full device would (after < 0 switches the hook off), so that
 * the out-of-memory paths can be tested without exhausting the device.  The environment variable
 * MRSIM_FAIL_ALLOC=<after> arms it in every context when the context is created (for programs
 * that cannot call this function).  The context's own status buffers are not counted. */
mrsim_status mrsim_debug_fail_alloc(mrsim_ctx *ctx, int32_t after);
/* Train maps (on by default).  A shaped pulse (Eq. 3.23) repeated with the same sub-pulse flips,
 * precession class and T1 class (the same pulse in every TR) composes, for each spin, to one
 * affine map of its state.  With maps on, mrsim_simulate[_ex], mrsim_simulate_coils,
 * mrsim_autotune and the batch calls build every spin's map once per launch (double-float arithmetic, float64 for MRSIM_FP64) and
 * apply it in place of the train's sub-pulses.  The result is the same composition with one
 * rounding of the map in place of one rounding per sub-pulse.  Such a call then needs
 * 12 x (map kinds) values per spin of device memory: a single-phantom call takes it from a
 * per-context stream-ordered pool and frees it after its kernel; a batch holds it from creation.
 * enable = 0 runs every train sub-pulse by sub-pulse (and needs no such memory).
 * mrsim_simulate_batch_static and the adjoint never use maps.  Affects the calls made after it;
 * batches created before it keep their setting. */
mrsim_status mrsim_context_set_train_maps(mrsim_ctx *ctx, int32_t enable);
/* Synchronise `stream` (cudaStream_t, NULL = legacy default stream) and report any device-side
 * status recorded by kernels of this context (e.g. MRSIM_ETIMEOUT); clears the status word. */
mrsim_status mrsim_stream_status(mrsim_ctx *ctx, void *stream);
/* Diagnostic: launches on `stream` one block that runs the kernels' bounded mbarrier wait on a
 * barrier nothing completes, with limit_ns (1e3 .. 1e9) instead of the 2 s of the op pipeline; the
 * wait runs out, the block records MRSIM_ETIMEOUT in the status word and ends.  This is how the
 * timeout path is tested without any fault; the context stays usable. */
mrsim_status mrsim_debug_wait_timeout(mrsim_ctx *ctx, int64_t limit_ns, void *stream);

/* ---- phantom: the object as a list of isochromats (§6.1.1, Eq. 6.2) ------------------- */

/* Copies n_spins isochromats from host arrays: position x,y,z [m], equilibrium magnetisation
 * M0 (rho), T1, T2 [s] (> 0, +INFINITY allowed = no relaxation), total off-resonance Δω [rad/s].
 * EINVAL on NaN/Inf positions, rho or dw, or T1/T2 <= 0.  n_spins = 0 is allowed. */
mrsim_status mrsim_phantom_create(mrsim_ctx *ctx, int64_t n_spins, const double *x, const double *y,
                                  const double *z, const double *rho, const double *t1, const double *t2,
                                  const double *dw, mrsim_phantom **out);
/* Same with the seven arrays in device memory (e.g. torch tensors); packing runs on `stream`,
 * which is synchronised before return so the caller may free the arrays afterwards. */
mrsim_status mrsim_phantom_create_device(mrsim_ctx *ctx, int64_t n_spins, const double *x, const double *y,
                                         const double *z, const double *rho, const double *t1,
                                         const double *t2, const double *dw, void *stream,
                                         mrsim_phantom **out);
/* Spin count of the phantom (-1 for NULL). */
int64_t mrsim_phantom_num_spins(const mrsim_phantom *p);
/* Frees the phantom's device memory (NULL is ignored) with cudaFree, which waits for the device's
 * outstanding work first. */
void mrsim_phantom_destroy(mrsim_phantom *p);

/* ---- sequence: elementary sequences (§4.1) compiled once in float64 ------------------- */

/* A compiled program on the host: the compilation step of mrsim_sequence_load on its own.  It
 * needs no context and no GPU, so a caller can compile the next request on another thread while
 * a context simulates the current one.  Different threads may compile at the same time. */
typedef struct mrsim_compiled mrsim_compiled;
/* Validates and compiles n_events events (host memory) with optional snapshots (see
 * mrsim_sequence_load_snapshots); same validation and error codes as mrsim_sequence_load.  On
 * failure *out = NULL and mrsim_compile_last_error() says why. */
mrsim_status mrsim_compile(int64_t n_events, const mrsim_event *events, double gamma_hz_per_t, int64_t n_snap,
                           const int64_t *snap_after, mrsim_compiled **out);
/* Message of the calling thread's last failed mrsim_compile ("" if none); valid until its next
 * mrsim_compile call. */
const char *mrsim_compile_last_error(void);
int64_t mrsim_compiled_num_adc(const mrsim_compiled *c);
/* Bytes mrsim_sequence_create copies to the device for this program: operations, class tables,
 * demodulation factors and sub-pulse tables in both precisions, in one image whose tables start
 * on 256-byte boundaries (one allocation, one copy). */
int64_t mrsim_compiled_upload_bytes(const mrsim_compiled *c);
void mrsim_compiled_destroy(mrsim_compiled *c);
/* Uploads a compiled program to ctx's device.  The sequence shares the program's host tables, so
 * c may be destroyed (or uploaded again, to any context) right after the call. */
mrsim_status mrsim_sequence_create(mrsim_ctx *ctx, const mrsim_compiled *c, mrsim_sequence **out);

/* Validates and compiles n_events events (host memory) with γ/2π = gamma_hz_per_t [Hz/T]:
 * gradient moments γ·G·Δt, RF rotation matrices (Eq. 3.19), relaxation intervals and the
 * recurring precession intervals are precomputed in float64 once, as the spin-independent terms
 * of the paper's master process (§6.3).  EINVAL on NaN/Inf fields, Δt < 0, adc not in {0,1},
 * reserved != 0 or gamma <= 0. */
mrsim_status mrsim_sequence_load(mrsim_ctx *ctx, int64_t n_events, const mrsim_event *events,
                                 double gamma_hz_per_t, mrsim_sequence **out);
/* As mrsim_sequence_load, and the program also records every spin's magnetisation after the
 * events snap_after[0..n_snap-1] (strictly increasing indices < n_events): the "magnetisation
 * data at arbitrary times" of §7.2.  The states are written to mrsim_options.snapshots in the
 * rotating (laboratory) frame, with T1 recovery up to the end of the event applied.  The signal is
 * the same as without snapshots. */
mrsim_status mrsim_sequence_load_snapshots(mrsim_ctx *ctx, int64_t n_events, const mrsim_event *events,
                                           double gamma_hz_per_t, int64_t n_snap, const int64_t *snap_after,
                                           mrsim_sequence **out);
/* Snapshots, samples (the length of the signal) and events of the compiled sequence (-1 for NULL). */
int64_t mrsim_sequence_num_snapshots(const mrsim_sequence *s);
int64_t mrsim_sequence_num_adc(const mrsim_sequence *s);
int64_t mrsim_sequence_num_events(const mrsim_sequence *s);
/* Number of compiled device operations (after merging runs of events); for diagnostics. */
int64_t mrsim_sequence_num_ops(const mrsim_sequence *s);
void mrsim_sequence_destroy(mrsim_sequence *s);

/* ---- simulation ----------------------------------------------------------------------- */

/* Forward simulation (§5.1.1): signal_out receives 2*n_adc doubles (re, im per sample), host or
 * device.  n_adc must equal mrsim_sequence_num_adc(seq).  With a device output the call is
 * asynchronous on `stream` (cudaStream_t); with a host output it synchronises. */
mrsim_status mrsim_simulate(mrsim_ctx *ctx, const mrsim_phantom *ph, const mrsim_sequence *seq,
                            mrsim_precision prec, void *stream, double *signal_out, int64_t n_adc);
/* As mrsim_simulate with launch controls, accumulation and state in/out (opt may be NULL).  State
 * in/out lets a long sequence run as consecutive sub-sequences (checkpoint / resume). */
mrsim_status mrsim_simulate_ex(mrsim_ctx *ctx, const mrsim_phantom *ph, const mrsim_sequence *seq,
                               mrsim_precision prec, void *stream, double *signal_out, int64_t n_adc,
                               const mrsim_options *opt);

/* ---- receive coils ------------------------------------------------------------------------- */

/* Signals of n_coils receive coils with inhomogeneous sensitivities.  Eq. 3.25 weights every
 * spin's magnetisation with the coil's receive sensitivity before the superposition (§6.1,
 * "Inhomogenitäten der Empfangssensitivität"; §9 names separate signals per array coil as the
 * wanted extension); for a transverse sensitivity the scalar product is the complex product
 *     signal_c[j] = exp(-j adc_phase_j) · Σ_s C[c][s] · (Mx + jMy)_s(t_j).
 * A homogeneous C = 1 gives mrsim_simulate's signal (§3.5.2).
 *   n_coils:    1..MRSIM_MAX_COILS
 *   sens:       C, n_coils x n_spins complex float64 interleaved (re, im), coil-major; host or
 *               device memory, read during the call (EINVAL if a value is not finite)
 *   signal_out: n_coils x 2*n_adc doubles, coil-major (re, im); host or device
 * Every spin starts in thermal equilibrium.  The rotations are computed once per spin and
 * shared by the coils.  Host output synchronises `stream`; device output is asynchronous. */
#define MRSIM_MAX_COILS 8
mrsim_status mrsim_simulate_coils(mrsim_ctx *ctx, const mrsim_phantom *ph, const mrsim_sequence *seq,
                                  mrsim_precision prec, void *stream, int32_t n_coils, const double *sens,
                                  double *signal_out, int64_t n_adc);

/* ---- K-t formalism: configuration populations of spin ensembles (§4.2) --------------------- */

/* The paper's second simulation method (§4.2; "eigenständige Simulationsmethode"): instead of
 * isochromats, an ensemble is described by the populations a_i of its transverse configurations
 * (orders i = -K..K) and b_i of its longitudinal ones (§4.2.1), M0 = 1, thermal equilibrium at
 * the start.  Each step is one elementary sequence: a hard pulse of flip B1·alpha and phase phi
 * mixes (a_i, a*_-i, b_i) with T'_HF of Eq. 4.2 (Eq. 4.14); over tau the interval's gradient
 * moves the transverse orders by `shift` (Eq. 4.17; populations beyond ±max_order are dropped),
 * relaxation scales a_i by E2 and b_i by E1 and adds 1 - E1 to b_0 (Eqs. 4.15, 4.16), and the
 * ensemble's off-resonance df turns the a_i by exp(-j 2π df tau).  A step with sample = 1
 * records a_0·exp(-j adc_phase), the ensemble's transverse magnetisation.  Many ensembles (e.g.
 * a dictionary over T1, T2, B1, Δf) run in parallel, one warp each. */
typedef struct mrsim_kt_step {
    double alpha;     /* flip angle [rad] before B1 scaling; 0 = no pulse */
    double phi;       /* pulse phase [rad] (Eq. 4.2) */
    double tau;       /* interval after the pulse [s], >= 0 */
    double adc_phase; /* receiver phase [rad] of this step's sample */
    int32_t shift;    /* order shift q of the interval's gradient moment q·Δk, |q| <= 64 */
    int32_t sample;   /* 1 = record a_0 at the end of the step, 0 = no sample */
} mrsim_kt_step;
#define MRSIM_KT_MAX_ORDER 255
/*   n_sets: ensembles; t1, t2 [s] (> 0, INFINITY allowed), b1 (flip scale; NULL = 1) and df
 *           [Hz] (NULL = 0): n_sets float64 each, host or device memory
 *   steps: host array of n_steps; max_order: K, 0..MRSIM_KT_MAX_ORDER
 *   signal_out: n_sets x 2*n_samples doubles (ensemble-major, (re, im)), host or device;
 *           n_samples must equal the number of steps with sample = 1
 * EINVAL for invalid steps or parameters.  Host output synchronises `stream`. */
mrsim_status mrsim_kt_simulate(mrsim_ctx *ctx, int64_t n_sets, const double *t1, const double *t2,
                               const double *b1, const double *df, int64_t n_steps, const mrsim_kt_step *steps,
                               int32_t max_order, mrsim_precision prec, void *stream, double *signal_out,
                               int64_t n_samples);

/* Spatial sampling check for spin-based simulation (§5.2.3): the largest |k| that any
 * configuration of the event list reaches, per axis (Eq. 5.1), in rad/m (k = γ·∫G dt).  A
 * configuration exists from the first pulse on; a pulse can conjugate it (so the moments of
 * consecutive inter-pulse segments add with one sign) or store it longitudinally, so
 * K_max = max over t of Σ|moment of each completed segment| + |moment of the current segment up
 * to t|.  Isochromats must be spaced below Δx_max = π / K_max (Eq. 5.2) along each axis for the
 * discrete spin sum to be free of aliasing; off-resonance spread adds to k and is not included.
 * Host only (no device needed).  EINVAL for invalid events. */
mrsim_status mrsim_max_config_k(int64_t n_events, const mrsim_event *events, double gamma_hz_per_t,
                                double kmax_rad_per_m[3]);

/* ---- batches: many phantoms with their own sequences in one persistent launch ---------- */

/* A batch borrows n phantom/sequence pairs (they must outlive it) and one device signal buffer
 * per pair (2*num_adc doubles each).  The work is split into tiles of spins (the paper's spin
 * blocks, §5.3.2); one persistent kernel, sized to the device (SMs x resident blocks), lets every
 * block pop (phantom, tile) items from a work queue, longest sequences first, until it is empty.
 * Batches of uneven spin counts and sequence lengths therefore keep every SM busy. */
typedef struct mrsim_batch mrsim_batch;
mrsim_status mrsim_batch_create(mrsim_ctx *ctx, int32_t n, const mrsim_phantom *const *phantoms,
                                const mrsim_sequence *const *seqs, mrsim_precision prec,
                                double *const *signals_out, mrsim_batch **out);
/* Work items (phantom, spin tile) of the batch in its current launch shape (-1 for NULL). */
int64_t mrsim_batch_num_items(const mrsim_batch *b);
/* Times every launch shape on the same fraction of every program (about 2e10 spin-steps in all),
 * then the three fastest on about 3e11, and keeps the fastest for this batch; returns it in best
 * (other fields zeroed).  Synchronises `stream`. */
mrsim_status mrsim_batch_autotune(mrsim_batch *b, void *stream, mrsim_options *best);
/* Sets the launch shape explicitly (EINVAL / EUNSUPPORTED as for mrsim_simulate_ex). */
mrsim_status mrsim_batch_set_shape(mrsim_batch *b, int32_t spins_per_thread, int32_t threads_per_block);
/* Enqueues on `stream`: zero the signal buffers, reset the work queue, run the persistent kernel.
 * Asynchronous; may itself be captured into a CUDA graph by the caller. */
mrsim_status mrsim_batch_launch(mrsim_batch *b, void *stream);
/* Same work as one CUDA graph: captured on the first call (and again after the shape changes),
 * replayed on `stream` afterwards. */
mrsim_status mrsim_batch_launch_graph(mrsim_batch *b, void *stream);
void mrsim_batch_destroy(mrsim_batch *b);
/* One-shot convenience: create, launch, synchronise `stream`, destroy. */
mrsim_status mrsim_simulate_batch(mrsim_ctx *ctx, int32_t n, const mrsim_phantom *const *phantoms,
                                  const mrsim_sequence *const *seqs, mrsim_precision prec, void *stream,
                                  double *const *signals_out);

/* ---- differentiation: adjoint (backward-in-time) gradients ---------------------------------- */

/* Gradients of a real loss L of the signal with respect to every spin's M0, T1, T2 and to
 * learnable RF flip angles, by the adjoint recursion through the elementary sequences (Eq. 4.1 is
 * affine in M, so the adjoint runs backward through the transposed steps: Eq. 3.19 rotations and
 * Eq. 3.5 precession/relaxation).  float64 throughout.  The forward pass stores each spin's state
 * every ckpt_every events; the backward pass recomputes the states between checkpoints.
 *   rf_param: NULL or n_events indices; event e's flip angle is rf_values[rf_param[e]] when
 *             rf_param[e] >= 0 (its rf_flip is then ignored), else the event's own rf_flip.
 *   ckpt_every: events per checkpoint segment, 1..128 (0 = 64); storage is
 *             ceil(n_events/ckpt_every) x 3 doubles per spin, allocated by the first forward call. */
typedef struct mrsim_adjoint mrsim_adjoint;
mrsim_status mrsim_adjoint_create(mrsim_ctx *ctx, int64_t n_events, const mrsim_event *events,
                                  double gamma_hz_per_t, const int32_t *rf_param, int32_t n_params,
                                  int32_t ckpt_every, mrsim_adjoint **out);
/* Samples of the adjoint's event list (the length of its signal; -1 for NULL). */
int64_t mrsim_adjoint_num_adc(const mrsim_adjoint *adj);
/* Forward simulation that also stores the checkpoints.  rf_values: device array of n_params flip
 * angles [rad] (may be NULL when n_params = 0); signal_out: device, 2*num_adc doubles.
 * Asynchronous on `stream`. */
mrsim_status mrsim_adjoint_forward(mrsim_adjoint *adj, const mrsim_phantom *ph, const double *rf_values,
                                   void *stream, double *signal_out);
/* Backward pass for the phantom and rf_values of the last forward call.  dl_dsignal: device,
 * 2*num_adc doubles (dL/dRe s_j, dL/dIm s_j).  Outputs (device, NULL to skip): d_rho, d_t1, d_t2
 * (n_spins each; dL/dT = 0 where T = INFINITY) and d_rf (n_params, overwritten).  Asynchronous. */
mrsim_status mrsim_adjoint_backward(mrsim_adjoint *adj, const mrsim_phantom *ph, const double *rf_values,
                                    const double *dl_dsignal, void *stream, double *d_rho, double *d_t1,
                                    double *d_t2, double *d_rf);
/* Arithmetic of the adjoint's forward and backward recursion: MRSIM_FP64 (the default) or
 * MRSIM_FP32_KAHAN, double-float pairs on the FP32 pipe (about 48 significant bits; GB300 runs
 * float64 at 1/64 of its float32 rate); MRSIM_FP32 gives MRSIM_EUNSUPPORTED.  The next forward
 * call recomputes the checkpoints. */
mrsim_status mrsim_adjoint_set_precision(mrsim_adjoint *adj, mrsim_precision prec);
/* Frees the adjoint's device tables and checkpoint storage (NULL is ignored). */
void mrsim_adjoint_destroy(mrsim_adjoint *adj);
/* One-shot gradient of a real loss L of the simulated signal (the same adjoint recursion as
 * mrsim_adjoint_create/forward/backward, Eq. 4.1 run backward through its transposed steps) for a
 * phantom and an already loaded sequence; the paper has no gradients, this differentiates its
 * forward method.  The call creates the adjoint program from the sequence's own event list,
 * runs the checkpointed forward pass with the pulses' own flips and the backward pass, copies
 * the results out and frees everything again, so it synchronises `stream`.
 *   prec:       MRSIM_FP64, or MRSIM_FP32_KAHAN (the recursion in double-float pairs, see
 *               mrsim_adjoint_set_precision); MRSIM_FP32 gives MRSIM_EUNSUPPORTED
 *   ckpt_every: events per checkpoint segment, 1..128 (0 = 64)
 *   dL_dsignal: 2*n_adc doubles (dL/dRe s_j, dL/dIm s_j), host or device
 *   d_rho, d_t1, d_t2: NULL or n_spins doubles each, host or device: dL/dM0, dL/dT1, dL/dT2 of
 *               every spin (dL/dT = 0 where T = INFINITY)
 *   d_rf_flip:  NULL or one double per pulse (event with rf_flip != 0) in event order, host or
 *               device: dL/dα of that pulse's flip angle
 * Needs device memory for the checkpoints (ceil(n_events/ckpt_every) x 3 doubles per spin) and
 * the signal; ENOMEM when it is not available. */
mrsim_status mrsim_simulate_adjoint(mrsim_ctx *ctx, const mrsim_phantom *ph, const mrsim_sequence *seq,
                                    mrsim_precision prec, int32_t ckpt_every, const double *dL_dsignal, void *stream,
                                    double *d_rho, double *d_t1, double *d_t2, double *d_rf_flip);
/* Pulses of a loaded sequence (events with rf_flip != 0): the length of mrsim_simulate_adjoint's
 * d_rf_flip (-1 for NULL). */
int64_t mrsim_sequence_num_pulses(const mrsim_sequence *s);

/* ---- non-parallel fields: local static-field direction, transverse gradient components ---- */

/* The static field at each spin may point along its own unit vector n_s (§3.2: the frame is
 * turned locally so that one axis lies along the static field, the Bloch equation is applied
 * there and the result turned back), and an elementary sequence's gradient field may have
 * components transverse to z (§3.4.3.2: a constant gradient field with transverse components
 * changes the direction of the total field, T1 relaxation follows that direction, and Eqs.
 * 3.14/3.15 hold in the turned frame).  Per spin and event, after the RF pulse of Eq. 3.19
 * (rotating frame, as in mrsim_simulate):
 *     b = (gtx.x, gty.x, G.x),   u = B0*n_s + b,   h = u/|u|
 *     θ = (γ (|u| - B0) + Δω) Δt
 *     M <- E2 (cos θ M⊥ - sin θ h × M⊥) + (E1 (M.h) + M0 (1 - E1)) h,   M⊥ = M - (M.h) h
 * (for n_s = z and no transverse components this is mrsim_simulate's step), and every spin
 * starts in equilibrium along its static field, M = M0 n_s.  Samples as in mrsim_simulate. */

/* Sets the phantom's static-field directions: b0_dir = 3*n_spins doubles (nx, ny, nz) per spin,
 * unit vectors (|n|^2 within 2e-9 of 1, else EINVAL naming the first bad spin), host or device;
 * the phantom keeps a device copy (3 doubles per spin).  A phantom without directions has its
 * field along z.  Synchronises `stream`. */
mrsim_status mrsim_phantom_set_b0_direction(mrsim_phantom *ph, const double *b0_dir, void *stream);
/* An event list prepared for mrsim_simulate_fields (the events are not compiled or merged as for
 * mrsim_simulate: one thread per spin runs every event):
 *   events:       n_events elementary sequences, host memory (validated as for mrsim_sequence_load)
 *   g_transverse: NULL, or 6*n_events doubles, host memory: per event gtx (3) and gty (3) [T/m],
 *                 the transverse field components Bx = gtx.x, By = gty.x during the event
 *   b0_tesla:     |B0| [T] > 0; it must exceed the gradient field at every spin (u != 0)
 * The records (float64 and float32, 192 bytes each per event) are uploaded once.  With the
 * context's train maps on at creation (mrsim_context_set_train_maps), a train (two or more
 * consecutive pulsed events without samples sharing one free interval, up to 256) that recurs at
 * least 4 times with the same pulses and interval runs, per spin, as one map composed at the
 * start of each simulation (double-float; float64 for MRSIM_FP64), which then needs
 * 12 x (map kinds) values per spin of device memory from the context's stream-ordered pool. */
typedef struct mrsim_fields mrsim_fields;
mrsim_status mrsim_fields_create(mrsim_ctx *ctx, int64_t n_events, const mrsim_event *events,
                                 const double *g_transverse, double gamma_hz_per_t, double b0_tesla,
                                 mrsim_fields **out);
/* Samples of the prepared list (the signal's length; -1 for NULL). */
int64_t mrsim_fields_num_adc(const mrsim_fields *f);
/* Train-map kinds of the prepared list (0: every train runs event by event; -1 for NULL). */
int32_t mrsim_fields_num_train_maps(const mrsim_fields *f);
void mrsim_fields_destroy(mrsim_fields *f);
/* Forward simulation with non-parallel fields: signal_out = 2*n_adc doubles, host or device
 * (device output: asynchronous on `stream`; host output synchronises).  float32 keeps the
 * phase's large part in float-float products; its error grows with the square root of the
 * number of events a spin's state carries (about 1e-7 rad per event). */
mrsim_status mrsim_simulate_fields(mrsim_ctx *ctx, const mrsim_phantom *ph, const mrsim_fields *f,
                                   mrsim_precision prec, void *stream, double *signal_out, int64_t n_adc);

/* ---- batches without allocation ---------------------------------------------------------- */

/* The paper has no counterpart: this entry point exists for callers that cannot allocate device
 * memory when they simulate (a plug-in whose host application owns every device allocation, a
 * real-time loop under a fixed memory budget).  It runs the same persistent batch kernel as
 * mrsim_batch_launch for n phantom/sequence pairs (handles created earlier; device signal
 * buffers of 2*num_adc doubles each, zeroed by the call), but allocates nothing: no cudaMalloc,
 * no cudaFree, no allocating library routine.  Its scratch (work-queue counter, per-phantom
 * descriptors, work items) is one file-scope device array of MRSIM_STATIC_SCRATCH_BYTES that
 * every GPU which loads the library holds until the process exits; the work list is staged
 * through a host buffer of the same size.  Limits: at most
 * (MRSIM_STATIC_SCRATCH_BYTES - 256) / sizeof(descriptor) phantoms and as many work items
 * (tiles of spins_per_thread x threads_per_block spins, 8 bytes each) as fit after them;
 * larger batches fail with MRSIM_EINVAL and a message saying which limit was hit.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress); with
 * lazy module loading (the CUDA default) that is also when the library's device code is loaded
 * on that device and the array is reserved there, i.e. the first call does take device memory
 * implicitly.  Make that first call at initialisation, e.g. with n = 0 (which does only this
 * set-up).  Every call shares the one array, which keeps the
 * last call's contents: calls whose work overlaps on the GPU (other streams, other host threads'
 * launches still running) race on it and must be serialised by the caller; host threads are
 * serialised inside the call.  spins_per_thread / threads_per_block: 0 = library default (which,
 * as in mrsim_batch_create, falls back to 1 x 64 and then 1 x 32 when it does not fit).  The
 * caller's current device is the same after the call as before it.  Train maps need device
 * memory per spin, so this call runs every shaped pulse sub-pulse by sub-pulse, as
 * mrsim_batch_launch does with maps switched off (mrsim_context_set_train_maps); with maps on, the
 * two differ by the rounding the maps remove, within the float32 tolerance.
 * Asynchronous on `stream`; errors of the kernel surface through mrsim_stream_status. */
#define MRSIM_STATIC_SCRATCH_BYTES (1u << 20)
mrsim_status mrsim_simulate_batch_static(mrsim_ctx *ctx, int32_t n, const mrsim_phantom *const *phantoms,
                                         const mrsim_sequence *const *seqs, mrsim_precision prec,
                                         void *stream, double *const *signals_out,
                                         int32_t spins_per_thread, int32_t threads_per_block);

/* ---- diagnostics ---------------------------------------------------------------------- */

/* Measured arithmetic rate of the device (the denominator of a roofline fraction for code bound
 * by an arithmetic pipe rather than by memory).  Launches, on `stream`, a kernel that fills every
 * SM (8 blocks of 256 threads per SM) in which every thread runs 8 independent fused
 * multiply-add chains with no memory traffic, once to calibrate and once sized to last about
 * target_ms (1 .. 1e4), and times the second launch with CUDA events:
 *   kind 0: float32 fmaf;  kind 1: float32 pairs, fma.rn.f32x2 (two lanes per instruction);
 *   kind 2: float64 fma.
 * *lane_ops_per_s receives the multiply-adds per second (one per lane, a pair counts two) at the
 * clock the device ran at; *kernel_ms (may be NULL) the timed launch's duration.  Synchronises
 * `stream`.  EINVAL for another kind or target. */
mrsim_status mrsim_measure_fma_rate(mrsim_ctx *ctx, int32_t kind, double target_ms, void *stream,
                                    double *lane_ops_per_s, double *kernel_ms);

/* Host-only compile of an event list (no device needed), for inspecting and testing the
 * sequence compiler.  On input each n_* field is the capacity of the matching array (ignored when
 * the pointer is NULL); on output it is the size the program needs.  Call once with NULL arrays
 * to get the sizes, then again with arrays of those sizes.  Same validation and error codes as
 * mrsim_sequence_load; EINVAL if a given array is too small. */
typedef struct mrsim_program_dump {
    void *ops;      /* float64 device operations, 128-byte records */
    int64_t n_ops;
    double *pcls;   /* 4 per precession class: kx, ky, kz [cycles/m], Δt [s] */
    int32_t n_pcls;
    int32_t n_e1;
    double *e1;     /* interval [s] per T1 class */
    double *e2;     /* interval [s] per T2 class */
    int32_t n_e2;
    int32_t n_train;
    double *train;  /* 2 per sub-pulse table entry: cos α, sin α */
    double *demod;  /* 2 per sample: the factor each sample's spin sum is multiplied by */
    int64_t n_adc;
} mrsim_program_dump;
mrsim_status mrsim_debug_compile(int64_t n_events, const mrsim_event *events, double gamma_hz_per_t,
                                 mrsim_program_dump *dump);
/* mrsim_debug_compile for a program with snapshots (as mrsim_sequence_load_snapshots). */
mrsim_status mrsim_debug_compile_snapshots(int64_t n_events, const mrsim_event *events, double gamma_hz_per_t,
                                           int64_t n_snap, const int64_t *snap_after, mrsim_program_dump *dump);

/* Autotuner: times every launch shape (spins per thread x threads per block) that fits the device
 * on a prefix of the compiled program (about 3e9 spin-steps, at least 256 operations) on `stream`,
 * and keeps the fastest in the context, keyed by precision, spin count and the compiled program's
 * size and class tables; later mrsim_simulate / mrsim_simulate_ex calls without an explicit shape
 * on any phantom/sequence with the same key use it.  Returns the shape in
 * best->spins_per_thread / best->threads_per_block (other fields zeroed).  Synchronises `stream`.
 * A key the context already holds is answered without timing.  With the environment variable
 * MRSIM_AUTOTUNE_CACHE naming a file, contexts load the shapes tuned on a device with the same SM
 * count from it when they are created and append every new one, so other processes skip the
 * timing. */
mrsim_status mrsim_autotune(mrsim_ctx *ctx, const mrsim_phantom *ph, const mrsim_sequence *seq,
                            mrsim_precision prec, void *stream, mrsim_options *best);

#ifdef __cplusplus
}
#endif
#endif /* MRSIM_H */
