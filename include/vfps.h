/*
 * vfps.h -- C ABI of the B300 (sm_103a) Vlasov-Fokker-Planck phase-space stepper.
 *
 * The library advances the longitudinal phase-space density psi(q, p) of an
 * electron bunch by time steps of the normalised Vlasov-Fokker-Planck
 * equation (Schoenfeldt et al., "A Parallelized Vlasov-Fokker-Planck-Solver
 * for Desktop PCs", Sec. II.A, Eq. VFP):
 *
 *     d psi/d theta + dH/dp d psi/dq - dH/dq d psi/dp = beta d/dp (p psi + d psi/dp),
 *     H = (q^2 + p^2)/2 + collective term,  beta = 1/(f_s tau_d).
 *
 * One time step is (Sec. III.B: f = f_rot + f_kick + f_damp,diff):
 *   1. bunch profile rho(q) = int psi dp and charge                 (Sec. II.B)
 *   2. wake V(q) = int Z(k) rho~(k) e^{ikq} dk by FFT, and the CSR
 *      power P = dkappa sum 2 Re(Z_k) |rho~_k|^2                     (Eq. wakepotential, Sec. IV.C)
 *   3. RotationMap: semi-Lagrangian rotation by 2 pi/steps_per_period
 *      with 2-D Lagrange interpolation on N_I x N_I nodes            (Sec. III.A-B)
 *   4. WakeKickMap: 1-D interpolated shift of each q column along p
 *      by dp = +S_csr V(q) * 2 pi/steps_per_period                   (Sec. III.B)
 *   5. FokkerPlanckMap: explicit step of beta (psi + p psi' + psi'')
 *      with the cubic derivative of Eq. cubic diff                   (Sec. III.B)
 *   6. renormalisation of the charge to 1 (not in the paper; optional)
 *
 * Grid: q_i = -L + i*Delta, p_j = -L + j*Delta, Delta = 2L/(n-1), i, j = 0..n-1.
 * psi is exchanged as n*n row-major doubles, index [i*n + j] = psi(q_i, p_j)
 * (p contiguous; the paper's flattened index z = N_y x + y, Sec. III.B).
 *
 * Conventions of every call:
 *  - returns 0 (VFPS_OK) or a negative VFPS_E* code; nothing else escapes;
 *  - host pointers are read or written before the call returns and stay
 *    owned by the caller; the library owns every device allocation;
 *  - a handle is not thread-safe; work is queued on the handle's stream;
 *  - calls that return data to the host synchronise that stream; state,
 *    status and series move through a pinned staging buffer of the calling
 *    thread (grown to the largest transfer, freed when the thread ends).
 */
#ifndef VFPS_H
#define VFPS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define VFPS_OK 0
#define VFPS_EINVAL (-1)   /* bad argument or parameter combination          */
#define VFPS_ENOMEM (-2)   /* device or host allocation failed               */
#define VFPS_ECUDA (-3)    /* a CUDA runtime call failed                     */
#define VFPS_ETIMEOUT (-4) /* a bounded device wait ran out                  */
#define VFPS_ENAN (-5)     /* non-finite or non-positive charge detected     */
#define VFPS_EBUSY (-6)    /* capacity exhausted (batch slots, HBM budget)   */
#define VFPS_EBOUNDS (-7)  /* debug build (VFPS_DEBUG) only: a shared-memory
                              index check failed; the site is named in
                              vfps_last_cuda_error()                         */
#define VFPS_ECONVERGE (-8) /* an iterative solve did not reach its tolerance  */

#define VFPS_IMPEDANCE_NONE 0            /* no collective effect                      */
#define VFPS_IMPEDANCE_FREE_SPACE 1      /* CSR in free space (Sec. II.B)             */
#define VFPS_IMPEDANCE_PARALLEL_PLATES 2 /* CSR shielded by parallel plates (Sec. II.B) */
#define VFPS_IMPEDANCE_TABLE 3           /* caller-supplied table                     */

typedef struct vfps_params {
    int32_t n;                /* grid points per axis, 8..2048                            */
    int32_t steps_per_period; /* time steps per synchrotron period, >= 2                  */
    int32_t interp_points;    /* N_I in {2, 3, 4}; 4 = cubic (default)                    */
    int32_t clamp;            /* 1: clamped interpolation (Eq. clamping); default 0       */
    int32_t fp_derivative;    /* 1: cubic derivative of Eq. cubic diff (default);
                                 0: central difference                                    */
    int32_t pad_factor;       /* zero padding: FFT length M = smallest power of two
                                 >= pad_factor*n; 2..64, pad_factor*n <= 16384; default 2 */
    int32_t precision;        /* 0: FP32 psi and column sums, FP64 charge and power sums (default); 1: FP64 throughout */
    int32_t renormalize;      /* 1: rescale the charge to 1 after every step (default)    */
    int32_t rotation;         /* 0: standard rotation (default); 1: Manhattan rotation of
                                 Sec. III.B: drift q -> q + h p, then RF kick p -> p - h q,
                                 each a 1-D interpolation, h = 2 sin(pi/steps_per_period)
                                 so that one period is exactly one turn                   */
    double half_width;        /* L: q, p in [-L, L]; default 6                            */
    double beta;              /* 1/(f_s tau_d) >= 0 (Eq. VFP); default 0                  */
} vfps_params;

typedef struct vfps_handle vfps_handle;

/* Fill *p with the defaults listed above (n = 256, steps_per_period = 1000). */
void vfps_params_default(vfps_params* p);

/* Create one simulation.
 *   psi0:  host, n*n doubles, [q][p] row-major, finite, with positive total
 *          charge; NULL = the unit Gaussian exp(-(q^2+p^2)/2).  The library
 *          normalises it to charge Delta^2 sum psi = 1 before upload.
 *   cuda_stream: a cudaStream_t to queue work on, or NULL for a library-owned
 *          stream.
 * The impedance starts as VFPS_IMPEDANCE_NONE with S_csr = 0.
 * Errors: EINVAL (parameters out of range, non-finite psi0 or charge <= 0),
 * ENOMEM, ECUDA. */
int vfps_create(const vfps_params* params, const double* psi0, void* cuda_stream,
                vfps_handle** out);

/* Select the collective wake (Sec. II.B) and its strength.
 *   model: VFPS_IMPEDANCE_*;  Pi: shielding parameter R^(1/2) sigma_z / h^(3/2)
 *          of parallel plates at +-h (model 2, > 0; the bursting threshold
 *          is near S_csr = 0.5 + 0.12 Pi);
 *   S_csr: normalised bunch current I_n R^(1/3) / sigma_z^(4/3) (any sign);
 *   table_re_im: model 3 only, host, (M/2+1) interleaved (re, im) doubles of
 *          the dimensionless impedance at kappa_k = 2 pi k/(M Delta).
 * The impedance is tabulated on the host in FP64 once per call.  Recomputes
 * the wake of the current state.  Errors: EINVAL, ECUDA. */
int vfps_set_impedance(vfps_handle* h, int model, double Pi, double S_csr,
                       const double* table_re_im);

/* Advance by nsteps >= 0 time steps (asynchronous on the handle's stream).
 * A simulation on the FP32 register-blocked kernel whose CTAs, plus one,
 * fit on the device at once steps in persistent cooperative launches of up
 * to 256 steps (vfps_step_mode): worker CTAs and one finaliser CTA meet on
 * two counters of the state word, so the wake transform of one step runs
 * while the workers load and rotate the next; the results are the same bits
 * as one launch per step.  Every device wait of such a launch is bounded
 * (VFPS_SPIN_LIMIT polls, about a second by default); a wait that runs out
 * ends the launch with status ETIMEOUT, after which the simulation's state
 * is undefined (destroy the handle; the CUDA context stays usable).
 * VFPS_PERSISTENT=0 in the environment at vfps_create keeps one launch per
 * step.
 * Errors: EINVAL, ECUDA, ENAN and ETIMEOUT (reported by the next
 * synchronising call). */
int vfps_step(vfps_handle* h, int64_t nsteps);

/* *persistent = 1 when vfps_step runs this simulation in persistent
 * launches, 0 when it launches one kernel (or CUDA graph node) per step.
 * Errors: EINVAL. */
int vfps_step_mode(vfps_handle* h, int32_t* persistent);

/* rho_out (host, n doubles): profile rho(q_i) = Delta sum_j psi_ij of the
 * current state.  Synchronises.  Errors: EINVAL, ECUDA, ENAN. */
int vfps_profile(vfps_handle* h, double* rho_out);

/* out (host, 4 doubles): bunch moments of the current state, computed on the
 * device -- {<q>, sigma_q, <p>, sigma_p} with <f> = sum f psi / sum psi over
 * the nodes (the bunch length and energy spread the paper plots, in units of
 * the natural sigma_z and sigma_delta).  One extra read of psi; FP32 (or FP64)
 * partials, FP64 sums.  Synchronises.  Errors: EINVAL, ECUDA, ENAN. */
int vfps_moments(vfps_handle* h, double* out);

/* out (host, length/2 + 1 doubles): power spectrum of the last `length` values
 * of the CSR-power series (one row of the paper's bursting spectrogram,
 * Sec. IV.C), computed on the device: mean removed, Hann window
 * (1 - cos(2 pi j/length))/2, out[k] = |sum_j ... exp(-2 pi i j k/length)|^2;
 * bin k is k steps_per_period/length cycles per synchrotron period.  length:
 * power of two, 16..8192, at most the steps done and at most the ring size
 * minus one (the series is read from the device ring, so it need not have been
 * drained).  FP32 transform of FP64-centred values.  Synchronises.  Errors:
 * EINVAL, ECUDA, ENAN. */
int vfps_power_spectrum(vfps_handle* h, int32_t length, double* out);

/* Record the bunch moments of the state every `every` steps (0: stop) as part
 * of the step itself: on a recording step the step kernel also sums p psi and
 * p^2 psi per column of the state it writes (FP32 lane partials, FP64 across
 * lanes), and the finaliser forms {<q>, sigma_q, <p>, sigma_p} of that state
 * (Sec. IV's bunch length and energy spread; <f> = sum f psi / sum psi over
 * the nodes, as vfps_moments) in FP64 from those sums and the column sums the
 * wake already needs -- no extra pass over psi.  States t >= 1 produced by
 * later steps with t a multiple of `every` are recorded; the records move to
 * the host with the CSR-power series.  A device ring of 32 bytes per ring
 * entry is allocated on first use.  Synchronises (draining what was
 * recorded so far).  Errors: EINVAL, ENOMEM, ECUDA. */
int vfps_record_moments(vfps_handle* h, int32_t every);

/* Drain the recorded moments: up to cap records of five doubles
 * {t, <q>, sigma_q, <p>, sigma_p}, oldest first; *n_written gets the
 * number of records.  Synchronises.  Errors: EINVAL, ECUDA, ENAN. */
int vfps_moment_series(vfps_handle* h, double* out, int64_t cap, int64_t* n_written);

/* Bursting spectrogram of the CSR-power series (Sec. IV.C: the Fourier
 * transform of P(t) over successive windows), on the device: `count` windows
 * of `length` values, `hop` steps apart, the last one ending at the newest
 * entry of the series; each window as vfps_power_spectrum (mean removed,
 * Hann window).  out (host): count x (length/2 + 1) doubles, oldest window
 * first.  length: power of two, 16..8192; hop >= 1; the span length + (count
 * - 1) hop at most the steps done and at most the ring size minus one.  One
 * launch, one CTA per window.  Synchronises.  Errors: EINVAL, ECUDA, ENAN. */
int vfps_spectrogram(vfps_handle* h, int32_t length, int32_t hop, int32_t count, double* out);

/* Drain the CSR-power series: out[k] = P(psi_t) for the steps t taken since
 * the last drain, oldest first (P of the state each step started from).
 * Writes min(cap, pending) values and *n_written; values beyond cap stay
 * queued.  Synchronises.  Errors: EINVAL, ECUDA, ENAN. */
int vfps_csr_power(vfps_handle* h, double* out, int64_t cap, int64_t* n_written);

/* Drain the series of the charge before renormalisation (one per step, same
 * order and rules as vfps_csr_power): the per-step charge leakage. */
int vfps_charge_series(vfps_handle* h, double* out, int64_t cap, int64_t* n_written);

/* Copy the current psi (normalised, n*n doubles) to host memory.  Synchronises. */
int vfps_get_state(vfps_handle* h, double* psi_out);

/* Replace psi by host psi (n*n doubles, normalised to charge 1 by the
 * library) and recompute its wake; the step counter is kept.  Errors: EINVAL. */
int vfps_set_state(vfps_handle* h, const double* psi);

/* Checkpoint and resume (the paper restarts runs from result files, Sec.
 * IV.C "adiabatic" scans; App. B option -i).  A checkpoint is the state
 * exactly as the device holds it between two steps -- the stored psi with its
 * pending renormalisation factor, the step count, the kick table and profile
 * of the next step, and the CSR power and charge of the current step -- so a
 * run resumed from it continues with the same bits as the uninterrupted run
 * (vfps_set_state, in contrast, takes a normalised psi and recomputes the
 * rest, which agrees only to rounding).  The loading handle must have been
 * created with the same parameters and impedance (model, Pi, S_csr);
 * anything else is refused with EINVAL.  After a load the step counter is the
 * checkpoint's and the series start again at that step.  buf: host memory of
 * at least vfps_checkpoint_bytes bytes, owned by the caller (raw bytes of this
 * library build; not a portable file format).  Both synchronise.
 * Errors: EINVAL, ECUDA, ENAN (the saved state had a bad charge). */
int vfps_checkpoint_bytes(vfps_handle* h, int64_t* bytes);
int vfps_save_checkpoint(vfps_handle* h, void* buf, int64_t bytes);
int vfps_load_checkpoint(vfps_handle* h, const void* buf, int64_t bytes);

/* Haissinski start (Appendix A names the equilibrium; Sec. II.B gives the
 * wake): replace the current state by psi = rho_H(q) g(p), with g the unit
 * Gaussian in p and rho_H the profile that solves
 *   rho(q) = A exp(-q^2/2 + S_csr int_{-L}^{q} V[rho] dq'),  Delta sum rho = 1,
 * for the simulation's own grid, impedance (set it first) and S_csr, V the
 * wake potential of the step (same FFT length and impedance table).  The
 * damped fixed-point iteration rho <- (rho + new)/2 from the unit Gaussian
 * runs on the device in FP64 (trapezoid rule for the integral) until
 * max|new - rho| < tol max rho, at most max_iter times; *iterations (may be
 * NULL) gets the count.  Below the instability threshold the run then starts
 * at equilibrium.  Synchronises.  Errors: EINVAL (tol <= 0, max_iter < 1,
 * shared memory), ECONVERGE (not converged; the state is unchanged), ECUDA. */
int vfps_haissinski(vfps_handle* h, double tol, int32_t max_iter, int32_t* iterations);

/* Number of steps taken so far. */
int vfps_steps_done(vfps_handle* h, int64_t* steps);

/* Free every resource of the handle (NULL is accepted). */
int vfps_destroy(vfps_handle* h);

/* Static description of an error code. */
const char* vfps_strerror(int code);

/* The calling thread's last failing CUDA call and its message, or the reason
 * vfps_step_static refused a request ("" if none); valid until that thread's
 * next library call. */
const char* vfps_last_cuda_error(void);

/* Host-only (needs no device): the library's FP64 impedance table for a grid,
 * the values vfps_set_impedance uploads.  out_re_im: (M/2+1) interleaved
 * (re, im) doubles at kappa_k = 2 pi k/(M Delta), M = pad_factor*n.
 * model: VFPS_IMPEDANCE_NONE, _FREE_SPACE or _PARALLEL_PLATES (Pi > 0).
 * Errors: EINVAL. */
int vfps_impedance_table(int model, int32_t n, double half_width, int32_t pad_factor,
                         double Pi, double* out_re_im);

/* One step without allocating device memory.  The paper has no counterpart:
 * this exists for callers that may not call cudaMalloc -- a plug-in inside an
 * application whose memory pool owns the device (allocating behind the pool
 * can fail or fragment it), or a latency-critical loop that cannot take
 * cudaMalloc's implicit synchronisation and failure path.
 *   psi_in:  device, n*n FP32 [q][p] row-major (any positive charge);
 *   psi_out: device, n*n FP32, distinct from psi_in; receives the next state
 *            normalised to charge 1 (as vfps_step with renormalize = 1; the
 *            renormalize field of params is not used);
 *            both 16-byte aligned when n is a multiple of 4;
 *   model, Pi, S_csr: as in vfps_set_impedance (models 0-2);
 *   power_out: host, NULL or one double: P(psi_in); when given, the call
 *            synchronises the stream and also reports VFPS_ENAN;
 *   cuda_stream: the stream to queue on (NULL = legacy default stream).
 * Only precision = 0.  Limits: n <= 1024 and FFT length <= 4096; larger
 * requests return VFPS_EINVAL with the reason in vfps_last_cuda_error().
 * Scratch lives in a fixed device array of about 80 KB inside the library
 * image (held by every GPU that loads the library until exit), looked up on
 * the first call on each device.  All calls share that array; calls whose
 * work overlaps on the GPU (other streams or host threads) race on it.  Host-side tables
 * (impedance, twiddles) use ordinary host memory. */
int vfps_step_static(const vfps_params* params, int model, double Pi, double S_csr,
                     const float* psi_in, float* psi_out, double* power_out, void* cuda_stream);

/* ---------------------------------------------------------------------------
 * Batch: many independent simulations of possibly different grid sizes that
 * advance together, one fused kernel launch per grid-size class per step.
 * Each slot behaves exactly like a handle with the same parameters: its
 * results do not depend on the other slots (no floating-point atomics; fixed
 * reduction order per slot).
 * ------------------------------------------------------------------------- */
typedef struct vfps_batch vfps_batch;

/* max_slots: slot capacity (>= 1).  budget_bytes: device-memory cap for the
 * slots' state (0 = no cap; admission also checks the free device memory).
 * cuda_stream: as in vfps_create.  Errors: EINVAL, ENOMEM, ECUDA. */
int vfps_batch_create(int32_t max_slots, int64_t budget_bytes, void* cuda_stream,
                      vfps_batch** out);

/* Add a simulation that will run nsteps steps.  Arguments as in vfps_create
 * and vfps_set_impedance.  *slot receives its id.
 * Errors: EINVAL, EBUSY (no free slot or over the memory budget), ENOMEM. */
int vfps_batch_add(vfps_batch* b, const vfps_params* params, const double* psi0,
                   int model, double Pi, double S_csr, const double* table_re_im,
                   int64_t nsteps, int32_t* slot);

/* Add `count` simulations of one set of parameters at once (a scan): one
 * host-to-device copy of all starting states, their charges summed and their
 * values normalised and converted on the device, then each slot's impedance
 * and wake -- the same states, bit for bit, as `count` vfps_batch_add calls.
 *   psi0: host, count consecutive n*n row-major states (NULL: unit
 *         Gaussians); pinned memory makes the copy run at link speed;
 *   model: 0, 1 or 2 for every slot; Pi, S_csr: host, count values each;
 *   slots: host, receives the count slot ids.
 * The slots share one device allocation, returned when the last of them is
 * removed (each slot's bytes still leave the budget when it is removed).
 * All or nothing: on any error no slot is added.  Errors: EINVAL (a
 * non-finite value or non-positive charge in any state, bad arguments),
 * EBUSY (free slots or memory budget), ENOMEM, ECUDA. */
int vfps_batch_add_many(vfps_batch* b, int32_t count, const vfps_params* params, const double* psi0,
                        int model, const double* Pi, const double* S_csr, int64_t nsteps, int32_t* slots);

/* Results of `count` slots at once: psi_out (host, may be NULL) receives the
 * states back to back (n*n doubles each, in the order of `slots`), gathered
 * and converted on the device and copied to the host in one transfer;
 * power_out (host, may be NULL) row i (power_cap doubles) receives slot i's
 * CSR-power series so far (as vfps_batch_take), n_power[i] its length.
 * Synchronises.  Errors: EINVAL, ECUDA, ENAN. */
int vfps_batch_take_many(vfps_batch* b, int32_t count, const int32_t* slots, double* psi_out,
                         double* power_out, int64_t power_cap, int64_t* n_power);

/* Bytes of device memory a slot with these parameters needs (for admission). */
int64_t vfps_batch_slot_bytes(const vfps_params* params);

/* Advance every unfinished slot by up to chunk_steps steps (asynchronous).
 * A slot stops exactly at its own nsteps. */
int vfps_batch_run(vfps_batch* b, int64_t chunk_steps);

/* Without blocking: *idle = 1 if every step and set-up queued on the batch
 * so far has finished on the device, else 0 (a serving loop polls this while
 * it admits arrivals; vfps_batch_add queues a new slot's set-up on its own
 * stream and never waits for the chunk in flight).  Errors: EINVAL, ECUDA. */
int vfps_batch_idle(vfps_batch* b, int32_t* idle);

/* Synchronise; list the finished slots not yet removed.  Writes up to cap ids. */
int vfps_batch_poll(vfps_batch* b, int32_t* done_slots, int32_t cap, int32_t* n_done);

/* Results of one slot (finished or not): psi_out (n*n, may be NULL), rho_out
 * (n, may be NULL), CSR-power series (all steps so far, up to power_cap
 * values, may be NULL), *n_power, *steps_done.  Synchronises. */
int vfps_batch_take(vfps_batch* b, int32_t slot, double* psi_out, double* rho_out,
                    double* power_out, int64_t power_cap, int64_t* n_power,
                    int64_t* steps_done);

/* out (host, 4 doubles): bunch moments of slot's current state, as
 * vfps_moments.  Synchronises the batch.  Errors: EINVAL, ECUDA, ENAN. */
int vfps_batch_moments(vfps_batch* b, int32_t slot, double* out);

/* out (host, length/2 + 1 doubles): vfps_power_spectrum of a slot.  Errors:
 * EINVAL, ECUDA, ENAN. */
int vfps_batch_power_spectrum(vfps_batch* b, int32_t slot, int32_t length, double* out);

/* vfps_record_moments for one slot (the slot leaves the pair kernel while it
 * records; its ring counts toward the batch's memory budget).  Errors as
 * vfps_record_moments. */
int vfps_batch_record_moments(vfps_batch* b, int32_t slot, int32_t every);

/* The slot's moment records so far (five doubles each, as
 * vfps_moment_series), up to cap, without consuming them.  Synchronises. */
int vfps_batch_moment_series(vfps_batch* b, int32_t slot, double* out, int64_t cap, int64_t* n_written);

/* vfps_spectrogram of several slots in one launch: out (host) holds nslots x
 * count x (length/2 + 1) doubles, slot-major in the order of `slots`.  Every
 * slot must have the span of steps.  Errors: EINVAL, ECUDA, ENAN. */
int vfps_batch_spectrogram(vfps_batch* b, const int32_t* slots, int32_t nslots, int32_t length, int32_t hop,
                           int32_t count, double* out);

/* Autotuner of the batch's FP32 launch groups (on = 1, the default; 0 keeps
 * the built-in rules).  For a group of a configuration not seen before in the
 * process -- key: n, precision, rotation, pairing, steps per period, group
 * size rounded up to a power of two -- the first steps of vfps_batch_run time
 * the candidate CTA widths W in {8, 4, 2} with strip lengths (1..32 tiles per
 * CTA) and with the balanced grid (one resident wave of CTAs, each taking an
 * equal run of the group's tiles), 16 back-to-back steps each after 16
 * warm-up steps, and keep the fastest for the rest of the process (a run
 * shorter than the tuning keeps tuning on its next call).  The timed steps
 * are ordinary steps: every candidate gives the same bits.  Setting
 * VFPS_AUTOTUNE=0 in the environment disables it everywhere.
 * Errors: EINVAL. */
int vfps_batch_autotune(vfps_batch* b, int32_t on);

/* Current launch groups of the batch: for each group, six int32 in out --
 * grid size n, instances, CTA width W, tiles per CTA strip (-1: balanced
 * grid), 1 if its shape is
 * final (tuned or fixed) or 0 while the autotuner is still timing it, 1 if
 * its CTAs advance pairs of simulations (see vfps_batch_pairing).  At most
 * cap groups; *n_groups gets the number written.  Errors: EINVAL, ENOMEM,
 * ECUDA. */
int vfps_batch_shapes(vfps_batch* b, int32_t* out, int32_t cap, int32_t* n_groups);

/* Pairing of simulations (on = 1; off, 0, is the default).  FP32
 * simulations of the standard rotation with cubic interpolation, no clamp,
 * n a multiple of 32, and equal grid, steps per period, damping, half width
 * and derivative rule share the rotation map and Fokker-Planck weights of
 * Sec. III; the batch runs them two at a time in one kernel that computes
 * both with packed FP32x2 arithmetic: about 40 % fewer instructions per cell,
 * at twice the registers and shared memory per warp (half the resident warps
 * of the single-simulation kernel).  Results are the same bits as unpaired
 * (up to the sign of zeros).  Takes effect at the next vfps_batch_run.
 * Errors: EINVAL. */
int vfps_batch_pairing(vfps_batch* b, int32_t on);

/* Fix the launch shape of the batch's FP32 groups: CTA width W (2, 4 or 8)
 * and tps tiles per CTA strip (1..256), or tps = -1 for the balanced grid,
 * instead of the autotuner's or the built-in choice, for groups where it fits
 * (shared memory, tps dividing the tiles per instance); W = tps = 0 releases
 * it.  Results do not depend on the shape.  Errors: EINVAL. */
int vfps_batch_pin_shape(vfps_batch* b, int32_t W, int32_t tps);

/* vfps_haissinski for one batch slot (before or between vfps_batch_run
 * calls).  Errors as vfps_haissinski. */
int vfps_batch_haissinski(vfps_batch* b, int32_t slot, double tol, int32_t max_iter, int32_t* iterations);

/* Free a slot (its memory returns to the budget). */
int vfps_batch_remove(vfps_batch* b, int32_t slot);

/* Kernel launches one batch step takes for the current set of unfinished
 * slots (one per launch group: precision, interpolation order, CTA width,
 * grid size; large groups are split in two to overlap their tails). */
int vfps_batch_launches_per_step(vfps_batch* b, int32_t* launches);

/* Number of active slots and device bytes they hold. */
int vfps_batch_usage(vfps_batch* b, int32_t* active, int64_t* bytes);

int vfps_batch_destroy(vfps_batch* b);

#ifdef __cplusplus
}
#endif
#endif /* VFPS_H */
