/*
 * spintrack -- spin-orbit tracking of a particle ensemble through a ring
 * lattice on one NVIDIA B300 (sm_103a).
 *
 * The tracked method is that of Abell, Meiser, Ranjbar, Barber, "Accurate and
 * efficient spin integration for particle accelerators" (arXiv:1501.03450):
 *   - orbit in the canonical variables z = (X, Px, Y, Py, T, Pt) of Sec. 2.1,
 *     Eqs. (1)-(3): X, Y, T in metres, Px, Py, Pt scaled by the reference
 *     momentum p0 (Pt by p0 c);
 *   - exact sector bends ("bend-kick", Sec. 3.1, Eq. (10)), matrix-kick
 *     quadrupoles (Sec. 3.3, Eqs. (21)-(27)), drift-kick-drift multipoles
 *     (Sec. 3.4, Eqs. (28)-(29)), exact drifts, thin Siberian snakes (Sec. 5);
 *   - spin precession from the Thomas-BMT equation in s (Sec. 2.2, Eq. (6b)),
 *     integrated per element by trapezoid-weighted edge rotations composed as
 *     unit quaternions, later slices on the left (Sec. 4.1, Eq. (37)), at the
 *     2^k sub-sampled step sizes of Eq. (38), extrapolated with the Romberg
 *     table of Eq. (39) and normalised per element (Sec. 4.3); or, for the
 *     comparisons of Sec. 5.3, piece-wise constant rotations with the
 *     precession vector at the middle of each slice (ST_SPIN_MID_HALF,
 *     ST_SPIN_MID_KICK below).
 *
 * Conventions of this library (the paper leaves them open):
 *   - quaternions are Hamilton, scalar first; the spin is rotated actively;
 *   - "spin_order" k is the number of Romberg iterations (result Q_kk);
 *   - the drift-kick-drift slice is half drift, kick, half drift; slice edges
 *     are the states between slices, edge 0 the element entrance;
 *   - particle gamma = gamma0 (1 + beta0 Pt) enters Eq. (6b);
 *   - a particle whose longitudinal momentum becomes imaginary is lost: its
 *     state is frozen at the entrance of that element and its lost flag set.
 *
 * All functions return ST_OK (0) or a negative error code; st_last_error()
 * gives a message for the calling thread.  No function throws.  One process,
 * one GPU; the library owns every device buffer it allocates.
 */
#ifndef SPINTRACK_H
#define SPINTRACK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---------------------------------------------------- */
#define ST_OK        0
#define ST_EINVAL   -1   /* invalid argument or lattice                          */
#define ST_ENOMEM   -2   /* device or host allocation failed                     */
#define ST_ECUDA    -3   /* CUDA runtime error (message in st_last_error)        */
#define ST_ETIMEOUT -4   /* a bounded device-side wait gave up (status word set) */
#define ST_ESTATE   -5   /* call out of order (e.g. track before upload)         */

/* ---- element kinds --------------------------------------------------- */
#define ST_DRIFT    0   /* exact drift, flow of H_drift (Eq. (29b)); no spin step      */
#define ST_MULT     1   /* normal quadrupole k1 + sextupole k2, drift-kick-drift slices
                           (Sec. 3.4); field b = (k1 Y + k2 X Y, k1 X + k2 (X^2-Y^2)/2)  */
#define ST_QUAD_MK  2   /* quadrupole k1, matrix-kick slices H_qL/2 H_qNL H_qL/2 (Eq. (27)) */
#define ST_SBEND    3   /* sector bend of curvature h = angle/L and field ratio eta
                           (Eq. (9)), exact map Eq. (10) per slice                       */
#define ST_SNAKE    4   /* thin, orbit-transparent spin rotation by snake_mu about the
                           horizontal axis (sin snake_phi, 0, cos snake_phi)            */
#define ST_SOLENOID 5   /* solenoid of body field k1 = b0/(B rho) (MAD ks), Sec. 3.7:
                           exact body map (Eq. (solenoid)) in n_slices slices, the
                           velocity taken along the kinetic momentum (Eq. (mgVSol)),
                           and thin-pancake fringes at both ends with the spin kicks of
                           Eq. (solFringe) (orbit unchanged across a fringe).  FP64
                           and mixed precision, single contexts and batches.          */

#define ST_RBEND    6   /* rectangular bend, Sec. 3.2: L = magnet length along its
                           Cartesian axis, angle = total bend, eta = field factor, e1 =
                           face asymmetry (the beam meets the entrance face at
                           angle/2 + e1 and the exit face at -angle/2 + e1).  Dynamic
                           rotations into and out of the magnet frame (Eq. (prot); the
                           spin components turn with the frame), thin-fringe orbit maps
                           (Eq. (dipolefringe), symplectic form) at both faces, the
                           exact body map (Eq. (rbend)) in n_slices slices, the offsets
                           of Eqs. (Xoffset), (Toffset); fringe = 1 adds the spin kicks
                           of Eq. (skfringeRB).  FP64 and mixed-precision contexts and
                           batches (the mixed kernels track it in FP64).               */

#define ST_TEAPOT   7   /* sector bend (h = angle/L, field ratio eta as ST_SBEND) integrated
                           by the TEAPOT drift-kick split, Sec. 3.6, Eqs. (DKsplit),
                           (teapotD): each slice is a curved drift of ds/2 (the flow of
                           -(1 + hX) Ps + Pt/beta0, including the reference time s/beta0),
                           the kick of the bend's uniform field over ds (dPx/ds =
                           -eta h (1 + hX), Eq. (sbendA)) and another curved drift;
                           split_order 4 composes it to fourth order.  eta = 0 is a
                           field-free curved frame.  The paper's comparison integrator:
                           less accurate than ST_SBEND at any slice count.  FP64 and
                           (second order) mixed precision, single contexts and
                           batches.                                                     */

#define ST_THIN_MULT 8  /* thin lens, Sec. 3.5: the ST_MULT multipole in the limit of zero
                           length at fixed integrated strengths, k1 = integrated quadrupole
                           strength k1 L [m^-1], k2 = integrated sextupole strength k2 L
                           [m^-2], L = 0.  Orbit: the kick of the integrated field (positions,
                           T and Pt unchanged).  Spin: sampled along the kick, n_slices
                           partial kicks of 1/n_slices each with Omega (Eq. (6b)) of the
                           integrated field at their edges, then the chosen spin scheme,
                           as for any element.  No fringe kicks, second-order only; FP64
                           and mixed-precision contexts.                                */

/* ---- spin integration schemes (spin_order arguments) ------------------ */
/* spin_order 0..4 is the number of Romberg iterations over slice-edge
 * samples.  Two negative values select the piece-wise constant rotation
 * R(ds Omega) per slice with Omega at the slice middle (Sec. 4.1, Eq. (37);
 * Sec. 5.3, Fig. oneTurnSpinErrs), on FP64 and mixed-precision contexts (the
 * mixed tracker runs them on its element kinds in its compensated
 * arithmetic), any n_slices, no fourth-order slice maps (ST_EINVAL
 * otherwise):                                                               */
#define ST_SPIN_MID_HALF  -1   /* each slice traversed as two half-slices of its own
                                  map, the rotation between them ("half-DKD, spin,
                                  half-DKD")                                        */
#define ST_SPIN_MID_KICK  -2   /* drift-kick (ST_MULT, ST_TEAPOT) and matrix-kick
                                  (ST_QUAD_MK) slices keep their map and rotate the
                                  spin between the two halves of the central kick
                                  ("half-drift, half-kick, spin, half-kick,
                                  half-drift"); exact maps as ST_SPIN_MID_HALF       */

/* ---- precision of a tracking context ---------------------------------- */
#define ST_FP64   0   /* all arithmetic in IEEE double                                 */
#define ST_MIXED  1   /* FP32 slice arithmetic with compensated coordinates, FP64
                         per-turn spin composition (see st_ctx_create)                 */

typedef struct st_lattice st_lattice;   /* opaque; immutable after creation          */
typedef struct st_ctx st_ctx;           /* opaque; particle state on the device      */

/* One beamline element.  Units: metres, radians; k1 = b2/(B rho) [m^-2],
 * k2 = B''/(B rho) [m^-3] (MAD convention).  n_slices is the number of
 * integration slices of a spin-carrying element (ST_MULT, ST_QUAD_MK,
 * ST_SBEND, ST_SOLENOID, ST_RBEND, ST_TEAPOT, ST_THIN_MULT) and must be a
 * multiple of 2^spin_order at st_track time (Romberg orders). */
typedef struct {
    int32_t type;
    int32_t n_slices;
    double L;
    double k1;
    double k2;
    double angle;
    double eta;
    double snake_phi;
    double snake_mu;
    int32_t fringe;    /* 1: thin fringe spin kicks at both ends of an ST_MULT, ST_QUAD_MK,
                        * ST_SBEND or ST_TEAPOT (Sec. 4.5, Eq. (skfringe)), or of an ST_RBEND
                        * (Eq. (skfringeRB), see ST_RBEND); for the others: a rotation about the
                        * longitudinal axis by -(+-)(1 + G) sum_m (b_m/(B rho)) Im (X + iY)^m / m,
                        * + at the entrance, - at the exit, with b_1/(B rho) = eta h,
                        * b_2/(B rho) = k1, b_3/(B rho) = k2/2; orbit unchanged.  0: none.
                        * Solenoids always carry their Sec. 4.4 fringe kicks; drifts and
                        * snakes must have 0 (ST_EINVAL otherwise).  Both trackers apply
                        * them (the mixed one on an ST_RBEND in its FP64 maps). */
    int32_t split_order; /* orbit slice map of an ST_MULT, ST_QUAD_MK or ST_TEAPOT: 0 or
                          * 2 = the symmetric second-order split of Eq. (27) (drift-kick-
                          * drift, matrix-kick, TEAPOT); 4 = Yoshida's fourth-order composition
                          * S2(x1 ds) S2(x0 ds) S2(x1 ds), x1 = 1/(2 - 2^(1/3)),
                          * x0 = 1 - 2 x1 (Sec. 3.3's higher-order versions).  Spin is
                          * still sampled at the slice edges.  Other types: 0 or 2
                          * (ST_EINVAL otherwise).  With 4 the midpoint schemes are
                          * refused (ST_EINVAL); FP64 and mixed precision. */
    double e1;           /* ST_RBEND only: face asymmetry (see ST_RBEND); ignored otherwise */
} st_element;

/* Reference particle: anomaly G and naive spin tune G*gamma0 of the scale
 * momentum p0 (gamma0 = Ggamma0/G, beta0 = sqrt(1 - 1/gamma0^2)); protons,
 * positive rigidity. */
typedef struct {
    double G;
    double Ggamma0;
} st_reference;

/* Build a lattice from n >= 1 elements (host array, copied).  Element tables
 * are deduplicated and packed with per-element constants, then copied to the
 * current CUDA device.  Errors: ST_EINVAL (n < 1, unknown type, L <= 0 or
 * n_slices < 1 for a spin-carrying element, angle == 0 or eta == 0 for a bend,
 * G*gamma0 <= G), ST_ENOMEM, ST_ECUDA.  *out is set only on success. */
int st_lattice_create(const st_element* elems, int32_t n, const st_reference* ref,
                      st_lattice** out);
int st_lattice_destroy(st_lattice* lat);

/* Create a tracking context for n_particles >= 1 particles on the current
 * device.  precision is ST_FP64 or ST_MIXED (every element kind runs in both).  cuda_stream is a cudaStream_t
 * (e.g. torch.cuda.current_stream().cuda_stream) or NULL for a stream owned by
 * the context.  Allocates the device state (orbit as (X,Px), (Y,Py), (T,Pt)
 * double2 arrays, spin, lost flags) and a staging buffer.  The lattice must
 * outlive the context. */
int st_ctx_create(const st_lattice* lat, int64_t n_particles, int32_t precision,
                  void* cuda_stream, st_ctx** out);
int st_ctx_destroy(st_ctx* ctx);

/* Load particle state.  z_soa is [6][n] doubles (X, Px, Y, Py, T, Pt rows);
 * spin_soa is [3][n] doubles (x, y, s components of unit spins).  Pointers are
 * host memory (src_is_device = 0; read during the call) or device memory of
 * the current device (src_is_device = 1; read asynchronously on the context
 * stream).  Clears the lost flags.  Errors: ST_EINVAL for NULL pointers. */
int st_particles_upload(st_ctx* ctx, const double* z_soa, const double* spin_soa,
                        int32_t src_is_device);

/* Track every particle for n_turns >= 0 turns with Romberg order spin_order
 * (0..4) or a midpoint scheme (ST_SPIN_MID_HALF, ST_SPIN_MID_KICK).
 * Asynchronous on the context stream.  Errors: ST_ESTATE before the first
 * upload, ST_EINVAL for n_turns < 0, spin_order outside -2..4, a
 * spin-carrying element whose n_slices is not a multiple of 2^spin_order, a
 * midpoint scheme with fourth-order slice maps, ST_ECUDA on a launch
 * failure. */
int st_track(st_ctx* ctx, int32_t n_turns, int32_t spin_order);

/* Track the orbits only (the maps of st_track without the spin step; spins
 * are left untouched) for n_turns >= 0 turns: FP64 for an ST_FP64 context,
 * the mixed tracker's compensated FP32 arithmetic for an ST_MIXED context.
 * Used by the learned spin map, which supplies the spin rotation per turn.
 * Asynchronous.  Errors as st_track. */
int st_track_orbit(st_ctx* ctx, int32_t n_turns);

/* Track one turn (as st_track with n_turns = 1) and write every particle's
 * one-turn spin rotation -- the element rotations of the turn composed and
 * renormalised, a unit quaternion (scalar first) -- to q_out (device double
 * [4][n]), with its sign chosen so that q . q_ref >= 0 (q_ref: host double[4]).
 * These are the (orbit at s = 0, one-turn map) pairs of the learned spin map.
 * Entries of particles already flagged lost are left unchanged; a particle
 * lost during the turn gets the rotation up to the element that lost it.
 * FP64 contexts only; spin_order as for st_track.  Asynchronous. */
int st_track_one_turn_map(st_ctx* ctx, int32_t spin_order, const double* q_ref, double* q_out);

/* Stroboscopic spin average: as st_track, and after every turn each
 * particle's spin at the start of the lattice (the fixed azimuth s = 0) is
 * added to spin_sum (device double [3][n], accumulated, not cleared), so that
 * spin_sum / n_turns is the turn-averaged spin <S>.  A particle lost during
 * a turn adds its spin for that turn (rotated up to the element that lost
 * it) and nothing in later turns.  FP64 contexts, and ST_MIXED contexts (the
 * mixed-precision tracker, Romberg orders 0..4 and the midpoint schemes; the
 * spin after each turn is its FP64 spin).  Asynchronous. */
int st_track_average(st_ctx* ctx, int32_t n_turns, int32_t spin_order, double* spin_sum);

/* Restore lost flags ([n] bytes, nonzero = lost; host or device memory as
 * st_particles_upload) after st_particles_upload, which clears them.  With
 * st_spins_download this checkpoints and resumes a run: the state between
 * launches is the FP64 orbit, the spins and the lost flags, so tracking
 * n1 turns, downloading, uploading into a new context and tracking n2 more
 * gives bit for bit the result of n1 + n2 turns in one context (FP64; the
 * mixed tracker too when the checkpoint falls on a launch boundary).
 * Errors: ST_EINVAL (NULL), ST_ESTATE (no particles uploaded), ST_ECUDA. */
int st_lost_upload(st_ctx* ctx, const uint8_t* lost, int32_t src_is_device);

/* Copy the tracked state out: spin_soa [3][n] (required), z_soa [6][n] and
 * lost [n] (each may be NULL), to host (dst_is_device = 0) or device memory.
 * Synchronises the context stream.  Returns ST_ETIMEOUT if a kernel reported
 * a bounded-wait failure, ST_ECUDA on an asynchronous CUDA error. */
int st_spins_download(st_ctx* ctx, double* spin_soa, double* z_soa, uint8_t* lost,
                      int32_t dst_is_device);

/* Launch shape used by st_track: threads per block (32..1024, multiple of 32)
 * and turns per kernel launch (>= 1).  0 keeps the current value.  These are
 * the knobs the autotuner sweeps. */
int st_ctx_set_launch(st_ctx* ctx, int32_t block_threads, int32_t turns_per_launch);

/* ---- batched jobs ----------------------------------------------------
 * Many independent tracking jobs (each its own lattice, particle count and
 * reference energy) tracked together by one persistent launch per chunk of
 * turns: work items of one block's worth of particles are ordered by cost
 * (largest first) and popped from a device work queue; each item's lattice is
 * staged into shared memory; every particle is tracked with the same
 * integrator as st_track, so results equal tracking each job alone.  The turn
 * loop is captured into a CUDA graph (per n_turns, spin order and launch
 * shape) and replayed. */
typedef struct st_batch st_batch;

/* n_jobs >= 1 jobs: lattices[j] (must outlive the batch) and n_particles[j]
 * (1..2^30).  precision ST_FP64 or ST_MIXED; cuda_stream as st_ctx_create.
 * Errors: ST_EINVAL, ST_ENOMEM, ST_ECUDA. */
int st_batch_create(const st_lattice* const* lattices, const int64_t* n_particles, int32_t n_jobs,
                    int32_t precision, void* cuda_stream, st_batch** out);
int st_batch_destroy(st_batch* batch);
/* Load job `job`'s particles ([6][n] orbit, [3][n] spins, as
 * st_particles_upload); synchronises the batch stream. */
int st_batch_upload(st_batch* batch, int32_t job, const double* z_soa, const double* spin_soa,
                    int32_t src_is_device);
/* Track every job for n_turns with Romberg order spin_order, or with a
 * midpoint scheme (ST_SPIN_MID_HALF, ST_SPIN_MID_KICK; batches without
 * fourth-order slice maps, FP64 or mixed precision), asynchronously.  Errors:
 * ST_ESTATE if a job has no particles, ST_EINVAL as st_track. */
int st_batch_track(st_batch* batch, int32_t n_turns, int32_t spin_order);
/* Copy job `job`'s state out (as st_spins_download); synchronises. */
int st_batch_download(st_batch* batch, int32_t job, double* spin_soa, double* z_soa, uint8_t* lost,
                      int32_t dst_is_device);
/* Launch shape: threads per block (32..128, multiple of 32; 0 keeps), turns
 * per launch (0 keeps), CUDA graph on/off (-1 keeps), register-budget
 * variant 0 (larger budget, fewer resident blocks; the default) or 1 (-1
 * keeps).  Defaults: 128 threads, 5 turns per launch, graph on, variant 0. */
int st_batch_set_launch(st_batch* batch, int32_t block_threads, int32_t turns_per_launch, int32_t use_graph,
                        int32_t variant);
/* Autotuner: times block size {64, 96, 128} x turns per launch {1,
 * trial_turns} x register variant {0, 1} on trial_turns turns of the live
 * state (restored after every trial), keeps the fastest shape and returns it
 * (any output pointer may be NULL).  Allocates a temporary backup buffer. */
int st_batch_autotune(st_batch* batch, int32_t spin_order, int32_t trial_turns, int32_t* best_block,
                      int32_t* best_tpl, int32_t* best_variant, float* best_ms);

/* Measure the current device's sustained fused-multiply-add throughput in
 * FP64 and in FP32 (flop/s, two flops per FMA) with independent FMA chains
 * timed by CUDA events (about 0.2 s).  These are the denominators of the
 * trackers' arithmetic roofline.  Errors: ST_EINVAL (NULL), ST_ECUDA. */
int st_measure_peaks(double* fp64_flops, double* fp32_flops);

/* The same FP32 measurement with Blackwell's packed FP32x2 fused
 * multiply-add (two per instruction, independent chains): *fp32_flops in
 * flop/s.  It shows whether the packed instructions raise the FP32 rate or
 * only save issue slots.  About 0.1 s.  Errors: ST_EINVAL (NULL), ST_ECUDA. */
int st_measure_fp32x2_peak(double* fp32_flops);

/* Failure-path self-test of the device-side bounded waits: one block waits,
 * with the library's bounded mbarrier wait, on a barrier that nothing ever
 * completes (no copy is issued, so nothing is left in flight).  The wait
 * gives up after limit_s seconds (1e-4 .. 2) and the call returns
 * ST_ETIMEOUT with the measured wait in *elapsed_s; the context stays usable.
 * Returns ST_OK only if the wait did not give up (which would be a bug).
 * Errors: ST_EINVAL, ST_ECUDA. */
int st_selftest_bounded_wait(double limit_s, double* elapsed_s);

/* Allocation-free FP64 tracking.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory (code running
 * inside an allocator or memory pool that owns the device memory, host
 * processes that forbid further allocations, latency-critical loops where a
 * cudaMalloc would stall).  It calls no cudaMalloc/cudaFree and no allocating
 * library routine: the packed lattice (at most 64 KiB: <= 512 distinct
 * elements, <= 16384 elements per turn) and the kernel status word live in
 * one file-scope device array of about 64 KiB that every GPU loading the
 * library holds until the process exits.
 *   elems, n_elems, ref: the lattice as for st_lattice_create (host memory).
 *   state: device (or managed) buffer of 9 n doubles, 16-byte aligned (it
 *          is read and written as pairs), updated in place, laid out as the
 *          tracker's native pairs: (X,Px)[n], (Y,Py)[n], (T,Pt)[n], (Sx,Sy)[n],
 *          then Sz[n];  lost: device (or managed) buffer of n flags (0 =
 *          tracked; set to 1 when a particle is lost; particles flagged on
 *          entry are skipped).  A misaligned state or a host pointer is
 *          refused with ST_EINVAL before anything is launched.
 *   n_turns >= 0, spin_order 0..4 (every spin-carrying element's n_slices a
 *   multiple of 2^spin_order) or a midpoint scheme (ST_SPIN_MID_HALF,
 *   ST_SPIN_MID_KICK; no fourth-order slice maps); cuda_stream may be NULL
 *   (legacy stream).
 * The first call on a device looks up the scratch array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  Every call shares the scratch and rewrites it;
 * calls that overlap on the GPU race.  On the host the lattice is packed
 * into a static 96 KiB buffer of the library under a mutex (no heap use), so
 * host threads calling at the same time take turns.  The call synchronises
 * the stream.
 * Errors: ST_EINVAL (arguments, alignment, non-device buffers, lattice too
 * large), ST_ECUDA, ST_ETIMEOUT. */
int st_track_fp64_noalloc(const st_element* elems, int32_t n_elems, const st_reference* ref,
                          double* state, uint8_t* lost, int64_t n_particles, int32_t n_turns,
                          int32_t spin_order, void* cuda_stream);

/* Slice-count tuner (Sec. 5.2.1, 5.3: the paper picks n_b and the Romberg
 * order against a finely sliced reference).  For a sample ensemble (z_soa
 * [6][n], spin_soa [3][n], host memory) every candidate discretisation --
 * every spin-carrying element cut into n_b = 1, 2, 4, ..., ST_TUNE_MAX_SLICES
 * slices, Romberg order K = 0 .. min(ST_TUNE_MAX_ORDER, log2 n_b) -- is
 * tracked for one turn by the FP64 tracker from the same state, its one-turn
 * Delta S of Sec. 5.3 (mean |S - S_ref| over the particles not lost) against
 * the reference (n_b = ST_TUNE_REF_SLICES, K = ST_TUNE_REF_ORDER) is measured,
 * and its turn is timed with CUDA events.  Returns the fastest candidate with
 * Delta S <= spin_error_bound (the reference itself if none is).  Outputs:
 * *n_slices_out, *spin_order_out (required); *dS_out, *ms_out,
 * *n_candidates_out (may be NULL); table_out (may be NULL) receives one row
 * (n_b, K, Delta S, ms) per candidate, at most ST_TUNE_MAX_CANDIDATES rows
 * (slicings that the lattice does not admit are skipped).
 * The elements' own n_slices are ignored.  Creates and destroys its own
 * lattices and contexts on the current device; synchronous.  Errors:
 * ST_EINVAL (NULL, n < 1, bound <= 0, invalid element, a lattice that the
 * FP64 tracker refuses), ST_ENOMEM, ST_ECUDA. */
#define ST_TUNE_MAX_SLICES     64
#define ST_TUNE_MAX_ORDER      3
#define ST_TUNE_REF_SLICES     128
#define ST_TUNE_REF_ORDER      3
#define ST_TUNE_MAX_CANDIDATES 22
int st_tune_slicing(const st_element* elems, int32_t n_elems, const st_reference* ref, const double* z_soa,
                    const double* spin_soa, int64_t n_particles, double spin_error_bound, int32_t* n_slices_out,
                    int32_t* spin_order_out, double* dS_out, float* ms_out, int32_t* n_candidates_out,
                    double* table_out);

/* BF16 tensor-core GEMM (tcgen05, TMA-fed, FP32 accumulation in tensor
 * memory): D[M][N] = A[M][K] . B[N][K]^T (+ bias[N] if bias != NULL).  All
 * pointers are device memory: A, B bf16 row-major, D and bias FP32; M a
 * multiple of 128, K of 64, N of 16; A, B and D 16-byte aligned.  Asynchronous on
 * cuda_stream; *status (device int32, caller-cleared) becomes nonzero if a
 * bounded wait expired.  This is the building block of the learned spin map's
 * kernels.  Errors: ST_EINVAL (shapes, alignment), ST_ECUDA. */
int st_gemm_bf16(const void* A, const void* B, float* D, int32_t M, int32_t N, int32_t K, const float* bias,
                 int32_t* status, void* cuda_stream);

/* ---- learned one-turn spin map ------------------------------------------
 * A multilayer perceptron 6 -> 256 -> 256 -> 256 -> 256 -> 4 with SiLU
 * activations maps a particle's orbit z = (X, Px, Y, Py, T, Pt) at the fixed
 * azimuth s = 0 to its one-turn spin rotation (the composed element rotations
 * of Sec. 4, Eqs. (37)-(39)) through an FP64 head
 *     u = q0 + P(x) + s y,   q = u / |u|,   x = in_scale * z,
 * q0 the closed-orbit one-turn quaternion, P a polynomial in x (degree <= 3,
 * fitted by st_mlp_fit_head; st_mlp_set_head installs a linear one), s the
 * output scales (one per component, s y componentwise) and y the network's
 * output.  Weights and activations are bf16
 * on the tensor cores (st_gemm_bf16's kernel) with FP32 accumulation; each
 * scaled input enters the first layer as two bf16 numbers (hi, and the bf16
 * rounding of x - hi) multiplying the same weight, so inputs are resolved to
 * about 2^-16.  Master weights and Adam moments are FP32.  All x / q / r
 * arrays below are device memory, row-major float [B][6] / [B][4].  The
 * parameter vector (host, float[st_mlp_param_count()]) is W1[256][6], b1,
 * W2[256][256], b2, W3, b3, W4, b4, W5[4][256], b5.
 * Monomials of P, in order: 1; x_0..x_5; x_i x_j (0 <= i <= j < 6, i the
 * outer loop); x_i x_j x_k (i <= j <= k) -- 1, 7, 28 or 84 terms for degree
 * 0..3. */
typedef struct st_mlp st_mlp;
int64_t st_mlp_param_count(void);
/* Buffers for batches of up to max_batch rows (padded to 128); parameters
 * start at zero; head q0 = (1,0,0,0), P = 0, s = 1, unit input scales.
 * cuda_stream as st_ctx_create. */
int st_mlp_create(int32_t max_batch, void* cuda_stream, st_mlp** out);
int st_mlp_destroy(st_mlp* mlp);
int st_mlp_set_params(st_mlp* mlp, const float* params);     /* host; resets Adam */
int st_mlp_get_params(st_mlp* mlp, float* params);           /* host */
/* Head: q0[4], P(x) = lin x with lin[4][6] (NULL = zero), out_scale > 0,
 * in_scale[6] >= 0 (0 removes a coordinate from P and from the network). */
int st_mlp_set_head(st_mlp* mlp, const double* q0, const double* lin, double out_scale, const double* in_scale);
/* Output scales s only, one per quaternion component: out_scale[4] > 0. */
int st_mlp_set_scale(st_mlp* mlp, const double* out_scale);
/* FP64 least-squares fit of q - q0 by P of the given degree (0..3) over n
 * tracked pairs: z_soa (device double [6][n], orbits at s = 0), q_soa (device
 * double [4][n], their one-turn quaternions from st_track_one_turn_map), lost
 * (device flags, may be NULL; flagged pairs are left out); q0 and in_scale as
 * last set.  The moments are summed on the device in FP64 and the normal
 * equations (monomials of coordinates with in_scale 0 dropped) solved on the
 * host by Cholesky.  Installs P in the head; writes its coefficients to
 * coef_out (host double [4][n_terms], may be NULL) and the RMS of each
 * residual component to rms_out (host double [4], may be NULL).  Synchronises
 * the network's stream.  Errors: ST_EINVAL (arguments, singular fit). */
int st_mlp_fit_head(st_mlp* mlp, int32_t degree, const double* z_soa, const double* q_soa, const uint8_t* lost,
                    int64_t n, double* coef_out, double* rms_out);
/* Training rows from tracked pairs (z_soa, q_soa as for st_mlp_fit_head):
 * x_rows = z (float [n][6]) and the residual targets
 * r_rows = (q - q0 - P(x)) / s (computed in FP64, float [n][4]) with the
 * current head.  Asynchronous. */
int st_mlp_make_targets(st_mlp* mlp, const double* z_soa, const double* q_soa, int64_t n, float* x_rows,
                        float* r_rows);
/* Inference: q[B][4] unit quaternions for x[B][6].  Asynchronous. */
int st_mlp_forward(st_mlp* mlp, const float* x, int32_t B, float* q_out);
/* Inference path of st_mlp_forward and st_track_surrogate: on != 0 (the
 * default) runs all five layers of each 128-row tile in one kernel, the
 * activations kept in shared memory and the accumulators in tensor memory;
 * 0 runs one GEMM per layer.  Both give the same results (same bf16
 * operands, accumulation order and epilogue).  Errors: ST_EINVAL (NULL). */
int st_mlp_set_fused_inference(st_mlp* mlp, int32_t on);
/* Loss L = mean_b |q_b - q_target_b|^2 of the normalised head output and its
 * gradient with respect to all parameters (kept on the device for
 * st_mlp_adam_step).  If loss / grads (host, may be NULL) are given they are
 * filled and the call synchronises. */
int st_mlp_loss_grad(st_mlp* mlp, const float* x, const float* q_target, int32_t B, float* loss, float* grads);
/* The same for the residual regression L = mean_b |y_b - r_b|^2 on the raw
 * network outputs y, with targets from st_mlp_make_targets. */
int st_mlp_loss_grad_residual(st_mlp* mlp, const float* x, const float* r_target, int32_t B, float* loss,
                              float* grads);
/* One Adam update with the last gradients; refreshes the bf16 weights. */
int st_mlp_adam_step(st_mlp* mlp, float lr, float beta1, float beta2, float eps);
/* A training schedule in one call: for k = 0 .. steps-1, the residual loss
 * and gradient (as st_mlp_loss_grad_residual) on the B rows starting at row
 * row_start[k] of x_rows [n_rows][6] / r_rows [n_rows][4] (device memory,
 * from st_mlp_make_targets), then one Adam update with learning rate lr[k]
 * (as st_mlp_adam_step).  row_start, lr: host arrays of `steps` entries;
 * loss_out: host double[steps] for every step's loss before its update, or
 * NULL.  The first step runs on the network's stream; the others are
 * replayed from one captured CUDA graph of a step (its rows and Adam schedule
 * read from device copies of row_start and lr) on streams the library
 * creates and joins back to the network's stream, with each layer's weight
 * and bias gradients beside the next layer's data gradient; the results are
 * those of stepping one step at a time.  Synchronises at the end and reports
 * a bounded-wait expiry of any step.  Errors: ST_EINVAL (arguments, a row
 * range outside [0, n_rows), lr <= 0), ST_ECUDA, ST_ETIMEOUT. */
int st_mlp_train(st_mlp* mlp, const float* x_rows, const float* r_rows, int64_t n_rows, int32_t B, int32_t steps,
                 const int64_t* row_start, const float* lr, float beta1, float beta2, float eps, double* loss_out);
/* Stroboscopic spin tracking with the learned map: per turn, the network
 * gives each particle's one-turn rotation from its FP64 orbit at s = 0 (head
 * in FP64), the spin is rotated by it (FP64), and the orbit is tracked
 * for one turn (st_track_orbit: FP64 or, for an ST_MIXED context, the mixed
 * tracker's compensated orbit).  spin_sum (device double [3][n], may be NULL)
 * accumulates S after every turn.  Needs n <= max_batch.  Asynchronous on the
 * context stream. */
int st_track_surrogate(st_ctx* ctx, st_mlp* mlp, int32_t n_turns, double* spin_sum);

/* Message describing the last error on the calling thread ("" if none). */
const char* st_last_error(void);

/* Library version string. */
const char* st_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SPINTRACK_H */
