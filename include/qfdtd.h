/*
 * qfdtd.h - C ABI of libqfdtd: the imaginary-time Schrodinger step of quantumfdtd v3
 * (Delgado, Steinbeisser, Strickland, Weber, arXiv 2211.10185) on one GB300 GPU.
 *
 * The library advances a complex wavefunction psi on an N^3 lattice (spacing a) in
 * imaginary time (Sec. 2, Eq. eq_iterat with the full H = H_K + V of Eq. eq_schro):
 *
 *     psi <- coef_A psi - coef_B dtau H_K psi,
 *     coef_A = (1 - dtau V/2)/(1 + dtau V/2),  coef_B = 1/(1 + dtau V/2),
 *
 * (the time discretisation is deferred by the paper to its references; this
 * Crank-Nicolson-in-V, explicit-in-H_K form is the reading implemented), with one of
 * four kinetic terms (Sec. 2): the FDTD 7-point Laplacian under Dirichlet boundaries
 * (Eq. HK0) or the FFT terms under periodic boundaries with the multipliers
 * k^2/(2 a^2 m) (Eq. HK1), 4 sin^2(k/2)/(2 a^2 m) (Eq. HK2) and
 * sqrt(4 sum sin^2(k/2) + (a m)^2)/a (Eq. HK3).  Energies are FP64 Rayleigh quotients,
 * excited states come from Gram-Schmidt over nearby snapshots (Sec. 1), and the parity
 * projectors are those of Sec. 3.
 *
 * Conventions for every call:
 *  - Every function returns a qf_status; nothing throws or aborts across the ABI.  On
 *    failure qf_last_error(handle) returns a NUL-terminated message owned by the handle.
 *  - Host pointers are borrowed for the duration of the call only; the call has
 *    finished reading or writing them when it returns.
 *  - Device memory is owned by the caller: qf_workspace_bytes() sizes one workspace
 *    that the caller allocates (e.g. a torch uint8 tensor) and passes to
 *    qf_create_lattice(); the library never allocates or frees device memory.
 *  - Host fields are FP64, interleaved (re, im), C order with x fastest: site
 *    (ix, iy, iz) at index (iz*N + iy)*N + ix, coordinate x_i = (i - N/2) a.
 *  - All GPU work of a handle is issued on the CUDA stream given at creation.  Calls
 *    that return host data synchronise that stream.  A handle is not thread safe.
 *  - N must be even, 8 <= N <= 512, and one of 8, 12, 16, 24, 32, 48, 64, 96, 128,
 *    192, 256, 384, 512 (the FFT plans built into the library; FDTD lattices accept any
 *    even N in [8, 1024]).  Odd N has no lattice momentum set (Sec. 2).
 */
#ifndef QFDTD_H
#define QFDTD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qf_lattice qf_lattice; /* opaque, library-owned host object */

typedef enum {
  QF_OK = 0,
  QF_EINVAL = 1,   /* bad argument (null pointer, size, enum value)                 */
  QF_ENOMEM = 2,   /* workspace too small                                           */
  QF_ECUDA = 3,    /* a CUDA call failed; the message names it                      */
  QF_ESTATE = 4,   /* call out of order (e.g. step before potential/kinetic/psi)    */
  QF_ETIMEOUT = 5, /* a bounded device wait ran out                                 */
  QF_ENOTCONV = 6  /* qf_step_n reached max_steps before the tolerance was met      */
} qf_status;

/* Kinetic terms of Sec. 2. */
typedef enum {
  QF_KIN_FDTD = 0,          /* Eq. HK0, Dirichlet planes at index 0                  */
  QF_KIN_FFT_NAIVE = 1,     /* Eq. HK1, multiplier k^2/(2 a^2 m), periodic           */
  QF_KIN_FFT_SYMANZIK = 2,  /* Eq. HK2, multiplier 4 sin^2(k/2)/(2 a^2 m), periodic  */
  QF_KIN_FFT_REL = 3        /* Eq. HK3, multiplier sqrt(4 sin^2(k/2) + (a m)^2)/a    */
} qf_kinetic;

/* Bulk precision: complex FP32 fields with FP64 reductions, or complex FP64 throughout. */
typedef enum { QF_PREC_C64 = 0, QF_PREC_C128 = 1 } qf_precision;

/* Parity projectors of Sec. 3, and d-wave projectors (listed by the paper as future
 * work; reading: products of single-axis mirror projectors).  R_i mirrors axis i
 * (site i -> (N - i) mod N); for QF_P_D_K and QF_P_D2_K, i and j are the two axes other
 * than k, and S_ij exchanges them. */
typedef enum {
  QF_P_PLUS = 0,     /* (psi(r) + psi(-r))/2                                             */
  QF_P_MINUS = 1,    /* (psi(r) - psi(-r))/2                                             */
  QF_P_MINUS_PK = 2, /* P^-_{p_k}: odd in axis k, even under flipping the other two; 1/4 */
  QF_P_D_K = 3,      /* (1 - R_i)(1 - R_j)(1 + R_k)/8: d_xy-like around axis k         */
  QF_P_D2_K = 4      /* (1 - S_ij)/2 (1 + R_i)(1 + R_j)(1 + R_k)/8: d_{x^2-y^2}-like     */
} qf_parity;

typedef struct {
  int n;              /* lattice sites per axis                                    */
  double a;           /* lattice spacing (the paper's A), > 0                      */
  int prec;           /* qf_precision                                              */
  int n_snap;         /* snapshot ring length, 1..3 (Gram-Schmidt uses up to 3)    */
  int plateau_slots;  /* 0..3 fields kept for the states at the plateau of E_i(tau)
                         (qf_track_excited); 0 keeps the energies only              */
} qf_lattice_desc;

typedef struct {
  double e_re, e_im;  /* Rayleigh quotient <psi|H|psi>/<psi|psi>                     */
  double norm;        /* <psi|psi> of the measured field                              */
  double de;          /* |E - E_previous check| (infinity before the second check)   */
  int64_t step;       /* step index t of the measured psi_t                           */
  double tau;         /* imaginary time of psi_t                                      */
} qf_energy;

typedef struct {
  double dtau;        /* time step in use                                            */
  int64_t step;       /* steps taken so far                                          */
  double tau;         /* imaginary time reached                                      */
  int kinetic;        /* qf_kinetic, -1 before qf_set_kinetic                         */
  int n_snapshots;    /* snapshots currently held (<= n_snap)                        */
  size_t workspace_bytes;
  int64_t launches;   /* kernels this handle has launched so far                     */
  int temporal_block; /* FDTD steps fused per pass (qf_set_temporal_blocking)         */
  int fft_passes;     /* HBM passes of a steady-state FFT step: 2 (N = 128 or 256
                         complex FP32, qf_use_two_pass_fft) or 4; 0 for FDTD          */
  int64_t field_exp2; /* the stored live field is 2^field_exp2 times the one
                         qf_get_wavefunction returns (see qf_step_n)                  */
} qf_info;

typedef struct {
  char name[24];      /* kernel kind, e.g. "fft_z_mid_T", "fft_x_inv_update"          */
  int64_t launches;   /* launches timed                                               */
  double total_ms;    /* summed CUDA-event duration of those launches                 */
} qf_kernel_stat;

/* Device workspace a lattice with this description needs (bytes, 256-byte aligned
 * start expected).  QF_EINVAL for an unsupported description. */
qf_status qf_workspace_bytes(const qf_lattice_desc* desc, size_t* bytes);

/* Creates a lattice on the current CUDA device.  dev_ws: device pointer to at least
 * qf_workspace_bytes() bytes, 256-byte aligned, owned by the caller and kept alive
 * until qf_destroy_lattice.  cuda_stream: a cudaStream_t (NULL = legacy default stream).
 * The fields start at zero; the potential and kinetic term are unset. */
qf_status qf_create_lattice(const qf_lattice_desc* desc, void* dev_ws, size_t ws_bytes, void* cuda_stream,
                            qf_lattice** out);

/* Releases the handle (never the caller's workspace).  NULL is accepted. */
qf_status qf_destroy_lattice(qf_lattice* lat);

/* V(r) of Eq. eq_schro from host FP64 arrays of N^3 values (v_im == NULL: real V,
 * stored as real).  Complex V is the non-equilibrium case of Sec. 1. */
qf_status qf_set_potential(qf_lattice* lat, const double* v_re, const double* v_im);

/* Kinetic term (qf_kinetic), mass m > 0 (the paper's M) and time step dtau.  dtau <= 0
 * selects 0.75 / T_max with T_max = 6/(m a^2) (HK0, HK2), 3 pi^2/(2 m a^2) (HK1),
 * sqrt(12 + (a m)^2)/a (HK3). */
qf_status qf_set_kinetic(qf_lattice* lat, int kinetic, double mass, double dtau);

/* Live psi from a host array of 2 N^3 doubles (interleaved re, im).  Values on the
 * Dirichlet planes are ignored by the FDTD term.  Cancels a pending renormalisation. */
qf_status qf_set_wavefunction(qf_lattice* lat, const double* re_im);

/* Copies a field to a host array of 2 N^3 doubles.  slot -1: live psi as stored;
 * 0..2: Gram-Schmidt state i; 100 + j: snapshot j (0 = latest); 200 + i: the state i
 * kept at its plateau by qf_track_excited (needs plateau_slots > i). */
qf_status qf_get_wavefunction(qf_lattice* lat, int slot, double* re_im);

/* Advances up to max_steps steps.  Step t maps psi_t to psi_{t+1}.  When
 * t % check_every == 0 (check_every > 0) the energy of psi_t is measured in the same
 * pass (FP64 sums), and the output of step t+1 is scaled by 1/sqrt(<psi_t|psi_t>).  The
 * call returns QF_OK right after a check with |E_t - E_{t-check_every}| < tol_abs, else
 * QF_ENOTCONV after max_steps.  After step t, when (t+1) % snap_every == 0
 * (snap_every > 0), psi_{t+1} enters the snapshot ring.  steps_done may be NULL.
 * Between checks psi shrinks by about the ground state's step multiplier per step (a
 * heavy relativistic term can take it below the complex-FP32 range within one check
 * interval); each step therefore also multiplies its output by an exact power of two 2^k,
 * k estimated at every check from the measured decay.  The library tracks the
 * accumulated power and removes it from every field it returns (qf_get_wavefunction,
 * norms in qf_energy), so results are those of the unscaled iteration; only the raw
 * device data of qf_field_pointer carries it (qf_info.field_exp2 for the live field). */
qf_status qf_step_n(qf_lattice* lat, int64_t max_steps, double tol_abs, int check_every, int snap_every,
                    int64_t* steps_done);

/* Result of the last check of qf_step_n.  QF_ESTATE before the first check. */
qf_status qf_energies(qf_lattice* lat, qf_energy* out);

/* Excited states (Sec. 1): classical Gram-Schmidt with one re-orthogonalisation pass
 * over the latest n_states snapshots (latest first, FP64 inner products), giving the
 * states 0..n_states-1 and E_i = <v_i|H|v_i> in out[0..n_states).  1 <= n_states <=
 * min(3, n_snap); QF_ESTATE when fewer snapshots are held. */
qf_status qf_project_excited(qf_lattice* lat, int n_states, qf_energy* out);

/* Plateau of the excited-state energies (Sec. 4: the saddle point of E_i(tau), made
 * automatic).  Runs qf_project_excited(lat, n_states, out) on the latest snapshots and
 * appends E_0..E_{n_states-1} to the handle's history as record j (j = 0, 1, ...).  For
 * each state i, record j >= 1 becomes the state's choice when |E_i(tau_j) -
 * E_i(tau_{j-1})| (complex modulus) is strictly smaller than the current choice's, so
 * the earliest minimiser wins; with plateau_slots > i the state v_i of that record is
 * copied into slot 200 + i.  Call it at successive snapshots (e.g. after each qf_step_n
 * chunk that ends on a snapshot).  Every call of one history uses the same n_states
 * (QF_EINVAL otherwise); qf_set_potential, qf_set_kinetic and qf_set_wavefunction start
 * a new history. */
qf_status qf_track_excited(qf_lattice* lat, int n_states, qf_energy* out);

/* The current choice for states 0..n_states-1: out[i] holds E_i at the chosen record,
 * with that record's step and tau, de = |E_i(tau_j) - E_i(tau_{j-1})| and norm 1;
 * record (may be NULL) receives j.  QF_ESTATE before two records, QF_EINVAL when
 * n_states exceeds the history's. */
qf_status qf_excited_plateau(qf_lattice* lat, int n_states, qf_energy* out, int* record);

/* Applies a parity projector (qf_parity; axis 1..3 = x, y, z for QF_P_MINUS_PK and the
 * d-wave projectors) to the live psi (target -1), to Gram-Schmidt state 0..2 or to a
 * plateau state 200 + i, in place, and renormalises it to unit norm (a zero result
 * stays zero).  Projection of the live psi cancels a pending renormalisation. */
qf_status qf_parity_project(qf_lattice* lat, int which, int axis, int target);

/* Momentum-space distribution of a field (slot as in qf_get_wavefunction; needs an
 * FFT size).  Psi(p) is the discrete Fourier transform of psi at p = 2 pi n/(N a),
 * n_l in (-N/2, N/2]; |Psi(p)|^2 is summed over shells b = round(|n|) and normalised to
 * total 1 (Parseval).  Sec. 3 compares momentum-space states through
 * y(p) = sqrt(4 pi) p Psi(p), whose square is the radial density; y[b] receives
 * sqrt(prob[b] / dp), dp = 2 pi/(N a), its magnitude from the shell probability.  *nbins
 * always receives the number of shells, round(sqrt(3) N/2) + 1; the arrays (p and y may
 * be NULL) need that many entries, else QF_EINVAL.  The scratch field is overwritten. */
qf_status qf_momentum_distribution(qf_lattice* lat, int slot, double* p, double* prob, double* y, int max_bins,
                                   int* nbins);

/* CUDA-graph replay in qf_step_n (on by default; no counterpart in the paper).  After a
 * check step, the check_every - 1 steps up to the next check issue the same launches
 * every time; they are captured once into a graph (per check interval and FDTD buffer
 * parity) and replayed.  Used when the handle's stream is not the legacy default stream
 * (which cannot be captured), the interval fits inside max_steps, snapshots fall at its
 * end (snap_every 0 or equal to check_every) and per-kernel profiling is off; if a
 * capture fails, the handle continues with ordinary launches.
 * Changing the potential or the kinetic term drops the captured graphs. */
qf_status qf_use_graphs(qf_lattice* lat, int enable);

/* Form of the FFT step (no counterpart in the paper; the paper's FFTW transforms are
 * replaced by GPU passes).  enable != 0, the default: complex-FP32 lattices with N = 128
 * or 256 run a steady-state step in two passes over HBM (the y transform split
 * (N/16) x 16 four-step fashion between the two passes; the scratch field holds a
 * blocked layout), other lattices in four.  enable == 0 selects the four-pass form for
 * N = 128 and 256 too.  Both
 * compute the same step to rounding; switching discards the scratch field's contents and
 * any captured graphs. */
qf_status qf_use_two_pass_fft(qf_lattice* lat, int enable);

/* Tile and radix-plan choice of the complex-FP32 four-pass FFT kernels for lattice size n
 * (no counterpart in the paper; every size, N = 128 and 256 when their four-pass form is
 * selected).  Variant 0 tiles about 4096 elements per block with up to 16 contiguous
 * columns; variant 1 half of both (more, smaller blocks per SM); the two compute the same
 * transforms (the fields agree bitwise; reductions may differ in their last bits).
 * Variants 2 and 3 are variants 0 and 1 with the size's second radix plan (a radix-16
 * first stage and 16 elements per thread: 16 x 2 for N = 32, 16 x 4 for N = 64,
 * 16 x 8 x 4 for N = 512; other sizes have none and reject them); the fields agree with
 * variants 0 and 1 to rounding.  variant -1, the default, lets the autotuner time every
 * variant of the size on the first FFT step of a lattice of that size and keep the
 * fastest for the process; 0-3 fixes it (process-wide, affects every handle).
 * qf_get_fft_tiles returns -1 while the choice is pending. */
qf_status qf_set_fft_tiles(int n, int variant);
qf_status qf_get_fft_tiles(int n, int* variant);

/* Temporal blocking of the FDTD step (the step of Sec. 2 with the Eq. HK0 term; no
 * counterpart in the paper).  k = 2, the default: on complex-FP32 lattices qf_step_n
 * runs two consecutive steps with no check at either and no snapshot after the first as
 * one pass over HBM (psi_t and V read once, psi_{t+2} written once, psi_{t+1} kept in
 * shared memory).  The fields are bitwise those of two single steps.  Requires the live
 * field to be zero on the Dirichlet planes, which holds after any FDTD step; the first
 * step after qf_set_wavefunction always runs alone.  k = 1 runs every step alone.  Other
 * precisions and kinetic terms ignore the setting.  QF_EINVAL unless k is 1 or 2. */
qf_status qf_set_temporal_blocking(qf_lattice* lat, int k);

/* Warm start across lattice sizes (no counterpart in the paper; it shortens solves by
 * starting from a converged coarser solution).  Sets the live psi of `fine` to the
 * trigonometric interpolation of the field `coarse_slot` of `coarse` (slot as in
 * qf_get_wavefunction): fine must have 2N sites, spacing a/2 (the same box) and the same
 * precision, and both sizes FFT plans.  Coarse DFT modes with |n_l| < N/2 are kept, each
 * axis' Nyquist coefficient is split between +-N/2, the rest of the fine spectrum is
 * zero; fine site 2j then equals coarse site j.  Both scratch fields are overwritten;
 * the call synchronises both streams. */
qf_status qf_prolong(qf_lattice* coarse, int coarse_slot, qf_lattice* fine);

/* Time step, counters and sizes of the handle. */
qf_status qf_get_info(qf_lattice* lat, qf_info* out);

/* Device pointer to a field (slot as in qf_get_wavefunction), for zero-copy access by
 * the caller on the handle's stream.  Elements are complex FP32 or FP64 pairs.  The
 * live field and the snapshots are stored times a power of two (see qf_step_n;
 * qf_info.field_exp2 for the live field); the states are normalised. */
qf_status qf_field_pointer(qf_lattice* lat, int slot, void** dev_ptr);

/* Per-kernel timing (no counterpart in the paper; measurement support).  enable != 0
 * brackets every kernel launch of this handle with CUDA events recorded on its stream
 * (event pool created on first use); enable == 0 stops and harvests.  Timing adds two
 * event records per launch and no device work. */
qf_status qf_profile(qf_lattice* lat, int enable);

/* Synchronises the handle's stream, folds finished timings into per-kind totals and
 * copies up to max of them to out; *count receives the number of kinds with launches.
 * reset != 0 clears the totals afterwards. */
qf_status qf_profile_read(qf_lattice* lat, qf_kernel_stat* out, int max, int* count, int reset);

/* One imaginary-time FFT step that allocates no device memory (the paper has no
 * counterpart: this is for callers that cannot allocate).  Some callers have no way to
 * obtain device memory when they call -- e.g. a plugin inside an application whose
 * allocator already owns the GPU, a loop that must not fail on out-of-memory midway,
 * or a plain-C caller holding only raw device pointers -- so they cannot provide the
 * workspace qf_create_lattice needs.  This call does the same work as one step of
 * qf_step_n for an FFT kinetic term (Eqs. HK1-HK3, complex FP32 fields) on arrays the
 * caller passes, and keeps its scratch (the transformed field, partial sums, tables) in
 * one fixed device array inside the library, present on every GPU that loads it until
 * the process exits.
 *   n: 8..64 and one of the FFT sizes listed above (QF_EINVAL otherwise: the fixed
 *      scratch holds at most a 64^3 complex FP32 field).
 *   kinetic: QF_KIN_FFT_NAIVE, _SYMANZIK or _REL; a, mass, dtau > 0 (no default rule).
 *   psi: device, n^3 complex FP32 (interleaved re, im), overwritten in place by
 *        out_scale * (coef_A psi - coef_B dtau H_K psi).
 *   v: device potential, n^3 FP32 values (v_complex == 0) or n^3 complex FP32 pairs.
 *   sums: NULL, or device array of 5 doubles that receives <psi|psi>, Re and Im
 *        <psi|H_K psi>, Re and Im <psi|V psi> of the input psi (FP64 sums).
 *   cuda_stream: stream for all work; the call returns without synchronising it.
 * The first call on a device looks up the array's device address; make that first call
 * before any stream capture.  All calls share the one array and it keeps the previous
 * call's contents (each call rewrites everything it reads), so calls whose GPU work
 * overlaps -- on different streams or from different threads on one device -- race. */
qf_status qf_fft_step_static(int n, double a, int kinetic, double mass, double dtau, void* psi, const void* v,
                             int v_complex, double out_scale, double* sums, void* cuda_stream);

/* ---- Batches (no counterpart in the paper: serving many independent solves) ------
 * A batch advances many resident lattices together.  Each step, complex-FP32 lattices
 * form groups, and each pass of a group is a single kernel launch over all its members
 * (up to 48 per launch): FDTD lattices of any sizes together (the stencil launch maps
 * its blocks to members through a table), FFT lattices of equal N, real/complex V and
 * check status; FP64 lattices run their own launches.  Every member computes
 * exactly what qf_step_n computes for it alone (same kernels, same blocks, same
 * reduction order), so its results do not depend on the other members.  A batch holds
 * no device memory; members keep their own workspaces.  During qf_batch_step all
 * members' work is issued on the batch's stream. */
typedef struct qf_batch qf_batch;
#define QF_BATCH_RUNNING (-1)

qf_status qf_batch_create(void* cuda_stream, qf_batch** out);
qf_status qf_batch_destroy(qf_batch* b); /* never destroys the members */

/* Adds a ready lattice (potential, kinetic term and psi set) with its own stopping rule:
 * it converges at a check with |E_t - E_prev| < tol_abs + tol_rel |E_t| and stops after
 * max_steps steps taken inside the batch.  The lattice must not be used on its own
 * while it is a member. */
qf_status qf_batch_add(qf_batch* b, qf_lattice* lat, int64_t max_steps, double tol_abs, double tol_rel);
qf_status qf_batch_remove(qf_batch* b, qf_lattice* lat);

/* Advances every running member by up to `steps` steps (check_every and snap_every as
 * in qf_step_n).  Members stop at convergence (status QF_OK) or at their step cap
 * (QF_ENOTCONV) and stay in the batch until removed; *n_running (may be NULL) receives
 * the number still running. */
qf_status qf_batch_step(qf_batch* b, int64_t steps, int check_every, int snap_every, int* n_running);

/* Stopping rules of batch members (the paper has no automatic convergence test; the
 * difference rule is the reading used by qf_step_n).  With d = |E_t - E_prev| at a check
 * and tol = tol_abs + tol_rel |E_t|:
 *   QF_STOP_DIFFERENCE (default): converged when d < tol.
 *   QF_STOP_EXTRAPOLATED: the check energies approach their limit geometrically, so
 *     while d shrinks (rho = d / d_prev < 1, d_prev the previous check's difference) the
 *     distance left to the limit is about d rho/(1 - rho); converged when
 *     max(d, d rho/(1 - rho)) < tol, never while d >= d_prev (d = 0 counts as
 *     converged).  The reported energy is then within about tol of the limit even when
 *     the contraction per check is slow, where the difference rule can stop far from it. */
typedef enum { QF_STOP_DIFFERENCE = 0, QF_STOP_EXTRAPOLATED = 1 } qf_stopping;

/* Selects the stopping rule (qf_stopping) for every member's following checks. */
qf_status qf_batch_set_stopping(qf_batch* b, int rule);

/* CUDA graphs of check-free intervals (on by default; no counterpart in the paper).
 * When every running member took a check at the previous step, the check_every - 1
 * steps up to the next check issue the same launches each time the batch holds the same
 * members in the same buffer state; they are captured once into a graph and replayed.
 * Needs check_every >= 3, snap_every 0 or equal to check_every, no member closer to its
 * step cap than the interval, no per-kernel profiling and a stream other than the legacy
 * default stream.  Adding or removing a member drops the captured graphs; a failed
 * capture leaves the batch on ordinary launches.  Results are bitwise those of ordinary
 * launches. */
qf_status qf_batch_use_graphs(qf_batch* b, int enable);

/* Graphs captured and graph replays so far. */
qf_status qf_batch_graph_info(qf_batch* b, int64_t* captures, int64_t* replays);

/* Members in insertion order: count, and per member (arrays of at least `max` entries,
 * may be NULL) its status (QF_BATCH_RUNNING, QF_OK, QF_ENOTCONV) and steps taken. */
qf_status qf_batch_members(qf_batch* b, int* count, int* status, int64_t* steps_done, int max);

/* Kernel launches the batch has issued. */
qf_status qf_batch_info(qf_batch* b, int64_t* launches);
const char* qf_batch_last_error(const qf_batch* b);

/* Message of the last failure of this handle ("" if none); static text for NULL. */
const char* qf_last_error(const qf_lattice* lat);

/* Self-test of the bounded device waits (no counterpart in the paper; failure
 * detection).  Launches, on the handle's stream, a kernel whose wait on a
 * shared-memory barrier can never complete; the wait gives up after its iteration limit
 * (about a second), the kernel records the failure and returns, and this call returns
 * QF_ETIMEOUT with the context still usable.  QF_OK would mean the limit did not work. */
qf_status qf_selftest_bounded_wait(qf_lattice* lat);

/* Library version string. */
const char* qf_version(void);

#ifdef __cplusplus
}
#endif

#endif /* QFDTD_H */
