/*
 * cosenu.h -- C ABI of the GB300 COSEnu engine (libcosenu.so).
 *
 * The engine advances the two-flavour neutrino quantum kinetic equations
 *     (d_t + v d_z) rho    = -i [H,    rho]
 *     (d_t + v d_z) rhobar = -i [Hbar, rhobar]
 * (arXiv:2203.12866, Sec. 2, Eq. (eom)) on a periodic z grid times N_v
 * velocity bins, with the Hamiltonian of Eq. (ham), 4th-order central
 * differences plus Kreiss-Oliger dissipation (Sec. 3.1) or the finite-volume
 * WENO7 flux (Sec. 3.2, Appendix A), and classic RK4 in time.
 *
 * Grid.  z in [-L/2, L/2), nz cells of width dz = L/nz, periodic (Sec. 4).
 * v bins: v_j = -1 + (j + 1/2) dv, dv = 2/nv, integrals over v are Riemann
 * sums with weight dv (Sec. 3).
 *
 * State layout (host and device): double [2][4][nz][nv]
 *   species (0 = nu, 1 = nubar) x component (0 = rho_ee, 1 = rho_xx,
 *   2 = Re rho_ex, 3 = Im rho_ex) x z x v, v fastest.
 * The stored neutrino state is g_nu(v) rho (Sec. 5); the stored antineutrino
 * state already carries the asymmetry factor: alpha g_nubar(v) rhobar.  The
 * Hamiltonian therefore uses the stored antineutrino state where Eq. (ham)
 * has alpha rhobar.
 *
 * Conventions.
 *   - Return codes: 0 on success, a negative COSENU_E* code on failure.  No
 *     C++ exception crosses this boundary.  cosenu_last_error() describes
 *     the most recent failure (per handle; thread-local for NULL handles).
 *   - A handle is not thread-safe; distinct handles are independent.
 *   - cosenu_step() only enqueues work on the handle's stream and returns;
 *     cosenu_get_state(), cosenu_moments(), cosenu_conserved() and
 *     cosenu_sync() wait for it.
 *   - Host pointers are read or written only during the call; the caller
 *     keeps ownership.  Device memory is owned by the library unless the
 *     handle was made by cosenu_create_external().
 *   - Requirements: nz >= 1; 4 <= nv <= 256 and nv a multiple of 4
 *     (rows are moved by 16-byte bulk copies).  Violations give COSENU_EINVAL.
 */
#ifndef COSENU_H
#define COSENU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define COSENU_VERSION 1

/* Spatial scheme: Sec. 3.1 (FD4 + Kreiss-Oliger r = 2), Sec. 3.2 (FV WENO7), or
 * FD4 + Kreiss-Oliger r = 3 (the general dissipation operator of Sec. 3.1 at
 * r = 3: right-hand side +(eps_ko / (64 dz)) (u_{-3} - 6u_{-2} + 15u_{-1}
 * - 20u_0 + 15u_{+1} - 6u_{+2} + u_{+3}); 3 halo rows). */
enum { COSENU_FDKO = 0, COSENU_WENO7 = 1, COSENU_FDKO3 = 2 };

/* Arithmetic.  COSENU_FP64: every operation in double.  COSENU_MIXED: the
 * state y and its RK4 update y += increment stay in double, the per-z
 * velocity moments that form H_nunu are kept as double running sums, and the
 * stencil / WENO / commutator arithmetic and the stage increments are float. */
enum { COSENU_FP64 = 0, COSENU_MIXED = 1 };

/* Error codes. */
enum {
  COSENU_OK = 0,
  COSENU_EINVAL = -1,      /* bad argument or unsupported size */
  COSENU_ENOMEM = -2,      /* device or host allocation failed */
  COSENU_ECUDA = -3,       /* a CUDA runtime call failed */
  COSENU_ENONFINITE = -4,  /* a non-finite value appeared in the state */
  COSENU_ETIMEOUT = -5,    /* a bounded device-side wait gave up */
  COSENU_ECANCELLED = -6,  /* a served run was cancelled */
  COSENU_PENDING = 1       /* a served run has not finished yet (not an error) */
};

/* Physical and numerical parameters (Sec. 2 and 3).
 *   mu       strength of H_nunu, Eq. (ham)                         default 1
 *   omega    vacuum oscillation frequency omega_vac                default 0
 *   theta    vacuum mixing angle theta_vac (radians)               default 0
 *   lambda   constant matter potential: +diag(lambda,0) for nu,
 *            -diag(lambda,0) for nubar (0 in the paper)          default 0
 *   ko_eps   Kreiss-Oliger strength eps_ko (Sec. 3.1, r = 2)       default 0.1
 *   weno_eps epsilon of the WENO weights, Eq. (weight)             default 1e-6
 *   dt       time step                            default 0.4 * dz (C_CFL 0.4) */
typedef struct {
  double mu, omega, theta, lambda, ko_eps, weno_eps, dt;
} cosenu_params;

/* Diagnostics (Sec. 2: P0, |P|; Sec. 5: M_0, delta P).  With
 * P(d) = (2 Re d_ex, -2 Im d_ex, d_ee - d_xx) for a 2x2 matrix d:
 *   tr_nu, tr_nubar  sum_{z,v} dv dz (rho_ee + rho_xx) of each species
 *   M[3]             sum_{z,v} dv dz P(S - Sbar^*)  (the lepton-number vector)
 *   M_vac            sin(2 theta) M[0] - cos(2 theta) M[2]
 *   dP_max           max over cells and species of | |P| / P0 - 1 |
 *   dP_mean          sum |P|/P0 - 1| P0 over nu cells / sum P0 over nu cells
 *   step             RK4 steps taken since the last cosenu_set_state. */
typedef struct {
  double tr_nu, tr_nubar;
  double M[3];
  double M_vac;
  double dP_max, dP_mean;
  int64_t step;
} cosenu_conserved_t;

typedef struct cosenu_s* cosenu_t;

/* Create a solver for an nz x nv grid on [-L/2, L/2) with the given scheme
 * and precision; allocates all device memory (see cosenu_workspace_bytes).
 * The state starts at zero and the parameters at their defaults.
 * Returns NULL on failure; cosenu_last_error(NULL) gives the reason. */
cosenu_t cosenu_create(int64_t nz, int32_t nv, double L, int scheme, int precision);

/* Bytes of device memory one solver needs (state, RK4 stage buffers, moment
 * sums, reduction scratch).  0 for invalid sizes. */
size_t cosenu_workspace_bytes(int64_t nz, int32_t nv, int scheme, int precision);

/* Like cosenu_create, but the solver lives in caller-owned device memory
 * `workspace` of at least cosenu_workspace_bytes() bytes, 256-byte aligned,
 * which must stay valid until cosenu_destroy.  Nothing is allocated on the
 * device. */
cosenu_t cosenu_create_external(int64_t nz, int32_t nv, double L, int scheme, int precision,
                                void* workspace, size_t workspace_bytes);

/* Release the handle and the device memory it allocated.  NULL is a no-op. */
void cosenu_destroy(cosenu_t h);

/* Velocity quadrature of the v integral of Eq. (ham) (and of the diagnostics).
 *   COSENU_MIDPOINT (default): nv bins of width 2/nv, beam at the bin midpoint,
 *     Riemann sum (Sec. 3);
 *   COSENU_TRAPEZOID: vertex points v_j = -1 + j h, h = 2/(nv - 1), trapezoid
 *     rule (Sec. 3.1);
 *   COSENU_SIMPSON: the same points, Simpson's rule (Sec. 3.1): the 1/3 rule on
 *     the first nv - 4 intervals and the 3/8 rule on the last three (nv - 1 is
 *     odd), exact for cubics.
 * Takes effect for later steps and diagnostics; the mixed path's running
 * moments are recomputed.  cosenu_velocities writes the nv beam velocities
 * and weights (either pointer may be NULL).  cosenu_set_state_collective
 * normalises g(v) with these weights. */
enum { COSENU_MIDPOINT = 0, COSENU_TRAPEZOID = 1, COSENU_SIMPSON = 2 };
int cosenu_set_quadrature(cosenu_t h, int32_t mode);
int cosenu_velocities(cosenu_t h, double* v, double* w);

/* Set / read the parameters.  dt <= 0 selects the default 0.4 * dz. */
int cosenu_set_params(cosenu_t h, const cosenu_params* p);
int cosenu_get_params(cosenu_t h, cosenu_params* p);

/* Use the given cudaStream_t (NULL = the legacy default stream) for all
 * later work of this handle. */
int cosenu_set_stream(cosenu_t h, void* stream);

/* Copy a host state (n = 8 nz nv doubles, layout above) into the solver and
 * reset the step counter.  Synchronous with respect to the host buffer. */
int cosenu_set_state(cosenu_t h, const double* host, size_t n);

/* Same from a device buffer of n doubles (stream-ordered, asynchronous). */
int cosenu_set_state_device(cosenu_t h, const double* dev, size_t n);

/* Set the initial state of the collective-oscillation runs of Sec. 5, built on
 * the device, and reset the step counter (waits):
 *   S_ee(z, v)    = g_nu(v),  Sbar_ee(z, v) = alpha g_nubar(v),  S_xx = Sbar_xx = 0,
 *   S_ex = Sbar_ex = eps0 exp(i phi(z)),
 * with g(v) proportional to exp(-(v - 1)^2 / (2 sigma^2)) at the beam velocities,
 * normalised so that sum_j w_j g(v_j) = 1 (quadrature weights, see
 * cosenu_set_quadrature), and the random phase
 * phi(z_i) = 2 pi u_i, u_i = (splitmix64(i XOR seed) >> 11) 2^-53 (splitmix64:
 * x += 0x9E3779B97F4A7C15; x = (x ^ x >> 30) * 0xBF58476D1CE4E5B9;
 * x = (x ^ x >> 27) * 0x94D049BB133111EB; x ^= x >> 31).
 * sigma_nu, sigma_nubar > 0; alpha, eps0 finite. */
int cosenu_set_state_collective(cosenu_t h, double alpha, double sigma_nu, double sigma_nubar,
                                double eps0, uint64_t seed);

/* Copy the current state to a host buffer of n = 8 nz nv doubles (waits). */
int cosenu_get_state(cosenu_t h, double* host, size_t n);

/* Copy rows z0 .. z0+nrows-1 (0 <= z0, z0 + nrows <= nz) of every species and
 * component to host: out[2][4][nrows][nv] doubles (waits).  For inspecting
 * large grids without moving the whole state. */
int cosenu_get_rows(cosenu_t h, int64_t z0, int64_t nrows, double* host);

/* Device pointer of the current state (layout above); valid until the next
 * cosenu_step / cosenu_set_state call. */
const double* cosenu_state_device(cosenu_t h);

/* Enqueue nsteps RK4 steps (4 fused stage kernels each) on the handle's
 * stream.  nsteps = 0 is a no-op. */
int cosenu_step(cosenu_t h, int64_t nsteps);

/* Wait for the handle's stream; report COSENU_ENONFINITE if a non-finite
 * value was written to the state, COSENU_ETIMEOUT if a device-side wait gave
 * up.  The device error flags are cleared after they are reported. */
int cosenu_sync(cosenu_t h);

/* z-averaged state zavg[2][4][nv] and per-z velocity moments of S - Sbar^*
 * vmom[nz][6] = (D3_0, D3_1, Dr_0, Dr_1, Di_0, Di_1) with
 *   D3_n = sum_j dv v_j^n [(S_ee - S_xx) - (Sbar_ee - Sbar_xx)],
 *   Dr_n = sum_j dv v_j^n (Re S_ex - Re Sbar_ex),
 *   Di_n = sum_j dv v_j^n (Im S_ex + Im Sbar_ex)   (Eq. (ham)).
 * Either output may be NULL.  Host buffers; waits. */
int cosenu_moments(cosenu_t h, double* zavg, double* vmom);

/* The per-z velocity moments from which the next stage kernel forms H_nunu,
 * vmom[nz][6] in the order of cosenu_moments (host buffer; waits).
 *   COSENU_MIXED: the double running sums D_n(y) the stage kernels read: set
 *     from y by cosenu_set_state (and cosenu_set_quadrature), then advanced each
 *     RK4 step by the v-sums of the step's float increment, which are summed in
 *     float per (species, component, z) row.  Comparing them with
 *     cosenu_moments' vmom, recomputed from y in double, measures how far the
 *     running sums have drifted.
 *   COSENU_FP64: the stage kernels sum the moments of each stage input in
 *     double from the state itself, so this equals cosenu_moments' vmom. */
int cosenu_running_moments(cosenu_t h, double* vmom);

/* Diagnostics of the current state (waits). */
int cosenu_conserved(cosenu_t h, cosenu_conserved_t* out);

/* delta P(z, v) = |P| / P0 - 1 of every cell (Sec. 5, the error map of the
 * collective runs), out[2 species][nz][nv] host doubles (0 where P0 <= 0),
 * with P = (2 Re rho_ex, -2 Im rho_ex, rho_ee - rho_xx), P0 = rho_ee + rho_xx
 * of the stored state (waits). */
int cosenu_dp_field(cosenu_t h, double* out);

/* Fourier spectrum over z (Sec. 5) of the perpendicular polarisation of one
 * beam, x(z_i) = P1 + i P2 = 2 (Re rho_ex - i Im rho_ex) of species `species`
 * and velocity bin `v_index`:
 *   X(m) = sum_{i=0}^{nz-1} x(z_i) exp(-2 pi i m i / nz),  m = m0 .. m0 + nk - 1
 * (wavenumber k = 2 pi m / L; m may be negative, taken modulo nz), written as
 * out[2 n] = Re X(m0 + n), out[2 n + 1] = Im X(m0 + n), host doubles.  Direct
 * transform, O(nk nz) work; 0 <= nk <= nz, nz <= 2^31 (waits). */
int cosenu_spectrum(cosenu_t h, int32_t species, int32_t v_index, int64_t m0, int64_t nk,
                    double* out);

/* Kernel timing.  With on != 0, every kernel launch of later cosenu_step calls
 * is bracketed by CUDA events on the handle's stream (and steps are launched
 * directly rather than replayed from a graph).  cosenu_stage_times waits for
 * the stream and returns, per kernel k of an RK4 step (k = 1..4: the fused
 * stage kernels; k = 5: the state-increment kernel that ends the step; in the
 * mixed path the small kernel after it that folds the increment's v-moments
 * into the running moments of y is not timed), the summed device time in
 * milliseconds ms[k-1] and the
 * number of timed launches n[k-1] since the last call (arrays of 5; either
 * pointer may be NULL), then clears the sums. */
int cosenu_set_stage_timing(cosenu_t h, int on);
int cosenu_stage_times(cosenu_t h, double* ms, int64_t* n);

/* Steps taken since the last cosenu_set_state. */
int64_t cosenu_steps_taken(cosenu_t h);

/* Description of the last error of h (of this thread for h = NULL). */
const char* cosenu_last_error(cosenu_t h);

/* Kernel launches the library has issued in this process (all handles). */
uint64_t cosenu_kernel_launches(void);

/* ------------------------------------------------------------------------
 * Batched solver: many independent grids advanced together.
 *
 * Every cell of every member is computed with exactly the arithmetic of a
 * single handle (the same kernels, the same summation order), so a member's
 * state after n batched steps is bit-identical to the same handle stepped n
 * times alone.  Members are grouped into classes of equal (scheme, precision,
 * nv); each class runs one fused kernel per RK4 stage over all of its members'
 * z rows (work items of whole or partial grids per CTA), plus one
 * state-increment kernel per class (and, mixed, one moment fold).  Classes are independent
 * chains of kernels, replayed from one CUDA graph as parallel branches.
 *
 * Member handles are created by the batch and share its stream.  Use the
 * single-handle calls on them for everything except stepping and stream
 * control: cosenu_set_params, cosenu_set_state(_device), cosenu_get_state,
 * cosenu_get_rows, cosenu_moments, cosenu_conserved (all ordered with the
 * batch's steps).  cosenu_step on a member steps that member alone.
 * cosenu_set_stream on a member fails with COSENU_EINVAL; cosenu_destroy
 * ignores a member (remove it with cosenu_batch_remove).  A batch is not
 * thread-safe.
 */
typedef struct cosenu_batch_s* cosenu_batch_t;

/* An empty batch on the current device, with its own stream.  NULL on
 * failure (reason in cosenu_last_error(NULL)). */
cosenu_batch_t cosenu_batch_create(void);

/* Destroy the batch and all of its members.  NULL is a no-op. */
void cosenu_batch_destroy(cosenu_batch_t b);

/* Add a member grid (arguments as cosenu_create); *member receives its handle.
 * The state starts at zero and the parameters at their defaults. */
int cosenu_batch_add(cosenu_batch_t b, int64_t nz, int32_t nv, double L, int scheme,
                     int precision, cosenu_t* member);

/* Remove a member and release its device memory (waits for the stream). */
int cosenu_batch_remove(cosenu_batch_t b, cosenu_t member);

/* Number of members. */
int32_t cosenu_batch_size(cosenu_batch_t b);

/* Device bytes held by the members' workspaces plus the batch's launch tables. */
size_t cosenu_batch_device_bytes(cosenu_batch_t b);

/* Enqueue nsteps RK4 steps of every member on the batch's stream and return.
 * The launch plan (classes, work items, graph) is rebuilt here when members or
 * their parameters changed since the last call. */
int cosenu_batch_step(cosenu_batch_t b, int64_t nsteps);

/* Wait for the batch's stream and check every member's error flags (then
 * clear them).  Returns COSENU_ENONFINITE / COSENU_ETIMEOUT like cosenu_sync;
 * *first_bad (may be NULL) receives the index (in cosenu_batch_member order)
 * of the first member with a flag, or -1. */
int cosenu_batch_sync(cosenu_batch_t b, int32_t* first_bad);

/* Handle of member i (0 <= i < cosenu_batch_size), in the order of addition
 * (removal closes the gap).  NULL if out of range. */
cosenu_t cosenu_batch_member(cosenu_batch_t b, int32_t i);

/* Empirical autotuner.  For every (class, stage) it times the candidate launch
 * shapes -- the ring shapes (rows per bulk copy, ring depth) with the best
 * copy sizes, and work items sized for 1, 2 or 4 times the resident CTAs --
 * on real steps of the batch (reps steps per candidate; the members advance by
 * these steps, with results that do not depend on the shape), keeps the
 * fastest, then times whole steps with the classes in series and as parallel
 * graph branches and keeps the faster.  *steps_taken (may be NULL) receives
 * the number of steps the members advanced.  The choice is kept per class key
 * (scheme, precision, nv) across later membership changes. */
int cosenu_batch_tune(cosenu_batch_t b, int32_t reps, int64_t* steps_taken);

/* Launch plan of class c (0 <= c < cosenu_batch_classes()), after the last
 * step or tune call.  Per stage s (index s - 1 for stages 1..4): rows per
 * bulk copy, ring slots, CTAs (work items), shared memory bytes and resident
 * CTAs per SM.  kernel_ms[k - 1]: mean device time of one launch of kernel k
 * (1..4 stages, 5 increment) in the steps timed before the last
 * cosenu_batch_stage_times call (0 if none). */
typedef struct {
  int32_t scheme, precision, nv, members;
  int64_t rows;  /* sum of the members' nz */
  int32_t rows_per_slot[4], ring[4], grid[4], smem[4], occupancy[4];
  int32_t concurrent; /* 1: classes run as parallel graph branches */
  double kernel_ms[5];
} cosenu_batch_class;
int32_t cosenu_batch_classes(cosenu_batch_t b);
int cosenu_batch_class_info(cosenu_batch_t b, int32_t c, cosenu_batch_class* out);

/* Kernel timing of batched steps, summed over classes, as cosenu_stage_times
 * (k = 1..4 the stage kernels, k = 5 the increment kernels).  Timed steps are
 * launched directly with the classes in series, so that each kernel's time is
 * its own. */
int cosenu_batch_set_stage_timing(cosenu_batch_t b, int on);
int cosenu_batch_stage_times(cosenu_batch_t b, double* ms, int64_t* n);

/* The batch's cudaStream_t (for events or for ordering other work with its
 * steps); owned by the batch. */
void* cosenu_batch_stream(cosenu_batch_t b);

/* Description of the last error of b (of this thread for b = NULL). */
const char* cosenu_batch_last_error(cosenu_batch_t b);

/* ------------------------------------------------------------------------
 * Serving: independent runs queued by any thread and executed by one batched
 * solver on the current device, under a device-memory budget (continuous
 * batching).  A worker thread repeats rounds: admit queued runs oldest first
 * while their workspaces (cosenu_workspace_bytes) fit in the budget and the
 * member limit allows -- the first that does not fit stops admission, so no
 * run is overtaken; set up each admitted run (member grid, parameters,
 * initial state); advance the batch by the fewest steps any run still needs,
 * capped at the round length; then retire the runs that reached their step
 * count or raised an error flag (diagnostics, optional copy of the final
 * state, device memory released).  A run's results are bit-identical to the
 * same grid stepped alone.  The calls below are thread-safe.
 */
typedef struct cosenu_server_s* cosenu_server_t;

/* One run.  state: host initial state [2][4][nz][nv], or NULL for the
 * collective initial state of cosenu_set_state_collective with the fields
 * alpha..seed.  out_state: host buffer of 8 nz nv doubles that receives the
 * final state, or NULL.  Both pointers must stay valid until the run has
 * finished (cosenu_poll / cosenu_wait returned 0) or was cancelled. */
typedef struct {
  int64_t nz;
  int32_t nv;
  double L;
  int32_t scheme, precision;
  cosenu_params params;  /* dt <= 0: the default 0.4 dz */
  int64_t nsteps;        /* RK4 steps to take (>= 0) */
  const double* state;
  double alpha, sigma_nu, sigma_nubar, eps0;
  uint64_t seed;
  double* out_state;
} cosenu_request;

/* Outcome of a run.  status: 0, COSENU_PENDING (not finished), or the run's
 * error (COSENU_ENONFINITE, COSENU_ETIMEOUT, COSENU_ECANCELLED, ...).
 * conserved: diagnostics of the final state (status 0).  Times in seconds
 * since the server was created (t_admit, t_done < 0 until they happen). */
typedef struct {
  int32_t status;
  int64_t steps;
  cosenu_conserved_t conserved;
  double t_submit, t_admit, t_done;
} cosenu_result;

typedef struct {
  int64_t submitted, admitted, finished, rounds, steps;
  int32_t queued, running;
  size_t bytes_in_use, peak_bytes, budget;  /* member workspaces */
} cosenu_server_stats;

/* budget_bytes: device memory the runs' workspaces may hold together (the
 * batch's launch tables, about 0.5 KB per run, come on top); max_running:
 * most runs in the batch at once (0 = no limit); round_steps: most steps per
 * round (0 = 64).  NULL on failure (cosenu_server_last_error(NULL)). */
cosenu_server_t cosenu_server_create(size_t budget_bytes, int32_t max_running,
                                     int32_t round_steps);

/* Stop the worker after its current round; runs not finished are cancelled. */
void cosenu_server_destroy(cosenu_server_t s);

/* Queue a run; *ticket identifies it.  COSENU_ENOMEM if its workspace alone
 * exceeds the budget, COSENU_EINVAL for an invalid request. */
int cosenu_submit(cosenu_server_t s, const cosenu_request* r, uint64_t* ticket);

/* COSENU_PENDING while the run is queued or running (*out shows its progress);
 * 0 once it has finished: *out receives the result and the ticket is released.
 * COSENU_EINVAL for an unknown (or already collected) ticket. */
int cosenu_poll(cosenu_server_t s, uint64_t ticket, cosenu_result* out);

/* Like cosenu_poll, but waits up to timeout_s seconds (< 0: no limit). */
int cosenu_wait(cosenu_server_t s, uint64_t ticket, double timeout_s, cosenu_result* out);

/* Cancel a run: a queued run is dropped, a running one leaves the batch at the
 * end of the current round; its result has status COSENU_ECANCELLED. */
int cosenu_cancel(cosenu_server_t s, uint64_t ticket);

int cosenu_server_get_stats(cosenu_server_t s, cosenu_server_stats* out);

/* Description of the last error of s (of this thread for s = NULL). */
const char* cosenu_server_last_error(cosenu_server_t s);

/* Conserved-quantity diagnostics without any device allocation.  (The paper has
 * no counterpart: this entry point exists for callers of this library.)
 *
 * Same quantities as cosenu_conserved, for a state the caller holds in device
 * memory: y_dev is the [2][4][nz][nv] double state (layout above) on an nz x nv
 * grid of length L, theta the vacuum mixing angle used for M_vac, and out_dev
 * a caller-owned device buffer of 8 doubles that receives
 *   tr_nu, tr_nubar, M[0], M[1], M[2], M_vac, dP_max, dP_mean.
 * The sums use the midpoint bins (weight 2/nv per beam): with no handle there is
 * no quadrature setting, so the results equal cosenu_conserved's only for
 * handles on the default COSENU_MIDPOINT quadrature.
 * The work is enqueued on `stream` (a cudaStream_t; NULL = legacy default
 * stream) and the call returns without waiting.
 *
 * Who needs it: callers that cannot call cudaMalloc -- a process whose device
 * memory is already fully handed to another allocator (a framework's caching
 * pool, a serving loop's fixed budget), where one more cudaMalloc would fail or
 * break the budget, and code on a latency-critical path that cannot afford the
 * device-wide synchronisation that cudaFree implies.
 * This function calls no cudaMalloc, cudaFree or other allocating routine.
 *
 * Scratch: the per-block partial sums live in one static device array of the
 * library (1 MiB, held on every GPU that loads the library until the process
 * exits).  Hence:
 *   - the grid may have at most 2^28 (z, v) cells (nz * nv <= 268435456);
 *     larger grids are rejected with COSENU_EINVAL and a message;
 *   - the first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress, with that device current) and keeps it for the
 *     life of the process; make that first call before any stream capture.
 *     The kept address does not survive a reset of the device's primary
 *     context (cudaDeviceReset): do not call this function after one;
 *   - every call on a device shares the array: calls whose work overlaps on the
 *     GPU (different streams without ordering) race and give wrong results.
 *     Each call writes every partial it reads, so no clearing is needed between
 *     calls.
 * Returns 0, COSENU_EINVAL (bad argument, grid too large) or COSENU_ECUDA; the
 * message is in cosenu_last_error(NULL). */
int cosenu_conserved_noalloc(const double* y_dev, int64_t nz, int32_t nv, double L, double theta,
                             double* out_dev, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* COSENU_H */
