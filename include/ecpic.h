/*
 * ecpic.h -- C ABI of libecpic, a GB300 (sm_103a) implementation of the
 * explicit energy-conserving particle-in-cell method (EC-PIC) for 1D3V
 * radio-frequency capacitively coupled discharges, after Powis & Kaganovich,
 * "Accuracy of the Explicit Energy-Conserving Particle-in-Cell Method for
 * Under-resolved Simulations of Capacitively Coupled Plasma Discharges"
 * (arXiv 2308.13092).  Section, equation and table numbers below refer to
 * that paper.
 *
 * Conventions
 *  - Every call returns an ecpic_status (0 = ECPIC_OK, negative = error);
 *    no C++ exception crosses this boundary.  ecpic_last_error() gives a
 *    human-readable message for the last failing call on a handle.
 *  - Host input arrays are copied; the caller keeps ownership.  Output
 *    buffers are allocated by the caller.  All device memory is owned by the
 *    handle that allocated it and released by its destroy call.
 *  - Pointers documented as "device" must point to memory of the handle's
 *    CUDA device; every other pointer is host memory.
 *  - Work is queued on the stream given at creation.  With NULL the handle
 *    creates its own non-blocking stream (the step graphs cannot be captured
 *    on the legacy default stream): work the caller queues on the legacy
 *    stream is not ordered with the library's, so order it through
 *    ecpic_sync() (or pass a stream of your own).  Calls marked "async"
 *    return before the GPU finishes and report device-side errors at the
 *    next ecpic_sync().
 *  - One handle must not be used from two host threads at once.
 *  - Calling out of order (for example step before init) returns
 *    ECPIC_ERR_STATE.
 *
 * Units are SI; energies in eV where noted.  Positions are cell-relative:
 * particle p lies at X = x[cell] + xi * (x[cell+1] - x[cell]), xi in [0,1).
 */
#ifndef ECPIC_H
#define ECPIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  ECPIC_OK = 0,
  ECPIC_ERR_ARG = -1,      /* invalid argument */
  ECPIC_ERR_STATE = -2,    /* call out of order */
  ECPIC_ERR_NOMEM = -3,    /* device allocation or memory budget */
  ECPIC_ERR_CAPACITY = -4, /* a fixed capacity was exceeded (species particles,
                              real-collision records, scratch size) */
  ECPIC_ERR_CUDA = -5,     /* CUDA runtime error */
  ECPIC_ERR_TIMEOUT = -6,  /* a bounded device wait gave up */
  ECPIC_ERR_NAN = -7       /* non-finite particle state detected */
} ecpic_status;

#define ECPIC_MAX_SPECIES 4
#define ECPIC_MAX_PROC 8
#define ECPIC_MAX_CELLS 2048

/* boundary conditions */
#define ECPIC_DIRICHLET_RF 0 /* phi_0 = RF waveform at x = 0, phi_N = 0 */
#define ECPIC_PERIODIC 1     /* periodic, uniform neutralising background */
/* field/gather scheme (Sec. 2a steps 3-4) */
#define ECPIC_SCHEME_EC 0 /* face field Eq. 5, shifted NGP gather Eq. 6-7 */
#define ECPIC_SCHEME_MC 1 /* centred node field, CIC gather */
/* higher-order EC (Sec. 2a: the field interpolation one order below the
 * charge deposit): quadratic-spline deposit, linear interpolation of the face
 * field; uniform grids; the ghost node beyond a wall is the wall node */
#define ECPIC_SCHEME_EC2 2
/* its momentum-conserving partner: the same quadratic deposit and a
 * quadratic-spline gather of the centred node field (uniform grids) */
#define ECPIC_SCHEME_MC2 3
/* collision processes (Sec. 2b) */
#define ECPIC_ELASTIC 0     /* electron-neutral elastic, neutral at rest */
#define ECPIC_EXCITATION 1  /* electron-impact excitation */
#define ECPIC_IONIZATION 2  /* electron-impact ionisation: births e + ion */
#define ECPIC_ION_ELASTIC 3 /* ion-neutral elastic, isotropic in CM frame */
#define ECPIC_CX 4          /* ion-neutral charge exchange */

typedef struct ecpic_run ecpic_run;

/* ------------------------------------------------------------------ */
/* Diagnostics (Sec. 3a: moments averaged at intervals; temperature is
 * the standard deviation of the x velocity distribution).  Scalars are
 * always filled; each array pointer may be NULL, else it must hold
 * n_species * (N+1) (per-species arrays) or N+1 (phi) doubles. */
typedef struct {
  int64_t step;                                /* time level reached */
  double time;                                 /* step * dt */
  int n_species;
  int n_cells;
  int64_t n_live[ECPIC_MAX_SPECIES];           /* particles now */
  int64_t absorbed[ECPIC_MAX_SPECIES][2];      /* at x=0 and x=L, total */
  int64_t births[ECPIC_MAX_SPECIES];           /* ionisation events */
  int64_t lost[ECPIC_MAX_SPECIES];             /* births dropped: capacity */
  int64_t candidates[ECPIC_MAX_SPECIES];       /* null-collision candidates */
  int64_t clamps[ECPIC_MAX_SPECIES];           /* nu_tot > nu_max seen */
  int64_t collisions[ECPIC_MAX_SPECIES][ECPIC_MAX_PROC];
  double ke[ECPIC_MAX_SPECIES]; /* sum 1/2 m w (vx^- vx^+ + vy^2 + vz^2), J/m^2,
                                   at the last sampled push */
  double fe;                    /* 1/2 eps0 sum_j E_j^2 dx_j at that level */
  int64_t n_samples;            /* samples in the averages */
  double* density;              /* [s][n] averaged density, m^-3 */
  double* phi;                  /* [n] averaged potential, V */
  double* temp_x;               /* [s][n] mean of per-sample T_x, eV */
  double* temp_x_mom;           /* [s][n] T_x of the averaged moments, eV */
  /* Tallies since the last ecpic_reset_averages (see ecpic_set_tallies):
   * bin counts (as doubles) of the central EEDF (species with q < 0, sample
   * steps) and of the impact energy and angle at x = 0 (q > 0, every step);
   * the power density J.E per cell (W/m^3), mean over samples. */
  int eedf_bins, iedf_bins, iad_bins;         /* filled by the library */
  int eedf_cell0, eedf_cell1;                 /* cells of the EEDF region */
  double eedf_dE, iedf_dE;                    /* bin widths, eV (angle: 90/iad_bins deg) */
  int64_t impacts_dropped[ECPIC_MAX_SPECIES]; /* beyond the per-step impact list */
  double* eedf;                               /* [s][eedf_bins] or NULL */
  double* iedf;                               /* [s][iedf_bins] or NULL */
  double* iad;                                /* [s][iad_bins] or NULL */
  double* power;                              /* [s][N] or NULL */
  /* particle rebalancing (ecpic_set_rebalance): groups of four merged,
   * particles split, cells left alone (above 4096 particles), since init */
  int64_t rb_merged[ECPIC_MAX_SPECIES];
  int64_t rb_split[ECPIC_MAX_SPECIES];
  int64_t rb_skipped[ECPIC_MAX_SPECIES];
} ecpic_diag;

/* ------------------------------------------------------------------ */
/* Single run.  Order: create -> set_grid -> set_scheme? -> add_species+
 * -> set_gas? -> add_process* -> init -> step / diagnostics / particles.
 * `device` is the CUDA ordinal; `cuda_stream` a cudaStream_t or NULL. */
int ecpic_create(ecpic_run** out, int device, void* cuda_stream);
void ecpic_destroy(ecpic_run* run);
const char* ecpic_last_error(const ecpic_run* run);

/* Grid and electrode bias (Sec. 2a step 2, Sec. 2b, Sec. 3c).  edges: N+1
 * strictly increasing node positions, edges[0] == 0, 2 <= N <=
 * ECPIC_MAX_CELLS; copied.  phi_0(t) = v_dc + v0 sin(2 pi f t + phase) at
 * x = 0 and phi_N = 0 (Dirichlet), or periodic. */
int ecpic_set_grid(ecpic_run* run, const double* edges, int n_edges, int bc,
                   double v0, double freq_hz, double phase_rad, double v_dc);
int ecpic_set_scheme(ecpic_run* run, int scheme);
/* Species (Eq. 2 charge q, mass m, macro-particle weight w in m^-2) with a
 * particle capacity (births beyond it are dropped and counted). */
int ecpic_add_species(ecpic_run* run, double q_C, double m_kg,
                      double weight_per_m2, int64_t capacity, int* species_out);
/* Background gas (Table 1: density, temperature) and its particle mass. */
int ecpic_set_gas(ecpic_run* run, double n_g_m3, double T_g_K, double m_g_kg);
/* Cross section sigma(E) tabulated at E = i*dE (eV), i < n, linear in
 * between, held at sigma[n-1] above, zero below threshold_eV.  All
 * processes of one species share (dE, n).  product_species: the species
 * receiving the ion of an ionisation (else ignored).  Copied. */
int ecpic_add_process(ecpic_run* run, int species, int kind, double threshold_eV,
                      double dE_eV, int n, const float* sigma_m2, int product_species);
/* Loader positions (before ecpic_init): 0 = uniform random from Philox
 * (default), 1 = quiet start, X_i = (i + 1/2) L / n for i < n per species.
 * The paper is silent on the loading; a quiet start keeps the initial charge
 * noise, and the field energy it holds, near zero (App. B heating tests). */
int ecpic_set_quiet_start(ecpic_run* run, int quiet);
/* Particle rebalancing (Sec. 3d: on a non-uniform grid, keep the particles
 * per cell near a target so that the cost follows the number of cells; the
 * paper proposes this and gives no algorithm -- the rule is this library's).
 * Before ecpic_init; EC and MC schemes.  Every particle then carries an
 * integer weight multiplier k (it stands for k particles of the base weight
 * w / m0, w the species weight given to ecpic_add_species); the deposit
 * (Eq. 2-3, in units of 2^-32 base particle), moments, energies and tallies
 * count k, and ionisation products inherit the parent's k.  Loaded particles
 * (and ecpic_set_particles) get k = m0 (1..65536).  Every `every` steps
 * (0: only ecpic_rebalance_now), after the field and the diagnostics sample
 * of that level, per species and cell with n particles:
 *  - n > hi (n <= 4096, else the cell is left alone and counted): order the
 *    particles by (vx, id), cut the order into floor(n/4) groups of four and
 *    merge the min(floor(n/4), ceil((n - target)/2)) groups nearest the
 *    middle of that order (ties: the slower group), skipping groups of total
 *    weight W > 65536; a group becomes two particles at its weighted centroid
 *    of weights a = ceil(W/2), b = W - a and velocities u + sqrt(b/a) d and
 *    u - sqrt(a/b) d (u the mean velocity, d = (s_x, +-s_y, +-s_z) the
 *    per-component standard deviations, signs from Philox with counter
 *    (id lo, id hi, level, (species << 8) | 0x10)), taking the group's two
 *    smallest ids: CIC node charges, momentum and each component's second
 *    moment (so the energy and the x temperature) are kept;
 *  - 0 < n < lo: the min(target - n, #{k >= 2}) heaviest particles (ties:
 *    smallest id) split in place into ceil(k/2) (same id) and floor(k/2)
 *    (id = child of the id at this level, tag 3): nothing changes but the
 *    count.
 * 0 <= lo <= target <= hi, target <= 4096.  Counted in ecpic_diag rb_merged/rb_split/
 * rb_skipped.  A plan that exceeds a species' capacity leaves the particles
 * as they were and fails the run with ECPIC_ERR_CAPACITY. */
int ecpic_set_rebalance(ecpic_run* run, int every, int target, int lo, int hi, uint32_t m0);
/* Rebalance the run now, at its current level (synchronises). */
int ecpic_rebalance_now(ecpic_run* run);
/* Weight multipliers of a species' live particles, in the order of
 * ecpic_get_particles (synchronises); ECPIC_ERR_ARG with *n set if cap is
 * too small.  Runs with ecpic_set_rebalance only. */
int ecpic_get_weights(ecpic_run* run, int species, uint32_t* k, int64_t cap, int64_t* n);
/* Replace the multipliers of the particles set by the last
 * ecpic_set_particles (n equal to its count; 1..65536 each); recomputes the
 * current field. */
int ecpic_set_weights(ecpic_run* run, int species, const uint32_t* k, int64_t n);
/* Diagnostic tallies (Sec. 3a, Fig. 1; before ecpic_init):
 *  - EEDF: on sample steps, kinetic energies (eV) of the particles of every
 *    species with q < 0 in the cells whose centres lie within
 *    eedf_center +- eedf_halfwidth (m; centre < 0: L/2; no such cell: the cell
 *    holding the centre), eedf_bins bins of eedf_dE, the last taking the rest;
 *  - impact energy and angle at the RF electrode: on every step, particles
 *    of every species with q > 0 absorbed at x = 0, energy (eV) in iedf_bins
 *    bins of iedf_dE, angle from the normal in iad_bins bins over 0..90 deg;
 *  - power density J.E per cell: on sample steps, q w E_i (v^{k-1/2} +
 *    v^{k+1/2}) / 2 / dx_j for each particle in cell j at level k (W/m^3).
 * Defaults: L/2 +- 0.5 mm, 0.5 eV x 100, 2 eV x 256, 90.  Read through
 * ecpic_diagnostics; cleared by ecpic_reset_averages. */
int ecpic_set_tallies(ecpic_run* run, double eedf_center_m, double eedf_halfwidth_m,
                      double eedf_dE_eV, int eedf_bins, double iedf_dE_eV, int iedf_bins,
                      int iad_bins);
/* Load n_per_species[s] particles uniformly in [0, L) with Maxwellian
 * velocities of T_eV[s] (Sec. 2b), ids 0..n-1, from the counter-based
 * Philox4x32-10 stream keyed on `seed`; time step dt; then deposit and
 * solve the field of step 0.  Allocates all device memory. */
int ecpic_init(ecpic_run* run, uint64_t seed, double dt_s,
               const int64_t* n_per_species, const double* T_eV);
/* Advance n_steps (async).  One step: EC (or MC) gather and leapfrog push
 * (Eq. 6-9), wall absorption, null-collision MCC, CIC deposit (Eq. 2-3),
 * Poisson (Eq. 4) and field (Eq. 5) of the next time level. */
int ecpic_step(ecpic_run* run, int64_t n_steps);
/* Wait for queued work; return the first device-side error of the run. */
int ecpic_sync(ecpic_run* run);
/* Restart the time averages; sample every `sample_every` steps (0 = off). */
int ecpic_reset_averages(ecpic_run* run, int sample_every);
int ecpic_diagnostics(ecpic_run* run, ecpic_diag* out);
/* Live particles of a species (synchronises).  Returns ECPIC_ERR_ARG with
 * *n set if cap is too small.  Any pointer may be NULL. */
int ecpic_get_particles(ecpic_run* run, int species, int32_t* cell, float* xi,
                        float* vx, float* vy, float* vz, uint64_t* id,
                        int64_t cap, int64_t* n);
/* Replace a species' particles (after init); recomputes the current field. */
int ecpic_set_particles(ecpic_run* run, int species, const int32_t* cell,
                        const float* xi, const float* vx, const float* vy,
                        const float* vz, const uint64_t* id, int64_t n);
/* Fields of the current time level: phi[N+1] (FP64), E[N] for EC or [N+1]
 * for MC (the FP32 values the push uses).  Either may be NULL. */
int ecpic_get_fields(ecpic_run* run, double* phi, float* E);
/* Null-collision bound of a species: nu_max (1/s) and the 24-bit candidate
 * threshold ceil((1 - exp(-nu_max dt)) 2^24). */
int ecpic_nu_max(ecpic_run* run, int species, double* nu_max, uint32_t* threshold24);
/* Counting-sort cadence in steps (>= 1; default 32). */
int ecpic_set_sort_every(ecpic_run* run, int sort_every);
/* Force a counting sort by cell now (compacts absorbed particles). */
int ecpic_sort_now(ecpic_run* run);
/* Particle memory grows with ionisation (Sec. 3a, the discharge's density
 * build-up): raise the capacity of one species of an initialised run to at
 * least `capacity` particles (< 2^31; never shrinks), keeping the run's
 * state.  A new device block is allocated on the run's stream, the run's
 * arrays are copied into it and the old block is freed; the call
 * synchronises the stream and belongs between steps.  ECPIC_ERR_NOMEM leaves
 * the run as it was.  The trajectory does not depend on the capacity. */
int ecpic_reserve(ecpic_run* run, int species, int64_t capacity);
/* on = 1: after every chunk of about 64 steps (whole sort cycles) ecpic_step
 * doubles the capacity of any species filled beyond 3/4 of it (as
 * ecpic_reserve), synchronising the stream at each chunk; on = 0 (the
 * default): ecpic_step stays asynchronous and a full species fails the run
 * with ECPIC_ERR_CAPACITY.  The engine always grows its runs this way. */
int ecpic_set_auto_grow(ecpic_run* run, int on);
/* Measurement: advance n_steps with plain launches (no graph), bracketing
 * each kernel phase with CUDA events on the run's stream; synchronises.
 * ms[0..3] = summed device time of the particle pass, the field solve, the
 * counting sort and the real-collision kernel; launches[0..3] = their launch
 * counts.  Same physics as ecpic_step. */
int ecpic_profile_step(ecpic_run* run, int64_t n_steps, double* ms, int64_t* launches);
/* Pass-kernel grid size override (0 = automatic); for tuning. */
int ecpic_set_pass_grid(ecpic_run* run, int ctas);
/* Autotuner over the sort cadence K and the particles per CTA: times the
 * graph-replayed step for each candidate pair of counting-sort cadence K in
 * {8, 16, 32, 64} and pass grid (automatic, one wave at full or half
 * occupancy, two or four waves), steps_per_trial steps each (at least 2K,
 * rounded up to whole sort cycles and, where their common multiple is at most
 * 8x that, whole energy-sample cycles of the resident runs), every pair
 * twice (in order, then in reverse order, so that the discharges' evolution
 * during the trials weighs on all pairs alike), and keeps the pair with the
 * least mean device time per particle-step.  The trials advance
 * the run for real; results do not depend on K or the grid (integer
 * deposit, id-keyed random numbers).  Outputs may be NULL: the chosen K, the
 * chosen grid (0 = automatic) and its ns per particle-step.  Synchronises. */
int ecpic_autotune(ecpic_run* run, int64_t steps_per_trial, int* sort_every, int* pass_ctas,
                   double* ns_per_particle_step);
/* As ecpic_autotune with the sort cadences to try given explicitly: ks[0..n_ks)
 * (1..4096 each, 1 <= n_ks <= 64), e.g. the divisors of a measurement window
 * so that the window holds whole sort cycles. */
int ecpic_autotune_ks(ecpic_run* run, int64_t steps_per_trial, const int* ks, int n_ks,
                      int* sort_every, int* pass_ctas, double* ns_per_particle_step);
/* Measurement of the stepping itself.  on = 1 captures the step graphs again
 * with an event-record node after every kernel phase (two instances of each
 * graph alternate, so that the host reads one while the other runs); every
 * step that ecpic_step advances from then on adds the device time of its
 * phases (CUDA events on the run's stream) to running sums.  The sums thus
 * come from the very replays that advance the run, not from a separate
 * profiling pass.  on = 0 restores the plain graphs (the sums are kept). */
int ecpic_set_phase_timing(ecpic_run* run, int on);
/* Read and clear the phase sums (waits for the timed steps): ms[0..3] = the
 * particle pass, the field solve, the counting sort, the real-collision
 * kernel; launches[0..3] their launch counts (a sort is four launches);
 * *steps and *sorts timed.  Any pointer may be NULL. */
int ecpic_phase_times(ecpic_run* run, double* ms, int64_t* launches, int64_t* steps,
                      int64_t* sorts);
/* The counting-sort cadence in steps and the steps taken since the last
 * sort (0: the next step starts a sort cycle).  Either pointer may be NULL. */
int ecpic_sort_state(ecpic_run* run, int* sort_every, int* since_sort);

/* ------------------------------------------------------------------ */
/* Batched and served runs.  An engine keeps up to max_slots independent
 * discharges resident on one GPU and advances all of them with one launch per
 * kernel phase (replayed from CUDA graphs); the runs may differ in grid, cell
 * count, particle count, voltage, pressure, scheme and time step.  Requests
 * are admitted first-fit, in submission order, as slots and the device-memory
 * budget allow; each run stops at its own step count and is retired with its
 * diagnostics.  The paper ran several simulations concurrently on one GPU
 * (Sec. 2b); this is that mode of use made first-class. */
typedef struct ecpic_engine ecpic_engine;

typedef struct {
  int species;          /* index within the run's species */
  int kind;             /* ECPIC_ELASTIC ... ECPIC_CX */
  double threshold_eV;
  double dE_eV;
  int n;                /* table entries */
  const float* sigma_m2;/* host, n entries; copied at submit */
  int product_species;  /* ionisation only */
} ecpic_process_desc;

typedef struct {
  const double* edges;  /* host, n_edges entries; copied at submit */
  int n_edges;
  int bc;
  double v0, freq_hz, phase_rad, v_dc;
  int scheme;
  int n_species;
  double q[ECPIC_MAX_SPECIES], m[ECPIC_MAX_SPECIES], w[ECPIC_MAX_SPECIES];
  int64_t capacity[ECPIC_MAX_SPECIES];
  int64_t n_init[ECPIC_MAX_SPECIES];
  double T_eV[ECPIC_MAX_SPECIES];
  double n_gas, T_gas, m_gas; /* n_gas = 0: no gas */
  int n_proc;
  const ecpic_process_desc* procs; /* host, n_proc entries; copied at submit */
  uint64_t seed;
  double dt;
  int sample_every;     /* diagnostics sampling cadence (0 = off) */
  int quiet_start;      /* 1: evenly spaced positions (ecpic_set_quiet_start) */
  /* tallies as ecpic_set_tallies; eedf_bins = 0 keeps every default */
  double eedf_center, eedf_halfwidth, eedf_dE;
  int eedf_bins;
  double iedf_dE;
  int iedf_bins, iad_bins;
  /* particle rebalancing as ecpic_set_rebalance; rb_m0 = 0 leaves it off */
  int rb_every, rb_target, rb_lo, rb_hi;
  uint32_t rb_m0;
} ecpic_run_config;

/* max_cells bounds N of every admitted run; species_per_run bounds their
 * species count; mem_budget_bytes bounds the particle and grid memory of the
 * resident runs at admission (0 = no limit; a resident run whose particle
 * capacity grows may take the total past it). */
int ecpic_engine_create(ecpic_engine** out, int device, void* cuda_stream,
                        size_t mem_budget_bytes, int max_slots, int max_cells,
                        int species_per_run);
void ecpic_engine_destroy(ecpic_engine* eng);
const char* ecpic_engine_last_error(const ecpic_engine* eng);
/* Queue a run for n_steps steps; *ticket identifies it.  Validates and
 * copies the configuration; ECPIC_ERR_NOMEM if it could never fit. */
int ecpic_engine_submit(ecpic_engine* eng, const ecpic_run_config* cfg, int64_t n_steps,
                        uint64_t* ticket);
/* One scheduling round: admit queued runs that fit (first fit in submission
 * order; the round's admissions are loaded, deposited and given their step-0
 * field together, in one launch of each kernel), advance every resident run
 * by up to max_steps steps (runs stop at their own step count; every about 64
 * steps, a species filled beyond 3/4 of its capacity has it doubled, see
 * ecpic_set_auto_grow), wait, and retire the runs that finished.
 * *n_resident (may be NULL) receives the number of runs resident after the
 * round, *n_queued the queue length. */
int ecpic_engine_pump(ecpic_engine* eng, int64_t max_steps, int* n_resident, int* n_queued);
/* State of a ticket: 0 queued, 1 resident, 2 finished, < 0 an ecpic_status
 * error of that run.  When finished, or resident (then read from the device:
 * synchronises), and out != NULL, fills its diagnostics (the profile arrays
 * of out, if not NULL, sized n_species*(N+1) / N+1).  *steps_done /
 * *particle_steps (may be NULL) report its progress as of the last pump. */
int ecpic_engine_poll(ecpic_engine* eng, uint64_t ticket, int* state, ecpic_diag* out,
                      int64_t* steps_done, int64_t* particle_steps);
/* Forget a finished ticket's stored results. */
int ecpic_engine_release(ecpic_engine* eng, uint64_t ticket);
/* Totals since creation: particle-steps advanced, runs finished, and the
 * device bytes currently held by resident runs. */
int ecpic_engine_stats(ecpic_engine* eng, int64_t* particle_steps, int64_t* runs_finished,
                       int64_t* bytes_resident);
/* Tuning: pass-kernel CTAs (0 = all SMs), counting-sort cadence. */
int ecpic_engine_tune(ecpic_engine* eng, int pass_ctas, int sort_every);
/* Autotuner over the resident runs, as ecpic_autotune (advances them; runs
 * that reach their end during the trials finish normally). */
int ecpic_engine_autotune(ecpic_engine* eng, int64_t steps_per_trial, int* sort_every,
                          int* pass_ctas, double* ns_per_particle_step);
/* Measurement: advance the resident runs n_steps with plain launches,
 * bracketing each kernel phase with CUDA events on the engine's stream (see
 * ecpic_profile_step: ms[0..3], launches[0..3]); synchronises.  No admission
 * or retirement. */
int ecpic_engine_profile(ecpic_engine* eng, int64_t n_steps, double* ms, int64_t* launches);
/* The engine's counterparts of ecpic_autotune_ks, ecpic_set_phase_timing,
 * ecpic_phase_times and ecpic_sort_state, over its resident runs. */
int ecpic_engine_autotune_ks(ecpic_engine* eng, int64_t steps_per_trial, const int* ks, int n_ks,
                             int* sort_every, int* pass_ctas, double* ns_per_particle_step);
int ecpic_engine_set_phase_timing(ecpic_engine* eng, int on);
int ecpic_engine_phase_times(ecpic_engine* eng, double* ms, int64_t* launches, int64_t* steps,
                             int64_t* sorts);
int ecpic_engine_sort_state(ecpic_engine* eng, int* sort_every, int* since_sort);

/* ------------------------------------------------------------------ */
/* Doubling non-uniform grid (Sec. 3c rules 1-4): buffers of dx_min cells of
 * total length >= L_buff at both electrodes, then cell sizes doubling up to
 * dx_max (sizes in units of dx_ref = L/n_ref).  Writes the N+1 edges (m) into
 * edges[cap] and returns N (> 0), or a negative ecpic_status. */
int ecpic_doubling_grid(int n_ref, double L, double L_buff, int dx_min, int dx_max,
                        double* edges, int cap);

/* ------------------------------------------------------------------ */
/* Kernel-level entry points on caller-owned device memory (tests, tools).
 * Fixed-point CIC deposit (Eq. 2-3 in units of 2^-32 particle): for each
 * particle r = floor(xi*2^32), S[cell] += 2^32 - r, S[cell+1] += r.
 * d_cell/d_xi: device, n entries; d_S: device, N+1 uint64, accumulated.
 * Particles with cell < 0 are skipped.  Async on cuda_stream. */
int ecpic_deposit_device(int N, int64_t n, const int32_t* d_cell, const float* d_xi,
                         uint64_t* d_S, void* cuda_stream);
/* Quadratic-spline fixed-point deposit of ECPIC_SCHEME_EC2: with r =
 * floor(xi 2^32), nearest node n0 = cell + (r >= 2^31) and offset U = r or
 * r - 2^32, nodes n0-1, n0, n0+1 receive a = floor((2^31-U)^2 / 2^33),
 * 2^32 - a - b, b = floor((2^31+U)^2 / 2^33), added to d_S (N+1 uint64).
 * bc: Dirichlet folds shares beyond a wall into the wall node; periodic wraps
 * (node N is node 0, and d_S[N] is set to d_S[0] afterwards).  Async. */
int ecpic_deposit_device2(int N, int bc, int64_t n, const int32_t* d_cell, const float* d_xi,
                          uint64_t* d_S, void* cuda_stream);
/* Bounds-check record of a library built with -DECPIC_CHECKS: out[0] = first
 * failing check site (0 = none), out[1] = its index, out[2] = its bound,
 * out[3] = number of failed checks.  Plain builds report zeros. */
int ecpic_debug_checks(int64_t* out4);
/* Philox4x32-10 on the device: out[4i..4i+3] = Philox(counter = ctr[4i..],
 * key = key[2i..]) for i < n.  All pointers device.  Async. */
int ecpic_philox_device(int64_t n, const uint32_t* d_ctr, const uint32_t* d_key,
                        uint32_t* d_out, void* cuda_stream);

/* ------------------------------------------------------------------ */
/* Allocation-free variant of ecpic_deposit_device.  The paper has no
 * counterpart: this is a service entry point of this library, not a step of
 * the method.
 *
 * It is for callers that must not allocate device memory while they run: a
 * process that handed all free HBM to its own pool at start-up (a cudaMalloc
 * would fail there), or a latency-bound loop that a cudaMalloc/cudaFree would
 * stall by synchronising the device.  It calls no cudaMalloc, cudaFree or
 * other allocating routine.  Its scratch is a fixed array of
 * ECPIC_NOALLOC_SCRATCH_BYTES (4 MiB) in the library's own device image,
 * holding per-block partial sums; nothing in it has to start at zero, since
 * each call writes every entry that it later reads.
 *
 * Arguments and result as ecpic_deposit_device: d_cell/d_xi device, n
 * entries (cell < 0 skipped, 0 <= xi < 1); d_S device, N+1 uint64, the
 * fixed-point sums are ADDED to it (a plain read-modify-write, not atomics).
 * Bit-identical to ecpic_deposit_device on the same input.  Async on
 * cuda_stream, which must belong to the current device.
 *
 * Limits and errors: 1 <= N <= ECPIC_NOALLOC_MAX_CELLS (2048), else
 * ECPIC_ERR_CAPACITY for N above it and ECPIC_ERR_ARG for bad arguments; n is
 * not limited.
 *
 * Set-up: the first call on each device (with that device current) looks up
 * the scratch array's address and keeps it; if you capture streams, make a
 * first call on each device before any capture begins.  That first lookup
 * also loads the library's device code, which commits the 4 MiB array (and
 * the code) in device memory: make the first call -- a call with n == 0 does
 * only this set-up -- before handing the device's free memory to a pool.  The
 * address is kept for the life of the process: after cudaDeviceReset (or
 * anything else that destroys the device's primary context) the kept address
 * is stale and this entry point must not be called again in that process.
 *
 * Races: all calls on a device share the one scratch array.  Calls that may
 * overlap -- on different streams or from different host threads without
 * ordering between them -- race on it and corrupt each other's results, and a
 * kernel writing d_S while a call runs races on d_S; order such calls on one
 * stream or with events. */
#define ECPIC_NOALLOC_SCRATCH_BYTES (4u << 20)
#define ECPIC_NOALLOC_MAX_CELLS 2048
int ecpic_deposit_device_noalloc(int N, int64_t n, const int32_t* d_cell, const float* d_xi,
                                 uint64_t* d_S, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif
