/*
 * ecpic_oracle.h -- plain FP64 CPU oracle for the 1D3V explicit
 * energy-conserving particle-in-cell method (EC-PIC) of Powis & Kaganovich,
 * "Accuracy of the Explicit Energy-Conserving Particle-in-Cell Method for
 * Under-resolved Simulations of Capacitively Coupled Plasma Discharges"
 * (arXiv 2308.13092).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  The GPU product
 * path never calls it, links it or shares code with it.
 *
 * Everything is FP64 with absolute particle positions X in [0, L].
 * Nodes x_0 = 0 < x_1 < ... < x_N = L; cell j = [x_j, x_{j+1}).
 *
 * All functions return 0 on success and a negative code on error:
 *   -1 bad argument, -2 call out of order, -3 out of memory,
 *   -4 particle capacity exceeded (births dropped; counted).
 */
#ifndef ECPIC_ORACLE_H
#define ECPIC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OR_MAX_SPECIES 4
#define OR_MAX_PROC 8

/* process kinds (Sec. 2b: e-n elastic, excitation, ionisation, ion-n elastic,
 * charge exchange) */
#define OR_ELASTIC 0
#define OR_EXCITATION 1
#define OR_IONIZATION 2
#define OR_ION_ELASTIC 3
#define OR_CX 4

#define OR_DIRICHLET 0
#define OR_PERIODIC 1
#define OR_SCHEME_EC 0
#define OR_SCHEME_MC 1
#define OR_SCHEME_EC2 2 /* quadratic-spline deposit, linear gather of the face field */
#define OR_SCHEME_MC2 3 /* quadratic-spline deposit and gather of the centred node field */

typedef struct or_run or_run;

/* ---- primitives exposed for pins ------------------------------------- */

/* Philox4x32-10 (Salmon et al., SC'11): out = bijection(ctr) under key. */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                          uint32_t out[4]);

/* id of a particle born in an ionisation event at step k:
 * mix(parent ^ mix(4k + tag)), mix = the splitmix64 output function,
 * tag 1 for the electron, 2 for the ion. */
uint64_t oracle_child_id(uint64_t parent, int64_t step, uint64_t tag);

/* Fixed-point CIC deposit rule (Eq. 2-3 in units of 2^-32 particle):
 * r = floor(xi32 * 2^32); S[cell] += 2^32 - r; S[cell+1] += r.
 * S has N+1 entries and is accumulated into (not cleared). */
int oracle_deposit_fixed(int N, int64_t n, const int32_t* cell,
                         const float* xi, uint64_t* S);
/* Quadratic-spline fixed-point deposit of EC2 (uniform grid): a particle at
 * p = cell + xi (cell units) with r = floor(xi * 2^32) has its nearest node
 * n0 = cell (r < 2^31) or cell + 1, offset U = r or r - 2^32 (2^-32 units);
 * nodes n0-1, n0, n0+1 receive a = floor((2^31 - U)^2 / 2^33), 2^32 - a - b,
 * b = floor((2^31 + U)^2 / 2^33) (exact integers, the shares of the
 * quadratic B-spline to 2^-32).  Beyond a Dirichlet wall the share folds
 * into the wall node; periodic indices wrap (node N is node 0). */
int oracle_deposit_fixed2(int N, int bc, int64_t n, const int32_t* cell, const float* xi,
                          uint64_t* S);

/* Finite-volume Poisson, Eq. 4 on a (possibly non-uniform) grid:
 * (phi_{n+1}-phi_n)/dx_n - (phi_n-phi_{n-1})/dx_{n-1} = -Q_n/eps0,
 * n = 1..N-1, phi_0 and phi_N given.  Q_n is charge per unit area in the
 * control volume of node n.  Thomas algorithm (tridiagonal LU). */
int oracle_poisson_thomas(int N, const double* x, const double* Q,
                          double phi0, double phiN, double* phi);
/* Same system by dense Gaussian elimination with partial pivoting
 * (cross-check for N <= 256). */
int oracle_poisson_dense(int N, const double* x, const double* Q,
                         double phi0, double phiN, double* phi);

/* Field from nodal potential.  EC (Eq. 5): E_j = -(phi_{j+1}-phi_j)/dx_j,
 * N values.  MC: centred node field, N+1 values.  bc: OR_DIRICHLET or
 * OR_PERIODIC (phi_N == phi_0). */
int oracle_field(int N, const double* x, const double* phi, int bc,
                 int scheme, double* E);

/* Doubling non-uniform grid of Sec. 3c.  Units of dx_ref = L/n_ref.  Writes
 * up to cap edges (meters) and returns the number of cells, or <0. */
int oracle_doubling_grid(int n_ref, double L, double L_buff, int dx_min,
                         int dx_max, double* edges, int cap);

/* ---- the simulation --------------------------------------------------- */

int oracle_create(or_run** out);
void oracle_destroy(or_run* r);
/* edges[0] must be 0; strictly increasing; n_edges = N+1 >= 3.
 * phi_0(t) = v_dc + v0*sin(2*pi*f*t + phase) at x = 0, phi_N = 0. */
int oracle_set_grid(or_run* r, const double* edges, int n_edges, int bc,
                    double v0, double freq_hz, double phase_rad, double v_dc);
int oracle_set_scheme(or_run* r, int scheme);
int oracle_add_species(or_run* r, double q, double m, double w,
                       int64_t capacity, int* species_out);
int oracle_set_gas(or_run* r, double n_g, double T_g, double m_g);
/* sigma tabulated at E = i*dE (eV), i = 0..n-1, linear interpolation,
 * held at sigma[n-1] above the table; zero below threshold_eV.
 * product_species: ion species that receives the ion of an ionisation. */
int oracle_add_process(or_run* r, int species, int kind, double threshold_eV,
                       double dE_eV, int n, const float* sigma,
                       int product_species);
/* Loader positions: 0 = uniform random (Philox, default), 1 = quiet start,
 * X_i = (i + 1/2) L / n for i < n per species (the paper is silent on the
 * loading; a quiet start keeps the initial charge noise, and the field energy
 * it holds, near zero).  Before oracle_init. */
int oracle_set_quiet_start(or_run* r, int quiet);
/* Tallies of the paper's diagnostics (Sec. 3a, Fig. 1, Sec. 3b-c):
 *  - EEDF: on sample steps, the kinetic energies (eV) of the particles of
 *    every species with q < 0 in the cells whose centres lie within
 *    eedf_center +- eedf_halfwidth (m; centre < 0: L/2), counted in
 *    eedf_bins bins of eedf_dE, the last bin taking everything above;
 *  - impact energy and angle: on every step, the particles of every species
 *    with q > 0 absorbed at x = 0 (the RF electrode), energy (eV) in
 *    iedf_bins bins of iedf_dE and angle from the normal in iad_bins bins
 *    over 0..90 degrees, from the velocity that carried them out;
 *  - J.E: on sample steps, q w E_i (v^{k-1/2} + v^{k+1/2}) / 2 / dx_j summed
 *    per cell j of the particle at level k (W/m^3), averaged over samples.
 * Before oracle_init; defaults: L/2 +- 0.5 mm, 0.5 eV x 100, 2 eV x 256, 90.
 * reset_averages clears them. */
int oracle_set_tallies(or_run* r, double eedf_center, double eedf_halfwidth, double eedf_dE,
                       int eedf_bins, double iedf_dE, int iedf_bins, int iad_bins);
/* shape5 = {eedf_bins, iedf_bins, iad_bins, first and last EEDF cell} */
int oracle_get_tally_shape(const or_run* r, int* shape5);
/* eedf [ns][eedf_bins], iedf [ns][iedf_bins], iad [ns][iad_bins] (counts),
 * power [ns][N] (W/m^3, mean over samples); any may be NULL.  Returns the
 * number of samples. */
int64_t oracle_get_tallies(const or_run* r, double* eedf, double* iedf, double* iad, double* power);
/* uniform positions + Maxwellian velocities from Philox; w per species is
 * the weight given to oracle_add_species. */
int oracle_init(or_run* r, uint64_t seed, double dt,
                const int64_t* n_per_species, const double* T_eV);
/* Replace a species' particles (X in meters, absolute). Recomputes the
 * charge and field of the current step. */
int oracle_set_particles(or_run* r, int species, const double* X,
                         const double* vx, const double* vy, const double* vz,
                         const uint64_t* id, int64_t n);
int oracle_get_particles(or_run* r, int species, double* X, double* vx,
                         double* vy, double* vz, uint64_t* id, int64_t cap,
                         int64_t* n);
/* Same, in the cell-relative form: X = x_cell + xi * dx_cell. */
int oracle_set_particles_cell(or_run* r, int species, const int32_t* cell,
                              const float* xi, const float* vx,
                              const float* vy, const float* vz,
                              const uint64_t* id, int64_t n);
/* cell j with x_j <= X < x_{j+1} and xi = (X - x_j)/dx_j in FP64. */
int oracle_get_particles_cell(or_run* r, int species, int32_t* cell,
                              double* xi, int64_t cap, int64_t* n);
int oracle_step(or_run* r, int64_t n_steps);
/* Time level k (RF phase and random stream follow it); field formed again. */
int oracle_set_step(or_run* r, int64_t k);
int oracle_reset_averages(or_run* r, int sample_every);

/* counters: out[0]=step, then per species s (OR_MAX_SPECIES slots of 16):
 * n, absorbed_left, absorbed_right, births, lost_capacity, clamps,
 * candidates, collisions[0..7], (unused). */
int oracle_get_counters(const or_run* r, int64_t* out, int cap);
/* instantaneous fields of the current step: phi[N+1], E[N or N+1],
 * Q[N+1] (charge per area in node control volumes). */
int oracle_get_fields(const or_run* r, double* phi, double* E, double* Q);
/* energy of the last completed push (time level of that push):
 * ke[s] = sum 1/2 m w (vx^{k-1/2} vx^{k+1/2} + vy^2 + vz^2), fe = field
 * energy 1/2 eps0 sum_j E_j^2 dx_j (face fields). */
int oracle_get_energy(const or_run* r, double* ke, double* fe);
/* time-averaged profiles over the samples taken so far:
 * density[s*(N+1)+n] (m^-3), phi[N+1], Tx[s*(N+1)+n] (eV, mean of
 * per-sample temperatures), Tx_mom[...] (eV, from averaged moments);
 * any pointer may be NULL.  Returns the number of samples. */
int64_t oracle_get_averages(const or_run* r, double* density, double* phi,
                            double* Tx, double* Tx_mom);
int oracle_nu_max(const or_run* r, int species, double* nu_max,
                  uint32_t* threshold24);

/* ---- particle rebalancing (Sec. 3d proposes it; the rule is this
 * project's design, described at or_rebalance in the source) ----------- */
/* Every particle carries an integer weight multiplier k (it stands for k
 * base particles); deposit, moments, energies and tallies count k.  Before
 * init: rebalance every `every` steps (0 = never), at level k+1 after the
 * field and the sample; merge in cells holding more than `hi` particles of a
 * species, split in cells holding fewer than `lo` (0 < n), aiming at
 * `target` (lo <= target <= hi, target <= 4096); loaded particles (and set_particles) get
 * multiplier m0 (1..65536) and base weight w / m0. */
int oracle_set_rebalance(or_run* r, int every, int target, int lo, int hi, uint32_t m0);
/* one rebalancing of every species now, at the current level */
int oracle_rebalance_now(or_run* r);
/* weight multipliers of a species' particles (order of get_particles) */
int oracle_get_weights(const or_run* r, int species, uint32_t* k, int64_t cap, int64_t* n);
/* replace them (n = the species' count; 1..65536 each); recomputes the field */
int oracle_set_weights(or_run* r, int species, const uint32_t* k, int64_t n);
/* per species s: out3[3s] groups merged, out3[3s+1] particles split,
 * out3[3s+2] cells skipped (above 4096 particles) */
int oracle_get_rebalance_counters(const or_run* r, int64_t* out3);
/* weighted fixed-point CIC rule: S[cell] += k (2^32 - r), S[cell+1] += k r,
 * r = floor(xi32 * 2^32) */
int oracle_deposit_fixed_w(int N, int64_t n, const int32_t* cell, const float* xi,
                           const uint32_t* k, uint64_t* S);

#ifdef __cplusplus
}
#endif
#endif
