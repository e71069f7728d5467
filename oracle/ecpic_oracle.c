/*
 * ecpic_oracle.c -- plain, slow, FP64 CPU oracle for the 1D3V EC-PIC hot
 * path of Powis & Kaganovich (arXiv 2308.13092).
 *
 * TEST INFRASTRUCTURE ONLY.  It is loaded by the tests, the smoke check and
 * the CPU-baseline leg of the benchmark; the GPU product never calls it.
 *
 * The time loop follows Sec. 2a (steps 1-7), rotated so that one call of
 * step() does: gather + leapfrog push (Eq. 6-9) -> wall absorption ->
 * Monte-Carlo collisions (step 6) -> CIC deposit (Eq. 2-3) -> Poisson (Eq. 4)
 * -> field (Eq. 5, or the centred MC field).  The first deposit, solve and
 * field are done at init.
 *
 * Readings of points the paper leaves open (node count, weights, boundary
 * volumes, wall rule, collision details, random-number layout) are listed in
 * the project design notes and repeated at the function that takes them.
 *
 * Parity status: every routine here is pinned by a CPU test against a closed
 * form, an invariant, a library routine or a printed table of the paper,
 * except the time-averaged profiles of a full RF-CCP run, whose parity with
 * the paper is unpinned (no figure data and no Turner cross sections exist
 * in this project; only GPU-vs-oracle agreement is tested there).
 */
#include "ecpic_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* CODATA 2018 */
#define OR_QE 1.602176634e-19
#define OR_EPS0 8.8541878128e-12
#define OR_KB 1.380649e-23

#define OR_TWO_PI 6.283185307179586476925286766559

typedef struct {
  int kind;
  double thr;    /* eV */
  double dE;     /* eV */
  int n;
  double* sigma; /* m^2, copied from the caller's float table */
  int product;   /* ion species of an ionisation, else -1 */
} or_process;

typedef struct {
  double q, m, w;
  double wb;        /* base weight: a particle of multiplier k weighs k * wb */
  int64_t cap, n;
  double *X, *vx, *vy, *vz;
  uint64_t* id;
  uint32_t* mw;     /* weight multipliers (all 1 without rebalancing) */
  int nproc;
  or_process proc[OR_MAX_PROC];
  int heavy;        /* has ion-neutral processes: sample the neutral */
  double nu_max;    /* 1/s */
  uint32_t thr24;   /* candidate iff (r0 >> 8) < thr24 */
  /* counters */
  int64_t absorbed[2], births, lost, clamps, candidates;
  int64_t coll[OR_MAX_PROC];
  int64_t rb_merged, rb_split, rb_skipped; /* groups merged, particles split, cells skipped */
  double ke;
  /* per-node deposit and moments at the current step */
  double *D, *M1, *M2;
  /* time averages */
  double *acc_n, *acc_T, *acc_M0, *acc_M1, *acc_M2;
  /* tallies (Sec. 3a diagnostics): EEDF of the central region on sample
   * steps (q < 0), impact energy and angle at x = 0 on every step (q > 0),
   * J.E per cell summed over sample steps */
  double *eedf, *iedf, *iad, *acc_P;
} or_species;

struct or_run {
  int N;
  double* x;  /* N+1 edges */
  double* dx; /* N cell widths */
  double* V;  /* N+1 node control volumes */
  double L;
  int bc;
  double v0, freq, phase, vdc;
  int scheme;
  int grid_set;
  int ns;
  or_species sp[OR_MAX_SPECIES];
  double ng, Tg, mg;
  int gas_set;
  uint64_t seed;
  double dt;
  int64_t step;
  int initialized;
  int quiet; /* loader: evenly spaced positions instead of random ones */
  /* tally set-up: EEDF region centre and half-width (m), bin widths (eV),
   * bin counts; eedf_c0..eedf_c1 the cells of the region */
  double eedf_xc, eedf_hw, eedf_dE, iedf_dE;
  int eedf_n, iedf_n, iad_n, eedf_c0, eedf_c1;
  double *Q, *phi, *E;
  double fe;
  int sample_every;
  int64_t n_samples;
  double* acc_phi;
  /* particle rebalancing (set before init): every rb_every steps; merge in
   * cells holding more than rb_hi particles of a species, split in cells
   * holding fewer than rb_lo; aim rb_target; loaded multiplier rb_m0 */
  int rb_every, rb_target, rb_lo, rb_hi;
  uint32_t rb_m0;
};

/* ------------------------------------------------------------------ */
/* Philox4x32-10, written from its definition in Salmon, Moraes, Dror &
 * Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11): ten rounds
 * of two 32x32->64 multiplications with the Weyl-sequence key schedule.   */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                          uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* splitmix64 output function (Steele, Lea & Flood, OOPSLA 2014). */
static uint64_t or_mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

uint64_t oracle_child_id(uint64_t parent, int64_t step, uint64_t tag) {
  return or_mix64(parent ^ or_mix64((uint64_t)step * 4u + tag));
}

/* 24-bit uniform in [0,1): (r >> 8) * 2^-24 */
static double or_u24(uint32_t r) { return (double)(r >> 8) * (1.0 / 16777216.0); }
/* 24-bit uniform in (0,1]: ((r >> 8) + 1) * 2^-24 */
static double or_u24_open(uint32_t r) {
  return (double)((r >> 8) + 1u) * (1.0 / 16777216.0);
}

/* Box-Muller: two standard normals from two uniforms (u1 in (0,1]). */
static void or_box_muller(double u1, double u2, double* z0, double* z1) {
  double rad = sqrt(-2.0 * log(u1));
  *z0 = rad * cos(OR_TWO_PI * u2);
  *z1 = rad * sin(OR_TWO_PI * u2);
}

/* isotropic unit vector from two uniforms: polar axis along x. */
static void or_isotropic(double ua, double ub, double d[3]) {
  double c = 1.0 - 2.0 * ua;
  double s = sqrt(fmax(0.0, 1.0 - c * c));
  double ph = OR_TWO_PI * ub;
  d[0] = c;
  d[1] = s * cos(ph);
  d[2] = s * sin(ph);
}

static void or_draw(const or_run* r, uint64_t id, uint32_t step_word,
                    uint32_t word3, uint32_t out[4]) {
  uint32_t ctr[4] = {(uint32_t)id, (uint32_t)(id >> 32), step_word, word3};
  uint32_t key[2] = {(uint32_t)r->seed, (uint32_t)(r->seed >> 32)};
  oracle_philox4x32_10(ctr, key, out);
}

/* ------------------------------------------------------------------ */
/* Deposit (Eq. 2-3) in fixed point.                                   */
int oracle_deposit_fixed(int N, int64_t n, const int32_t* cell,
                         const float* xi, uint64_t* S) {
  if (N < 1 || n < 0 || (n > 0 && (!cell || !xi)) || !S) return -1;
  for (int64_t i = 0; i < n; ++i) {
    int j = cell[i];
    float f = xi[i];
    if (j < 0 || j >= N || !(f >= 0.0f) || !(f < 1.0f)) return -1;
    uint32_t rgt = (uint32_t)((double)f * 4294967296.0); /* floor, f < 1 */
    uint64_t lft = 4294967296ull - (uint64_t)rgt;
    S[j] += lft;
    S[j + 1] += (uint64_t)rgt;
  }
  return 0;
}

/* ------------------------------------------------------------------ */
/* Poisson, Eq. 4 in finite-volume form (exact Eq. 4 times dx on a uniform
 * grid).  Row n (1..N-1): a_n phi_{n-1} + b_n phi_n + c_n phi_{n+1} = d_n. */
static void or_poisson_rows(int N, const double* x, const double* Q,
                            double phi0, double phiN, double* a, double* b,
                            double* c, double* d) {
  for (int n = 1; n <= N - 1; ++n) {
    double dl = x[n] - x[n - 1];
    double dr = x[n + 1] - x[n];
    a[n] = 1.0 / dl;
    c[n] = 1.0 / dr;
    b[n] = -(1.0 / dl + 1.0 / dr);
    d[n] = -Q[n] / OR_EPS0;
  }
  d[1] -= a[1] * phi0;
  d[N - 1] -= c[N - 1] * phiN;
}

int oracle_poisson_thomas(int N, const double* x, const double* Q,
                          double phi0, double phiN, double* phi) {
  if (N < 2 || !x || !Q || !phi) return -1;
  double* a = malloc(sizeof(double) * (size_t)(N + 1));
  double* b = malloc(sizeof(double) * (size_t)(N + 1));
  double* c = malloc(sizeof(double) * (size_t)(N + 1));
  double* d = malloc(sizeof(double) * (size_t)(N + 1));
  if (!a || !b || !c || !d) {
    free(a); free(b); free(c); free(d);
    return -3;
  }
  or_poisson_rows(N, x, Q, phi0, phiN, a, b, c, d);
  /* forward elimination (L of the tridiagonal LU) */
  for (int n = 2; n <= N - 1; ++n) {
    double m = a[n] / b[n - 1];
    b[n] -= m * c[n - 1];
    d[n] -= m * d[n - 1];
  }
  /* back substitution (U) */
  phi[0] = phi0;
  phi[N] = phiN;
  phi[N - 1] = d[N - 1] / b[N - 1];
  for (int n = N - 2; n >= 1; --n) phi[n] = (d[n] - c[n] * phi[n + 1]) / b[n];
  free(a); free(b); free(c); free(d);
  return 0;
}

int oracle_poisson_dense(int N, const double* x, const double* Q,
                         double phi0, double phiN, double* phi) {
  if (N < 2 || N > 256 || !x || !Q || !phi) return -1;
  int m = N - 1;
  double* A = calloc((size_t)m * (size_t)(m + 1), sizeof(double));
  double* a = malloc(sizeof(double) * (size_t)(N + 1));
  double* b = malloc(sizeof(double) * (size_t)(N + 1));
  double* c = malloc(sizeof(double) * (size_t)(N + 1));
  double* d = malloc(sizeof(double) * (size_t)(N + 1));
  if (!A || !a || !b || !c || !d) {
    free(A); free(a); free(b); free(c); free(d);
    return -3;
  }
  or_poisson_rows(N, x, Q, phi0, phiN, a, b, c, d);
  /* augmented matrix, unknown k <-> node k+1 */
  for (int r = 0; r < m; ++r) {
    int n = r + 1;
    if (r > 0) A[r * (m + 1) + (r - 1)] = a[n];
    A[r * (m + 1) + r] = b[n];
    if (r < m - 1) A[r * (m + 1) + (r + 1)] = c[n];
    A[r * (m + 1) + m] = d[n];
  }
  for (int col = 0; col < m; ++col) {
    int piv = col;
    for (int r = col + 1; r < m; ++r)
      if (fabs(A[r * (m + 1) + col]) > fabs(A[piv * (m + 1) + col])) piv = r;
    if (piv != col)
      for (int k = 0; k <= m; ++k) {
        double t = A[col * (m + 1) + k];
        A[col * (m + 1) + k] = A[piv * (m + 1) + k];
        A[piv * (m + 1) + k] = t;
      }
    for (int r = col + 1; r < m; ++r) {
      double f = A[r * (m + 1) + col] / A[col * (m + 1) + col];
      for (int k = col; k <= m; ++k) A[r * (m + 1) + k] -= f * A[col * (m + 1) + k];
    }
  }
  for (int r = m - 1; r >= 0; --r) {
    double s = A[r * (m + 1) + m];
    for (int k = r + 1; k < m; ++k) s -= A[r * (m + 1) + k] * phi[k + 1];
    phi[r + 1] = s / A[r * (m + 1) + r];
  }
  phi[0] = phi0;
  phi[N] = phiN;
  free(A); free(a); free(b); free(c); free(d);
  return 0;
}

/* Field.  EC: Eq. 5, one value per cell (face-centred on the staggered
 * reading of Sec. 2a).  MC: centred difference at interior nodes,
 * one-sided at Dirichlet end nodes, wrapped when periodic. */
int oracle_field(int N, const double* x, const double* phi, int bc,
                 int scheme, double* E) {
  if (N < 2 || !x || !phi || !E) return -1;
  if (scheme == OR_SCHEME_EC) {
    for (int j = 0; j < N; ++j) E[j] = -(phi[j + 1] - phi[j]) / (x[j + 1] - x[j]);
    return 0;
  }
  for (int n = 1; n <= N - 1; ++n)
    E[n] = -(phi[n + 1] - phi[n - 1]) / (x[n + 1] - x[n - 1]);
  if (bc == OR_PERIODIC) {
    double dl = x[N] - x[N - 1], dr = x[1] - x[0];
    E[0] = -(phi[1] - phi[N - 1]) / (dl + dr);
    E[N] = E[0];
  } else {
    E[0] = -(phi[1] - phi[0]) / (x[1] - x[0]);
    E[N] = -(phi[N] - phi[N - 1]) / (x[N] - x[N - 1]);
  }
  return 0;
}

/* ------------------------------------------------------------------ */
/* Doubling grid (Sec. 3c rules 1-4; L_buff = 5 cm for Table 2).
 * Half-domain of H = n_ref/2 reference cells: ceil(L_buff/dx_min) cells of
 * dx_min from the wall, then greedily the next cell is twice the previous one
 * when that stays <= dx_max and the current position is a multiple of the
 * doubled size; otherwise the previous size.  Mirrored about the centre. */
int oracle_doubling_grid(int n_ref, double L, double L_buff, int dx_min,
                         int dx_max, double* edges, int cap) {
  if (n_ref < 2 || (n_ref & 1) || L <= 0 || L_buff < 0 || dx_min < 1 ||
      dx_max < dx_min || !edges)
    return -1;
  double dx_ref = L / (double)n_ref;
  int H = n_ref / 2;
  int* size = malloc(sizeof(int) * (size_t)H);
  if (!size) return -3;
  int nh = 0, pos = 0;
  int nb = (int)ceil(L_buff / (dx_min * dx_ref) - 1e-9);
  for (int i = 0; i < nb && pos < H; ++i) {
    int s = dx_min;
    if (pos + s > H) s = H - pos;
    size[nh++] = s;
    pos += s;
  }
  int prev = dx_min;
  while (pos < H) {
    int s = prev;
    if (2 * prev <= dx_max && pos % (2 * prev) == 0) s = 2 * prev;
    while (pos + s > H && s > dx_min) s /= 2;
    if (pos + s > H) s = H - pos;
    size[nh++] = s;
    pos += s;
    prev = s;
  }
  int ncell = 2 * nh;
  if (ncell + 1 > cap) {
    free(size);
    return -1;
  }
  int u = 0;
  edges[0] = 0.0;
  for (int i = 0; i < nh; ++i) {
    u += size[i];
    edges[i + 1] = u * dx_ref;
  }
  for (int i = nh - 1; i >= 0; --i) {
    u += size[i];
    edges[ncell - i] = u * dx_ref;
  }
  edges[ncell] = L;
  free(size);
  return ncell;
}

/* ------------------------------------------------------------------ */
static void or_free_species(or_species* s) {
  free(s->X); free(s->vx); free(s->vy); free(s->vz); free(s->id); free(s->mw);
  free(s->D); free(s->M1); free(s->M2);
  free(s->eedf); free(s->iedf); free(s->iad); free(s->acc_P);
  free(s->acc_n); free(s->acc_T); free(s->acc_M0); free(s->acc_M1);
  free(s->acc_M2);
  for (int k = 0; k < s->nproc; ++k) free(s->proc[k].sigma);
  memset(s, 0, sizeof(*s));
}

int oracle_create(or_run** out) {
  if (!out) return -1;
  or_run* r = calloc(1, sizeof(or_run));
  if (!r) return -3;
  r->rb_m0 = 1;
  *out = r;
  return 0;
}

void oracle_destroy(or_run* r) {
  if (!r) return;
  for (int s = 0; s < r->ns; ++s) or_free_species(&r->sp[s]);
  free(r->x); free(r->dx); free(r->V); free(r->Q); free(r->phi); free(r->E);
  free(r->acc_phi);
  free(r);
}

static int or_alloc_node_arrays(or_run* r, or_species* s) {
  size_t nn = (size_t)r->N + 1;
  s->D = calloc(nn, sizeof(double));
  s->M1 = calloc(nn, sizeof(double));
  s->M2 = calloc(nn, sizeof(double));
  s->acc_n = calloc(nn, sizeof(double));
  s->acc_T = calloc(nn, sizeof(double));
  s->acc_M0 = calloc(nn, sizeof(double));
  s->acc_M1 = calloc(nn, sizeof(double));
  s->acc_M2 = calloc(nn, sizeof(double));
  if (!s->D || !s->M1 || !s->M2 || !s->acc_n || !s->acc_T || !s->acc_M0 ||
      !s->acc_M1 || !s->acc_M2)
    return -3;
  return 0;
}

int oracle_set_grid(or_run* r, const double* edges, int n_edges, int bc,
                    double v0, double freq_hz, double phase_rad, double v_dc) {
  if (!r || !edges || n_edges < 3 || (bc != OR_DIRICHLET && bc != OR_PERIODIC))
    return -1;
  if (r->ns > 0) return -2; /* grid before species */
  if (edges[0] != 0.0) return -1;
  for (int i = 1; i < n_edges; ++i)
    if (!(edges[i] > edges[i - 1])) return -1;
  free(r->x); free(r->dx); free(r->V); free(r->Q); free(r->phi); free(r->E);
  free(r->acc_phi);
  int N = n_edges - 1;
  r->N = N;
  r->x = malloc(sizeof(double) * (size_t)(N + 1));
  r->dx = malloc(sizeof(double) * (size_t)N);
  r->V = malloc(sizeof(double) * (size_t)(N + 1));
  r->Q = calloc((size_t)N + 1, sizeof(double));
  r->phi = calloc((size_t)N + 1, sizeof(double));
  r->E = calloc((size_t)N + 1, sizeof(double));
  r->acc_phi = calloc((size_t)N + 1, sizeof(double));
  if (!r->x || !r->dx || !r->V || !r->Q || !r->phi || !r->E || !r->acc_phi)
    return -3;
  memcpy(r->x, edges, sizeof(double) * (size_t)(N + 1));
  for (int j = 0; j < N; ++j) r->dx[j] = r->x[j + 1] - r->x[j];
  r->L = r->x[N];
  /* node control volumes: half cells at Dirichlet end nodes; the two end
   * nodes are one node when periodic */
  for (int n = 1; n < N; ++n) r->V[n] = 0.5 * (r->dx[n - 1] + r->dx[n]);
  if (bc == OR_PERIODIC) {
    r->V[0] = r->V[N] = 0.5 * (r->dx[N - 1] + r->dx[0]);
  } else {
    r->V[0] = 0.5 * r->dx[0];
    r->V[N] = 0.5 * r->dx[N - 1];
  }
  r->bc = bc;
  r->v0 = v0; r->freq = freq_hz; r->phase = phase_rad; r->vdc = v_dc;
  r->grid_set = 1;
  return 0;
}

static int or_uniform(const or_run* r) {
  for (int j = 0; j < r->N; ++j)
    if (fabs(r->dx[j] - r->dx[0]) > 1e-9 * r->dx[0]) return 0;
  return 1;
}

int oracle_set_scheme(or_run* r, int scheme) {
  if (!r || scheme < OR_SCHEME_EC || scheme > OR_SCHEME_MC2) return -1;
  /* the quadratic deposit is written for uniform cells */
  if (scheme >= OR_SCHEME_EC2 && r->grid_set && !or_uniform(r)) return -1;
  r->scheme = scheme;
  return 0;
}

/* node index of a quadratic share: folded at Dirichlet walls, wrapped when
 * periodic (node N is node 0) */
static int or_node2(int n, int N, int bc) {
  if (bc == OR_PERIODIC) {
    n %= N;
    return n < 0 ? n + N : n;
  }
  return n < 0 ? 0 : (n > N ? N : n);
}

int oracle_deposit_fixed2(int N, int bc, int64_t n, const int32_t* cell, const float* xi,
                          uint64_t* S) {
  if (N < 1 || n < 0 || (n > 0 && (!cell || !xi)) || !S) return -1;
  for (int64_t i = 0; i < n; ++i) {
    int j = cell[i];
    float f = xi[i];
    if (j < 0 || j >= N || !(f >= 0.0f) || !(f < 1.0f)) return -1;
    uint32_t r32 = (uint32_t)((double)f * 4294967296.0); /* floor, f < 1 */
    int n0 = r32 < 2147483648u ? j : j + 1;
    int64_t U = r32 < 2147483648u ? (int64_t)r32 : (int64_t)r32 - 4294967296LL;
    unsigned __int128 A = (unsigned __int128)(uint64_t)(2147483648LL - U);
    unsigned __int128 B = (unsigned __int128)(uint64_t)(2147483648LL + U);
    uint64_t a = (uint64_t)((A * A) >> 33), b = (uint64_t)((B * B) >> 33);
    uint64_t m = 4294967296ull - a - b;
    S[or_node2(n0 - 1, N, bc)] += a;
    S[or_node2(n0, N, bc)] += m;
    S[or_node2(n0 + 1, N, bc)] += b;
  }
  if (bc == OR_PERIODIC) S[N] = S[0];
  return 0;
}

int oracle_add_species(or_run* r, double q, double m, double w,
                       int64_t capacity, int* species_out) {
  if (!r || m <= 0 || w < 0 || capacity < 1) return -1;
  if (!r->grid_set || r->initialized) return -2;
  if (r->ns >= OR_MAX_SPECIES) return -1;
  or_species* s = &r->sp[r->ns];
  memset(s, 0, sizeof(*s));
  s->q = q; s->m = m; s->w = w; s->wb = w; s->cap = capacity;
  size_t c = (size_t)capacity;
  s->X = malloc(sizeof(double) * c);
  s->vx = malloc(sizeof(double) * c);
  s->vy = malloc(sizeof(double) * c);
  s->vz = malloc(sizeof(double) * c);
  s->id = malloc(sizeof(uint64_t) * c);
  s->mw = malloc(sizeof(uint32_t) * c);
  if (!s->X || !s->vx || !s->vy || !s->vz || !s->id || !s->mw) return -3;
  if (or_alloc_node_arrays(r, s)) return -3;
  if (species_out) *species_out = r->ns;
  r->ns++;
  return 0;
}

int oracle_set_gas(or_run* r, double n_g, double T_g, double m_g) {
  if (!r || n_g < 0 || T_g < 0 || m_g <= 0) return -1;
  if (r->initialized) return -2;
  r->ng = n_g; r->Tg = T_g; r->mg = m_g;
  r->gas_set = 1;
  return 0;
}

int oracle_add_process(or_run* r, int species, int kind, double threshold_eV,
                       double dE_eV, int n, const float* sigma,
                       int product_species) {
  if (!r || species < 0 || species >= r->ns || kind < OR_ELASTIC ||
      kind > OR_CX || dE_eV <= 0 || n < 2 || !sigma || threshold_eV < 0)
    return -1;
  if (r->initialized) return -2;
  or_species* s = &r->sp[species];
  if (s->nproc >= OR_MAX_PROC) return -1;
  /* all processes of one species share one energy grid */
  if (s->nproc > 0 && (s->proc[0].dE != dE_eV || s->proc[0].n != n)) return -1;
  int heavy = (kind == OR_ION_ELASTIC || kind == OR_CX);
  if (s->nproc > 0 && heavy != s->heavy) return -1;
  if (kind == OR_IONIZATION &&
      (product_species < 0 || product_species >= r->ns || product_species == species))
    return -1;
  for (int i = 0; i < n; ++i)
    if (!(sigma[i] >= 0.0f) || !isfinite(sigma[i])) return -1;
  or_process* p = &s->proc[s->nproc];
  p->kind = kind;
  p->thr = threshold_eV;
  p->dE = dE_eV;
  p->n = n;
  p->product = (kind == OR_IONIZATION) ? product_species : -1;
  p->sigma = malloc(sizeof(double) * (size_t)n);
  if (!p->sigma) return -3;
  for (int i = 0; i < n; ++i) p->sigma[i] = (double)sigma[i];
  s->heavy = heavy;
  s->nproc++;
  return 0;
}

/* sigma(E): linear interpolation in the uniform-energy table, held at the
 * last entry above the table, zero below the threshold. */
static double or_sigma(const or_process* p, double E) {
  if (E < p->thr) return 0.0;
  double u = E / p->dE;
  double fi = floor(u);
  if (fi >= (double)(p->n - 1)) return p->sigma[p->n - 1];
  int i = (int)fi;
  double t = u - fi;
  return p->sigma[i] + t * (p->sigma[i + 1] - p->sigma[i]);
}

/* Null-collision frequency bound: on every table segment [E_i, E_{i+1}],
 * n_g * max(sigma_tot(E_i), sigma_tot(E_{i+1})) * speed(E_{i+1}); the max over
 * segments.  Candidate probability P = 1 - exp(-nu_max dt) becomes the
 * 24-bit integer threshold ceil(P * 2^24). */
static void or_null_rate(or_run* r, or_species* s) {
  s->nu_max = 0.0;
  s->thr24 = 0;
  if (s->nproc == 0 || !r->gas_set || r->ng <= 0) return;
  int n = s->proc[0].n;
  double dE = s->proc[0].dE;
  double best = 0.0;
  for (int i = 0; i + 1 < n; ++i) {
    double a = 0.0, b = 0.0;
    for (int k = 0; k < s->nproc; ++k) {
      a += s->proc[k].sigma[i];
      b += s->proc[k].sigma[i + 1];
    }
    double sig = a > b ? a : b;
    double v = sqrt(2.0 * (double)(i + 1) * dE * OR_QE / s->m);
    if (sig * v > best) best = sig * v;
  }
  s->nu_max = r->ng * best;
  double P = 1.0 - exp(-s->nu_max * r->dt);
  double t = ceil(P * 16777216.0);
  if (t > 16777216.0) t = 16777216.0;
  s->thr24 = (uint32_t)t;
}

int oracle_nu_max(const or_run* r, int species, double* nu_max,
                  uint32_t* threshold24) {
  if (!r || species < 0 || species >= r->ns) return -1;
  if (nu_max) *nu_max = r->sp[species].nu_max;
  if (threshold24) *threshold24 = r->sp[species].thr24;
  return 0;
}

/* ------------------------------------------------------------------ */
static int or_locate(const or_run* r, double X) {
  int lo = 0, hi = r->N; /* x[lo] <= X < x[hi] */
  while (hi - lo > 1) {
    int mid = (lo + hi) / 2;
    if (r->x[mid] <= X) lo = mid; else hi = mid;
  }
  return lo;
}

static double or_rf(const or_run* r, int64_t k) {
  double t = (double)k * r->dt;
  return r->vdc + r->v0 * sin(OR_TWO_PI * r->freq * t + r->phase);
}

/* Step 1 (Eq. 2-3): per-species CIC shares D_s,n, and the first and second
 * vx moments.  Periodic: node N is node 0. */
static void or_deposit(or_run* r) {
  int N = r->N;
  for (int si = 0; si < r->ns; ++si) {
    or_species* s = &r->sp[si];
    memset(s->D, 0, sizeof(double) * (size_t)(N + 1));
    memset(s->M1, 0, sizeof(double) * (size_t)(N + 1));
    memset(s->M2, 0, sizeof(double) * (size_t)(N + 1));
    for (int64_t i = 0; i < s->n; ++i) {
      int j = or_locate(r, s->X[i]);
      double xi = (s->X[i] - r->x[j]) / r->dx[j];
      double v = s->vx[i];
      double k = (double)s->mw[i]; /* weight multiplier: k base particles */
      if (r->scheme >= OR_SCHEME_EC2) {
        /* quadratic B-spline charge shares about the nearest node n0 */
        int n0 = xi < 0.5 ? j : j + 1;
        double u = xi < 0.5 ? xi : xi - 1.0;
        double a = 0.5 * (0.5 - u) * (0.5 - u), b = 0.5 * (0.5 + u) * (0.5 + u);
        s->D[or_node2(n0 - 1, N, r->bc)] += k * a;
        s->D[or_node2(n0, N, r->bc)] += k * (0.75 - u * u);
        s->D[or_node2(n0 + 1, N, r->bc)] += k * b;
      } else {
        s->D[j] += k * (1.0 - xi);
        s->D[j + 1] += k * xi;
      }
      s->M1[j] += k * (1.0 - xi) * v;
      s->M1[j + 1] += k * xi * v;
      s->M2[j] += k * (1.0 - xi) * v * v;
      s->M2[j + 1] += k * xi * v * v;
    }
    if (r->bc == OR_PERIODIC) {
      if (r->scheme < OR_SCHEME_EC2) s->D[0] += s->D[N];
      s->D[N] = s->D[0];
      s->M1[0] += s->M1[N]; s->M1[N] = s->M1[0];
      s->M2[0] += s->M2[N]; s->M2[N] = s->M2[0];
    }
  }
  for (int n = 0; n <= N; ++n) {
    double q = 0.0;
    for (int si = 0; si < r->ns; ++si) q += r->sp[si].q * r->sp[si].wb * r->sp[si].D[n];
    r->Q[n] = q;
  }
}

/* Steps 2-3: Poisson (Eq. 4) and field (Eq. 5 or centred) at step k.
 * Periodic: a uniform neutralising background (Q_n -= V_n * sum Q / L),
 * phi_0 = phi_N = 0. */
static int or_solve(or_run* r, int64_t k) {
  int N = r->N;
  double* Qs = malloc(sizeof(double) * (size_t)(N + 1));
  if (!Qs) return -3;
  double phi0, phiN;
  if (r->bc == OR_PERIODIC) {
    double tot = 0.0;
    for (int n = 0; n < N; ++n) tot += r->Q[n];
    for (int n = 0; n <= N; ++n) Qs[n] = r->Q[n] - r->V[n] * tot / r->L;
    phi0 = phiN = 0.0;
  } else {
    memcpy(Qs, r->Q, sizeof(double) * (size_t)(N + 1));
    phi0 = or_rf(r, k);
    phiN = 0.0;
  }
  int rc = oracle_poisson_thomas(N, r->x, Qs, phi0, phiN, r->phi);
  free(Qs);
  if (rc) return rc;
  return oracle_field(N, r->x, r->phi, r->bc,
                      (r->scheme == OR_SCHEME_MC || r->scheme == OR_SCHEME_MC2) ? OR_SCHEME_MC : OR_SCHEME_EC,
                      r->E);
}

/* histogram bin of value v for bins of width d: floor(v / d), the last bin
 * collecting everything above */
static int or_bin(double v, double d, int n) {
  double b = floor(v / d);
  if (!(b >= 0.0)) return 0;
  if (b >= (double)(n - 1)) return n - 1;
  return (int)b;
}

/* an ion of species s reaching x = 0 with velocity (vx, vy, vz): energy
 * (eV) and angle from the electrode normal (degrees, 0..90) */
static void or_tally_impact(const or_run* r, or_species* s, double vx, double vy, double vz,
                            double k) {
  double E = 0.5 * s->m * (vx * vx + vy * vy + vz * vz) / OR_QE;
  double th = atan2(sqrt(vy * vy + vz * vz), fabs(vx)) * (180.0 / 3.14159265358979323846);
  s->iedf[or_bin(E, r->iedf_dE, r->iedf_n)] += k;
  s->iad[or_bin(th, 90.0 / r->iad_n, r->iad_n)] += k;
}

static void or_sample(or_run* r) {
  int N = r->N;
  for (int si = 0; si < r->ns; ++si) {
    or_species* s = &r->sp[si];
    if (!(s->q < 0.0)) continue;
    for (int64_t i = 0; i < s->n; ++i) {
      int j = or_locate(r, s->X[i]);
      if (j < r->eedf_c0 || j > r->eedf_c1) continue;
      double E = 0.5 * s->m * (s->vx[i] * s->vx[i] + s->vy[i] * s->vy[i] + s->vz[i] * s->vz[i]) / OR_QE;
      s->eedf[or_bin(E, r->eedf_dE, r->eedf_n)] += (double)s->mw[i];
    }
  }
  for (int si = 0; si < r->ns; ++si) {
    or_species* s = &r->sp[si];
    for (int n = 0; n <= N; ++n) {
      double D = s->D[n];
      s->acc_n[n] += s->wb * D / r->V[n];
      double T = 0.0;
      if (D > 0.0) {
        double m1 = s->M1[n] / D, m2 = s->M2[n] / D;
        T = s->m * (m2 - m1 * m1) / OR_QE;
      }
      s->acc_T[n] += T;
      s->acc_M0[n] += D;
      s->acc_M1[n] += s->M1[n];
      s->acc_M2[n] += s->M2[n];
    }
  }
  for (int n = 0; n <= N; ++n) r->acc_phi[n] += r->phi[n];
  r->n_samples++;
}

static int or_refresh(or_run* r) {
  or_deposit(r);
  return or_solve(r, r->step);
}

/* ------------------------------------------------------------------ */
int oracle_init(or_run* r, uint64_t seed, double dt,
                const int64_t* n_per_species, const double* T_eV) {
  if (!r || !n_per_species || !T_eV || !(dt > 0)) return -1;
  if (!r->grid_set || r->ns == 0) return -2;
  for (int si = 0; si < r->ns; ++si)
    if (n_per_species[si] < 0 || n_per_species[si] > r->sp[si].cap || T_eV[si] < 0)
      return -1;
  if (r->scheme >= OR_SCHEME_EC2 && !or_uniform(r)) return -1;
  r->seed = seed;
  r->dt = dt;
  r->step = 0;
  /* Sec. 2b: uniform density, Maxwellian temperature.  Position from
   * 32-bit word 0 of the block with word3 = (s<<8)|0x80 (or, for a quiet
   * start, X = (i + 1/2) L / n); velocities from the block with
   * word3 = (s<<8)|0x81 (Box-Muller on 32-bit uniforms). */
  for (int si = 0; si < r->ns; ++si) {
    or_species* s = &r->sp[si];
    double sd = sqrt(OR_QE * T_eV[si] / s->m);
    s->n = n_per_species[si];
    /* a loaded particle of weight w holds rb_m0 base particles of weight wb */
    s->wb = s->w / (double)r->rb_m0;
    for (int64_t i = 0; i < s->n; ++i) {
      uint32_t a[4], b[4];
      or_draw(r, (uint64_t)i, 0xFFFFFFFFu, ((uint32_t)si << 8) | 0x80u, a);
      or_draw(r, (uint64_t)i, 0xFFFFFFFFu, ((uint32_t)si << 8) | 0x81u, b);
      double u = (double)a[0] * (1.0 / 4294967296.0);
      if (r->quiet) u = ((double)i + 0.5) / (double)s->n;
      s->X[i] = u * r->L;
      double z0, z1, z2, z3;
      or_box_muller(((double)b[0] + 1.0) * (1.0 / 4294967296.0),
                    (double)b[1] * (1.0 / 4294967296.0), &z0, &z1);
      or_box_muller(((double)b[2] + 1.0) * (1.0 / 4294967296.0),
                    (double)b[3] * (1.0 / 4294967296.0), &z2, &z3);
      s->vx[i] = sd * z0;
      s->vy[i] = sd * z1;
      s->vz[i] = sd * z2;
      s->id[i] = (uint64_t)i;
      s->mw[i] = r->rb_m0;
    }
    memset(s->absorbed, 0, sizeof(s->absorbed));
    memset(s->coll, 0, sizeof(s->coll));
    s->births = s->lost = s->clamps = s->candidates = 0;
    s->rb_merged = s->rb_split = s->rb_skipped = 0;
    s->ke = 0.0;
  }
  for (int si = 0; si < r->ns; ++si) or_null_rate(r, &r->sp[si]);
  /* tallies: defaults, the EEDF region's cells (centres within the region,
   * else the cell holding its centre), zeroed arrays */
  if (!(r->eedf_n > 0)) {
    r->eedf_xc = -1.0; r->eedf_hw = 0.5e-3; r->eedf_dE = 0.5; r->eedf_n = 100;
    r->iedf_dE = 2.0; r->iedf_n = 256; r->iad_n = 90;
  }
  double xc = r->eedf_xc < 0.0 ? 0.5 * r->L : r->eedf_xc;
  r->eedf_c0 = r->N;
  r->eedf_c1 = -1;
  for (int j = 0; j < r->N; ++j) {
    double cj = 0.5 * (r->x[j] + r->x[j + 1]);
    if (cj >= xc - r->eedf_hw && cj <= xc + r->eedf_hw) {
      if (j < r->eedf_c0) r->eedf_c0 = j;
      r->eedf_c1 = j;
    }
  }
  if (r->eedf_c0 > r->eedf_c1) r->eedf_c0 = r->eedf_c1 = or_locate(r, xc < r->L ? xc : 0.0);
  for (int si = 0; si < r->ns; ++si) {
    or_species* s = &r->sp[si];
    free(s->eedf); free(s->iedf); free(s->iad); free(s->acc_P);
    s->eedf = calloc((size_t)r->eedf_n, sizeof(double));
    s->iedf = calloc((size_t)r->iedf_n, sizeof(double));
    s->iad = calloc((size_t)r->iad_n, sizeof(double));
    s->acc_P = calloc((size_t)r->N, sizeof(double));
    if (!s->eedf || !s->iedf || !s->iad || !s->acc_P) return -3;
  }
  r->initialized = 1;
  r->fe = 0.0;
  return or_refresh(r);
}

int oracle_set_quiet_start(or_run* r, int quiet) {
  if (!r || (quiet != 0 && quiet != 1)) return -1;
  if (r->initialized) return -2;
  r->quiet = quiet;
  return 0;
}

int oracle_set_particles(or_run* r, int species, const double* X,
                         const double* vx, const double* vy, const double* vz,
                         const uint64_t* id, int64_t n) {
  if (!r || species < 0 || species >= r->ns || n < 0) return -1;
  if (!r->initialized) return -2;
  or_species* s = &r->sp[species];
  if (n > s->cap) return -1;
  for (int64_t i = 0; i < n; ++i) {
    if (!(X[i] >= 0.0) || !(X[i] < r->L)) return -1;
    s->X[i] = X[i];
    s->vx[i] = vx[i];
    s->vy[i] = vy[i];
    s->vz[i] = vz[i];
    s->id[i] = id[i];
    s->mw[i] = r->rb_m0;
  }
  s->n = n;
  return or_refresh(r);
}

int oracle_get_particles(or_run* r, int species, double* X, double* vx,
                         double* vy, double* vz, uint64_t* id, int64_t cap,
                         int64_t* n) {
  if (!r || species < 0 || species >= r->ns || !n) return -1;
  or_species* s = &r->sp[species];
  *n = s->n;
  if (cap < s->n) return -1;
  for (int64_t i = 0; i < s->n; ++i) {
    if (X) X[i] = s->X[i];
    if (vx) vx[i] = s->vx[i];
    if (vy) vy[i] = s->vy[i];
    if (vz) vz[i] = s->vz[i];
    if (id) id[i] = s->id[i];
  }
  return 0;
}

int oracle_set_particles_cell(or_run* r, int species, const int32_t* cell,
                              const float* xi, const float* vx,
                              const float* vy, const float* vz,
                              const uint64_t* id, int64_t n) {
  if (!r || species < 0 || species >= r->ns || n < 0) return -1;
  if (!r->initialized) return -2;
  or_species* s = &r->sp[species];
  if (n > s->cap) return -1;
  for (int64_t i = 0; i < n; ++i) {
    int j = cell[i];
    if (j < 0 || j >= r->N || !(xi[i] >= 0.0f) || !(xi[i] < 1.0f)) return -1;
    double X = r->x[j] + (double)xi[i] * r->dx[j];
    if (X >= r->L) X = r->x[j];
    s->X[i] = X;
    s->vx[i] = (double)vx[i];
    s->vy[i] = (double)vy[i];
    s->vz[i] = (double)vz[i];
    s->id[i] = id[i];
    s->mw[i] = r->rb_m0;
  }
  s->n = n;
  return or_refresh(r);
}

int oracle_get_particles_cell(or_run* r, int species, int32_t* cell,
                              double* xi, int64_t cap, int64_t* n) {
  if (!r || species < 0 || species >= r->ns || !n) return -1;
  or_species* s = &r->sp[species];
  *n = s->n;
  if (cap < s->n) return -1;
  for (int64_t i = 0; i < s->n; ++i) {
    int j = or_locate(r, s->X[i]);
    if (cell) cell[i] = j;
    if (xi) xi[i] = (s->X[i] - r->x[j]) / r->dx[j];
  }
  return 0;
}

static int or_append(or_species* s, double X, double vx, double vy, double vz,
                     uint64_t id, uint32_t k) {
  if (s->n >= s->cap) {
    s->lost++;
    return -4;
  }
  s->X[s->n] = X; s->vx[s->n] = vx; s->vy[s->n] = vy; s->vz[s->n] = vz;
  s->id[s->n] = id;
  s->mw[s->n] = k;
  s->n++;
  return 0;
}

/* Step 6: null-collision Monte Carlo (Vahedi & Surendra) for one particle.
 * Draws: block A = Philox(ctr = (id, step, (s<<8)|0)): r0 candidate,
 * r1 process, r2/r3 scattering direction.  Heavy species: block B (|1) gives
 * the target neutral's Maxwellian velocity.  Electron ionisation: block B
 * gives the energy split (s0) and the secondary's direction (s1, s2), and
 * block C (|2) the new ion's Maxwellian velocity. */
static int or_collide(or_run* r, int si, int64_t i, int64_t k) {
  or_species* s = &r->sp[si];
  if (s->nproc == 0 || s->thr24 == 0) return 0;
  uint64_t id = s->id[i];
  uint32_t A[4];
  or_draw(r, id, (uint32_t)k, (uint32_t)si << 8, A);
  if ((A[0] >> 8) >= s->thr24) return 0;
  s->candidates++;
  double v[3] = {s->vx[i], s->vy[i], s->vz[i]};
  double vn[3] = {0.0, 0.0, 0.0};
  uint32_t B[4];
  int haveB = 0;
  if (s->heavy) {
    or_draw(r, id, (uint32_t)k, ((uint32_t)si << 8) | 1u, B);
    haveB = 1;
    double z0, z1, z2, z3;
    or_box_muller(or_u24_open(B[0]), or_u24(B[1]), &z0, &z1);
    or_box_muller(or_u24_open(B[2]), or_u24(B[3]), &z2, &z3);
    double sd = sqrt(OR_KB * r->Tg / r->mg);
    vn[0] = sd * z0; vn[1] = sd * z1; vn[2] = sd * z2;
  }
  double g[3] = {v[0] - vn[0], v[1] - vn[1], v[2] - vn[2]};
  double g2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
  double gm = sqrt(g2);
  double E = 0.5 * s->m * g2 / OR_QE;
  double nu[OR_MAX_PROC];
  double tot = 0.0;
  for (int p = 0; p < s->nproc; ++p) {
    nu[p] = r->ng * or_sigma(&s->proc[p], E) * gm;
    tot += nu[p];
  }
  if (tot > s->nu_max) s->clamps++;
  double R = or_u24(A[1]) * s->nu_max;
  int chosen = -1;
  double cum = 0.0;
  for (int p = 0; p < s->nproc; ++p) {
    cum += nu[p];
    if (R < cum) {
      chosen = p;
      break;
    }
  }
  if (chosen < 0) return 0; /* null collision */
  s->coll[chosen]++;
  const or_process* pr = &s->proc[chosen];
  double d[3];
  or_isotropic(or_u24(A[2]), or_u24(A[3]), d);
  int rc = 0;
  switch (pr->kind) {
    case OR_ELASTIC: {
      /* neutral at rest; energy loss (2m/M)(1 - cos chi) E */
      double cchi = (gm > 0.0) ? (g[0] * d[0] + g[1] * d[1] + g[2] * d[2]) / gm : 1.0;
      double E1 = E * (1.0 - 2.0 * s->m / r->mg * (1.0 - cchi));
      double sp = sqrt(2.0 * E1 * OR_QE / s->m);
      v[0] = sp * d[0]; v[1] = sp * d[1]; v[2] = sp * d[2];
      break;
    }
    case OR_EXCITATION: {
      double E1 = E - pr->thr;
      double sp = sqrt(2.0 * E1 * OR_QE / s->m);
      v[0] = sp * d[0]; v[1] = sp * d[1]; v[2] = sp * d[2];
      break;
    }
    case OR_IONIZATION: {
      if (!haveB) or_draw(r, id, (uint32_t)k, ((uint32_t)si << 8) | 1u, B);
      double Erem = E - pr->thr;
      double f = or_u24(B[0]);
      double E1 = f * Erem, E2 = (1.0 - f) * Erem;
      double sp1 = sqrt(2.0 * E1 * OR_QE / s->m);
      double sp2 = sqrt(2.0 * E2 * OR_QE / s->m);
      v[0] = sp1 * d[0]; v[1] = sp1 * d[1]; v[2] = sp1 * d[2];
      double d2[3];
      or_isotropic(or_u24(B[1]), or_u24(B[2]), d2);
      uint32_t C[4];
      or_draw(r, id, (uint32_t)k, ((uint32_t)si << 8) | 2u, C);
      double z0, z1, z2, z3;
      or_box_muller(or_u24_open(C[0]), or_u24(C[1]), &z0, &z1);
      or_box_muller(or_u24_open(C[2]), or_u24(C[3]), &z2, &z3);
      double sd = sqrt(OR_KB * r->Tg / r->mg);
      double X = s->X[i];
      s->births++;
      /* both products carry the parent's weight (charge conserved) */
      uint32_t kw = s->mw[i];
      if (or_append(s, X, sp2 * d2[0], sp2 * d2[1], sp2 * d2[2],
                    oracle_child_id(id, k, 1), kw))
        rc = -4;
      if (or_append(&r->sp[pr->product], X, sd * z0, sd * z1, sd * z2,
                    oracle_child_id(id, k, 2), kw))
        rc = -4;
      break;
    }
    case OR_ION_ELASTIC: {
      /* isotropic in the centre-of-mass frame */
      double M = s->m + r->mg;
      double gm_new = gm;
      for (int c = 0; c < 3; ++c) {
        double vcm = (s->m * v[c] + r->mg * vn[c]) / M;
        v[c] = vcm + (r->mg / M) * gm_new * d[c];
      }
      break;
    }
    case OR_CX: {
      v[0] = vn[0]; v[1] = vn[1]; v[2] = vn[2];
      break;
    }
  }
  s->vx[i] = v[0]; s->vy[i] = v[1]; s->vz[i] = v[2];
  return rc;
}

/* EC2 gather: linear interpolation of the face fields about the nearest node
 * n0 (faces n0-1 at n0-1/2 and n0 at n0+1/2), the derivative of the
 * quadratic-spline potential; the face beyond a Dirichlet wall carries no
 * field (its ghost node is the wall node), periodic faces wrap. */
static double or_gather2(const or_run* r, int j, double xi) {
  int N = r->N;
  int n0 = xi < 0.5 ? j : j + 1;
  double u = xi < 0.5 ? xi : xi - 1.0;
  int fl = n0 - 1, fr = n0;
  double El, Er;
  if (r->bc == OR_PERIODIC) {
    El = r->E[(fl + N) % N];
    Er = r->E[fr % N];
  } else {
    El = fl < 0 ? 0.0 : r->E[fl];
    Er = fr >= N ? 0.0 : r->E[fr];
  }
  return (0.5 - u) * El + (0.5 + u) * Er;
}

/* MC2 gather: the quadratic-spline weights of the deposit applied to the
 * centred node field (the transpose of the deposit: shares folded into a
 * wall node read that node's field, periodic nodes wrap). */
static double or_gather2_mc(const or_run* r, int j, double xi) {
  int N = r->N;
  int n0 = xi < 0.5 ? j : j + 1;
  double u = xi < 0.5 ? xi : xi - 1.0;
  double w[3] = {0.5 * (0.5 - u) * (0.5 - u), 0.75 - u * u, 0.5 * (0.5 + u) * (0.5 + u)};
  double e = 0.0;
  for (int q = 0; q < 3; ++q) e += w[q] * r->E[or_node2(n0 - 1 + q, N, r->bc)];
  return e;
}

/* ------------------------------------------------------------------ */
/* Particle rebalancing on non-uniform grids (Sec. 3d: keep the number of
 * particles per cell near a target so that the cost follows the cell count;
 * the paper proposes this and gives no algorithm -- the rule below is this
 * project's design).  Every particle carries an integer weight multiplier k
 * (it stands for k base particles of weight wb), and the deposit, moments,
 * energies and tallies count k.  At a rebalancing level, per species and
 * cell j with n particles:
 *   - n > rb_hi (merge; cells above OR_RB_MAX_CELL are left alone and
 *     counted): order the particles by (vx, id), cut the order into
 *     floor(n/4) consecutive groups of four (the n mod 4 fastest stay
 *     apart), and merge the G = min(floor(n/4), ceil((n - rb_target)/2))
 *     groups nearest the middle of that order (ties: the slower group),
 *     skipping groups whose weight exceeds OR_RB_MAX_WEIGHT.  A group of
 *     weight W = sum k, mean velocity u = sum k v / W and per-component
 *     standard deviations s_x, s_y, s_z becomes two particles at the
 *     weighted centroid X_c = sum k X / W, of weights a = ceil(W/2) and
 *     b = W - a, with velocities u + sqrt(b/a) d and u - sqrt(a/b) d,
 *     d = (s_x, +-s_y, +-s_z), the signs from Philox; they take the group's
 *     two smallest ids.  CIC node charges (linear in the offset within the
 *     cell), momentum and each velocity component's second moment -- hence
 *     the energy and the x temperature -- are those of the group.
 *   - 0 < n < rb_lo (split): the S = min(rb_target - n, #{k >= 2})
 *     particles of largest k (ties: smallest id) each become two at the same
 *     position and velocity, of weights ceil(k/2) (keeping the id) and
 *     floor(k/2) (id child_id(id, level, 3)): every node charge, the
 *     momentum and the energy are unchanged exactly.
 * Random numbers: Philox with counter (id_min lo, id_min hi, level,
 * (s << 8) | 0x10), word 0 bit 0 (y sign) and bit 1 (z sign). */
#define OR_RB_MAX_CELL 4096
#define OR_RB_MAX_WEIGHT 65536u

typedef struct {
  double vx;
  uint64_t id;
  int64_t i;
} or_rb_key;

static int or_rb_cmp_v(const void* a, const void* b) {
  const or_rb_key* p = (const or_rb_key*)a;
  const or_rb_key* q = (const or_rb_key*)b;
  if (p->vx < q->vx) return -1;
  if (p->vx > q->vx) return 1;
  return (p->id < q->id) ? -1 : (p->id > q->id);
}

typedef struct {
  uint32_t k;
  uint64_t id;
  int64_t i;
} or_rb_wkey;

static int or_rb_cmp_w(const void* a, const void* b) {
  const or_rb_wkey* p = (const or_rb_wkey*)a;
  const or_rb_wkey* q = (const or_rb_wkey*)b;
  if (p->k != q->k) return (p->k > q->k) ? -1 : 1; /* heaviest first */
  return (p->id < q->id) ? -1 : (p->id > q->id);
}

typedef struct {
  int dist; /* |2g - (ng - 1)| */
  int g;
} or_rb_group;

static int or_rb_cmp_g(const void* a, const void* b) {
  const or_rb_group* p = (const or_rb_group*)a;
  const or_rb_group* q = (const or_rb_group*)b;
  if (p->dist != q->dist) return p->dist < q->dist ? -1 : 1;
  return p->g < q->g ? -1 : (p->g > q->g);
}

/* rebalance species si in cell j holding the particles idx[0..n): the new
 * particles are written to the output arrays of the species at *out */
typedef struct {
  double *X, *vx, *vy, *vz;
  uint64_t* id;
  uint32_t* mw;
  int64_t n, cap;
} or_rb_out;

static int or_rb_put(or_rb_out* o, double X, double vx, double vy, double vz, uint64_t id,
                     uint32_t k) {
  if (o->n >= o->cap) return -4;
  o->X[o->n] = X; o->vx[o->n] = vx; o->vy[o->n] = vy; o->vz[o->n] = vz;
  o->id[o->n] = id; o->mw[o->n] = k;
  o->n++;
  return 0;
}

static int or_rb_cell(or_run* r, int si, const int64_t* idx, int64_t n, or_rb_out* o) {
  or_species* s = &r->sp[si];
  int rc = 0;
  int64_t merge_groups = 0, splits = 0;
  if (n > r->rb_hi) {
    if (n > OR_RB_MAX_CELL) {
      s->rb_skipped++;
    } else {
      int64_t ng = n / 4;
      int64_t want = (n - r->rb_target + 1) / 2;
      merge_groups = ng < want ? ng : want;
    }
  } else if (n > 0 && n < r->rb_lo) {
    int64_t heavy = 0;
    for (int64_t t = 0; t < n; ++t) heavy += s->mw[idx[t]] >= 2u;
    splits = r->rb_target - n < heavy ? r->rb_target - n : heavy;
  }
  if (merge_groups > 0) {
    or_rb_key* key = malloc(sizeof(or_rb_key) * (size_t)n);
    int64_t ng = n / 4;
    or_rb_group* grp = malloc(sizeof(or_rb_group) * (size_t)ng);
    char* merged = calloc((size_t)ng, 1);
    if (!key || !grp || !merged) { free(key); free(grp); free(merged); return -3; }
    for (int64_t t = 0; t < n; ++t) {
      key[t].vx = s->vx[idx[t]];
      key[t].id = s->id[idx[t]];
      key[t].i = idx[t];
    }
    qsort(key, (size_t)n, sizeof(or_rb_key), or_rb_cmp_v);
    for (int64_t g = 0; g < ng; ++g) {
      int64_t d = 2 * g - (ng - 1);
      grp[g].dist = (int)(d < 0 ? -d : d);
      grp[g].g = (int)g;
    }
    qsort(grp, (size_t)ng, sizeof(or_rb_group), or_rb_cmp_g);
    int64_t taken = 0;
    for (int64_t t = 0; t < ng && taken < merge_groups; ++t) {
      int g = grp[t].g;
      uint64_t W = 0;
      for (int q = 0; q < 4; ++q) W += s->mw[key[4 * g + q].i];
      if (W > OR_RB_MAX_WEIGHT) continue;
      merged[g] = 1;
      taken++;
    }
    for (int64_t g = 0; g < ng; ++g) {
      if (!merged[g]) continue;
      double W = 0.0, Xc = 0.0, u[3] = {0.0, 0.0, 0.0}, m2[3] = {0.0, 0.0, 0.0};
      uint64_t id0 = UINT64_MAX, id1 = UINT64_MAX;
      uint32_t Wi = 0;
      for (int q = 0; q < 4; ++q) {
        int64_t i = key[4 * g + q].i;
        double k = (double)s->mw[i];
        Wi += s->mw[i];
        W += k;
        Xc += k * s->X[i];
        u[0] += k * s->vx[i];
        u[1] += k * s->vy[i];
        u[2] += k * s->vz[i];
        uint64_t id = s->id[i];
        if (id < id0) { id1 = id0; id0 = id; } else if (id < id1) { id1 = id; }
      }
      Xc /= W;
      for (int c = 0; c < 3; ++c) u[c] /= W;
      for (int q = 0; q < 4; ++q) {
        int64_t i = key[4 * g + q].i;
        double k = (double)s->mw[i];
        double v[3] = {s->vx[i] - u[0], s->vy[i] - u[1], s->vz[i] - u[2]};
        for (int c = 0; c < 3; ++c) m2[c] += k * v[c] * v[c];
      }
      uint32_t A[4];
      or_draw(r, id0, (uint32_t)r->step, ((uint32_t)si << 8) | 0x10u, A);
      double d[3] = {sqrt(m2[0] / W), sqrt(m2[1] / W), sqrt(m2[2] / W)};
      if (A[0] & 1u) d[1] = -d[1];
      if (A[0] & 2u) d[2] = -d[2];
      uint32_t ka = (Wi + 1u) / 2u, kb = Wi - ka;
      double fa = sqrt((double)kb / (double)ka), fb = sqrt((double)ka / (double)kb);
      /* the centroid of positions in one cell stays in that cell */
      if (or_rb_put(o, Xc, u[0] + fa * d[0], u[1] + fa * d[1], u[2] + fa * d[2], id0, ka)) rc = -4;
      if (or_rb_put(o, Xc, u[0] - fb * d[0], u[1] - fb * d[1], u[2] - fb * d[2], id1, kb)) rc = -4;
      s->rb_merged++;
    }
    /* the particles that stay as they are */
    for (int64_t t = 0; t < n; ++t) {
      int64_t g = t / 4;
      if (g < ng && merged[g]) continue;
      int64_t i = key[t].i;
      if (or_rb_put(o, s->X[i], s->vx[i], s->vy[i], s->vz[i], s->id[i], s->mw[i])) rc = -4;
    }
    free(key); free(grp); free(merged);
    return rc;
  }
  if (splits > 0) {
    or_rb_wkey* key = malloc(sizeof(or_rb_wkey) * (size_t)n);
    if (!key) return -3;
    for (int64_t t = 0; t < n; ++t) {
      key[t].k = s->mw[idx[t]];
      key[t].id = s->id[idx[t]];
      key[t].i = idx[t];
    }
    qsort(key, (size_t)n, sizeof(or_rb_wkey), or_rb_cmp_w);
    for (int64_t t = 0; t < n; ++t) {
      int64_t i = key[t].i;
      uint32_t k = s->mw[i];
      if (t < splits) {
        uint32_t ka = (k + 1u) / 2u, kb = k - ka;
        if (or_rb_put(o, s->X[i], s->vx[i], s->vy[i], s->vz[i], s->id[i], ka)) rc = -4;
        if (or_rb_put(o, s->X[i], s->vx[i], s->vy[i], s->vz[i],
                      oracle_child_id(s->id[i], r->step, 3), kb)) rc = -4;
        s->rb_split++;
      } else {
        if (or_rb_put(o, s->X[i], s->vx[i], s->vy[i], s->vz[i], s->id[i], k)) rc = -4;
      }
    }
    free(key);
    return rc;
  }
  for (int64_t t = 0; t < n; ++t) {
    int64_t i = idx[t];
    if (or_rb_put(o, s->X[i], s->vx[i], s->vy[i], s->vz[i], s->id[i], s->mw[i])) rc = -4;
  }
  return rc;
}

/* one rebalancing of every species at the current level (particles gathered
 * by cell; the output replaces the species' arrays, cell by cell) */
static int or_rebalance(or_run* r) {
  int rc = 0;
  int N = r->N;
  for (int si = 0; si < r->ns; ++si) {
    or_species* s = &r->sp[si];
    int64_t n = s->n;
    int64_t* cnt = calloc((size_t)N + 1, sizeof(int64_t));
    int64_t* order = malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int* cellof = malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    or_rb_out o;
    o.cap = s->cap;
    o.n = 0;
    o.X = malloc(sizeof(double) * (size_t)s->cap);
    o.vx = malloc(sizeof(double) * (size_t)s->cap);
    o.vy = malloc(sizeof(double) * (size_t)s->cap);
    o.vz = malloc(sizeof(double) * (size_t)s->cap);
    o.id = malloc(sizeof(uint64_t) * (size_t)s->cap);
    o.mw = malloc(sizeof(uint32_t) * (size_t)s->cap);
    if (!cnt || !order || !cellof || !o.X || !o.vx || !o.vy || !o.vz || !o.id || !o.mw) {
      free(cnt); free(order); free(cellof);
      free(o.X); free(o.vx); free(o.vy); free(o.vz); free(o.id); free(o.mw);
      return -3;
    }
    for (int64_t i = 0; i < n; ++i) {
      cellof[i] = or_locate(r, s->X[i]);
      cnt[cellof[i] + 1]++;
    }
    for (int j = 0; j < N; ++j) cnt[j + 1] += cnt[j];
    {
      int64_t* pos = malloc(sizeof(int64_t) * (size_t)N);
      if (!pos) return -3;
      for (int j = 0; j < N; ++j) pos[j] = cnt[j];
      for (int64_t i = 0; i < n; ++i) order[pos[cellof[i]]++] = i;
      free(pos);
    }
    for (int j = 0; j < N; ++j) {
      int e = or_rb_cell(r, si, order + cnt[j], cnt[j + 1] - cnt[j], &o);
      if (e == -4) { rc = -4; s->lost++; }
      else if (e) return e;
    }
    free(s->X); free(s->vx); free(s->vy); free(s->vz); free(s->id); free(s->mw);
    s->X = o.X; s->vx = o.vx; s->vy = o.vy; s->vz = o.vz; s->id = o.id; s->mw = o.mw;
    s->n = o.n;
    free(cnt); free(order); free(cellof);
  }
  return rc;
}

static int or_step_once(or_run* r) {
  int64_t k = r->step;
  int N = r->N;
  int rc = 0;
  /* field energy at time level k: face fields from phi^k */
  double fe = 0.0;
  for (int j = 0; j < N; ++j) {
    double Ej = -(r->phi[j + 1] - r->phi[j]) / r->dx[j];
    fe += 0.5 * OR_EPS0 * Ej * Ej * r->dx[j];
  }
  r->fe = fe;
  /* steps 4-5 (Eq. 6-9), then the walls */
  const int sampled = r->sample_every > 0 && (k + 1) % r->sample_every == 0;
  for (int si = 0; si < r->ns; ++si) {
    or_species* s = &r->sp[si];
    double qm = s->q / s->m;
    double ke = 0.0;
    int64_t keep = 0;
    for (int64_t i = 0; i < s->n; ++i) {
      double X = s->X[i];
      int j = or_locate(r, X);
      double xi = (X - r->x[j]) / r->dx[j];
      double Ei = (r->scheme == OR_SCHEME_EC) ? r->E[j]
                : (r->scheme == OR_SCHEME_EC2) ? or_gather2(r, j, xi)
                : (r->scheme == OR_SCHEME_MC2) ? or_gather2_mc(r, j, xi)
                                               : (1.0 - xi) * r->E[j] + xi * r->E[j + 1];
      double vold = s->vx[i];
      double vnew = vold + qm * Ei * r->dt;
      double wi = s->wb * (double)s->mw[i];
      ke += 0.5 * s->m * wi * (vold * vnew + s->vy[i] * s->vy[i] + s->vz[i] * s->vz[i]);
      /* J.E of the push: q w E_i (v^{k-1/2} + v^{k+1/2})/2 per unit volume of cell j */
      if (sampled) s->acc_P[j] += s->q * wi * Ei * 0.5 * (vold + vnew) / r->dx[j];
      double Xn = X + vnew * r->dt;
      if (r->bc == OR_DIRICHLET) {
        if (Xn <= 0.0) {
          s->absorbed[0]++;
          if (s->q > 0.0) or_tally_impact(r, s, vnew, s->vy[i], s->vz[i], (double)s->mw[i]);
          continue;
        }
        if (Xn >= r->L) { s->absorbed[1]++; continue; }
      } else {
        Xn = Xn - r->L * floor(Xn / r->L);
        if (Xn >= r->L || Xn < 0.0) Xn = 0.0;
      }
      s->X[keep] = Xn;
      s->vx[keep] = vnew;
      s->vy[keep] = s->vy[i];
      s->vz[keep] = s->vz[i];
      s->id[keep] = s->id[i];
      s->mw[keep] = s->mw[i];
      keep++;
    }
    s->n = keep;
    s->ke = ke;
  }
  /* step 6 on the survivors; particles born now are not collided now */
  int64_t n0[OR_MAX_SPECIES];
  for (int si = 0; si < r->ns; ++si) n0[si] = r->sp[si].n;
  for (int si = 0; si < r->ns; ++si)
    for (int64_t i = 0; i < n0[si]; ++i)
      if (or_collide(r, si, i, k)) rc = -4;
  /* steps 1-3 at k+1 */
  r->step = k + 1;
  int e = or_refresh(r);
  if (e) return e;
  if (r->sample_every > 0 && r->step % r->sample_every == 0) or_sample(r);
  /* particle rebalancing at level k+1, after the field and the sample: it
   * keeps every node's charge (see or_rebalance), so the field stands */
  if (r->rb_every > 0 && r->step % r->rb_every == 0) {
    e = or_rebalance(r);
    if (e == -4) rc = -4;
    else if (e) return e;
  }
  return rc;
}

int oracle_step(or_run* r, int64_t n_steps) {
  if (!r || n_steps < 0) return -1;
  if (!r->initialized) return -2;
  int rc = 0;
  for (int64_t t = 0; t < n_steps; ++t) {
    int e = or_step_once(r);
    if (e == -4) rc = -4;
    else if (e) return e;
  }
  return rc;
}

/* Move the run to time level k: the electrode potential (Sec. 2a, the RF
 * bias at t = k dt) and the random stream (keyed on the level) follow it,
 * so a state taken from the middle of a run continues from its own level.
 * The field is formed again for level k. */
int oracle_set_step(or_run* r, int64_t k) {
  if (!r || k < 0) return -1;
  if (!r->initialized) return -2;
  r->step = k;
  return or_refresh(r);
}

int oracle_reset_averages(or_run* r, int sample_every) {
  if (!r || sample_every < 0) return -1;
  if (!r->grid_set) return -2;
  r->sample_every = sample_every;
  r->n_samples = 0;
  size_t nn = (size_t)r->N + 1;
  memset(r->acc_phi, 0, sizeof(double) * nn);
  for (int si = 0; si < r->ns; ++si) {
    or_species* s = &r->sp[si];
    memset(s->acc_n, 0, sizeof(double) * nn);
    memset(s->acc_T, 0, sizeof(double) * nn);
    memset(s->acc_M0, 0, sizeof(double) * nn);
    memset(s->acc_M1, 0, sizeof(double) * nn);
    memset(s->acc_M2, 0, sizeof(double) * nn);
    if (s->eedf) memset(s->eedf, 0, sizeof(double) * (size_t)r->eedf_n);
    if (s->iedf) memset(s->iedf, 0, sizeof(double) * (size_t)r->iedf_n);
    if (s->iad) memset(s->iad, 0, sizeof(double) * (size_t)r->iad_n);
    if (s->acc_P) memset(s->acc_P, 0, sizeof(double) * (size_t)r->N);
  }
  return 0;
}

int oracle_set_tallies(or_run* r, double eedf_center, double eedf_halfwidth, double eedf_dE,
                       int eedf_bins, double iedf_dE, int iedf_bins, int iad_bins) {
  if (!r || !(eedf_halfwidth >= 0.0) || !(eedf_dE > 0.0) || eedf_bins < 1 || !(iedf_dE > 0.0) ||
      iedf_bins < 1 || iad_bins < 1)
    return -1;
  if (r->initialized) return -2;
  r->eedf_xc = eedf_center; r->eedf_hw = eedf_halfwidth; r->eedf_dE = eedf_dE;
  r->eedf_n = eedf_bins; r->iedf_dE = iedf_dE; r->iedf_n = iedf_bins; r->iad_n = iad_bins;
  return 0;
}

int oracle_get_tally_shape(const or_run* r, int* shape5) {
  if (!r || !shape5) return -1;
  if (!r->initialized) return -2;
  shape5[0] = r->eedf_n; shape5[1] = r->iedf_n; shape5[2] = r->iad_n;
  shape5[3] = r->eedf_c0; shape5[4] = r->eedf_c1;
  return 0;
}

int64_t oracle_get_tallies(const or_run* r, double* eedf, double* iedf, double* iad, double* power) {
  if (!r) return -1;
  if (!r->initialized) return -2;
  double inv = r->n_samples > 0 ? 1.0 / (double)r->n_samples : 0.0;
  for (int si = 0; si < r->ns; ++si) {
    const or_species* s = &r->sp[si];
    for (int b = 0; b < r->eedf_n; ++b) if (eedf) eedf[(size_t)si * r->eedf_n + b] = s->eedf[b];
    for (int b = 0; b < r->iedf_n; ++b) if (iedf) iedf[(size_t)si * r->iedf_n + b] = s->iedf[b];
    for (int b = 0; b < r->iad_n; ++b) if (iad) iad[(size_t)si * r->iad_n + b] = s->iad[b];
    for (int j = 0; j < r->N; ++j) if (power) power[(size_t)si * r->N + j] = s->acc_P[j] * inv;
  }
  return r->n_samples;
}

int oracle_get_counters(const or_run* r, int64_t* out, int cap) {
  if (!r || !out || cap < 1 + 16 * OR_MAX_SPECIES) return -1;
  memset(out, 0, sizeof(int64_t) * (size_t)cap);
  out[0] = r->step;
  for (int si = 0; si < r->ns; ++si) {
    const or_species* s = &r->sp[si];
    int64_t* o = out + 1 + 16 * si;
    o[0] = s->n;
    o[1] = s->absorbed[0];
    o[2] = s->absorbed[1];
    o[3] = s->births;
    o[4] = s->lost;
    o[5] = s->clamps;
    o[6] = s->candidates;
    for (int p = 0; p < OR_MAX_PROC; ++p) o[7 + p] = s->coll[p];
  }
  return 0;
}

int oracle_get_fields(const or_run* r, double* phi, double* E, double* Q) {
  if (!r || !r->grid_set) return -1;
  int N = r->N;
  if (phi) memcpy(phi, r->phi, sizeof(double) * (size_t)(N + 1));
  if (E) memcpy(E, r->E, sizeof(double) * (size_t)((r->scheme == OR_SCHEME_MC || r->scheme == OR_SCHEME_MC2) ? N + 1 : N));
  if (Q) memcpy(Q, r->Q, sizeof(double) * (size_t)(N + 1));
  return 0;
}

int oracle_get_energy(const or_run* r, double* ke, double* fe) {
  if (!r) return -1;
  if (ke)
    for (int si = 0; si < r->ns; ++si) ke[si] = r->sp[si].ke;
  if (fe) *fe = r->fe;
  return 0;
}

int64_t oracle_get_averages(const or_run* r, double* density, double* phi,
                            double* Tx, double* Tx_mom) {
  if (!r || !r->grid_set) return -1;
  int64_t ns = r->n_samples;
  int N = r->N;
  double inv = ns > 0 ? 1.0 / (double)ns : 0.0;
  for (int si = 0; si < r->ns; ++si) {
    const or_species* s = &r->sp[si];
    for (int n = 0; n <= N; ++n) {
      size_t o = (size_t)si * (size_t)(N + 1) + (size_t)n;
      if (density) density[o] = s->acc_n[n] * inv;
      if (Tx) Tx[o] = s->acc_T[n] * inv;
      if (Tx_mom) {
        double M0 = s->acc_M0[n];
        double T = 0.0;
        if (M0 > 0.0) {
          double m1 = s->acc_M1[n] / M0, m2 = s->acc_M2[n] / M0;
          T = s->m * (m2 - m1 * m1) / OR_QE;
        }
        Tx_mom[o] = T;
      }
    }
  }
  if (phi)
    for (int n = 0; n <= N; ++n) phi[n] = r->acc_phi[n] * inv;
  return ns;
}

/* ------------------------------------------------------------------ */
int oracle_set_rebalance(or_run* r, int every, int target, int lo, int hi, uint32_t m0) {
  if (!r || every < 0 || target < 1 || target > OR_RB_MAX_CELL || lo < 0 || hi < target ||
      lo > target || m0 < 1 || m0 > OR_RB_MAX_WEIGHT)
    return -1;
  if (r->initialized) return -2;
  r->rb_every = every; r->rb_target = target; r->rb_lo = lo; r->rb_hi = hi; r->rb_m0 = m0;
  return 0;
}

int oracle_rebalance_now(or_run* r) {
  if (!r) return -1;
  if (!r->initialized) return -2;
  return or_rebalance(r);
}

int oracle_get_weights(const or_run* r, int species, uint32_t* k, int64_t cap, int64_t* n) {
  if (!r || species < 0 || species >= r->ns || !n) return -1;
  const or_species* s = &r->sp[species];
  *n = s->n;
  if (cap < s->n) return -1;
  if (k) memcpy(k, s->mw, sizeof(uint32_t) * (size_t)s->n);
  return 0;
}

int oracle_set_weights(or_run* r, int species, const uint32_t* k, int64_t n) {
  if (!r || species < 0 || species >= r->ns || !k) return -1;
  if (!r->initialized) return -2;
  or_species* s = &r->sp[species];
  if (n != s->n) return -1;
  for (int64_t i = 0; i < n; ++i)
    if (k[i] < 1u || k[i] > OR_RB_MAX_WEIGHT) return -1;
  memcpy(s->mw, k, sizeof(uint32_t) * (size_t)n);
  return or_refresh(r);
}

int oracle_get_rebalance_counters(const or_run* r, int64_t* out3) {
  if (!r || !out3) return -1;
  for (int si = 0; si < OR_MAX_SPECIES; ++si) {
    const or_species* s = &r->sp[si];
    int on = si < r->ns;
    out3[3 * si] = on ? s->rb_merged : 0;
    out3[3 * si + 1] = on ? s->rb_split : 0;
    out3[3 * si + 2] = on ? s->rb_skipped : 0;
  }
  return 0;
}

int oracle_deposit_fixed_w(int N, int64_t n, const int32_t* cell, const float* xi,
                           const uint32_t* k, uint64_t* S) {
  if (N < 1 || n < 0 || (n > 0 && (!cell || !xi || !k)) || !S) return -1;
  for (int64_t i = 0; i < n; ++i) {
    int j = cell[i];
    float f = xi[i];
    if (j < 0 || j >= N || !(f >= 0.0f) || !(f < 1.0f)) return -1;
    uint64_t rgt = (uint64_t)(uint32_t)((double)f * 4294967296.0); /* floor, f < 1 */
    S[j] += (uint64_t)k[i] * (4294967296ull - rgt);
    S[j + 1] += (uint64_t)k[i] * rgt;
  }
  return 0;
}
