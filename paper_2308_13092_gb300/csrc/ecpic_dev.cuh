// ecpic_dev.cuh -- device-side state layout and helpers of libecpic.
//
// HBM layout (one "batch" holds up to max_slots independent discharge runs):
//   * particles: structure of arrays per (slot, species) segment, two buffer
//     sets (the counting sort scatters from one to the other):
//       int32 cell | f32 xi in [0,1) | f32 vx, vy, vz (m/s) | u64 id
//     28 B per particle.  cell < 0 marks an absorbed particle until the next
//     sort compacts it away.
//   * per run: FP64 edges/volumes, FP32 per-cell dt/dx and neighbour width
//     ratios, FP32 field E (what the push reads), FP64 potential, the
//     fixed-point deposit S (u64, N+1 per species), FP64 diagnostics.
// Device-mutable counters live in RunState/SegState so that CUDA graphs
// replay without host updates.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/ecpic.h"

namespace ecpic {

constexpr int kMaxSpecies = ECPIC_MAX_SPECIES;
constexpr int kMaxProc = ECPIC_MAX_PROC;
constexpr int kMaxCells = ECPIC_MAX_CELLS;
constexpr int kMaxSeg = 1024;  // slots * species per batch
constexpr int kNumCtr = 20;    // counters per species, see Ctr

// per-species counters in RunState::ctr
enum Ctr {
  C_ABS_L = 0, C_ABS_R = 1, C_BIRTHS = 2, C_LOST = 3, C_CLAMPS = 4, C_CAND = 5,
  C_NAN = 6, C_IMP_LOST = 7, C_COLL0 = 8,  // C_COLL0 + p, p < kMaxProc
  C_RB_MERGED = 16, C_RB_SPLIT = 17, C_RB_SKIPPED = 18  // particle rebalancing
};

// particle rebalancing limits: cells above kRbMaxCell particles of a species
// are left alone, groups heavier than kRbMaxWeight base particles are not
// merged (the weighted deposit's 64-bit sums stay far from overflow)
constexpr int kRbMaxCell = 4096;
constexpr unsigned kRbMaxWeight = 65536u;

struct ProcDev {
  int kind;
  float thr;             // eV
  int product_seg;       // ionisation: segment of the ion species in this run
  int product_species;
};

struct SpeciesDev {
  double q, m, w;
  double cw;            // q w 2^-32: the charge of one 2^-32 deposit share (C m^-2)
  float qm_dt;          // (q/m) dt: the push adds qm_dt * E
  float half_m_over_e;  // E[eV] = half_m_over_e * |g|^2
  float two_e_over_m;   // |v| = sqrt(two_e_over_m * E[eV])
  float two_m_over_M;   // electron elastic energy-loss factor 2m/M
  float m_frac;         // m_gas / (m + m_gas)
  float mass_frac;      // m / (m + m_gas)
  float nu_max;         // 1/s (FP32 copy of the host FP64 value)
  float nu_bnd;         // n_g * max over nodes of the summed cross sections, padded by
                        // 2^-16 so that nu_bnd * |g| bounds the FP32 total rate
  uint32_t thr24;       // candidate iff (r0 >> 8) < thr24
  float dE_inv;
  int ntab;
  int nproc;
  int heavy;            // samples the target neutral's velocity
  int np4;              // groups of four processes per table node: (nproc + 3) / 4
  // cross sections (m^2) of all processes interleaved by node: entry
  // [node * np4 + g] holds processes 4g..4g+3 (zero past nproc)
  const float4* sig4;
  float thr_all[kMaxProc];  // thresholds (eV), FLT_MAX past nproc
  ProcDev proc[kMaxProc];
};

struct RunDev {
  int active;
  int N, bc, scheme, uniform, ns;
  int seg0;             // first segment of this run (segments seg0..seg0+ns-1)
  int sample_every;
  // field solve: every species' q w is equal up to sign (field_pm), so one
  // signed integer sum of the deposits per node serves all; bit s of
  // field_neg: species s has the opposite sign of species 0
  int field_pm, field_neg;
  // particle rebalancing: weight multipliers on (the segments' wt arrays),
  // every rb_every steps (0: only on demand), merge above rb_hi particles of
  // a species in a cell, split below rb_lo, aiming at rb_target
  int rb, rb_every, rb_target, rb_lo, rb_hi, rb_pad;
  double L, dt;
  float dtdx_u;         // dt/dx on a uniform grid
  float ng;             // gas density
  float vth_gas;        // sqrt(kT/m_gas)
  float pad0;
  const double* x;      // N+1 edges
  const double* dx;     // N widths
  const double* V;      // N+1 node control volumes
  const double* invV;   // N+1: 1/V
  const double* mcw;    // N+1: centred-field weight dx_n/(dx_{n-1}+dx_n) (MC scheme)
  const double* cumV;   // N+1: sum_{m=1..n} V_m (periodic neutralising background)
  double* g;            // N: (phi_{n+1}-phi_n)/dx_n of the current field, FP64
  double inv_L;
  const float* dtdx;    // N: dt/dx_j
  const float* rp;      // N: dx_j / dx_{j+1} (wrapped when periodic)
  const float* rm;      // N: dx_j / dx_{j-1}
  double v0, freq, phase, vdc;
  uint64_t seed;
  float* E;             // N (EC) or N+1 (MC)
  double* phi;          // N+1
  unsigned long long* S;  // ns * (N+1) fixed-point deposit
  float* mom;           // ns * 2 * (N+1): sample-step vx moments (FP32 partials)
  double* momd;         // ns * 2 * (N+1): sample-step vx moments (FP64 totals)
  double* acc;          // diagnostics accumulators, see kAcc*
  // tallies: EEDF of cells eedf_c0..eedf_c1 (species with q < 0, sample
  // steps), impact energy and angle at x = 0 (q > 0, every step); per
  // species tal[s * tal_stride + ...] = eedf | iedf | iad counts
  unsigned long long* tal;
  double* pw;           // ns * N: sum over samples of (v^- + v^+) E_i per cell
  int tal_stride, eedf_n, iedf_n, iad_n, eedf_c0, eedf_c1;
  float eedf_dEinv, iedf_dEinv, iad_binv;  // bins per eV, per eV, per degree
  SpeciesDev sp[kMaxSpecies];
};

// diagnostics accumulator offsets, in units of (N+1) doubles, species-major
//   [0, ns)      density        [ns, 2ns)  temperature
//   [2ns, 3ns)   M0   [3ns, 4ns) M1   [4ns, 5ns) M2   [5ns] phi
inline __host__ __device__ int acc_size(int ns) { return 5 * ns + 1; }

struct RunState {
  long long step;       // current time level k
  long long step_end;   // stepping stops at this level
  int status;           // first device-side error (ecpic_status)
  int fresh;            // admitted in a wave, its particles and step-0 field not yet formed
  long long n_samples;
  double ke_acc[kMaxSpecies];   // accumulating during a sampled push
  double ke[kMaxSpecies];       // of the last sampled push
  double fe_field;              // field energy of the current field
  double fe;                    // at the level of the last sampled push
  double phi0;                  // electrode potential of the current field
  long long phi_level;          // time level of the potential held in phi
  long long rb_level;           // level of the last rebalancing (-1: none)
  int rb_force;                 // rebalance at the current level whatever the cadence
  int rb_pad;
  unsigned long long psteps;    // particle-steps advanced (live at the start of each step)
  unsigned long long ctr[kMaxSpecies][kNumCtr];
};

// A real collision recorded by the pass for the collision kernel, with the
// particle's state after the push (48 B, written and read as three 16-byte
// words).
struct __align__(16) RealRec {
  uint64_t id;
  int i;            // index in the current buffer set
  int chosen;       // process
  float En, gm;     // energy (eV) and relative speed (m/s) of the null-collision test
  float vx, vy, vz;
  int c;
  float f;
  unsigned k;       // weight multiplier (1 without rebalancing)
};
static_assert(sizeof(RealRec) == 48, "RealRec layout");

struct SegDev {
  int32_t* cell[2];
  float* xi[2];
  float* vx[2];
  float* vy[2];
  float* vz[2];
  uint64_t* id[2];
  uint32_t* wt[2];      // weight multipliers (rebalancing runs only, else null)
  long long cap;
  int run;              // slot index
  int species;
  int hoff;             // offset of this segment's histogram (N ints)
  int pad;
  // real collisions of the current step, recorded by the pass for the
  // collision kernel
  RealRec* real;
  long long real_cap;
  // particles of a q > 0 species absorbed at x = 0 this step (indices), for
  // the impact tallies of the collision kernel; overflow is counted
  int* imp;
  long long imp_cap;
};

struct SegState {
  long long n_proc;     // particles processed by this step's pass
  long long n_alloc;    // append cursor for births (>= n_proc)
  long long n_live;     // written by the sort scan
  long long n_dead;     // slots below n_proc marked absorbed since the last sort
  long long n_real;     // records in SegDev::real this step (reset by the field kernel)
  long long n_imp;      // entries in SegDev::imp this step (reset by the field kernel)
  int cur;              // current buffer set
  int rb_over;          // rebalancing: the planned particles exceed the capacity
  long long n_rb;       // rebalancing: particles after the merges and splits
};

// kernel modes for the segment-walking kernels
enum PassMode { MODE_STEP = 0, MODE_REFRESH = 1, MODE_SORT = 2, MODE_REBAL = 3 };

// ------------------------------------------------------------------ Philox
// Philox4x32-10 (Salmon et al., SC'11): ten rounds, Weyl key schedule.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
    const uint32_t lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

__device__ __forceinline__ uint4 draw(uint64_t seed, uint64_t id, uint32_t step_word,
                                      uint32_t word3) {
  return philox4x32_10(make_uint4((uint32_t)id, (uint32_t)(id >> 32), step_word, word3),
                       make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
}

// 24-bit uniforms, exact in FP32
__device__ __forceinline__ float u24(uint32_t r) { return (float)(r >> 8) * 5.9604644775390625e-8f; }
__device__ __forceinline__ float u24_open(uint32_t r) {
  return (float)((r >> 8) + 1u) * 5.9604644775390625e-8f;
}

// kinetic energy (eV) from vx and vy^2 + vz^2, rounded the same way wherever
// a tally bins it (the pass and the collision kernel must agree)
__device__ __forceinline__ float yz2(float vy, float vz) { return __fadd_rn(__fmul_rn(vy, vy), __fmul_rn(vz, vz)); }
__device__ __forceinline__ float kin_eV(float half_m_over_e, float vx, float yz) {
  return __fmul_rn(half_m_over_e, __fadd_rn(__fmul_rn(vx, vx), yz));
}
__device__ __forceinline__ int tally_bin(float v, float inv_width, int n) {
  const float b = floorf(__fmul_rn(v, inv_width));
  if (!(b >= 0.0f)) return 0;
  if (b >= (float)(n - 1)) return n - 1;
  return (int)b;
}

// splitmix64 output function (Steele, Lea & Flood 2014)
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
// id of an ionisation child born at step k: mix(parent ^ mix(4k + tag))
__device__ __forceinline__ uint64_t child_id(uint64_t parent, long long step, uint64_t tag) {
  return mix64(parent ^ mix64((uint64_t)step * 4u + tag));
}

}  // namespace ecpic
