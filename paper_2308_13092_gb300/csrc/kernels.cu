// kernels.cu -- the sm_103a kernels of libecpic.
//
// One time step of every resident run is two launches:
//   k_pass   fused gather (Eq. 6-7, or CIC for the MC scheme) -> leapfrog
//            push (Eq. 8-9) in cell-relative FP32 -> wall absorption ->
//            null-collision MCC (Sec. 2a step 6) -> fixed-point CIC deposit
//            (Eq. 2-3) of the new positions, over all (run, species)
//            segments, load-balanced by particle count;
//   k_field  per run: charge from the deposit, Poisson (Eq. 4) in its
//            two-scan form, field (Eq. 5 or centred), potential, sampling.
// Every K steps a counting sort by cell (k_hist, k_scan, k_scatter,
// k_finalize) restores cell order and drops absorbed particles.
#include <cfloat>
#include <climits>

#include "kernels.h"

namespace ecpic {

// Checked builds (-DECPIC_CHECKS): indexed accesses are validated against
// their bounds; the first violation (site, index, bound) and a violation count
// are recorded and the access is skipped.  Plain builds compile the checks
// away.
__device__ unsigned long long g_check[4];

namespace {

#ifdef ECPIC_CHECKS
__device__ __noinline__ bool chk(bool ok, int where, long long idx, long long bound) {
  if (!ok) {
    if (atomicCAS(&g_check[0], 0ull, (unsigned long long)where) == 0ull) {
      g_check[1] = (unsigned long long)idx;
      g_check[2] = (unsigned long long)bound;
    }
    atomicAdd(&g_check[3], 1ull);
  }
  return ok;
}
#else
__device__ __forceinline__ bool chk(bool, int, long long, long long) { return true; }
#endif

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr double kEps0 = 8.8541878128e-12;
constexpr double kTwoPi = 6.283185307179586476925286766559;

// ----------------------------------------------------------------- reductions
template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T t = __shfl_up_sync(kFull, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// exclusive scan over the block (blockDim a multiple of 32); wsm >= 32 entries
template <typename T>
__device__ T block_excl_scan(T v, T* wsm, T* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const T inc = warp_incl_scan(v);
  if (lane == 31) wsm[w] = inc;
  __syncthreads();
  if (w == 0) {
    T t = lane < nw ? wsm[lane] : T(0);
    t = warp_incl_scan(t);
    if (lane < nw) wsm[lane] = t;
  }
  __syncthreads();
  const T off = w > 0 ? wsm[w - 1] : T(0);
  *total = wsm[nw - 1];
  __syncthreads();
  return off + inc - v;
}

template <typename T>
__device__ T block_sum(T v, T* wsm) {
  T total;
  block_excl_scan(v, wsm, &total);
  return total;
}

// in-place inclusive scan of a[0..n) held in shared memory (fixed partition,
// so the FP64 rounding is deterministic)
template <typename T>
__device__ void block_incl_scan_array(T* a, int n, T* wsm) {
  const int per = (n + blockDim.x - 1) / blockDim.x;
  const int beg = min(n, (int)threadIdx.x * per), end = min(n, beg + per);
  T loc = T(0);
  for (int i = beg; i < end; ++i) loc += a[i];
  T total;
  T run = block_excl_scan(loc, wsm, &total);
  for (int i = beg; i < end; ++i) {
    run += a[i];
    a[i] = run;
  }
  __syncthreads();
}

// ----------------------------------------------------------------- segments
__device__ __forceinline__ bool run_live(const RunDev& R, const RunState& S, int mode, int only,
                                         int slot) {
  if (!R.active) return false;
  if (mode == MODE_REFRESH) return only == kOnlyFresh ? S.fresh != 0 : slot == only;
  if (S.status != 0) return false;
  if (mode == MODE_STEP) return S.step < S.step_end;
  if (mode == MODE_REBAL)  // a rebalancing run at a rebalancing level (once per level)
    return R.rb && (S.rb_force || (R.rb_every > 0 && S.step > 0 && S.step % R.rb_every == 0 &&
                                   S.rb_level != S.step));
  return true;
}

// exclusive prefix of the work of all segments (particles, groups of `unit`
// particles, or recorded real collisions): pre[0..nseg]
// (with meta: per segment its run slot, buffer index and real-collision
// count, meta[3 s .. 3 s + 2], so that the records' consumers need no
// dependent global loads for them)
__device__ long long seg_prefix(const BatchView& b, int mode, int only, long long* pre,
                                long long* wsm, int unit = 1, bool reals = false,
                                int* meta = nullptr) {
  const int per = (b.nseg + blockDim.x - 1) / blockDim.x;
  const int s0 = threadIdx.x * per;
  long long loc = 0;
  for (int k = 0; k < per; ++k) {
    const int s = s0 + k;
    if (s < b.nseg) {
      const int slot = b.segs[s].run;
      const bool live = run_live(b.runs[slot], b.rst[slot], mode, only, slot);
      // records past a list's capacity were never written (the pass failed
      // the run with ECPIC_ERR_CAPACITY): only the stored ones count
      const long long nr = reals ? min(b.sst[s].n_real, b.segs[s].real_cap) : 0;
      const long long c = !live ? 0
                          : reals ? nr + min(b.sst[s].n_imp, b.segs[s].imp_cap)
                                  : (b.sst[s].n_proc + unit - 1) / unit;
      pre[s] = c;
      loc += c;
      if (meta) {
        meta[3 * s] = slot;
        meta[3 * s + 1] = b.sst[s].cur;
        meta[3 * s + 2] = live ? (int)nr : 0;
      }
    }
  }
  long long total;
  long long run = block_excl_scan(loc, wsm, &total);
  for (int k = 0; k < per; ++k) {
    const int s = s0 + k;
    if (s < b.nseg) {
      const long long c = pre[s];
      pre[s] = run;
      run += c;
    }
  }
  if (threadIdx.x == 0) pre[b.nseg] = total;
  __syncthreads();
  return total;
}

// first segment s with pre[s] <= v < pre[s+1]
__device__ __forceinline__ int seg_find(const long long* pre, int nseg, long long v) {
  int lo = 0, hi = nseg;  // pre[lo] <= v, answer in [lo, hi)
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (pre[mid] <= v) lo = mid; else hi = mid;
  }
  return lo;
}

// ----------------------------------------------------------------- deposit
// Fixed-point CIC deposit (Eq. 2-3) in units of 2^-32 particle: a particle at
// (c, xi) with r = floor(xi 2^32) (xi * 2^32 is exact in FP32; rz truncation
// = floor) adds 2^32 - r to node c and r to node c+1.  In shared memory each
// cell keeps three 32-bit sums, updated with native 32-bit atomics: its
// particle count, and the sums of the low and high 16 bits of r.  The flush
// forms the node values, S[c] += cnt 2^32 - R and S[c+1] += R with
// R = hi 2^16 + lo.  With at most kFlushParticles particles between flushes
// no sum reaches 2^32.
constexpr int kFlushParticles = 65536;
constexpr int kFlushIters = kFlushParticles / (4 * kPassBlock);  // quad iterations of a block

// Adds four particles (cells c[j] < 0 skipped); a thread's consecutive
// particles in the same cell are merged first, so sorted data costs one
// atomic triple per run.
__device__ __forceinline__ void dep_add4(uint32_t* dcnt, uint32_t* dlo, uint32_t* dhi, const int c[4],
                                         const float f[4]) {
  unsigned lo[4], hi[4], cn[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const bool v = c[j] >= 0;
    const unsigned r = v ? __float2uint_rz(f[j] * 4294967296.0f) : 0u;
    lo[j] = r & 0xFFFFu;
    hi[j] = r >> 16;
    cn[j] = v ? 1u : 0u;
  }
#pragma unroll
  for (int j = 3; j >= 1; --j) {
    if (c[j] >= 0 && c[j] == c[j - 1]) {
      lo[j - 1] += lo[j];
      hi[j - 1] += hi[j];
      cn[j - 1] += cn[j];
      cn[j] = 0u;
    }
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    if (cn[j]) {
      atomicAdd(dcnt + c[j], cn[j]);
      atomicAdd(dlo + c[j], lo[j]);
      atomicAdd(dhi + c[j], hi[j]);
    }
  }
}

// Adds the shared sums of cells [a, e) to the node array S in HBM and clears
// them.  Every thread of the block calls it, between barriers.
__device__ void dep_flush(uint32_t* dcnt, uint32_t* dlo, uint32_t* dhi, int a, int e,
                          unsigned long long* S) {
  for (int c = a + (int)threadIdx.x; c < e; c += (int)blockDim.x) {
    const uint32_t n = dcnt[c];
    if (n) {
      const unsigned long long R = ((unsigned long long)dhi[c] << 16) + (unsigned long long)dlo[c];
      atomicAdd(S + c, ((unsigned long long)n << 32) - R);
      if (R) atomicAdd(S + c + 1, R);
      dcnt[c] = 0u;
      dlo[c] = 0u;
      dhi[c] = 0u;
    }
  }
}

// ---- weighted CIC deposit (rebalancing runs) -----------------------------
// A particle of weight multiplier k adds k (2^32 - r) to node c and k r to
// node c+1.  Shared 64-bit atomics are compare-and-swap loops on this part
// and the lanes of a warp share a few cells on sorted data, so the sums stay
// in native 32-bit atomics: with r = rh 2^16 + rl, k rl = a1 2^16 + a0 and
// k rh = b1 2^16 + b0 (k <= 2^16, so every piece is below 2^16), each cell
// keeps K = sum k, A = sum a0, M = sum (a1 + b0), B = sum b1, and
// R = sum k r = 2^32 B + 2^16 M + A.  Flushed at least every
// kFlushParticles / 2 = 2^15 particles, K stays <= 2^31 and M < 2^32.
// Four arrays keep the pass at four CTAs per SM on 1024-cell batches.
struct DepW {
  uint32_t *k, *a, *m, *b;  // (nmax + 1) each
};

__device__ __forceinline__ void depw_add4(const DepW& d, const int c[4], const float f[4],
                                          const unsigned kq[4]) {
  unsigned K[4], A[4], M[4], B[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const bool v = c[j] >= 0;
    const unsigned r = v ? __float2uint_rz(f[j] * 4294967296.0f) : 0u;
    const unsigned k = v ? kq[j] : 0u;
    const unsigned p = k * (r & 0xFFFFu), q = k * (r >> 16);
    K[j] = k;
    A[j] = p & 0xFFFFu;
    M[j] = (p >> 16) + (q & 0xFFFFu);
    B[j] = q >> 16;
  }
#pragma unroll
  for (int j = 3; j >= 1; --j) {
    if (c[j] >= 0 && c[j] == c[j - 1]) {
      K[j - 1] += K[j];
      A[j - 1] += A[j];
      M[j - 1] += M[j];
      B[j - 1] += B[j];
      K[j] = 0u;
    }
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    if (K[j]) {
      atomicAdd(d.k + c[j], K[j]);
      atomicAdd(d.a + c[j], A[j]);
      atomicAdd(d.m + c[j], M[j]);
      atomicAdd(d.b + c[j], B[j]);
    }
  }
}

// Adds the sums of cells [a, e) to the node array S (cell c to nodes c and
// c+1) and clears them; every thread of the block calls it, between barriers.
__device__ void depw_flush(const DepW& d, int a, int e, unsigned long long* S) {
  for (int c = a + (int)threadIdx.x; c < e; c += (int)blockDim.x) {
    const uint32_t K = d.k[c];
    if (K) {
      const unsigned long long R = ((unsigned long long)d.b[c] << 32) +
                                   ((unsigned long long)d.m[c] << 16) + d.a[c];
      atomicAdd(S + c, ((unsigned long long)K << 32) - R);
      if (R) atomicAdd(S + c + 1, R);
      d.k[c] = 0u;
      d.a[c] = 0u;
      d.m[c] = 0u;
      d.b[c] = 0u;
    }
  }
}

// ---- quadratic-spline deposit of the EC2 scheme (uniform grids) ----------
// A particle at cell + xi with r = floor(xi 2^32) has its nearest node
// n0 = cell + (r >= 2^31) and offset U = r or r - 2^32 (2^-32 cell units);
// nodes n0-1, n0, n0+1 get a = floor((2^31-U)^2 / 2^33), 2^32 - a - b,
// b = floor((2^31+U)^2 / 2^33): the quadratic B-spline weights to 2^-32,
// exact integers summing to 2^32.
__device__ __forceinline__ void spline2_shares(float f, int c, int* n0, unsigned* a, unsigned* b) {
  const unsigned r = __float2uint_rz(f * 4294967296.0f);
  const bool up = r >= 0x80000000u;
  *n0 = c + (up ? 1 : 0);
  const long long U = up ? (long long)r - 4294967296LL : (long long)r;
  const unsigned long long A = (unsigned long long)(2147483648LL - U);
  const unsigned long long B = (unsigned long long)(2147483648LL + U);
  *a = (unsigned)((__umul64hi(A, A) << 31) | ((A * A) >> 33));
  *b = (unsigned)((__umul64hi(B, B) << 31) | ((B * B) >> 33));
}

// node of a share beyond the cells: folded into the wall node (Dirichlet: the
// ghost node beyond a wall is the wall node), wrapped when periodic (node N
// and node 0 are one node for the field solve)
__device__ __forceinline__ int node2(int n, int N, bool periodic) {
  if (periodic) return n < 0 ? n + N : (n > N ? n - N : n);
  return n < 0 ? 0 : (n > N ? N : n);
}

// Adds four particles to two 32-bit sums per node (the low and high 16 bits
// of the shares it receives, after folding or wrapping); runs of equal
// nearest node merged first.  A wall node can receive two shares of one
// particle, and a run's middle share can reach 2^34, so the EC2 pass flushes
// every kFlushParticles / 4 particles: no sum reaches 2^32.
__device__ __forceinline__ void dep2_add4(uint32_t* dlo, uint32_t* dhi, int N, bool periodic,
                                          const int c[4], const float f[4]) {
  int n0[4];
  unsigned long long A[4], M[4], B[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    unsigned a = 0u, b = 0u;
    n0[j] = -1;
    if (c[j] >= 0) spline2_shares(f[j], c[j], &n0[j], &a, &b);
    A[j] = a;
    B[j] = b;
    M[j] = c[j] >= 0 ? 4294967296ull - a - b : 0ull;
  }
#pragma unroll
  for (int j = 3; j >= 1; --j) {
    if (n0[j] >= 0 && n0[j] == n0[j - 1]) {
      A[j - 1] += A[j];
      M[j - 1] += M[j];
      B[j - 1] += B[j];
      n0[j] = -1;
    }
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    if (n0[j] >= 0) {
      const int nl = node2(n0[j] - 1, N, periodic), nr = node2(n0[j] + 1, N, periodic);
      atomicAdd(dlo + nl, (unsigned)(A[j] & 0xFFFFu));
      atomicAdd(dhi + nl, (unsigned)(A[j] >> 16));
      atomicAdd(dlo + n0[j], (unsigned)(M[j] & 0xFFFFu));
      atomicAdd(dhi + n0[j], (unsigned)(M[j] >> 16));
      atomicAdd(dlo + nr, (unsigned)(B[j] & 0xFFFFu));
      atomicAdd(dhi + nr, (unsigned)(B[j] >> 16));
    }
  }
}

// Adds the sums of nodes [a, e] to S and clears them; every thread of the
// block calls it, between barriers.
__device__ void dep2_flush(uint32_t* dlo, uint32_t* dhi, int a, int e, unsigned long long* S) {
  for (int n = a + (int)threadIdx.x; n <= e; n += (int)blockDim.x) {
    const unsigned long long v = ((unsigned long long)dhi[n] << 16) + dlo[n];
    if (v) {
      atomicAdd(S + n, v);
      dlo[n] = 0u;
      dhi[n] = 0u;
    }
  }
}

__device__ __forceinline__ void deposit2_one(unsigned long long* S, int c, float f, int N, bool periodic) {
  int n0;
  unsigned a, b;
  spline2_shares(f, c, &n0, &a, &b);
  atomicAdd(S + node2(n0 - 1, N, periodic), (unsigned long long)a);
  atomicAdd(S + n0, 4294967296ull - a - b);
  atomicAdd(S + node2(n0 + 1, N, periodic), (unsigned long long)b);
}

__device__ __forceinline__ void deposit_one(unsigned long long* S, int c, float f, unsigned k = 1u) {
  const unsigned r = __float2uint_rz(f * 4294967296.0f);
  atomicAdd(S + c, (unsigned long long)k * (4294967296ull - (unsigned long long)r));
  atomicAdd(S + c + 1, (unsigned long long)k * (unsigned long long)r);
}

// ----------------------------------------------------------------- MCC helpers
// Collision frequencies nu_p = n_g sigma_p(E) |g| of a species' processes, in
// process order, from its node-interleaved table: linear interpolation
// between nodes dE apart, the last node's value past the table, zero below a
// process threshold.  Returns the first p whose running sum exceeds Rr (the
// selection of Sec. 2a step 6; -1 for a null collision) and the total in *tot.
__device__ __forceinline__ int select_process(const SpeciesDev* SP, float E, float gm, float ng,
                                              float Rr, float* tot) {
  const int n = SP->ntab, np4 = SP->np4;
  const float u = E * SP->dE_inv;
  const float fi = floorf(u);
  const bool top = fi >= (float)(n - 1);
  int i = top ? n - 1 : (int)fi;
  if (!chk(i >= 0 && i < n, 17, i, n)) i = 0;
  const int i1 = top ? i : i + 1;
  const float t = top ? 0.0f : u - fi;
  const float4* tab = SP->sig4;
  float cum = 0.0f;
  int chosen = -1;
  for (int g = 0; g < np4; ++g) {
    const float4 a = __ldg(tab + (size_t)i * np4 + g);
    const float4 b = __ldg(tab + (size_t)i1 * np4 + g);
    const float sg[4] = {a.x + t * (b.x - a.x), a.y + t * (b.y - a.y), a.z + t * (b.z - a.z),
                         a.w + t * (b.w - a.w)};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int p = 4 * g + q;
      const float sig = E < SP->thr_all[p] ? 0.0f : sg[q];
      cum += ng * sig * gm;
      if (chosen < 0 && Rr < cum) chosen = p;
    }
  }
  *tot = cum;
  return chosen;
}

__device__ __forceinline__ void box_muller(float u1, float u2, float& z0, float& z1) {
  const float rad = sqrtf(-2.0f * logf(u1));
  float s, c;
  sincospif(2.0f * u2, &s, &c);
  z0 = rad * c;
  z1 = rad * s;
}

// unit vector uniform on the sphere, polar axis along x
__device__ __forceinline__ void isotropic(float ua, float ub, float& d0, float& d1, float& d2) {
  const float c = 1.0f - 2.0f * ua;
  const float s = sqrtf(fmaxf(0.0f, 1.0f - c * c));
  float sp, cp;
  sincospif(2.0f * ub, &sp, &cp);
  d0 = c;
  d1 = s * cp;
  d2 = s * sp;
}

__device__ __forceinline__ void set_status(RunState* st, int code) {
  atomicCAS(&st->status, 0, code);
}

// append a particle to a segment (births); false if the capacity is full
__device__ __forceinline__ bool append_particle(const SegDev& G, SegState* ss, int c, float f,
                                                float vx, float vy, float vz, uint64_t id,
                                                unsigned k = 1u) {
  const long long idx = (long long)atomicAdd((unsigned long long*)&ss->n_alloc, 1ull);
  if (idx >= G.cap) return false;
  const int cur = ss->cur;
  G.cell[cur][idx] = c;
  G.xi[cur][idx] = f;
  G.vx[cur][idx] = vx;
  G.vy[cur][idx] = vy;
  G.vz[cur][idx] = vz;
  G.id[cur][idx] = id;
  if (G.wt[cur]) G.wt[cur][idx] = k;
  return true;
}

// cell walk on a non-uniform grid: g = xi + vx dt/dx_c, carried into the
// neighbours with their width ratios; FP32 rounding to 1.0f puts the particle
// on the next face (xi = 0)
__device__ __forceinline__ void walk_nonuniform(int& c, float& f, float g, int N, int bc,
                                                const float* rp, const float* rm) {
  int guard = 0;
  while (g >= 1.0f) {
    if (c == N - 1 && bc != ECPIC_PERIODIC) { c = N; g = 0.0f; break; }
    g = (g - 1.0f) * __ldg(rp + c);
    c = (c == N - 1) ? 0 : c + 1;
    if (++guard > N) { g = 0.0f; break; }
  }
  while (g < 0.0f) {
    if (c == 0 && bc != ECPIC_PERIODIC) { c = -1; g = 0.0f; break; }
    g = 1.0f + g * __ldg(rm + c);
    c = (c == 0) ? N - 1 : c - 1;
    if (g >= 1.0f) {
      c = (c == N - 1) ? 0 : c + 1;
      g = 0.0f;
    }
    if (++guard > N) { g = 0.0f; break; }
  }
  f = g;
}

constexpr int kRing = 160;  // candidate ring per warp: >= 31 left over + 4 * 32 added

struct PassShared {
  unsigned long long ctr[kNumCtr];
  long long wsm[32];
  double dsm[32];
  int lohi[2];
  int qcount;
};

// Ionisation of the electron at (c, f) with energy Erem above threshold
// left to share (Sec. 2a step 6): the two electrons split it by a uniform
// fraction, the primary leaving along (d0, d1, d2), the secondary isotropic;
// the ion is drawn from the gas Maxwellian.  The secondary is appended to
// this segment, the ion to its species' segment; both are deposited (and,
// on sample steps, enter the vx moments) in HBM.  Returns the primary's new
// velocity.
__device__ __noinline__ float3 ionize(const BatchView& b, int s, int chosen, int c, float f, uint64_t id,
                                      long long k, float Erem, bool sample, float d0, float d1,
                                      float d2, unsigned kw) {
  const SegDev& G = b.segs[s];
  const int slot = G.run, sp = G.species;
  const RunDev* R = b.runs + slot;
  RunState* st = b.rst + slot;
  SegState* ss = b.sst + s;
  const SpeciesDev* SP = &R->sp[sp];
  const int N = R->N;
  const uint64_t seed = R->seed;
  const uint4 B = draw(seed, id, (uint32_t)k, ((uint32_t)sp << 8) | 1u);
  const float fr = u24(B.x);
  const float v1 = sqrtf(SP->two_e_over_m * (fr * Erem));
  const float v2 = sqrtf(SP->two_e_over_m * ((1.0f - fr) * Erem));
  float e0, e1, e2;
  isotropic(u24(B.y), u24(B.z), e0, e1, e2);
  const uint4 Cw = draw(seed, id, (uint32_t)k, ((uint32_t)sp << 8) | 2u);
  float z0, z1, z2, z3;
  box_muller(u24_open(Cw.x), u24(Cw.y), z0, z1);
  box_muller(u24_open(Cw.z), u24(Cw.w), z2, z3);
  const float sd = R->vth_gas;
  atomicAdd(&st->ctr[sp][C_BIRTHS], 1ull);
  // secondary electron: same segment and species; both products carry the
  // parent's weight multiplier kw (charge conserved)
  const float vb = v2 * e0;
  const float fk = (float)kw;
  if (append_particle(G, ss, c, f, vb, v2 * e1, v2 * e2, child_id(id, k, 1), kw)) {
    if (R->scheme >= ECPIC_SCHEME_EC2)
      deposit2_one(R->S + (size_t)sp * (N + 1), c, f, N, R->bc == ECPIC_PERIODIC);
    else
      deposit_one(R->S + (size_t)sp * (N + 1), c, f, kw);
    if (sample && SP->q < 0.0 && c >= R->eedf_c0 && c <= R->eedf_c1)
      atomicAdd(R->tal + (size_t)sp * R->tal_stride +
                    tally_bin(kin_eV(SP->half_m_over_e, vb, yz2(v2 * e1, v2 * e2)), R->eedf_dEinv, R->eedf_n),
                (unsigned long long)kw);
    if (sample) {
      double* md = R->momd + (size_t)sp * 2 * (N + 1);
      atomicAdd(md + c, (double)(fk * ((1.0f - f) * vb)));
      atomicAdd(md + c + 1, (double)(fk * (f * vb)));
      atomicAdd(md + (N + 1) + c, (double)(fk * ((1.0f - f) * vb * vb)));
      atomicAdd(md + (N + 1) + c + 1, (double)(fk * (f * vb * vb)));
    }
  } else {
    atomicAdd(&st->ctr[sp][C_LOST], 1ull);
    set_status(st, ECPIC_ERR_CAPACITY);
  }
  // ion: the product species' segment
  const int ps = SP->proc[chosen].product_seg;
  if (chk(ps >= 0 && ps < b.nseg, 18, ps, b.nseg)) {
    const int pspec = SP->proc[chosen].product_species;
    const float ivx = sd * z0;
    if (append_particle(b.segs[ps], b.sst + ps, c, f, ivx, sd * z1, sd * z2, child_id(id, k, 2), kw)) {
      if (R->scheme >= ECPIC_SCHEME_EC2)
        deposit2_one(R->S + (size_t)pspec * (N + 1), c, f, N, R->bc == ECPIC_PERIODIC);
      else
        deposit_one(R->S + (size_t)pspec * (N + 1), c, f, kw);
      if (sample) {
        double* md = R->momd + (size_t)pspec * 2 * (N + 1);
        atomicAdd(md + c, (double)(fk * ((1.0f - f) * ivx)));
        atomicAdd(md + c + 1, (double)(fk * (f * ivx)));
        atomicAdd(md + (N + 1) + c, (double)(fk * ((1.0f - f) * ivx * ivx)));
        atomicAdd(md + (N + 1) + c + 1, (double)(fk * (f * ivx * ivx)));
      }
    } else {
      atomicAdd(&st->ctr[pspec][C_LOST], 1ull);
      set_status(st, ECPIC_ERR_CAPACITY);
    }
  }
  return make_float3(v1 * d0, v1 * d1, v1 * d2);
}

// Impact tallies of an ion absorbed at x = 0 this step: energy (eV) and
// angle from the electrode normal (degrees) of the velocity that carried it
// out; the absorbed slot keeps that velocity until the next sort.
__device__ __noinline__ void tally_impact(const BatchView& b, int s, int slot, int cur, int i) {
  const SegDev& G = b.segs[s];
  const RunDev* R = b.runs + slot;
  const int sp = G.species;
  if (!chk(i >= 0 && i < G.cap, 26, i, G.cap)) return;
  const float vx = G.vx[cur][i], yz = yz2(G.vy[cur][i], G.vz[cur][i]);
  const float E = kin_eV(R->sp[sp].half_m_over_e, vx, yz);
  const float th = atan2f(sqrtf(yz), fabsf(vx)) * 57.295779513082323f;
  const unsigned long long kw = G.wt[cur] ? (unsigned long long)G.wt[cur][i] : 1ull;
  unsigned long long* tal = R->tal + (size_t)sp * R->tal_stride + R->eedf_n;
  atomicAdd(tal + tally_bin(E, R->iedf_dEinv, R->iedf_n), kw);
  atomicAdd(tal + R->iedf_n + tally_bin(th, R->iad_binv, R->iad_n), kw);
}

// A real (non-null) collision as recorded by the pass (Sec. 2a step 6):
// process, energy En and relative speed gm of the null-collision test, and
// the particle's pushed state.  Redraws Philox block A (scattering angles)
// and, for heavy species, block B (the target neutral's velocity), scatters
// and writes the new velocity.  On sample steps the pass has already added
// the pre-collision vx moments; the change is added here.
__device__ __forceinline__ void collide_real(const BatchView& b, int s, int slot, int cur,
                                             const RealRec& rec) {
  const int i = rec.i, chosen = rec.chosen;
  const float En = rec.En, gm = rec.gm;
  const SegDev& G = b.segs[s];
  const int sp = G.species;
  const RunDev* R = b.runs + slot;
  const RunState* st = b.rst + slot;
  const SpeciesDev* SP = &R->sp[sp];
  const long long k = st->step;
  const bool sample = R->sample_every > 0 && ((k + 1) % R->sample_every) == 0;
  const int N = R->N;
  const uint64_t seed = R->seed;
  if (!chk(i >= 0 && i < G.cap && chosen >= 0 && chosen < SP->nproc, 6, i, G.cap)) return;
  const int c = rec.c;
  if (!chk(c >= 0 && c < N, 7, c, N)) return;
  const float f = rec.f;
  float vx = rec.vx, vy = rec.vy, vz = rec.vz;
  const float vx_old = vx;
  const uint64_t id = rec.id;
  const uint4 A = draw(seed, id, (uint32_t)k, (uint32_t)sp << 8);
  float gx = vx, gy = vy, gz = vz, vnx = 0.f, vny = 0.f, vnz = 0.f;
  if (SP->heavy) {
    const uint4 B = draw(seed, id, (uint32_t)k, ((uint32_t)sp << 8) | 1u);
    float z0, z1, z2, z3;
    box_muller(u24_open(B.x), u24(B.y), z0, z1);
    box_muller(u24_open(B.z), u24(B.w), z2, z3);
    const float sd = R->vth_gas;
    vnx = sd * z0;
    vny = sd * z1;
    vnz = sd * z2;
    gx -= vnx;
    gy -= vny;
    gz -= vnz;
  }
  float d0, d1, d2;
  isotropic(u24(A.z), u24(A.w), d0, d1, d2);
  const int kind = SP->proc[chosen].kind;
  const float thr = SP->proc[chosen].thr;
  if (kind == ECPIC_ELASTIC) {
    const float cchi = gm > 0.0f ? (gx * d0 + gy * d1 + gz * d2) / gm : 1.0f;
    const float E1 = En * (1.0f - SP->two_m_over_M * (1.0f - cchi));
    const float v1 = sqrtf(SP->two_e_over_m * E1);
    vx = v1 * d0; vy = v1 * d1; vz = v1 * d2;
  } else if (kind == ECPIC_EXCITATION) {
    const float v1 = sqrtf(SP->two_e_over_m * (En - thr));
    vx = v1 * d0; vy = v1 * d1; vz = v1 * d2;
  } else if (kind == ECPIC_IONIZATION) {
    const float3 v1 = ionize(b, s, chosen, c, f, id, k, En - thr, sample, d0, d1, d2, rec.k);
    vx = v1.x; vy = v1.y; vz = v1.z;
  } else if (kind == ECPIC_ION_ELASTIC) {
    const float h = SP->m_frac * gm;
    vx = SP->mass_frac * vx + SP->m_frac * vnx + h * d0;
    vy = SP->mass_frac * vy + SP->m_frac * vny + h * d1;
    vz = SP->mass_frac * vz + SP->m_frac * vnz + h * d2;
  } else {  // ECPIC_CX
    vx = vnx; vy = vny; vz = vnz;
  }
  G.vx[cur][i] = vx;
  G.vy[cur][i] = vy;
  G.vz[cur][i] = vz;
  if (sample && SP->q < 0.0 && c >= R->eedf_c0 && c <= R->eedf_c1) {
    // the pass binned the pre-collision energy of this central particle
    const int b0 = tally_bin(kin_eV(SP->half_m_over_e, rec.vx, yz2(rec.vy, rec.vz)), R->eedf_dEinv, R->eedf_n);
    const int b1 = tally_bin(kin_eV(SP->half_m_over_e, vx, yz2(vy, vz)), R->eedf_dEinv, R->eedf_n);
    if (b0 != b1) {
      unsigned long long* tal = R->tal + (size_t)sp * R->tal_stride;
      atomicAdd(tal + b0, 0ull - (unsigned long long)rec.k);  // minus k, modulo 2^64
      atomicAdd(tal + b1, (unsigned long long)rec.k);
    }
  }
  if (sample) {
    double* md = R->momd + (size_t)sp * 2 * (N + 1);
    const float fk = (float)rec.k;
    const float d1v = vx - vx_old, d2v = vx * vx - vx_old * vx_old;
    atomicAdd(md + c, (double)(fk * ((1.0f - f) * d1v)));
    atomicAdd(md + c + 1, (double)(fk * (f * d1v)));
    atomicAdd(md + (N + 1) + c, (double)(fk * ((1.0f - f) * d2v)));
    atomicAdd(md + (N + 1) + c + 1, (double)(fk * (f * d2v)));
  }
}

// Segmented sums across the lanes of a warp for the sample steps' per-node
// float sums (vx moments, J.E).  Adding every particle's share to shared
// memory made a sample step's pass ten times an ordinary one: float atomics
// on shared memory retry while lanes contend, and on cell-sorted particles
// the 32 lanes of a warp add to the same few cells.  A lane whose particles
// all lie in one cell takes that cell as its key; consecutive lanes with
// equal keys form a segment, their values are summed down the segment in
// five shuffle steps, and the segment's first lane adds the sum to shared
// memory.  A lane whose particles lie in several cells (drifting electrons
// some steps after a sort) has key -1 and adds each of its runs of equal
// cells straight to the run's FP64 sums in HBM.  Called by all lanes.
__device__ __forceinline__ unsigned warp_seg_heads(int key, bool* head) {
  const int lane = threadIdx.x & 31;
  const int prev = __shfl_up_sync(0xFFFFFFFFu, key, 1);
  *head = lane == 0 || key != prev;
  return __ballot_sync(0xFFFFFFFFu, *head);
}

// On return, a segment's first lane holds the segment's sum.
__device__ __forceinline__ float warp_seg_sum(float x, unsigned heads) {
  const int lane = threadIdx.x & 31;
  const unsigned long long hb = heads;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float y = __shfl_down_sync(0xFFFFFFFFu, x, o);
    // lanes lane+1 .. lane+o start no segment: lane+o is in this one
    const unsigned long long span = ((1ull << o) - 1ull) << (lane + 1);
    if (lane + o < 32 && (hb & span) == 0ull) x += y;
  }
  return x;
}

// The key of a lane's valid entries c[j] >= 0: their common cell, -1 if they
// lie in several cells or there are none.
__device__ __forceinline__ int lane_cell_key(const int c[4]) {
  int k = -1;
  bool multi = false;
#pragma unroll
  for (int j = 0; j < 4; ++j)
    if (c[j] >= 0) {
      if (k < 0) k = c[j];
      else if (c[j] != k) multi = true;
    }
  return multi ? -1 : k;
}

// L2 prefetch of a byte range (one bulk instruction; 16-byte aligned start,
// size a multiple of 16)
__device__ __forceinline__ void l2_prefetch(const void* p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Streaming part of one piece: quads [qbeg, qend) of segment s, four
// particles per thread with 16-byte loads.  Gather (Eq. 6-7 / CIC), leapfrog
// (Eq. 8-9) in cell units, walls, the Philox candidate test, fixed-point
// deposit of X^{k+1} (Eq. 2-3).  Collision candidates (Sec. 2a step 6)
// enter a per-warp ring with their selection word and |g|^2 (or vx); the
// warp drains it 32 at a time (all lanes busy) with the null-collision test.
// The few real collisions are recorded for k_collide, which scatters them
// with its own register budget.  vy, vz are streamed when a species'
// candidate probability is 1/16 or more (its candidates then touch most
// 32-byte sectors anyway) and on energy-sample steps; otherwise the test
// reads them per candidate.
//
// Compiled five times (KIND): 0 = ordinary steps of the linear schemes (the
// common case), 1 = their energy-sample steps (moments, energy, EEDF, J.E),
// 2 = the EC2 scheme with the sample decision taken at run time, 3 and 4 =
// the linear schemes with per-particle weight multipliers (rebalancing
// runs), ordinary and sample steps.  Keeping the rare code out of the
// common instances keeps their loops small in the instruction cache and
// their registers free of the sample-step state.
template <int KIND, bool STAGE>
__device__ __forceinline__ void pass_piece(const BatchView& b, int s, long long qbeg, long long qend, int mode,
                           uint32_t* dep, float* Msm, unsigned char* ring, PassShared& sh) {
  const SegDev& G = b.segs[s];
  const int slot = G.run, sp = G.species;
  const RunDev* R = b.runs + slot;
  RunState* st = b.rst + slot;
  SegState* ss = b.sst + s;
  const int N = R->N, scheme = R->scheme, bc = R->bc, uniform = R->uniform;
  const int cur = ss->cur;
  const long long n = ss->n_proc;
  if (!chk(n <= G.cap && N <= b.nmax && (cur == 0 || cur == 1), 14, n, G.cap)) return;
  int32_t* pc = G.cell[cur];
  float* pxi = G.xi[cur];
  float* pvx = G.vx[cur];
  const float* pvy = G.vy[cur];
  const float* pvz = G.vz[cur];
  const uint64_t* pid = G.id[cur];
  const long long k = st->step;
  const bool stepping = (mode == MODE_STEP);
  constexpr bool weighted = KIND == 3 || KIND == 4;
  const uint32_t* pwt = weighted ? G.wt[cur] : nullptr;
  const bool sample = KIND == 1 || KIND == 4 ||
                      (KIND == 2 && stepping && R->sample_every > 0 &&
                       ((k + 1) % R->sample_every) == 0);
  const SpeciesDev* SP = &R->sp[sp];
  const float qm_dt = SP->qm_dt, dtdx_u = R->dtdx_u;
  // the run's field staged in shared memory for the gather (after the rings)
  float* Esm = reinterpret_cast<float*>(ring + sizeof(int) * (size_t)(3 * kRing) * (kPassBlock / 32));
  // (launches whose CTAs take only an iteration or two read the field from
  // L1/L2 instead: the staging's barrier and round trip would not pay)
  if (STAGE) {
    const int ne = (scheme == ECPIC_SCHEME_MC || scheme == ECPIC_SCHEME_MC2) ? N + 1 : N;
    for (int q = threadIdx.x; q < ne; q += kPassBlock) Esm[q] = R->E[q];
    __syncthreads();
  }
  const float* E = STAGE ? Esm : R->E;
  const uint32_t thr24 = SP->thr24;
  const bool mcc = stepping && SP->nproc > 0 && thr24 > 0;
  const bool heavy = SP->heavy != 0;
  const bool yz_stream = mcc && !heavy && thr24 >= (1u << 20);
  const bool load_yz = sample || yz_stream;
  const bool walls = bc != ECPIC_PERIODIC;
  constexpr bool order2 = KIND == 2;
  const bool eedf_on = sample && SP->q < 0.0;
  const bool imp_on = stepping && walls && SP->q > 0.0 && G.imp_cap > 0;
  const int ec0 = R->eedf_c0, ec1 = R->eedf_c1;
  unsigned long long* tal = R->tal + (size_t)sp * R->tal_stride;
  float* Psm = Msm + 2 * (b.nmax + 1);
  const uint64_t seed = R->seed;
  const int lane = threadIdx.x & 31;
  const unsigned lt_mask = (1u << lane) - 1u;

  int my_lo = INT_MAX, my_hi = -1;
  // kinetic energy of sample steps: each quad's four terms in FP32, the
  // quads summed in FP64 (one FP64 add per four particles: FP64 is slow on
  // this part), so the error per particle is a few FP32 roundings whatever
  // the number of particles a thread handles
  double ke = 0.0;
  unsigned ncand = 0, nlive = 0, nabs_l = 0, nabs_r = 0, nnan = 0, nimp_lost = 0;
  // this warp's candidate ring: index, Philox word A.y, |g|^2 or vx
  int* qi = reinterpret_cast<int*>(ring) + (threadIdx.x >> 5) * (3 * kRing);
  uint32_t* qr = reinterpret_cast<uint32_t*>(qi + kRing);
  float* qw = reinterpret_cast<float*>(qi + 2 * kRing);
  int head = 0, wcount = 0;  // warp-uniform
  uint32_t* dcnt = dep;
  uint32_t* dlo = dep + (b.nmax + 1);
  uint32_t* dhi = dep + 2 * (b.nmax + 1);
  // weighted runs: four 32-bit sums per cell (dep holds four arrays when the
  // batch has weighted runs)
  const DepW dw{dep, dep + (b.nmax + 1), dep + 2 * (b.nmax + 1), dep + 3 * (b.nmax + 1)};
  unsigned long long* Sg = R->S + (size_t)sp * (N + 1);
  int since_flush = 0;

  // block-uniform trip count (warp collectives below need full warps); the
  // pass after the last quad empties both rings
  for (long long base = qbeg;; base += kPassBlock) {
    const bool more = base < qend;
    if (more) {
      if (threadIdx.x == 0) {
        // the next iteration's particle records into L2
        const long long nb = base + kPassBlock;
        if (nb < qend) {
          const long long p0 = 4 * nb;
          long long p1 = 4 * min(qend, nb + kPassBlock);
          p1 = min(p1, n);
          if (p1 > p0) {
            const unsigned b4 = (unsigned)(((p1 - p0) * 4) & ~15ll);
            if (b4) {
              l2_prefetch(pc + p0, b4);
              l2_prefetch(pxi + p0, b4);
              l2_prefetch(pvx + p0, b4);
              if (load_yz) {
                l2_prefetch(pvy + p0, b4);
                l2_prefetch(pvz + p0, b4);
              }
              if (mcc) l2_prefetch(pid + p0, (unsigned)(((p1 - p0) * 8) & ~15ll));
              if (weighted) l2_prefetch(pwt + p0, b4);
            }
          }
        }
      }
      const long long q = base + (long long)threadIdx.x;
      const long long i0 = 4 * q;
      const bool inq = q < qend && chk(i0 < G.cap, 2, i0, G.cap);
      const bool full = inq && (i0 + 3 < n) && chk(i0 + 3 < G.cap, 3, i0 + 3, G.cap);
      int c[4];
      float f[4], v[4];
      if (full) {
        const int4 c4 = *reinterpret_cast<const int4*>(pc + i0);
        const float4 f4 = *reinterpret_cast<const float4*>(pxi + i0);
        const float4 v4 = *reinterpret_cast<const float4*>(pvx + i0);
        c[0] = c4.x; c[1] = c4.y; c[2] = c4.z; c[3] = c4.w;
        f[0] = f4.x; f[1] = f4.y; f[2] = f4.z; f[3] = f4.w;
        v[0] = v4.x; v[1] = v4.y; v[2] = v4.z; v[3] = v4.w;
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const bool in = inq && (i0 + j < n);
          c[j] = in ? pc[i0 + j] : -1;
          f[j] = in ? pxi[i0 + j] : 0.0f;
          v[j] = in ? pvx[i0 + j] : 0.0f;
        }
      }
      // weight multipliers: read here on sample steps (the moments use them),
      // else just before the deposit (a shorter live range)
      unsigned kq[4] = {1u, 1u, 1u, 1u};
      if (weighted && sample) {
        if (full) {
          const uint4 k4 = *reinterpret_cast<const uint4*>(pwt + i0);
          kq[0] = k4.x; kq[1] = k4.y; kq[2] = k4.z; kq[3] = k4.w;
        } else {
#pragma unroll
          for (int j = 0; j < 4; ++j) kq[j] = (inq && i0 + j < n) ? pwt[i0 + j] : 1u;
        }
      }
      bool cand[4] = {false, false, false, false};
      bool hit[4] = {false, false, false, false};  // absorbed at x = 0 (impact tallies)
#pragma unroll
      for (int j = 0; j < 4; ++j) nlive += c[j] >= 0 ? 1u : 0u;
      if (stepping) {
        uint64_t id[4] = {0, 0, 0, 0};
        if (mcc) {
          if (full) {
            const ulonglong2 a = *reinterpret_cast<const ulonglong2*>(pid + i0);
            const ulonglong2 bq = *reinterpret_cast<const ulonglong2*>(pid + i0 + 2);
            id[0] = a.x; id[1] = a.y; id[2] = bq.x; id[3] = bq.y;
          } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) id[j] = c[j] >= 0 ? pid[i0 + j] : 0ull;
          }
        }
        // vy^2 + vz^2 (collisions do not change it before the push reads it)
        float yz[4] = {0.f, 0.f, 0.f, 0.f};
        if (load_yz) {
          if (full) {
            const float4 y4 = *reinterpret_cast<const float4*>(pvy + i0);
            const float4 z4 = *reinterpret_cast<const float4*>(pvz + i0);
            yz[0] = yz2(y4.x, z4.x);
            yz[1] = yz2(y4.y, z4.y);
            yz[2] = yz2(y4.z, z4.z);
            yz[3] = yz2(y4.w, z4.w);
          } else {
#pragma unroll
            for (int j = 0; j < 4; ++j)
              if (c[j] >= 0) yz[j] = yz2(pvy[i0 + j], pvz[i0 + j]);
          }
        }
        // gather (Eq. 6-7; CIC for MC) and push (Eq. 8), branch-free over the
        // four particles so the loads and arithmetic overlap
        float Ei[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const bool ok = c[j] >= 0 && chk(c[j] < N, 4, c[j], N);
          if (!ok) c[j] = -1;
          const int cc = ok ? c[j] : 0;
          if (scheme == ECPIC_SCHEME_EC) {
            Ei[j] = E[cc];
          } else if (order2 && scheme == ECPIC_SCHEME_MC2) {
            // the deposit's quadratic weights on the centred node field (its
            // transpose: folded and wrapped nodes read their field)
            const bool up = f[j] >= 0.5f;
            const int n0 = cc + (up ? 1 : 0);
            const float u = up ? f[j] - 1.0f : f[j];
            const float wl = 0.5f * (0.5f - u) * (0.5f - u), wr = 0.5f * (0.5f + u) * (0.5f + u);
            Ei[j] = wl * E[node2(n0 - 1, N, !walls)] + (0.75f - u * u) * E[n0] +
                    wr * E[node2(n0 + 1, N, !walls)];
          } else if (order2) {
            // linear between the faces about the nearest node n0 (faces
            // n0-1 and n0): the derivative of the quadratic-spline potential
            const bool up = f[j] >= 0.5f;
            const int n0 = cc + (up ? 1 : 0);
            const float u = up ? f[j] - 1.0f : f[j];
            float El, Er;
            if (walls) {
              El = n0 >= 1 ? E[n0 - 1] : 0.0f;
              Er = n0 < N ? E[n0] : 0.0f;
            } else {
              El = E[n0 >= 1 ? n0 - 1 : N - 1];
              Er = E[n0 < N ? n0 : 0];
            }
            Ei[j] = (0.5f - u) * El + (0.5f + u) * Er;
          } else {
            const float e0 = E[cc], e1 = E[cc + 1];
            Ei[j] = e0 + f[j] * (e1 - e0);
          }
        }
        float keq = 0.0f;
        float pje[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float vnew = v[j] + qm_dt * Ei[j];
          if (sample) {
            const float fk = weighted ? (float)kq[j] : 1.0f;
            if (c[j] >= 0) keq += fk * (v[j] * vnew + yz[j]);
            // J.E of the push, per cell at level k (scaled by q w / 2 dx later)
            pje[j] = c[j] >= 0 ? fk * ((v[j] + vnew) * Ei[j]) : 0.0f;
          }
          v[j] = vnew;
        }
        if (sample) {
          ke += (double)keq;
          // J.E per cell of level k: per lane, then down each segment
          const int key = lane_cell_key(c);
          float pl = 0.0f;
          int cc = -1;
          double* pwg = R->pw + (size_t)sp * N;
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            if (c[j] < 0) continue;
            if (key < 0 && c[j] != cc) {
              if (cc >= 0) atomicAdd(pwg + cc, (double)pl);
              cc = c[j];
              pl = 0.0f;
            }
            pl += pje[j];
          }
          if (key < 0 && cc >= 0) {
            atomicAdd(pwg + cc, (double)pl);
            pl = 0.0f;
          }
          bool head;
          const unsigned heads = warp_seg_heads(key, &head);
          pl = warp_seg_sum(pl, heads);
          if (head && key >= 0) atomicAdd(Psm + key, pl);
        }
        // Philox block A of all four: independent chains the scheduler
        // interleaves; A.x decides the candidate, A.y selects the process
        uint32_t r0[4] = {0u, 0u, 0u, 0u}, ry[4] = {0u, 0u, 0u, 0u};
        if (mcc) {
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const uint4 A = draw(seed, id[j], (uint32_t)k, (uint32_t)sp << 8);
            r0[j] = A.x;
            ry[j] = A.y;
          }
        }
        // Eq. 9 in cell units, then the walls: absorbed when X <= 0 or X >= L
        if (uniform) {
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const bool live = c[j] >= 0;
            const bool bad = live && !(fabsf(v[j]) < 3.0e8f);
            float g = f[j] + v[j] * dtdx_u;
            const float fl = floorf(g);
            int cj = c[j] + (int)fl;
            g -= fl;
            const bool up = g >= 1.0f;  // g - floor(g) rounded to 1
            cj += up ? 1 : 0;
            g = up ? 0.0f : g;
            if (!walls && (cj < 0 || cj >= N)) {
              cj %= N;
              if (cj < 0) cj += N;
            }
            const bool out = walls && (cj < 0 || cj >= N || (cj == 0 && g == 0.0f));
            const bool ok = live && !bad && !out;
            nnan += bad ? 1u : 0u;
            nabs_r += (live && !bad && out && cj >= N) ? 1u : 0u;
            nabs_l += (live && !bad && out && cj < N) ? 1u : 0u;
            hit[j] = imp_on && live && !bad && out && cj < N;
            c[j] = ok ? cj : -1;
            f[j] = g;
            cand[j] = mcc && ok && (r0[j] >> 8) < thr24;
          }
        } else {
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            if (c[j] < 0) continue;
            if (!(fabsf(v[j]) < 3.0e8f)) {
              ++nnan;
              c[j] = -1;
              continue;
            }
            int cj = c[j];
            float fj = f[j];
            walk_nonuniform(cj, fj, fj + v[j] * __ldg(R->dtdx + cj), N, bc, R->rp, R->rm);
            if (walls && (cj < 0 || cj >= N || (cj == 0 && fj == 0.0f))) {
              nabs_r += cj >= N ? 1u : 0u;
              nabs_l += cj >= N ? 0u : 1u;
              hit[j] = imp_on && cj < N;
              c[j] = -1;
              continue;
            }
            c[j] = cj;
            f[j] = fj;
            cand[j] = mcc && (r0[j] >> 8) < thr24;
          }
        }
        if (full) {
          *reinterpret_cast<int4*>(pc + i0) = make_int4(c[0], c[1], c[2], c[3]);
          *reinterpret_cast<float4*>(pxi + i0) = make_float4(f[0], f[1], f[2], f[3]);
          *reinterpret_cast<float4*>(pvx + i0) = make_float4(v[0], v[1], v[2], v[3]);
        } else {
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (inq && i0 + j < n) {
              pc[i0 + j] = c[j];
              pxi[i0 + j] = f[j];
              pvx[i0 + j] = v[j];
            }
        }
        // ions absorbed at x = 0: their indices, for the impact tallies of the
        // collision kernel (the absorbed slot keeps its velocity until the sort)
        if (imp_on && __any_sync(kFull, hit[0] || hit[1] || hit[2] || hit[3])) {
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const unsigned m = __ballot_sync(kFull, hit[j]);
            if (m) {
              const int lead = __ffs(m) - 1;
              unsigned long long base = 0ull;
              if (lane == lead) base = atomicAdd((unsigned long long*)&ss->n_imp, (unsigned long long)__popc(m));
              base = __shfl_sync(kFull, base, lead);
              if (hit[j]) {
                const long long idx = (long long)base + __popc(m & lt_mask);
                if (idx < G.imp_cap) G.imp[idx] = (int)(i0 + j);
                else ++nimp_lost;
              }
            }
          }
        }
        // EEDF of the central cells on sample steps (pre-collision; the
        // collision kernel moves the particles that collide)
        if (eedf_on) {
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (c[j] >= ec0 && c[j] <= ec1)
              atomicAdd(tal + tally_bin(kin_eV(SP->half_m_over_e, v[j], yz[j]), R->eedf_dEinv, R->eedf_n),
                        (unsigned long long)kq[j]);
        }
        if (mcc) {
          // a candidate with Rr >= nu_bnd |g| is a null collision whatever its
          // energy (the total rate never exceeds nu_bnd |g|): where |g| is at
          // hand, only the others go on to the cross-section test
          const float nu_max = SP->nu_max, nu_bnd = SP->nu_bnd;
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const bool test = cand[j] && (!yz_stream ||
                u24(ry[j]) * nu_max < nu_bnd * sqrtf(v[j] * v[j] + yz[j]));
            ncand += cand[j] ? 1u : 0u;
            cand[j] = test;
          }
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const unsigned m = __ballot_sync(kFull, cand[j]);
            if (cand[j]) {
              int pos = head + wcount + __popc(m & lt_mask);
              if (pos >= kRing) pos -= kRing;
              if (chk(pos >= 0 && pos < kRing, 5, pos, kRing)) {
                qi[pos] = (int)(i0 + j);
                qr[pos] = ry[j];
                qw[pos] = yz_stream ? v[j] * v[j] + yz[j] : v[j];
              }
            }
            wcount += __popc(m);
          }
        }
      }
      // fixed-point CIC deposit of the new positions (Eq. 2-3); vx moments
      // (pre-collision: the collision adds the change)
      if (order2)
        dep2_add4(dlo, dhi, N, !walls, c, f);
      else if (weighted) {
        if (!sample) {
          if (full) {
            const uint4 k4 = *reinterpret_cast<const uint4*>(pwt + i0);
            kq[0] = k4.x; kq[1] = k4.y; kq[2] = k4.z; kq[3] = k4.w;
          } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) kq[j] = (inq && i0 + j < n) ? pwt[i0 + j] : 1u;
          }
        }
        depw_add4(dw, c, f, kq);
      }
      else
        dep_add4(dcnt, dlo, dhi, c, f);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (c[j] >= 0) {
          my_lo = min(my_lo, c[j]);
          my_hi = max(my_hi, c[j] + 1);
        }
      }
      if (sample) {
        // vx moments at the nodes of the new cell (CIC shares): per lane
        // summed where its particles share a cell, then down each segment
        const int Nm = b.nmax + 1;
        int cm[4];
#pragma unroll
        for (int j = 0; j < 4; ++j)
          cm[j] = (c[j] >= 0 && chk(c[j] + 1 <= b.nmax, 20, c[j], b.nmax)) ? c[j] : -1;
        const int key = lane_cell_key(cm);
        float a1 = 0.0f, b1 = 0.0f, a2 = 0.0f, b2 = 0.0f;
        int cc = -1;  // spread lanes: the current run of equal cells
        double* mdg = R->momd + (size_t)sp * 2 * (N + 1);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          if (cm[j] < 0) continue;
          const float fk = weighted ? (float)kq[j] : 1.0f;
          const float lo = fk * ((1.0f - f[j]) * v[j]), hi = fk * (f[j] * v[j]);
          if (key < 0 && cm[j] != cc) {
            // spread over cells: each run of equal cells straight to the
            // run's FP64 sums in HBM
            if (cc >= 0) {
              atomicAdd(mdg + cc, (double)a1);
              atomicAdd(mdg + cc + 1, (double)b1);
              atomicAdd(mdg + (N + 1) + cc, (double)a2);
              atomicAdd(mdg + (N + 1) + cc + 1, (double)b2);
            }
            cc = cm[j];
            a1 = b1 = a2 = b2 = 0.0f;
          }
          a1 += lo;
          b1 += hi;
          a2 += lo * v[j];
          b2 += hi * v[j];
        }
        if (key < 0 && cc >= 0) {
          atomicAdd(mdg + cc, (double)a1);
          atomicAdd(mdg + cc + 1, (double)b1);
          atomicAdd(mdg + (N + 1) + cc, (double)a2);
          atomicAdd(mdg + (N + 1) + cc + 1, (double)b2);
          a1 = b1 = a2 = b2 = 0.0f;
        }
        bool head;
        const unsigned heads = warp_seg_heads(key, &head);
        a1 = warp_seg_sum(a1, heads);
        b1 = warp_seg_sum(b1, heads);
        a2 = warp_seg_sum(a2, heads);
        b2 = warp_seg_sum(b2, heads);
        if (head && key >= 0) {
          atomicAdd(Msm + key, a1);
          atomicAdd(Msm + key + 1, b1);
          atomicAdd(Msm + Nm + key, a2);
          atomicAdd(Msm + Nm + key + 1, b2);
        }
      }
    }
    if (mcc) {
      __syncwarp();
      while (wcount >= 32 || (!more && wcount > 0)) {
        // null-collision test of up to 32 candidates
        const int take = min(wcount, 32);
        const bool act = lane < take;
        int pos = head + lane;
        if (pos >= kRing) pos -= kRing;
        int i = 0;
        uint32_t ryv = 0u;
        float w = 0.0f;
        if (act) {
          i = qi[pos];
          ryv = qr[pos];
          w = qw[pos];
        }
        float g2 = w;
        if (heavy) {
          // relative speed to a target neutral drawn from the gas Maxwellian
          if (act) {
            const float vx = pvx[i], vy = pvy[i], vz = pvz[i];
            const uint4 B = draw(seed, pid[i], (uint32_t)k, ((uint32_t)sp << 8) | 1u);
            float z0, z1, z2, z3;
            box_muller(u24_open(B.x), u24(B.y), z0, z1);
            box_muller(u24_open(B.z), u24(B.w), z2, z3);
            const float sd = R->vth_gas;
            const float gx = vx - sd * z0, gy = vy - sd * z1, gz = vz - sd * z2;
            g2 = gx * gx + gy * gy + gz * gz;
          }
        } else if (!yz_stream) {
          if (act) {
            const float vy = pvy[i], vz = pvz[i];
            g2 = w * w + (vy * vy + vz * vz);
          }
        }
        const float gm = sqrtf(g2), En = SP->half_m_over_e * g2;
        const float nu_max = SP->nu_max;
        const float Rr = u24(ryv) * nu_max;
        float tot = 0.0f;
        int chosen = -1;
        if (act && Rr < SP->nu_bnd * gm) chosen = select_process(SP, En, gm, R->ng, Rr, &tot);
        if (tot > nu_max) atomicAdd(&sh.ctr[C_CLAMPS], 1ull);
        // real collisions: a record each, with the particle's pushed state
        // (still in L1/L2 here), for the collision kernel
        const unsigned m = __ballot_sync(kFull, chosen >= 0);
        if (m) {
          const int lead = __ffs(m) - 1;
          unsigned long long base = 0ull;
          if (lane == lead) base = atomicAdd((unsigned long long*)&ss->n_real, (unsigned long long)__popc(m));
          base = __shfl_sync(kFull, base, lead);
          if (chosen >= 0) {
            const long long idx = (long long)base + __popc(m & lt_mask);
            if (idx < G.real_cap) {
              const uint64_t id = pid[i];
              int4* dst = reinterpret_cast<int4*>(G.real + idx);  // RealRec field order
              dst[0] = make_int4((int)(uint32_t)id, (int)(uint32_t)(id >> 32), i, chosen);
              dst[1] = make_int4(__float_as_int(En), __float_as_int(gm), __float_as_int(pvx[i]),
                                 __float_as_int(pvy[i]));
              dst[2] = make_int4(__float_as_int(pvz[i]), pc[i], __float_as_int(pxi[i]),
                                 weighted ? (int)pwt[i] : 1);
            } else {
              set_status(st, ECPIC_ERR_CAPACITY);
            }
          }
        }
        head += take;
        if (head >= kRing) head -= kRing;
        wcount -= take;
        __syncwarp();
      }
    }
    if (!more) break;
    if (++since_flush == (order2 ? kFlushIters / 4 : weighted ? kFlushIters / 2 : kFlushIters)) {
      __syncthreads();
      if (order2)
        dep2_flush(dlo, dhi, 0, N, Sg);
      else if (weighted)
        depw_flush(dw, 0, N, Sg);
      else
        dep_flush(dcnt, dlo, dhi, 0, N, Sg);
      __syncthreads();
      since_flush = 0;
    }
  }

  // piece epilogue: node range, energy, counters, flush to HBM
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    my_lo = min(my_lo, __shfl_xor_sync(kFull, my_lo, o));
    my_hi = max(my_hi, __shfl_xor_sync(kFull, my_hi, o));
  }
  ncand = warp_sum(ncand);
  nlive = warp_sum(nlive);
  nabs_l = warp_sum(nabs_l);
  nabs_r = warp_sum(nabs_r);
  nnan = warp_sum(nnan);
  nimp_lost = warp_sum(nimp_lost);
  if (lane == 0 && stepping && nlive) atomicAdd(&st->psteps, (unsigned long long)nlive);
  if (lane == 0) {
    if (my_hi >= 0) {
      atomicMin(&sh.lohi[0], my_lo);
      atomicMax(&sh.lohi[1], my_hi);
    }
    if (ncand) atomicAdd(&sh.ctr[C_CAND], (unsigned long long)ncand);
    if (nabs_l) atomicAdd(&sh.ctr[C_ABS_L], (unsigned long long)nabs_l);
    if (nabs_r) atomicAdd(&sh.ctr[C_ABS_R], (unsigned long long)nabs_r);
    if (nimp_lost) atomicAdd(&sh.ctr[C_IMP_LOST], (unsigned long long)nimp_lost);
    if (nnan) {
      atomicAdd(&sh.ctr[C_NAN], (unsigned long long)nnan);
      set_status(st, ECPIC_ERR_NAN);
    }
  }
  if (sample) {
    const double kes = block_sum(ke, sh.dsm);
    if (threadIdx.x == 0) atomicAdd(&st->ke_acc[sp], 0.5 * SP->m * SP->w * kes);
  }
  __syncthreads();
  const int flo = sh.lohi[0], fhi = chk(sh.lohi[1] <= N, 8, sh.lohi[1], N) ? sh.lohi[1] : N;
  const int Nm = b.nmax + 1;
  double* md = R->momd + (size_t)sp * 2 * (N + 1);
  // an empty range (no live particle in the piece) is (INT_MAX, -1): skip it
  // before forming flo + threadIdx.x, which would overflow
  if (flo < fhi) {
    if (order2)  // shares reach one node beyond the range, or wrap
      dep2_flush(dlo, dhi, walls ? max(flo - 1, 0) : 0, walls ? min(fhi + 1, N) : N, Sg);
    else if (weighted)
      depw_flush(dw, flo, fhi, Sg);
    else
      dep_flush(dcnt, dlo, dhi, flo, fhi, Sg);
  }
  const int nbeg = flo <= fhi ? flo + (int)threadIdx.x : fhi + 1;
  if (sample) {
    double* pwg = R->pw + (size_t)sp * N;
    for (int j = threadIdx.x; j < N; j += kPassBlock) {
      const float pj = Psm[j];
      if (pj != 0.0f) {
        atomicAdd(pwg + j, (double)pj);
        Psm[j] = 0.0f;
      }
    }
  }
  for (int nn = nbeg; nn <= fhi && sample; nn += kPassBlock) {
    const float m1 = Msm[nn], m2 = Msm[Nm + nn];
    if (m1 != 0.0f) atomicAdd(md + nn, (double)m1);
    if (m2 != 0.0f) atomicAdd(md + (N + 1) + nn, (double)m2);
    Msm[nn] = 0.0f;
    Msm[Nm + nn] = 0.0f;
  }
  if (threadIdx.x == 0) {
    const unsigned long long dead = sh.ctr[C_ABS_L] + sh.ctr[C_ABS_R] + sh.ctr[C_NAN];
    if (dead) atomicAdd((unsigned long long*)&ss->n_dead, dead);
  }
  __syncthreads();
  if (threadIdx.x < kNumCtr) {
    const unsigned long long val = sh.ctr[threadIdx.x];
    if (val) {
      atomicAdd(&st->ctr[sp][threadIdx.x], val);
      sh.ctr[threadIdx.x] = 0ull;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    sh.lohi[0] = INT_MAX;
    sh.lohi[1] = -1;
  }
  __syncthreads();
}

// WEIGHTED: the batch holds rebalancing runs (weight multipliers).  Their
// instance of the pass is compiled into a kernel of its own so that the
// kernel of unweighted batches keeps its register allocation.
template <bool STAGE, bool WEIGHTED>
__global__ void __launch_bounds__(kPassBlock, 4) k_pass(BatchView b, int mode, int only) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  long long* pre = reinterpret_cast<long long*>(smem_raw);
  // deposit sums, 3 (nmax+1): count, lo, hi (linear); -, lo, hi per node (EC2);
  // four when the batch has weighted runs
  uint32_t* dep = reinterpret_cast<uint32_t*>(pre + b.nseg + 1);
  const int ndep = b.weighted ? 4 : 3;
  float* Msm = reinterpret_cast<float*>(dep + ndep * (b.nmax + 1));
  unsigned char* ring = reinterpret_cast<unsigned char*>(Msm + 3 * (b.nmax + 1));  // Msm: M1 | M2 | J.E
  __shared__ PassShared sh;
  for (int i = threadIdx.x; i <= b.nmax; i += kPassBlock) {
    for (int q = 0; q < ndep; ++q) dep[q * (b.nmax + 1) + i] = 0u;
    Msm[i] = 0.0f;
    Msm[b.nmax + 1 + i] = 0.0f;
    Msm[2 * (b.nmax + 1) + i] = 0.0f;
  }
  if (threadIdx.x < kNumCtr) sh.ctr[threadIdx.x] = 0ull;
  if (threadIdx.x == 0) {
    sh.lohi[0] = INT_MAX;
    sh.lohi[1] = -1;
    sh.qcount = 0;
  }
  // the work is split in quads of particles, equal quads per CTA
  const long long T = seg_prefix(b, mode, only, pre, sh.wsm, 4);
  if (T == 0) return;
  const long long lo = T * (long long)blockIdx.x / gridDim.x;
  const long long hi = T * (long long)(blockIdx.x + 1) / gridDim.x;
  if (lo >= hi) return;
  for (int s = seg_find(pre, b.nseg, lo); s < b.nseg && pre[s] < hi; ++s) {
    const long long beg = max(lo, pre[s]) - pre[s];
    const long long end = min(hi, pre[s + 1]) - pre[s];
    if (beg >= end) continue;
    if (!chk(b.segs[s].run >= 0 && b.segs[s].run < b.max_slots, 23, s, b.nseg)) continue;
    // which instance: a sampled step of a stepping pass
    const SegDev& G = b.segs[s];
    const RunDev& R = b.runs[G.run];
    const bool stepping = mode == MODE_STEP;
    const long long k = b.rst[G.run].step;
    const bool smp = stepping && R.sample_every > 0 && ((k + 1) % R.sample_every) == 0;
    if (R.scheme >= ECPIC_SCHEME_EC2)  // EC2, MC2
      pass_piece<2, STAGE>(b, s, beg, end, mode, dep, Msm, ring, sh);
    else if (WEIGHTED && R.rb && smp)  // weight multipliers
      pass_piece<WEIGHTED ? 4 : 1, STAGE>(b, s, beg, end, mode, dep, Msm, ring, sh);
    else if (WEIGHTED && R.rb)
      pass_piece<WEIGHTED ? 3 : 0, STAGE>(b, s, beg, end, mode, dep, Msm, ring, sh);
    else if (smp)
      pass_piece<1, STAGE>(b, s, beg, end, mode, dep, Msm, ring, sh);
    else
      pass_piece<0, STAGE>(b, s, beg, end, mode, dep, Msm, ring, sh);
  }
}

// Real collisions recorded by this step's pass, then its impact records,
// all segments, equal records per warp.  Process counters are summed over the lanes that share a
// (segment, process) before one atomic each.
__global__ void __launch_bounds__(kCollideBlock) k_collide(BatchView b) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  long long* pre = reinterpret_cast<long long*>(smem_raw);
  int* meta = reinterpret_cast<int*>(pre + b.nseg + 1);  // slot, buffer, reals per segment
  __shared__ long long wsm[32];
  const long long T = seg_prefix(b, MODE_STEP, -1, pre, wsm, 1, true, meta);
  const int lane = threadIdx.x & 31;
  const long long stride = (long long)gridDim.x * kCollideBlock;
  for (long long w0 = (long long)blockIdx.x * kCollideBlock + (threadIdx.x & ~31); w0 < T; w0 += stride) {
    const long long r = w0 + lane;
    const bool valid = r < T;
    int s = 0, slot = 0, cur = 0;
    RealRec rec;
    rec.chosen = -1;
    int imp_i = -1;  // an impact record instead: the absorbed ion's index
    if (valid) {
      s = seg_find(pre, b.nseg, r);
      slot = meta[3 * s];
      cur = meta[3 * s + 1];
      const long long j = r - pre[s];
      const long long nr = meta[3 * s + 2];
      if (j >= nr) {
        const long long ii = j - nr;
        if (ii < b.segs[s].imp_cap) imp_i = b.segs[s].imp[ii];
      } else if (chk(j >= 0 && j < b.segs[s].real_cap, 25, j, b.segs[s].real_cap)) {
        const int4* src = reinterpret_cast<const int4*>(b.segs[s].real + j);  // RealRec field order
        const int4 w0 = src[0], w1 = src[1], w2 = src[2];
        rec.id = (uint64_t)(uint32_t)w0.x | ((uint64_t)(uint32_t)w0.y << 32);
        rec.i = w0.z;
        rec.chosen = w0.w;
        rec.En = __int_as_float(w1.x);
        rec.gm = __int_as_float(w1.y);
        rec.vx = __int_as_float(w1.z);
        rec.vy = __int_as_float(w1.w);
        rec.vz = __int_as_float(w2.x);
        rec.c = w2.y;
        rec.f = __int_as_float(w2.z);
        rec.k = (unsigned)w2.w;
      }
    }
    const bool ok = valid && rec.chosen >= 0 && rec.chosen < kMaxProc;
    const unsigned key = ok ? ((unsigned)s << 4) | (unsigned)rec.chosen : 0xFFFFFFFFu;
    const unsigned grp = __match_any_sync(kFull, key);
    if (ok && lane == __ffs(grp) - 1) {
      const SegDev& G = b.segs[s];
      atomicAdd(&b.rst[slot].ctr[G.species][C_COLL0 + rec.chosen], (unsigned long long)__popc(grp));
    }
    if (ok) collide_real(b, s, slot, cur, rec);
    if (imp_i >= 0) tally_impact(b, s, slot, cur, imp_i);
  }
}

// ----------------------------------------------------------------- field
// 1/D in FP64 from an FP32 seed and two Newton steps (no FP64 division,
// which is slow on this part); D > 0.
__device__ __forceinline__ double recip(double D) {
  double r = (double)__frcp_rn((float)D);
  r = r * (2.0 - D * r);
  r = r * (2.0 - D * r);
  return r;
}

// Poisson (Eq. 4 in finite-volume form) solved through Gauss's law: with
// g_n = (phi_{n+1}-phi_n)/dx_n, Eq. 4 reads g_n - g_{n-1} = -Q_n/eps0, so
// g_n = g_0 - C_n/eps0 with C_n = sum_{m=1..n} Q_m, and the boundary values
// fix g_0 = (phi_N - phi_0 + sum_n dx_n C_n / eps0) / L.  This is the exact
// solution of the same tridiagonal system that a Thomas sweep solves.  The
// prefix sums of the fixed-point deposit are taken in 64-bit integers (exact),
// so FP64 enters only once per node.  EC field E_j = -g_j (Eq. 5).
// One CTA per run; each thread owns a run of consecutive nodes and all
// species are scanned together, so that a step costs a few barriers and
// global round trips (FP64 is slow on this part: the node loop keeps its
// FP64 operations few).  The potential and the field energy are formed only
// on the steps that sample them (and on refresh).
__global__ void __launch_bounds__(kFieldBlock, 2) k_field(BatchView b, int advance, int only) {
  const int slot = blockIdx.x;
  if (slot >= b.max_slots) return;
  const RunDev* R = b.runs + slot;
  RunState* st = b.rst + slot;
  // every scalar this kernel needs, loaded before the first branch so that
  // the loads travel together
  const int active = R->active;
  const int status0 = st->status;
  const int fresh = st->fresh;
  const long long step0 = st->step, step_end = st->step_end;
  const int N = R->N, ns = R->ns, seg0 = R->seg0;
  const int se = R->sample_every;
  const bool periodic = (R->bc == ECPIC_PERIODIC);
  const bool face = R->scheme == ECPIC_SCHEME_EC || R->scheme == ECPIC_SCHEME_EC2;
  const double* dx = R->dx;
  unsigned long long* Sall = R->S;
  const double inv_L = R->inv_L;
  const int field_pm = R->field_pm, field_neg = R->field_neg;
  if (!active) return;
  if (advance) {
    if (status0 != 0 || step0 >= step_end) return;
  } else if ((only >= 0 && slot != only) || (only == kOnlyFresh && !fresh)) {
    return;
  }
  if (only == kOnlyFresh) {
    __syncthreads();  // every thread has read the flag
    if (threadIdx.x == 0) st->fresh = 0;
  }
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* C = reinterpret_cast<double*>(smem_raw);  // N+1
  __shared__ double dsm[32];
  __shared__ unsigned long long wtot[kFieldBlock / 32][kMaxSpecies];
  __shared__ double phi0_sh;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const long long kn = advance ? step0 + 1 : step0;
  const bool sample = advance && se > 0 && (kn % se) == 0;
  // the push of level kn samples the energy when (kn + 1) % se == 0
  const bool want_fe = !advance || (se > 0 && ((kn + 1) % se) == 0);
  const bool want_phi = !advance || sample;
  constexpr double kInvEps0 = 1.0 / kEps0;
  constexpr double kInvQe = 1.0 / 1.602176634e-19;
  constexpr double k2m32 = 2.3283064365386963e-10;  // 2^-32
  // the charge of one deposit share per species (q w 2^-32, formed on the
  // host: FP64 is slow on this part, and every thread would repeat it)
  double cw[kMaxSpecies];
#pragma unroll
  for (int s = 0; s < kMaxSpecies; ++s) cw[s] = s < ns ? R->sp[s].cw : 0.0;
  // this thread's segment (species tid), for the size update at the end;
  // nothing changes the sizes while this kernel runs
  SegState* my_ss = nullptr;
  long long my_cap = 0, my_alloc = 0;
  if (advance && tid < ns) {
    const int sg = seg0 + tid;
    my_ss = b.sst + sg;
    my_cap = b.segs[sg].cap;
    my_alloc = my_ss->n_alloc;
  }

  if (tid == kFieldBlock - 1) {
    double p0 = 0.0;
    if (!periodic) {
      const double t = (double)kn * R->dt;
      const double arg = __dadd_rn(__dmul_rn(__dmul_rn(kTwoPi, R->freq), t), R->phase);
      p0 = R->vdc + R->v0 * sin(arg);
    }
    phi0_sh = p0;
  }

  // sampled moments (Sec. 3a: density and x temperature per node)
  if (sample) {
    double* acc = R->acc;
    for (int n = tid; n <= N; n += kFieldBlock) {
      for (int s = 0; s < ns; ++s) {
        const unsigned long long* S = Sall + (size_t)s * (N + 1);
        const double* md = R->momd + (size_t)s * 2 * (N + 1);
        double D, M1, M2;
        if (periodic && (n == 0 || n == N)) {
          D = (double)(S[0] + S[N]);
          M1 = md[0] + md[N];
          M2 = md[N + 1] + md[N + 1 + N];
        } else {
          D = (double)S[n];
          M1 = md[n];
          M2 = md[N + 1 + n];
        }
        D *= k2m32;
        double T = 0.0;
        if (D > 0.0) {
          const double iD = recip(D);
          const double a = M1 * iD;
          T = R->sp[s].m * (M2 * iD - a * a) * kInvQe;
        }
        acc[(size_t)s * (N + 1) + n] += R->sp[s].w * D * R->invV[n];
        acc[(size_t)(ns + s) * (N + 1) + n] += T;
        acc[(size_t)(2 * ns + s) * (N + 1) + n] += D;
        acc[(size_t)(3 * ns + s) * (N + 1) + n] += M1;
        acc[(size_t)(4 * ns + s) * (N + 1) + n] += M2;
      }
    }
    __syncthreads();
    for (int n = tid; n <= N; n += kFieldBlock)
      for (int s = 0; s < ns; ++s) {
        double* md = R->momd + (size_t)s * 2 * (N + 1);
        md[n] = 0.0;
        md[N + 1 + n] = 0.0;
      }
  }

  // C_n = sum_s q_s w_s 2^-32 * sum_{m=1..n} S_s,m, the integer prefix exact:
  // thread t owns nodes [beg, end); one block scan for all species
  const int per = (N + 1 + kFieldBlock - 1) / kFieldBlock;
  const int beg = min(N + 1, tid * per), end = min(N + 1, beg + per);
  unsigned long long run[kMaxSpecies], s0[kMaxSpecies];
#pragma unroll
  for (int s = 0; s < kMaxSpecies; ++s) {
    run[s] = 0ull;
    s0[s] = 0ull;
    if (s < ns) {
      const unsigned long long* S = Sall + (size_t)s * (N + 1);
      unsigned long long loc = 0ull;
      for (int n = max(beg, 1); n < end; ++n) loc += S[n];
      s0[s] = S[0];  // node 0 only enters the total
      const unsigned long long inc = warp_incl_scan(loc);
      if (lane == 31) wtot[w][s] = inc;
      run[s] = inc - loc;
    }
  }
  __syncthreads();
  // Species whose weights q_s w_s are all equal up to sign (electrons and an
  // ion species of the same weight) take the signed integer sum of their
  // prefixes first, so that one conversion to FP64 per node serves them all:
  // C_n = cs * C'_n with cs = 2^-32 q_0 w_0 and C'_n that integer.  The sum is
  // exact while the species' totals stay below 2^63 together.
  unsigned long long tot[kMaxSpecies];
  bool pm = field_pm != 0;
  unsigned long long sum_tot = 0ull;
#pragma unroll
  for (int s = 0; s < kMaxSpecies; ++s) {
    tot[s] = 0ull;
    if (s < ns) {
      unsigned long long off = 0ull, t = 0ull;
#pragma unroll
      for (int q = 0; q < kFieldBlock / 32; ++q) {
        const unsigned long long v = wtot[q][s];
        off += q < w ? v : 0ull;
        t += v;
      }
      run[s] += off;
      tot[s] = t + s0[s];
      pm = pm && tot[s] < (1ull << 62);
      sum_tot += tot[s] >> 2;
    }
  }
  pm = pm && sum_tot < (1ull << 61) - 4ull;
  const double cs = pm ? cw[0] : 1.0;
  // total charge (in units of cs) for the uniform neutralising background of
  // a periodic system: Q_n -= V_n Qtot / L
  double qtot = 0.0;
  if (pm) {
    unsigned long long qi = 0ull;
#pragma unroll
    for (int s = 0; s < kMaxSpecies; ++s)
      if (s < ns) qi += ((field_neg >> s) & 1) ? 0ull - tot[s] : tot[s];
    qtot = (double)(long long)qi;
  } else {
#pragma unroll
    for (int s = 0; s < kMaxSpecies; ++s)
      if (s < ns) qtot += cw[s] * (double)tot[s];
  }
  const double a = periodic ? qtot * inv_L : 0.0;
  double loc = 0.0;
  for (int n = beg; n < end; ++n) {
    double c = 0.0;
    unsigned long long qi = 0ull;
#pragma unroll
    for (int s = 0; s < kMaxSpecies; ++s) {
      if (s < ns) {
        unsigned long long* S = Sall + (size_t)s * (N + 1);
        if (n > 0) run[s] += S[n];
        S[n] = 0ull;
        if (pm)
          qi += ((field_neg >> s) & 1) ? 0ull - run[s] : run[s];
        else
          c += cw[s] * (double)run[s];
      }
    }
    if (pm) c = (double)(long long)qi;
    if (n < N) {
      if (periodic) c -= a * R->cumV[n];
      C[n] = c;
      loc += dx[n] * c;
    }
  }
  const double A = cs * block_sum(loc, dsm);
  const double phi0 = phi0_sh;
  const double g0 = (A * kInvEps0 - phi0) * inv_L;
  const double kc = cs * kInvEps0;
  double fe = 0.0;
  double* gst = R->g;
  float* E = R->E;
  for (int n = beg; n < min(end, N); ++n) {
    const double gn = g0 - C[n] * kc;
    C[n] = gn;
    gst[n] = gn;
    if (face) E[n] = (float)(-gn);  // face field
    if (want_fe) fe += gn * gn * dx[n];
  }
  if (!face) {
    __syncthreads();
    const double* wgt = R->mcw;
    for (int n = tid; n <= N; n += kFieldBlock) {
      double e;
      if (n > 0 && n < N) {
        e = -(C[n] * wgt[n] + C[n - 1] * (1.0 - wgt[n]));
      } else if (periodic) {
        e = -(C[0] * wgt[0] + C[N - 1] * (1.0 - wgt[0]));
      } else {
        e = (n == 0) ? -C[0] : -C[N - 1];
      }
      E[n] = (float)e;
    }
  }
  double fe_tot = 0.0;
  if (want_fe) fe_tot = 0.5 * kEps0 * block_sum(fe, dsm);
  if (want_phi) {
    // potential: phi_n = phi_0 + sum_{m<n} g_m dx_m
    __syncthreads();
    for (int n = tid; n < N; n += kFieldBlock) C[n] *= dx[n];
    __syncthreads();
    block_incl_scan_array(C, N, dsm);
    double* phi = R->phi;
    for (int n = tid; n <= N; n += kFieldBlock) {
      double p;
      if (n == 0) p = phi0;
      else if (n == N) p = 0.0;
      else p = phi0 + C[n - 1];
      phi[n] = p;
      if (sample) R->acc[(size_t)(5 * ns) * (N + 1) + n] += p;
    }
  }
  if (tid == 0) {
    st->phi0 = phi0;
    st->phi_level = want_phi ? kn : st->phi_level;
    if (sample) {
      st->fe = st->fe_field;
      for (int s = 0; s < ns; ++s) {
        st->ke[s] = st->ke_acc[s];
        st->ke_acc[s] = 0.0;
      }
      st->n_samples += 1;
    }
    if (want_fe) st->fe_field = fe_tot;
    if (advance) st->step = kn;
  }
  if (my_ss) {
    // the step's births are kept up to the capacity; the next pass's records start empty
    const long long n = my_alloc < my_cap ? my_alloc : my_cap;
    my_ss->n_proc = n;
    my_ss->n_alloc = n;
    my_ss->n_real = 0;
    my_ss->n_imp = 0;
  }
}

// potential of the current field of one run from the stored g (host reads)
__global__ void __launch_bounds__(kFieldBlock) k_phi(BatchView b, int slot) {
  const RunDev* R = b.runs + slot;
  if (!R->active) return;
  RunState* st = b.rst + slot;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* C = reinterpret_cast<double*>(smem_raw);
  __shared__ double dsm[32];
  const int N = R->N;
  for (int n = threadIdx.x; n < N; n += kFieldBlock) C[n] = R->g[n] * R->dx[n];
  __syncthreads();
  block_incl_scan_array(C, N, dsm);
  const double phi0 = st->phi0;
  for (int n = threadIdx.x; n <= N; n += kFieldBlock)
    R->phi[n] = (n == 0) ? phi0 : (n == N ? 0.0 : phi0 + C[n - 1]);
  if (threadIdx.x == 0) st->phi_level = st->step;
}

// ----------------------------------------------------------------- sort
__global__ void __launch_bounds__(kPassBlock) k_hist(BatchView b, int mode) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  long long* pre = reinterpret_cast<long long*>(smem_raw);
  int* H = reinterpret_cast<int*>(pre + b.nseg + 1);
  __shared__ long long wsm[32];
  __shared__ int lohi[2];
  for (int i = threadIdx.x; i <= b.nmax; i += kPassBlock) H[i] = 0;
  if (threadIdx.x == 0) {
    lohi[0] = INT_MAX;
    lohi[1] = -1;
  }
  // quads of four particles per thread, as in the pass
  const long long T = seg_prefix(b, mode, -1, pre, wsm, 4);
  if (T == 0) return;
  const long long lo = T * (long long)blockIdx.x / gridDim.x;
  const long long hi = T * (long long)(blockIdx.x + 1) / gridDim.x;
  if (lo >= hi) return;
  const int lane = threadIdx.x & 31;
  for (int s = seg_find(pre, b.nseg, lo); s < b.nseg && pre[s] < hi; ++s) {
    const long long beg = max(lo, pre[s]) - pre[s];
    const long long end = min(hi, pre[s + 1]) - pre[s];
    if (beg >= end) continue;
    const SegDev& G = b.segs[s];
    const int32_t* pc = G.cell[b.sst[s].cur];
    const long long n = b.sst[s].n_proc;
    const int Nr = b.runs[G.run].N;
    int my_lo = INT_MAX, my_hi = -1;
    for (long long base = beg + (long long)(threadIdx.x & ~31); base < end; base += kPassBlock) {
      const long long i0 = 4 * (base + lane);
      int c[4];
      if (base + lane < end && i0 + 3 < n && chk(i0 + 3 < G.cap, 26, i0, G.cap)) {
        const int4 c4 = *reinterpret_cast<const int4*>(pc + i0);
        c[0] = c4.x; c[1] = c4.y; c[2] = c4.z; c[3] = c4.w;
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) c[j] = (base + lane < end && i0 + j < n) ? pc[i0 + j] : -1;
      }
      // a thread's consecutive particles in one cell (most quads of sorted
      // data) are counted together: one shared atomic per run of equal cells
      int cur = -1, cnt = 0;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int cj = c[j] < Nr ? c[j] : -1;
        if (cj >= 0) {
          my_lo = min(my_lo, cj);
          my_hi = max(my_hi, cj);
        }
        if (cj != cur) {
          if (cur >= 0 && chk(cur <= b.nmax, 9, cur, b.nmax)) atomicAdd(H + cur, cnt);
          cur = cj;
          cnt = 0;
        }
        ++cnt;
      }
      if (cur >= 0 && chk(cur <= b.nmax, 9, cur, b.nmax)) atomicAdd(H + cur, cnt);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      my_lo = min(my_lo, __shfl_xor_sync(kFull, my_lo, o));
      my_hi = max(my_hi, __shfl_xor_sync(kFull, my_hi, o));
    }
    if (lane == 0 && my_hi >= 0) {
      atomicMin(&lohi[0], my_lo);
      atomicMax(&lohi[1], my_hi);
    }
    __syncthreads();
    const int flo = lohi[0], fhi = lohi[1];
    const int nbeg = flo <= fhi ? flo + (int)threadIdx.x : fhi + 1;  // empty range: skip
    for (int n = nbeg; n <= fhi; n += kPassBlock) {
      const int v = H[n];
      if (v) {
        atomicAdd(b.hist + G.hoff + n, v);
        H[n] = 0;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      lohi[0] = INT_MAX;
      lohi[1] = -1;
    }
    __syncthreads();
  }
}

// per segment: counts -> exclusive cursors; live total
__global__ void __launch_bounds__(kPassBlock) k_scan(BatchView b, int mode) {
  const int s = blockIdx.x;
  if (s >= b.nseg) return;
  const SegDev& G = b.segs[s];
  const int slot = G.run;
  if (!run_live(b.runs[slot], b.rst[slot], mode, -1, slot)) return;
  __shared__ long long wsm[32];
  const int N = b.runs[slot].N;
  int* h = b.hist + G.hoff;
  const int per = (N + kPassBlock - 1) / kPassBlock;
  const int beg = min(N, (int)threadIdx.x * per), end = min(N, beg + per);
  long long loc = 0;
  for (int i = beg; i < end; ++i) loc += h[i];
  long long total;
  long long run = block_excl_scan(loc, wsm, &total);
  for (int i = beg; i < end; ++i) {
    const int c = h[i];
    h[i] = (int)run;
    run += c;
  }
  if (threadIdx.x == 0) b.sst[s].n_live = total;
}

// Counting-sort scatter (the order within a cell is not kept), one CTA
// iteration of kScatQ particles at a time: the chunk's cells are counted in
// shared memory (a range [clo, chi] of its run's cells), each cell present
// reserves its slice of the destination with one global atomic per CTA
// iteration, the records are staged in shared memory in cell order, and
// consecutive threads then write consecutive destinations of each cell, so
// the stores fill whole sectors.  The next iteration's source records are
// prefetched into L2.  Launched as one wave (scatter_grid).
constexpr int kScatQ = 4 * kPassBlock;  // particles per CTA iteration

size_t scatter_smem_bytes(int nseg, int nmax) {
  return sizeof(long long) * (size_t)(nseg + 1) +
         (size_t)kScatQ * (sizeof(unsigned long long) + 6 * sizeof(int)) +
         3 * sizeof(int) * (size_t)(nmax + 1);
}

__global__ void __launch_bounds__(kPassBlock) k_scatter(BatchView b, int mode) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  long long* pre = reinterpret_cast<long long*>(smem_raw);
  unsigned long long* st_id = reinterpret_cast<unsigned long long*>(pre + b.nseg + 1);
  int* st_c = reinterpret_cast<int*>(st_id + kScatQ);
  float* st_x = reinterpret_cast<float*>(st_c + kScatQ);
  float* st_u = st_x + kScatQ;
  float* st_v = st_u + kScatQ;
  float* st_w = st_v + kScatQ;
  uint32_t* st_k = reinterpret_cast<uint32_t*>(st_w + kScatQ);
  const int M = b.nmax + 1;
  int* cnt = reinterpret_cast<int*>(st_k + kScatQ);  // per cell of the chunk's range
  int* lpre = cnt + M;                               // its exclusive prefix
  int* gbase = lpre + M;                             // its reserved destination
  __shared__ long long wsm[32];
  __shared__ int wsi[32];
  __shared__ int lohi[2];
  for (int i = threadIdx.x; i < M; i += kPassBlock) cnt[i] = 0;
  if (threadIdx.x == 0) {
    lohi[0] = INT_MAX;
    lohi[1] = -1;
  }
  const long long T = seg_prefix(b, mode, -1, pre, wsm, 4);  // ends with a barrier
  if (T == 0) return;
  const long long lo = T * (long long)blockIdx.x / gridDim.x;
  const long long hi = T * (long long)(blockIdx.x + 1) / gridDim.x;
  if (lo >= hi) return;
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  for (int s = seg_find(pre, b.nseg, lo); s < b.nseg && pre[s] < hi; ++s) {
    const long long beg = max(lo, pre[s]) - pre[s];
    const long long end = min(hi, pre[s + 1]) - pre[s];
    if (beg >= end) continue;
    const SegDev& G = b.segs[s];
    const int src = b.sst[s].cur, dst = src ^ 1;
    const long long n = b.sst[s].n_proc;
    int* cursor = b.hist + G.hoff;
    const int Nr = b.runs[G.run].N;
    const int32_t* sc = G.cell[src];
    const float* sx = G.xi[src];
    const float* su = G.vx[src];
    const float* sv = G.vy[src];
    const float* sw = G.vz[src];
    const uint64_t* si = G.id[src];
    const uint32_t* sk = G.wt[src];  // weight multipliers (rebalancing runs)
    int32_t* dc = G.cell[dst];
    float* dx_ = G.xi[dst];
    float* du = G.vx[dst];
    float* dv = G.vy[dst];
    float* dw = G.vz[dst];
    uint64_t* di = G.id[dst];
    uint32_t* dk = G.wt[dst];
    // block-uniform trip count: the barriers below need every thread
    for (long long base = beg; base < end; base += kPassBlock) {
      if (threadIdx.x == 0) {
        const long long nb = base + kPassBlock;
        if (nb < end) {
          const long long p0 = 4 * nb;
          const long long p1 = min(4 * min(end, nb + kPassBlock), n);
          if (p1 > p0) {
            const unsigned b4 = (unsigned)(((p1 - p0) * 4) & ~15ll);
            if (b4) {
              l2_prefetch(sc + p0, b4);
              l2_prefetch(sx + p0, b4);
              l2_prefetch(su + p0, b4);
              l2_prefetch(sv + p0, b4);
              l2_prefetch(sw + p0, b4);
              l2_prefetch(si + p0, (unsigned)(((p1 - p0) * 8) & ~15ll));
              if (sk) l2_prefetch(sk + p0, b4);
            }
          }
        }
      }
      const long long q = base + threadIdx.x;
      const long long i0 = 4 * q;
      int c[4];
      float x[4], u[4], v[4], w[4];
      uint64_t id[4];
      unsigned kq[4] = {1u, 1u, 1u, 1u};
      if (q < end && i0 + 3 < n && chk(i0 + 3 < G.cap, 27, i0, G.cap)) {
        const int4 c4 = *reinterpret_cast<const int4*>(sc + i0);
        const float4 x4 = *reinterpret_cast<const float4*>(sx + i0);
        const float4 u4 = *reinterpret_cast<const float4*>(su + i0);
        const float4 v4 = *reinterpret_cast<const float4*>(sv + i0);
        const float4 w4 = *reinterpret_cast<const float4*>(sw + i0);
        const ulonglong2 a = *reinterpret_cast<const ulonglong2*>(si + i0);
        const ulonglong2 a2 = *reinterpret_cast<const ulonglong2*>(si + i0 + 2);
        c[0] = c4.x; c[1] = c4.y; c[2] = c4.z; c[3] = c4.w;
        x[0] = x4.x; x[1] = x4.y; x[2] = x4.z; x[3] = x4.w;
        u[0] = u4.x; u[1] = u4.y; u[2] = u4.z; u[3] = u4.w;
        v[0] = v4.x; v[1] = v4.y; v[2] = v4.z; v[3] = v4.w;
        w[0] = w4.x; w[1] = w4.y; w[2] = w4.z; w[3] = w4.w;
        id[0] = a.x; id[1] = a.y; id[2] = a2.x; id[3] = a2.y;
        if (sk) {
          const uint4 k4 = *reinterpret_cast<const uint4*>(sk + i0);
          kq[0] = k4.x; kq[1] = k4.y; kq[2] = k4.z; kq[3] = k4.w;
        }
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const bool in = q < end && i0 + j < n && chk(i0 + j < G.cap, 27, i0 + j, G.cap);
          c[j] = in ? sc[i0 + j] : -1;
          x[j] = in ? sx[i0 + j] : 0.f;
          u[j] = in ? su[i0 + j] : 0.f;
          v[j] = in ? sv[i0 + j] : 0.f;
          w[j] = in ? sw[i0 + j] : 0.f;
          id[j] = in ? si[i0 + j] : 0ull;
          if (sk && in) kq[j] = sk[i0 + j];
        }
      }
      // the chunk's cell range (absorbed particles, cell < 0, are dropped)
      int my_lo = INT_MAX, my_hi = -1;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        c[j] = c[j] < Nr ? c[j] : -1;
        if (c[j] >= 0) {
          my_lo = min(my_lo, c[j]);
          my_hi = max(my_hi, c[j]);
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        my_lo = min(my_lo, __shfl_xor_sync(kFull, my_lo, o));
        my_hi = max(my_hi, __shfl_xor_sync(kFull, my_hi, o));
      }
      if (lane == 0 && my_hi >= 0) {
        atomicMin(&lohi[0], my_lo);
        atomicMax(&lohi[1], my_hi);
      }
      __syncthreads();
      const int clo = lohi[0], chi = lohi[1];
      const int R = chi >= clo ? chi - clo + 1 : 0;
      // rank of each particle among the chunk's particles of its cell
      int r[4] = {0, 0, 0, 0};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const unsigned grp = __match_any_sync(kFull, c[j] >= 0 ? (unsigned)c[j] : 0xFFFFFFFFu);
        if (c[j] >= 0 && chk(c[j] - clo < M, 28, c[j] - clo, M)) {
          const int leader = __ffs(grp) - 1;
          int b0 = 0;
          if (lane == leader) b0 = atomicAdd(cnt + (c[j] - clo), __popc(grp));
          b0 = __shfl_sync(grp, b0, leader);
          r[j] = b0 + __popc(grp & lt);
        }
      }
      __syncthreads();
      // local prefix of the range's counts; each cell present reserves its
      // destination slice
      const int per = (R + kPassBlock - 1) / kPassBlock;
      const int kb = min(R, (int)threadIdx.x * per), ke = min(R, kb + per);
      int loc = 0;
      for (int k = kb; k < ke; ++k) loc += cnt[k];
      int m;
      int run = block_excl_scan(loc, wsi, &m);
      for (int k = kb; k < ke; ++k) {
        const int ck = cnt[k];
        lpre[k] = run;
        run += ck;
        gbase[k] = ck ? atomicAdd(cursor + clo + k, ck) : 0;
      }
      __syncthreads();
      // stage in cell order
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (c[j] < 0) continue;
        const int p = lpre[c[j] - clo] + r[j];
        if (!chk(p >= 0 && p < kScatQ, 29, p, kScatQ)) continue;
        st_c[p] = c[j];
        st_x[p] = x[j];
        st_u[p] = u[j];
        st_v[p] = v[j];
        st_w[p] = w[j];
        st_id[p] = id[j];
        st_k[p] = kq[j];
      }
      __syncthreads();
      for (int t = threadIdx.x; t < m; t += kPassBlock) {
        const int cc = st_c[t];
        const int k = cc - clo;
        const long long d = (long long)gbase[k] + (t - lpre[k]);
        if (!chk(d >= 0 && d < G.cap, 10, d, G.cap)) continue;
        dc[d] = cc;
        dx_[d] = st_x[t];
        du[d] = st_u[t];
        dv[d] = st_v[t];
        dw[d] = st_w[t];
        di[d] = st_id[t];
        if (dk) dk[d] = st_k[t];
      }
      for (int k = threadIdx.x; k < R; k += kPassBlock) cnt[k] = 0;
      if (threadIdx.x == 0) {
        lohi[0] = INT_MAX;
        lohi[1] = -1;
      }
      __syncthreads();
    }
  }
}

__global__ void __launch_bounds__(kPassBlock) k_finalize(BatchView b) {
  // (the counting sort's last phase; rebalancing ends with k_rb_finalize)
  const int s = blockIdx.x;
  if (s >= b.nseg) return;
  const SegDev& G = b.segs[s];
  const int slot = G.run;
  if (!run_live(b.runs[slot], b.rst[slot], MODE_SORT, -1, slot)) return;
  const int N = b.runs[slot].N;
  for (int i = threadIdx.x; i < N; i += kPassBlock) b.hist[G.hoff + i] = 0;
  if (threadIdx.x == 0) {
    SegState* ss = b.sst + s;
    ss->cur ^= 1;
    ss->n_proc = ss->n_live;
    ss->n_alloc = ss->n_live;
    ss->n_dead = 0;
  }
}

// ----------------------------------------------------------------- rebalancing
// Particle rebalancing (Sec. 3d proposes keeping the particles per cell near a
// target on non-uniform grids; the rule is this library's design, the same as
// the oracle's).  It runs for the runs due at their current level (after the
// field kernel of that level): a counting sort by cell into the other buffer
// set (k_hist, k_scan, k_scatter in MODE_REBAL), then per (segment, cell):
//   - more than rb_hi particles (at most kRbMaxCell): order them by (vx, id),
//     cut the order into floor(n/4) groups of four, merge the
//     G = min(floor(n/4), ceil((n - target)/2)) groups nearest the middle of
//     the order (ties: the slower), skipping groups heavier than
//     kRbMaxWeight; a group becomes two particles at its weighted centroid
//     with velocities u + sqrt(b/a) d, u - sqrt(a/b) d (u the mean velocity,
//     d the per-component standard deviations with Philox signs for y and z,
//     a = ceil(W/2), b = W - a), taking the group's two smallest ids;
//   - fewer than rb_lo (and some): split the min(target - n, #{k >= 2})
//     heaviest (ties: smallest id) in place into ceil(k/2) (same id) and
//     floor(k/2) (id child_id(id, level, 3));
//   - otherwise copied.
// k_rb_classify lists the cells that merge or split and counts the others,
// k_rb_cells counts each listed cell's output, k_rb_scan places the cells,
// k_rb_copy streams the unchanged cells' particles back into the current
// buffer set and k_rb_cells writes the listed cells there, k_rb_finalize and
// k_rb_mark set the sizes and the run's rebalancing level.
constexpr int kRbBlock = 256;
constexpr int kRbListCells = 4096;  // list entry = segment * kRbListCells + cell
constexpr int kRbGroups = kRbMaxCell / 4;

struct RbSmem {
  unsigned long long k2[kRbMaxCell];  // second key: id
  uint32_t k1[kRbMaxCell];            // first key: monotone vx bits, or ~k
  uint16_t ix[kRbMaxCell];            // index within the cell
  uint16_t pref[kRbGroups];           // eligible groups before each order position
  uint8_t el[kRbGroups];              // group at an order position may merge
  unsigned kmax;                      // the cell's largest weight multiplier
};

// FP32 bits ordered like the values (+0 and -0 as one value)
__device__ __forceinline__ uint32_t rb_fkey(float v) {
  const uint32_t u = __float_as_uint(v == 0.0f ? 0.0f : v);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// ascending bitonic sort of P (a power of two) entries by (k1, k2)
__device__ void rb_bitonic(RbSmem& sm, int P) {
  for (int size = 2; size <= P; size <<= 1)
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int t = threadIdx.x; t < (P >> 1); t += blockDim.x) {
        const int i = 2 * stride * (t / stride) + (t % stride);
        const int j = i + stride;
        const bool up = (i & size) == 0;
        const bool gt = sm.k1[i] > sm.k1[j] || (sm.k1[i] == sm.k1[j] && sm.k2[i] > sm.k2[j]);
        if (gt == up) {
          const uint32_t a = sm.k1[i]; sm.k1[i] = sm.k1[j]; sm.k1[j] = a;
          const unsigned long long c = sm.k2[i]; sm.k2[i] = sm.k2[j]; sm.k2[j] = c;
          const uint16_t x = sm.ix[i]; sm.ix[i] = sm.ix[j]; sm.ix[j] = x;
        }
      }
      __syncthreads();
    }
}

// order position of merge group g among ng groups: by distance from the
// middle of the velocity order, the slower group first on a tie
__device__ __forceinline__ int rb_pos(int g, int ng) {
  const int d = 2 * g - (ng - 1);
  return (d < 0 ? -d : d) - (d < 0 ? 1 : 0);
}

__device__ __forceinline__ void rb_copy(const SegDev& G, int in, int out, long long i, long long o) {
  G.cell[out][o] = G.cell[in][i];
  G.xi[out][o] = G.xi[in][i];
  G.vx[out][o] = G.vx[in][i];
  G.vy[out][o] = G.vy[in][i];
  G.vz[out][o] = G.vz[in][i];
  G.id[out][o] = G.id[in][i];
  G.wt[out][o] = G.wt[in][i];
}

// One cell: the particles [start, start + n) of buffer set `in` (sorted by
// cell).  Returns the cell's output count; when write, the output goes to
// buffer set `out` from position obase and the counters are updated.  Every
// thread of the block calls it (block-uniform arguments).
__device__ int rb_cell(const BatchView& b, int s, int c, long long start, int n, bool write,
                       long long obase, RbSmem& sm, long long* wsm) {
  const SegDev& G = b.segs[s];
  const int slot = G.run, sp = G.species;
  const RunDev* R = b.runs + slot;
  RunState* st = b.rst + slot;
  const int out = b.sst[s].cur, in = out ^ 1;
  const int T = R->rb_target;
  int mode = 0;  // 0 copy, 1 merge, 2 split, 3 skip (copy, counted)
  if (n > R->rb_hi) mode = n > kRbMaxCell ? 3 : 1;
  else if (n > 0 && n < R->rb_lo) mode = 2;
  const int tid = threadIdx.x;
  if (mode == 2) {
    long long heavy = 0;
    for (int t = tid; t < n; t += blockDim.x) heavy += G.wt[in][start + t] >= 2u ? 1 : 0;
    heavy = block_sum(heavy, wsm);
    const int S = (int)min((long long)(T - n), heavy);
    if (S <= 0) {
      mode = 0;
    } else {
      if (!write) return n + S;
      int P = 1;
      while (P < n) P <<= 1;
      for (int t = tid; t < P; t += blockDim.x) {
        if (t < n) {
          sm.k1[t] = ~G.wt[in][start + t];  // heaviest first
          sm.k2[t] = G.id[in][start + t];
          sm.ix[t] = (uint16_t)t;
        } else {
          sm.k1[t] = 0xFFFFFFFFu;
          sm.k2[t] = ~0ull;
          sm.ix[t] = 0;
        }
      }
      __syncthreads();
      rb_bitonic(sm, P);
      const long long k_lvl = st->step;
      for (int t = tid; t < n; t += blockDim.x) {
        const long long i = start + sm.ix[t];
        if (t < S) {
          const long long o = obase + 2 * t;
          rb_copy(G, in, out, i, o);
          rb_copy(G, in, out, i, o + 1);
          const unsigned k = G.wt[in][i];
          G.wt[out][o] = (k + 1u) / 2u;
          G.wt[out][o + 1] = k / 2u;
          G.id[out][o + 1] = child_id(G.id[in][i], k_lvl, 3);
        } else {
          rb_copy(G, in, out, i, obase + S + t);
        }
      }
      if (tid == 0) atomicAdd(&st->ctr[sp][C_RB_SPLIT], (unsigned long long)S);
      __syncthreads();
      return n + S;
    }
  }
  if (mode == 0 || mode == 3) {
    // (listed cells only: a split cell with nothing to split)
    if (write)
      for (int t = tid; t < n; t += blockDim.x) rb_copy(G, in, out, start + t, obase + t);
    return n;
  }
  // merge: order by (vx, id), groups of four, the ones nearest the middle
  const int ng = n / 4;
  const int Gw = min(ng, (n - T + 1) / 2);
  if (!write) {
    // with no multiplier above kRbMaxWeight / 4 every group is eligible
    // (W <= kRbMaxWeight), so the count needs no ordering
    if (tid == 0) sm.kmax = 0u;
    __syncthreads();
    unsigned km = 0u;
    for (int t = tid; t < n; t += blockDim.x) km = max(km, G.wt[in][start + t]);
    km = __reduce_max_sync(0xFFFFFFFFu, km);
    if ((tid & 31) == 0) atomicMax(&sm.kmax, km);
    __syncthreads();
    const unsigned kmax = sm.kmax;
    __syncthreads();  // every thread has read it before the next cell resets it
    if (kmax <= kRbMaxWeight / 4u) return n - 2 * Gw;
  }
  int P = 1;
  while (P < n) P <<= 1;
  for (int t = tid; t < P; t += blockDim.x) {
    if (t < n) {
      sm.k1[t] = rb_fkey(G.vx[in][start + t]);
      sm.k2[t] = G.id[in][start + t];
      sm.ix[t] = (uint16_t)t;
    } else {
      sm.k1[t] = 0xFFFFFFFFu;
      sm.k2[t] = ~0ull;
      sm.ix[t] = 0;
    }
  }
  __syncthreads();
  rb_bitonic(sm, P);
  for (int g = tid; g < ng; g += blockDim.x) {
    unsigned W = 0u;
    for (int q = 0; q < 4; ++q) W += G.wt[in][start + sm.ix[4 * g + q]];
    sm.el[rb_pos(g, ng)] = W <= kRbMaxWeight ? 1 : 0;
  }
  __syncthreads();
  // eligible groups before each order position (block scan; ng <= 1024)
  {
    const int per = (ng + blockDim.x - 1) / blockDim.x;
    const int a = min(ng, tid * per), e = min(ng, a + per);
    long long loc = 0;
    for (int q = a; q < e; ++q) loc += sm.el[q];
    long long tot;
    long long run = block_excl_scan(loc, wsm, &tot);
    for (int q = a; q < e; ++q) {
      sm.pref[q] = (uint16_t)run;
      run += sm.el[q];
    }
    __syncthreads();
    const int chosen = (int)min((long long)Gw, tot);
    if (!write) return n - 2 * chosen;
  }
  // output offsets: a chosen group's first particle emits two, its others
  // none, every other particle one.  They are scanned in shared memory (the
  // sort keys are no longer needed), so that consecutive threads take
  // consecutive order positions and their stores coalesce.
  auto emits = [&](int t) -> int {
    const int g = t / 4;
    if (g >= ng) return 1;
    const int ps = rb_pos(g, ng);
    const bool ch = sm.el[ps] && (int)sm.pref[ps] < Gw;
    return ch ? ((t & 3) == 0 ? 2 : 0) : 1;
  };
  long long* opos = reinterpret_cast<long long*>(sm.k2);
  for (int t = tid; t < n; t += blockDim.x) opos[t] = emits(t);
  __syncthreads();
  block_incl_scan_array(opos, n, wsm);
  const long long tot = opos[n - 1];
  const long long k_lvl = st->step;
  unsigned long long merged = 0;
  // single particles: consecutive threads, consecutive positions
  for (int t = tid; t < n; t += blockDim.x)
    if (emits(t) == 1) rb_copy(G, in, out, start + sm.ix[t], obase + opos[t] - 1);
  // chosen groups, one per thread (the FP64 merge arithmetic is a long
  // dependent chain on this part's slow FP64 pipe: spread it over the block)
  for (int g = tid; g < ng; g += blockDim.x) {
    const int t = 4 * g;
    if (emits(t) != 2) continue;
    const long long pos = opos[t] - 2;
    {
      // the group's weighted centroid, mean velocity and spreads (FP64)
      double W = 0.0, X = 0.0, u[3] = {0.0, 0.0, 0.0}, m2[3] = {0.0, 0.0, 0.0};
      unsigned Wi = 0u;
      unsigned long long id0 = ~0ull, id1 = ~0ull;
      long long ii[4];
      for (int q = 0; q < 4; ++q) {
        const long long i = start + sm.ix[t + q];
        ii[q] = i;
        const unsigned k = G.wt[in][i];
        const double kd = (double)k;
        Wi += k;
        W += kd;
        X += kd * (double)G.xi[in][i];
        u[0] += kd * (double)G.vx[in][i];
        u[1] += kd * (double)G.vy[in][i];
        u[2] += kd * (double)G.vz[in][i];
        const unsigned long long id = G.id[in][i];
        if (id < id0) { id1 = id0; id0 = id; } else if (id < id1) { id1 = id; }
      }
      X /= W;
      for (int q = 0; q < 3; ++q) u[q] /= W;
      for (int q = 0; q < 4; ++q) {
        const long long i = ii[q];
        const double kd = (double)G.wt[in][i];
        const double dv[3] = {(double)G.vx[in][i] - u[0], (double)G.vy[in][i] - u[1],
                              (double)G.vz[in][i] - u[2]};
        for (int r = 0; r < 3; ++r) m2[r] += kd * dv[r] * dv[r];
      }
      const uint4 A = draw(R->seed, id0, (uint32_t)k_lvl, ((uint32_t)sp << 8) | 0x10u);
      double d[3] = {sqrt(m2[0] / W), sqrt(m2[1] / W), sqrt(m2[2] / W)};
      if (A.x & 1u) d[1] = -d[1];
      if (A.x & 2u) d[2] = -d[2];
      const unsigned ka = (Wi + 1u) / 2u, kb = Wi - ka;
      const double fa = sqrt((double)kb / (double)ka), fb = sqrt((double)ka / (double)kb);
      float xc = (float)X;
      if (xc >= 1.0f) xc = 0.99999994f;  // the centroid lies in the cell
      const long long o = obase + pos;
      const int cc = G.cell[in][ii[0]];
      G.cell[out][o] = cc;
      G.cell[out][o + 1] = cc;
      G.xi[out][o] = xc;
      G.xi[out][o + 1] = xc;
      G.vx[out][o] = (float)(u[0] + fa * d[0]);
      G.vy[out][o] = (float)(u[1] + fa * d[1]);
      G.vz[out][o] = (float)(u[2] + fa * d[2]);
      G.vx[out][o + 1] = (float)(u[0] - fb * d[0]);
      G.vy[out][o + 1] = (float)(u[1] - fb * d[1]);
      G.vz[out][o + 1] = (float)(u[2] - fb * d[2]);
      G.id[out][o] = id0;
      G.id[out][o + 1] = id1;
      G.wt[out][o] = ka;
      G.wt[out][o + 1] = kb;
      ++merged;
    }
  }
  merged = warp_sum(merged);
  if ((tid & 31) == 0 && merged) atomicAdd(&st->ctr[sp][C_RB_MERGED], merged);
  __syncthreads();
  return (int)tot;
}

// Per (segment, cell) of a due run, one thread: a cell that merges or splits
// (more than rb_hi particles, at most kRbMaxCell; fewer than rb_lo) goes on
// the list for k_rb_cells; the others keep their particles, so their output
// count is their count and k_rb_copy moves them (mode 0; 2: above kRbMaxCell,
// counted as skipped).
__global__ void __launch_bounds__(kPassBlock) k_rb_classify(BatchView b) {
  const int s = blockIdx.y;
  const int c = blockIdx.x * kPassBlock + threadIdx.x;
  if (s >= b.nseg) return;
  const SegDev& G = b.segs[s];
  const int slot = G.run;
  const RunDev& R = b.runs[slot];
  if (!run_live(R, b.rst[slot], MODE_REBAL, -1, slot) || c >= R.N || c >= kRbListCells) return;
  const int* h = b.hist + G.hoff;  // after the scatter: the end of each cell
  const int n = h[c] - (c > 0 ? h[c - 1] : 0);
  const bool listed = (n > R.rb_hi && n <= kRbMaxCell) || (n > 0 && n < R.rb_lo);
  b.rbmode[G.hoff + c] = listed ? 1 : (n > R.rb_hi ? 2 : 0);
  if (listed) {
    // at most one entry per (segment, cell): within nseg * nmax by construction
    const int k = atomicAdd(b.rbnum, 1);
    const bool fits = k < b.nseg * b.nmax;
    chk(fits, 30, k, (long long)b.nseg * b.nmax);
    if (fits) b.rblist[k] = s * kRbListCells + c;
  } else {
    b.rbcnt[G.hoff + c] = n;
  }
}

// write = 0: each listed cell's output count into rbcnt; write = 1: the
// listed cells' particles into the current buffer set at the scanned offsets
__global__ void __launch_bounds__(kRbBlock) k_rb_cells(BatchView b, int write) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  RbSmem& sm = *reinterpret_cast<RbSmem*>(smem_raw);
  __shared__ long long wsm[32];
  const int num = *b.rbnum;
  for (int item = blockIdx.x; item < num; item += gridDim.x) {
    const int e = b.rblist[item];
    const int s = e / kRbListCells, c = e % kRbListCells;
    if (!chk(s >= 0 && s < b.nseg, 31, s, b.nseg)) continue;
    const SegDev& G = b.segs[s];
    if (write && b.sst[s].rb_over) continue;
    const int* h = b.hist + G.hoff;
    const long long end = h[c];
    const long long start = c > 0 ? h[c - 1] : 0;
    // (an unconditional guard: the writes below index by this range)
    if (!(start >= 0 && end >= start && end <= G.cap)) continue;
    int* oc = b.rbcnt + G.hoff;
    const int cnt = rb_cell(b, s, c, start, (int)(end - start), write != 0, write ? oc[c] : 0, sm, wsm);
    if (!write && threadIdx.x == 0) oc[c] = cnt;
  }
}

// The particles of the cells that keep them (mode 0 and 2), streamed from the
// sorted buffer set into the current one at their cell's scanned offset:
// consecutive particles of a cell, consecutive positions.  Segments of due
// runs whose plan did not overflow the capacity.
__global__ void __launch_bounds__(kPassBlock) k_rb_copy(BatchView b) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  long long* pre = reinterpret_cast<long long*>(smem_raw);
  __shared__ long long wsm[32];
  {
    const int per = (b.nseg + blockDim.x - 1) / blockDim.x;
    const int s0 = threadIdx.x * per;
    long long loc = 0;
    for (int k = 0; k < per; ++k) {
      const int sg = s0 + k;
      if (sg < b.nseg) {
        const int slot = b.segs[sg].run;
        const bool due = run_live(b.runs[slot], b.rst[slot], MODE_REBAL, -1, slot) &&
                         !b.sst[sg].rb_over;
        const long long cnt = due ? b.sst[sg].n_live : 0;
        pre[sg] = cnt;
        loc += cnt;
      }
    }
    long long total;
    long long run = block_excl_scan(loc, wsm, &total);
    for (int k = 0; k < per; ++k) {
      const int sg = s0 + k;
      if (sg < b.nseg) {
        const long long cnt = pre[sg];
        pre[sg] = run;
        run += cnt;
      }
    }
    if (threadIdx.x == 0) pre[b.nseg] = total;
    __syncthreads();
  }
  const long long T = pre[b.nseg];
  if (T == 0) return;
  const long long lo = T * (long long)blockIdx.x / gridDim.x;
  const long long hi = T * (long long)(blockIdx.x + 1) / gridDim.x;
  if (lo >= hi) return;
  for (int s = seg_find(pre, b.nseg, lo); s < b.nseg && pre[s] < hi; ++s) {
    const long long beg = max(lo, pre[s]) - pre[s];
    const long long end = min(hi, pre[s + 1]) - pre[s];
    if (beg >= end) continue;
    const SegDev& G = b.segs[s];
    const int out = b.sst[s].cur, in = out ^ 1;
    const int N = b.runs[G.run].N;
    const int* h = b.hist + G.hoff;
    const int* oc = b.rbcnt + G.hoff;
    const uint8_t* md = b.rbmode + G.hoff;
    for (long long i = beg + threadIdx.x; i < end; i += blockDim.x) {
      if (!chk(i < G.cap, 32, i, G.cap)) continue;
      const int c = G.cell[in][i];
      if (!chk(c >= 0 && c < N, 33, c, N)) continue;
      if (md[c] == 1) continue;  // listed: written by k_rb_cells
      const long long o = (long long)oc[c] + (i - (c > 0 ? h[c - 1] : 0));
      // (an unconditional guard, as in k_rb_cells: the writes index by o)
      const bool ok = o >= 0 && o < G.cap;
      chk(ok, 34, o, G.cap);
      if (ok) rb_copy(G, in, out, i, o);
    }
  }
}

// per segment: output counts -> exclusive offsets; the total (capacity check)
__global__ void __launch_bounds__(kPassBlock) k_rb_scan(BatchView b) {
  const int s = blockIdx.x;
  if (s >= b.nseg) return;
  const SegDev& G = b.segs[s];
  const int slot = G.run;
  if (!run_live(b.runs[slot], b.rst[slot], MODE_REBAL, -1, slot)) return;
  __shared__ long long wsm[32];
  const int N = b.runs[slot].N;
  int* h = b.rbcnt + G.hoff;
  const int per = (N + kPassBlock - 1) / kPassBlock;
  const int beg = min(N, (int)threadIdx.x * per), end = min(N, beg + per);
  long long loc = 0;
  for (int i = beg; i < end; ++i) loc += h[i];
  long long total;
  long long run = block_excl_scan(loc, wsm, &total);
  for (int i = beg; i < end; ++i) {
    const int c = h[i];
    h[i] = (int)run;
    run += c;
  }
  if (threadIdx.x == 0) {
    b.sst[s].n_rb = total;
    b.sst[s].rb_over = total > G.cap ? 1 : 0;
  }
}

// per segment: sizes after the rebalancing (or, if the plan overflowed the
// capacity, the sorted particles unchanged); cell arrays cleared
__global__ void __launch_bounds__(kPassBlock) k_rb_finalize(BatchView b) {
  const int s = blockIdx.x;
  if (s >= b.nseg) return;
  const SegDev& G = b.segs[s];
  const int slot = G.run;
  if (!run_live(b.runs[slot], b.rst[slot], MODE_REBAL, -1, slot)) return;
  const int N = b.runs[slot].N;
  const bool over = b.sst[s].rb_over != 0;
  unsigned long long skipped = 0;
  for (int i = threadIdx.x; i < N; i += kPassBlock) {
    b.hist[G.hoff + i] = 0;
    b.rbcnt[G.hoff + i] = 0;
    skipped += (!over && b.rbmode[G.hoff + i] == 2) ? 1ull : 0ull;
    b.rbmode[G.hoff + i] = 0;
  }
  skipped = warp_sum(skipped);
  if ((threadIdx.x & 31) == 0 && skipped)
    atomicAdd(&b.rst[slot].ctr[G.species][C_RB_SKIPPED], skipped);
  __syncthreads();  // every thread has read rb_over
  if (threadIdx.x == 0) {
    SegState* ss = b.sst + s;
    if (ss->rb_over) {
      ss->cur ^= 1;  // the sorted buffer set
      ss->n_proc = ss->n_live;
      ss->n_alloc = ss->n_live;
    } else {
      ss->n_proc = ss->n_rb;
      ss->n_alloc = ss->n_rb;
    }
    ss->n_dead = 0;
  }
}

// per run: the level rebalanced; a capacity overflow fails the run
__global__ void k_rb_mark(BatchView b) {
  const int slot = blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= b.max_slots) return;
  RunState* st = b.rst + slot;
  const RunDev& R = b.runs[slot];
  if (!run_live(R, *st, MODE_REBAL, -1, slot)) return;
  bool over = false;
  for (int q = 0; q < R.ns; ++q) {
    SegState* ss = b.sst + R.seg0 + q;
    over = over || ss->rb_over;
    ss->rb_over = 0;
  }
  st->rb_level = st->step;
  st->rb_force = 0;
  if (over) {
    set_status(st, ECPIC_ERR_CAPACITY);
  }
}

// ----------------------------------------------------------------- loader
// Uniform positions and Maxwellian velocities (Sec. 2b) from Philox blocks
// (id = i, step word 0xFFFFFFFF, word3 = (s<<8)|0x80 for X, |0x81 for v),
// in FP64 so that the cell index matches the FP64 definition exactly.
__device__ __forceinline__ void init_run(const BatchView& b, int slot, const InitParams& p) {
  const RunDev* R = b.runs + slot;
  const int sp = blockIdx.y;
  if (sp >= R->ns) return;
  const int s = R->seg0 + sp;
  const SegDev& G = b.segs[s];
  const int cur = b.sst[s].cur;
  const int N = R->N;
  const double L = R->L;
  const double* x = R->x;
  const double* dx = R->dx;
  const double sd = p.sd[sp];
  const long long n = p.n[sp];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const uint4 A = draw(R->seed, (uint64_t)i, 0xFFFFFFFFu, ((uint32_t)sp << 8) | 0x80u);
    const uint4 B = draw(R->seed, (uint64_t)i, 0xFFFFFFFFu, ((uint32_t)sp << 8) | 0x81u);
    const double u = p.quiet ? __ddiv_rn((double)i + 0.5, (double)n)
                             : (double)A.x * 2.3283064365386963e-10;
    const double X = __dmul_rn(u, L);
    int lo = 0, hi = N;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (x[mid] <= X) lo = mid; else hi = mid;
    }
    int c = lo;
    float f = __double2float_rn(__ddiv_rn(__dsub_rn(X, x[c]), dx[c]));
    if (f >= 1.0f) {
      if (c + 1 < N) {
        c += 1;
        f = 0.0f;
      } else {
        f = 0.99999994f;
      }
    }
    const double u1a = __dmul_rn((double)B.x + 1.0, 2.3283064365386963e-10);
    const double u2a = __dmul_rn((double)B.y, 2.3283064365386963e-10);
    const double u1b = __dmul_rn((double)B.z + 1.0, 2.3283064365386963e-10);
    const double u2b = __dmul_rn((double)B.w, 2.3283064365386963e-10);
    const double ra = sqrt(__dmul_rn(-2.0, log(u1a)));
    const double rb = sqrt(__dmul_rn(-2.0, log(u1b)));
    const double aa = __dmul_rn(kTwoPi, u2a), ab = __dmul_rn(kTwoPi, u2b);
    const double z0 = __dmul_rn(ra, cos(aa)), z1 = __dmul_rn(ra, sin(aa));
    const double z2 = __dmul_rn(rb, cos(ab));
    if (!chk(i < G.cap && c >= 0 && c < N, 11, i, G.cap)) continue;
    G.cell[cur][i] = c;
    G.xi[cur][i] = f;
    G.vx[cur][i] = __double2float_rn(__dmul_rn(sd, z0));
    G.vy[cur][i] = __double2float_rn(__dmul_rn(sd, z1));
    G.vz[cur][i] = __double2float_rn(__dmul_rn(sd, z2));
    G.id[cur][i] = (uint64_t)i;
    if (G.wt[cur]) G.wt[cur][i] = p.rb_m0;
  }
}

__global__ void k_init(BatchView b, int slot, InitParams p) { init_run(b, slot, p); }

// A wave of admitted runs: blockIdx.z indexes the list of slots.
__global__ void k_init_many(BatchView b, const int* slots, const InitParams* ps, int count) {
  if ((int)blockIdx.z >= count) return;
  const int slot = slots[blockIdx.z];
  if (slot < 0 || slot >= b.max_slots) return;
  init_run(b, slot, ps[blockIdx.z]);
}

// ----------------------------------------------------------------- test kernels
__global__ void __launch_bounds__(kPassBlock) k_deposit_device(int N, long long n, const int* cell,
                                                               const float* xi,
                                                               unsigned long long* S) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint32_t* dcnt = reinterpret_cast<uint32_t*>(smem_raw);
  uint32_t* dlo = dcnt + (N + 1);
  uint32_t* dhi = dcnt + 2 * (N + 1);
  for (int i = threadIdx.x; i < 3 * (N + 1); i += kPassBlock) dcnt[i] = 0u;
  __syncthreads();
  const long long nq = (n + 3) / 4;
  int since_flush = 0;
  // block-uniform trip count: the periodic flush needs every thread
  for (long long base = (long long)blockIdx.x * kPassBlock; base < nq;
       base += (long long)gridDim.x * kPassBlock) {
    const long long q = base + threadIdx.x;
    int c[4];
    float f[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const long long i = 4 * q + j;
      const int cc = (q < nq && i < n) ? cell[i] : -1;
      const bool ok = cc >= 0 && cc < N;
      c[j] = ok ? cc : -1;
      f[j] = ok ? xi[i] : 0.0f;
    }
    dep_add4(dcnt, dlo, dhi, c, f);
    if (++since_flush == kFlushIters) {
      __syncthreads();
      dep_flush(dcnt, dlo, dhi, 0, N, S);
      __syncthreads();
      since_flush = 0;
    }
  }
  __syncthreads();
  dep_flush(dcnt, dlo, dhi, 0, N, S);
}

// EC2 quadratic deposit of caller-owned (cell, xi) arrays straight to S
// (tests): the pass's integer shares; periodic node N is node 0 here and is
// mirrored after the deposit
__global__ void k_deposit2_device(int N, int periodic, long long n, const int* cell, const float* xi,
                                  unsigned long long* S) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int c = cell[i];
    if (c < 0 || c >= N) continue;
    int n0;
    unsigned a, b;
    spline2_shares(xi[i], c, &n0, &a, &b);
    int nodes[3] = {n0 - 1, n0, n0 + 1};
    for (int q = 0; q < 3; ++q) {
      int m = nodes[q];
      if (periodic) m = ((m % N) + N) % N;
      else m = m < 0 ? 0 : (m > N ? N : m);
      nodes[q] = m;
    }
    atomicAdd(S + nodes[0], (unsigned long long)a);
    atomicAdd(S + nodes[1], 4294967296ull - a - b);
    atomicAdd(S + nodes[2], (unsigned long long)b);
  }
}

__global__ void k_mirror_node(int N, unsigned long long* S) { S[N] = S[0]; }

__global__ void k_philox_device(long long n, const uint32_t* ctr, const uint32_t* key,
                                uint32_t* out) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const uint4 c = make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]);
    const uint4 r = philox4x32_10(c, make_uint2(key[2 * i], key[2 * i + 1]));
    out[4 * i] = r.x;
    out[4 * i + 1] = r.y;
    out[4 * i + 2] = r.z;
    out[4 * i + 3] = r.w;
  }
}

}  // namespace

// ----------------------------------------------------------------- launchers
size_t pass_smem_bytes(const BatchView& b) {
  return sizeof(long long) * (size_t)(b.nseg + 1) +
         (b.weighted ? 4 : 3) * sizeof(uint32_t) * (size_t)(b.nmax + 1) +
         sizeof(float) * 3 * (size_t)(b.nmax + 1) +
         sizeof(int) * (size_t)(3 * kRing) * (kPassBlock / 32) + sizeof(float) * (size_t)(b.nmax + 1);
}

size_t field_smem_bytes(const BatchView& b) { return sizeof(double) * (size_t)(b.nmax + 1); }

static void set_smem_attr(const void* fn, size_t bytes) {
  if (bytes > 48 * 1024) cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <bool W>
static int pass_occupancy(size_t sm) {
  set_smem_attr((const void*)k_pass<true, W>, sm);
  set_smem_attr((const void*)k_pass<false, W>, sm);
  int n = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_pass<true, W>, kPassBlock, sm);
  return n > 0 ? n : 1;
}

int pass_max_ctas_per_sm(const BatchView& b) {
  const size_t sm = pass_smem_bytes(b);
  return b.weighted ? pass_occupancy<true>(sm) : pass_occupancy<false>(sm);
}

template <bool W>
static void launch_pass_w(const BatchView& b, int grid, int mode, int only, cudaStream_t s,
                          bool stage_field, size_t sm) {
  if (stage_field) {
    set_smem_attr((const void*)k_pass<true, W>, sm);
    k_pass<true, W><<<grid, kPassBlock, sm, s>>>(b, mode, only);
  } else {
    set_smem_attr((const void*)k_pass<false, W>, sm);
    k_pass<false, W><<<grid, kPassBlock, sm, s>>>(b, mode, only);
  }
}

void launch_pass(const BatchView& b, int grid, int mode, int only, cudaStream_t s, bool stage_field) {
  const size_t sm = pass_smem_bytes(b);
  if (b.weighted)
    launch_pass_w<true>(b, grid, mode, only, s, stage_field, sm);
  else
    launch_pass_w<false>(b, grid, mode, only, s, stage_field, sm);
}

void launch_collide(const BatchView& b, int grid, cudaStream_t s) {
  const size_t sm = sizeof(long long) * (size_t)(b.nseg + 1) + 3 * sizeof(int) * (size_t)b.nseg;
  set_smem_attr((const void*)k_collide, sm);
  k_collide<<<grid, kCollideBlock, sm, s>>>(b);
}

void launch_field(const BatchView& b, int advance, int only, cudaStream_t s) {
  const size_t sm = field_smem_bytes(b);
  set_smem_attr((const void*)k_field, sm);
  k_field<<<b.max_slots, kFieldBlock, sm, s>>>(b, advance, only);
}

void launch_phi(const BatchView& b, int slot, cudaStream_t s) {
  const size_t sm = field_smem_bytes(b);
  set_smem_attr((const void*)k_phi, sm);
  k_phi<<<1, kFieldBlock, sm, s>>>(b, slot);
}

// The scatter's grid: one wave of as many CTAs as fit on the device at its
// shared-memory size (every CTA takes an equal share of the particles, so a
// partial second wave would leave most SMs idle while it runs).
static int scatter_grid(size_t sms) {
  int dev = 0, nsm = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_scatter, kPassBlock, sms);
  return (occ > 0 ? occ : 1) * (nsm > 0 ? nsm : 1);
}

void launch_sort_phase(const BatchView& b, int grid, int phase, cudaStream_t s) {
  if (phase == 0) {
    const size_t smh = sizeof(long long) * (size_t)(b.nseg + 1) + sizeof(int) * (size_t)(b.nmax + 1);
    set_smem_attr((const void*)k_hist, smh);
    k_hist<<<grid, kPassBlock, smh, s>>>(b, MODE_SORT);
  } else if (phase == 1) {
    k_scan<<<b.nseg, kPassBlock, 0, s>>>(b, MODE_SORT);
  } else if (phase == 2) {
    const size_t sms = scatter_smem_bytes(b.nseg, b.nmax);
    set_smem_attr((const void*)k_scatter, sms);
    k_scatter<<<scatter_grid(sms), kPassBlock, sms, s>>>(b, MODE_SORT);
  } else {
    k_finalize<<<b.nseg, kPassBlock, 0, s>>>(b);
  }
}

void launch_sort(const BatchView& b, int grid, cudaStream_t s) {
  for (int ph = 0; ph < 4; ++ph) launch_sort_phase(b, grid, ph, s);
}

void launch_rebalance(const BatchView& b, int grid, cudaStream_t s) {
  const size_t smh = sizeof(long long) * (size_t)(b.nseg + 1) + sizeof(int) * (size_t)(b.nmax + 1);
  set_smem_attr((const void*)k_hist, smh);
  k_hist<<<grid, kPassBlock, smh, s>>>(b, MODE_REBAL);
  k_scan<<<b.nseg, kPassBlock, 0, s>>>(b, MODE_REBAL);
  const size_t sms = scatter_smem_bytes(b.nseg, b.nmax);
  set_smem_attr((const void*)k_scatter, sms);
  k_scatter<<<scatter_grid(sms), kPassBlock, sms, s>>>(b, MODE_REBAL);
  cudaMemsetAsync(b.rbnum, 0, sizeof(int), s);
  k_rb_classify<<<dim3((unsigned)((b.nmax + kPassBlock - 1) / kPassBlock), (unsigned)b.nseg), kPassBlock, 0,
                  s>>>(b);
  const size_t smr = sizeof(RbSmem);
  set_smem_attr((const void*)k_rb_cells, smr);
  k_rb_cells<<<grid, kRbBlock, smr, s>>>(b, 0);
  k_rb_scan<<<b.nseg, kPassBlock, 0, s>>>(b);
  // (a latency-bound stream: four times the persistent grid in flight)
  const size_t smc = sizeof(long long) * (size_t)(b.nseg + 1);
  set_smem_attr((const void*)k_rb_copy, smc);
  k_rb_copy<<<4 * grid, kPassBlock, smc, s>>>(b);
  k_rb_cells<<<grid, kRbBlock, smr, s>>>(b, 1);
  k_rb_finalize<<<b.nseg, kPassBlock, 0, s>>>(b);
  k_rb_mark<<<(b.max_slots + 127) / 128, 128, 0, s>>>(b);
}

void launch_init(const BatchView& b, int slot, const InitParams& p, cudaStream_t s) {
  long long nmax = 0;
  for (int i = 0; i < kMaxSpecies; ++i) nmax = p.n[i] > nmax ? p.n[i] : nmax;
  long long blocks = (nmax + 255) / 256;
  if (blocks < 1) blocks = 1;
  if (blocks > 4096) blocks = 4096;
  k_init<<<dim3((unsigned)blocks, kMaxSpecies), 256, 0, s>>>(b, slot, p);
}

void launch_init_many(const BatchView& b, const int* slots, const InitParams* ps, int count,
                      long long nmax, cudaStream_t s) {
  if (count <= 0) return;
  long long blocks = (nmax + 255) / 256;
  if (blocks < 1) blocks = 1;
  if (blocks > 4096) blocks = 4096;
  for (int off = 0; off < count; off += 65535) {
    const int c = count - off < 65535 ? count - off : 65535;
    k_init_many<<<dim3((unsigned)blocks, kMaxSpecies, (unsigned)c), 256, 0, s>>>(b, slots + off, ps + off, c);
  }
}

void launch_deposit_device(int N, long long n, const int* cell, const float* xi,
                           unsigned long long* S, cudaStream_t s) {
  long long blocks = (n + kPassBlock * 8 - 1) / (kPassBlock * 8);
  if (blocks < 1) blocks = 1;
  if (blocks > 304) blocks = 304;
  const size_t sm = 3 * sizeof(uint32_t) * (size_t)(N + 1);
  set_smem_attr((const void*)k_deposit_device, sm);
  k_deposit_device<<<(unsigned)blocks, kPassBlock, sm, s>>>(N, n, cell, xi, S);
}

void launch_deposit2_device(int N, int periodic, long long n, const int* cell, const float* xi,
                            unsigned long long* S, cudaStream_t s) {
  long long blocks = (n + 255) / 256;
  if (blocks < 1) blocks = 1;
  if (blocks > 1216) blocks = 1216;
  k_deposit2_device<<<(unsigned)blocks, 256, 0, s>>>(N, periodic, n, cell, xi, S);
  if (periodic) k_mirror_node<<<1, 1, 0, s>>>(N, S);
}

void launch_philox_device(long long n, const uint32_t* ctr, const uint32_t* key, uint32_t* out,
                          cudaStream_t s) {
  long long blocks = (n + 255) / 256;
  if (blocks < 1) blocks = 1;
  if (blocks > 4096) blocks = 4096;
  k_philox_device<<<(unsigned)blocks, 256, 0, s>>>(n, ctr, key, out);
}

}  // namespace ecpic

namespace ecpic {
void read_checks(unsigned long long out[4]) {
  cudaMemcpyFromSymbol(out, g_check, sizeof(unsigned long long) * 4);
}
}  // namespace ecpic
