// runtime.cu -- host runtime of libecpic (device memory, uploads, graphs).
#include "runtime.h"

#include <algorithm>
#include <utility>
#include <cfloat>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstddef>
#include <cstring>

namespace ecpic {

namespace {
constexpr double kQe = 1.602176634e-19;
constexpr double kKb = 1.380649e-23;
constexpr size_t kAlign = 256;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

struct Carve {
  char* base;
  size_t off = 0;
  template <typename T>
  T* take(size_t count) {
    T* p = reinterpret_cast<T*>(base + off);
    off += align_up(sizeof(T) * (count ? count : 1));
    return p;
  }
};

// Records (48 B) for the real collisions of one step: at most one per candidate,
// and the candidate count of n <= cap particles is binomial with the
// null-collision probability P; mean + 12 standard deviations + 256 is never
// exceeded in practice (an overflow fails the run with ECPIC_ERR_CAPACITY).
long long real_capacity(const HostSpecies& sp, const RunSpec& s) {
  double nu = 0.0;
  uint32_t thr = 0;
  null_rate(sp, s, &nu, &thr);
  if (thr == 0 || sp.cap <= 0) return 0;
  const double mean = (double)sp.cap * ((double)thr / 16777216.0);
  const double bound = std::ceil(mean + 12.0 * std::sqrt(mean) + 256.0);
  return bound < (double)sp.cap ? (long long)bound : (long long)sp.cap;
}

// Impact records per step: absorbed ions at x = 0 are few per step in a
// discharge; 4096 + cap/64 per species, the excess counted as dropped.
long long impact_capacity(const HostSpecies& sp) { return sp.q > 0.0 ? 4096 + sp.cap / 64 : 0; }

// cells whose centres lie within centre +- halfwidth, else the cell holding
// the centre (the EEDF region)
void eedf_cells(const RunSpec& s, int* c0, int* c1) {
  const size_t N = s.edges.size() - 1;
  const double L = s.edges[N];
  const double xc = s.eedf_center < 0.0 ? 0.5 * L : s.eedf_center;
  *c0 = (int)N;
  *c1 = -1;
  for (size_t j = 0; j < N; ++j) {
    const double cj = 0.5 * (s.edges[j] + s.edges[j + 1]);
    if (cj >= xc - s.eedf_halfwidth && cj <= xc + s.eedf_halfwidth) {
      *c0 = std::min(*c0, (int)j);
      *c1 = (int)j;
    }
  }
  if (*c0 > *c1) {
    const double x = xc < L ? xc : 0.0;
    size_t j = 0;
    while (j + 1 < N && s.edges[j + 1] <= x) ++j;
    *c0 = *c1 = (int)j;
  }
}

size_t layout_bytes(const RunSpec& s) {
  const size_t N = s.edges.size() - 1, ns = s.species.size();
  size_t b = 0;
  auto add = [&](size_t bytes) { b += align_up(bytes ? bytes : 1); };
  add(8 * (N + 1));       // x
  add(8 * N);             // dx
  add(8 * (N + 1));       // V
  add(8 * (N + 1));       // invV
  add(8 * (N + 1));       // mcw
  add(8 * (N + 1));       // cumV
  add(8 * N);             // g
  add(4 * N);             // dtdx
  add(4 * N);             // rp
  add(4 * N);             // rm
  add(4 * (N + 1));       // E
  add(8 * (N + 1));       // phi
  add(8 * ns * (N + 1));  // S
  add(8 * ns * 2 * (N + 1));  // momd
  add(8 * (size_t)acc_size((int)ns) * (N + 1));
  for (const auto& sp : s.species)
    if (!sp.procs.empty()) add(16 * sp.procs[0].sigma.size() * ((sp.procs.size() + 3) / 4));
  for (const auto& sp : s.species)
    for (int buf = 0; buf < 2; ++buf) {
      const size_t c = (size_t)sp.cap;
      add(4 * c); add(4 * c); add(4 * c); add(4 * c); add(4 * c); add(8 * c);
      if (s.rb) add(4 * c);  // weight multipliers
    }
  for (const auto& sp : s.species) add(sizeof(RealRec) * (size_t)real_capacity(sp, s));
  for (const auto& sp : s.species) add(sizeof(int) * (size_t)impact_capacity(sp));
  add(8 * ns * (size_t)(s.eedf_bins + s.iedf_bins + s.iad_bins));  // tallies
  add(8 * ns * N);                                                  // J.E sums
  return b;
}

// Pointers of every array of one run inside its device block, in a fixed
// order: the arrays that do not depend on the particle capacities come first
// (the host-built grid arrays and cross-section tables, ending at *data_end,
// then the field, deposit, accumulators and tallies that start from zero),
// so a block carved again with larger capacities keeps their offsets.  Sets
// the pointer fields of R and of the run's spc segment descriptors; returns
// the size of that capacity-independent prefix and, in *total, of the whole.
size_t carve_layout(const RunSpec& spec, char* base, RunDev* R, SegDev* segs, int spc,
                    size_t* total, size_t* data_end = nullptr) {
  Carve cv{base};
  const size_t N = spec.edges.size() - 1, ns = spec.species.size();
  // uploaded from the host: grid, cell-walk factors, cross-section tables
  R->x = cv.take<double>(N + 1);
  R->dx = cv.take<double>(N);
  R->V = cv.take<double>(N + 1);
  R->invV = cv.take<double>(N + 1);
  R->mcw = cv.take<double>(N + 1);
  R->cumV = cv.take<double>(N + 1);
  R->dtdx = cv.take<float>(N);
  R->rp = cv.take<float>(N);
  R->rm = cv.take<float>(N);
  for (size_t s = 0; s < ns; ++s) {
    const HostSpecies& hs = spec.species[s];
    R->sp[s].sig4 = nullptr;
    if (!hs.procs.empty())
      R->sp[s].sig4 = cv.take<float4>(hs.procs[0].sigma.size() * ((hs.procs.size() + 3) / 4));
  }
  if (data_end) *data_end = cv.off;
  // starting from zero: field, deposit, moments, accumulators, tallies
  R->g = cv.take<double>(N);
  R->E = cv.take<float>(N + 1);
  R->phi = cv.take<double>(N + 1);
  R->S = cv.take<unsigned long long>(ns * (N + 1));
  R->momd = cv.take<double>(ns * 2 * (N + 1));
  R->acc = cv.take<double>((size_t)acc_size((int)ns) * (N + 1));
  R->mom = nullptr;
  R->tal = cv.take<unsigned long long>(ns * (size_t)(spec.eedf_bins + spec.iedf_bins + spec.iad_bins));
  R->pw = cv.take<double>(ns * N);
  const size_t prefix = cv.off;
  for (int s = 0; s < spc; ++s) {
    SegDev& G = segs[s];
    if (s < (int)ns) {
      const size_t c = (size_t)spec.species[s].cap;
      for (int buf = 0; buf < 2; ++buf) {
        G.cell[buf] = cv.take<int32_t>(c);
        G.xi[buf] = cv.take<float>(c);
        G.vx[buf] = cv.take<float>(c);
        G.vy[buf] = cv.take<float>(c);
        G.vz[buf] = cv.take<float>(c);
        G.id[buf] = cv.take<uint64_t>(c);
        G.wt[buf] = spec.rb ? cv.take<uint32_t>(c) : nullptr;
      }
      G.cap = (long long)c;
    } else {
      std::memset(G.cell, 0, sizeof(G.cell));
      std::memset(G.xi, 0, sizeof(G.xi));
      std::memset(G.vx, 0, sizeof(G.vx));
      std::memset(G.vy, 0, sizeof(G.vy));
      std::memset(G.vz, 0, sizeof(G.vz));
      std::memset(G.id, 0, sizeof(G.id));
      std::memset(G.wt, 0, sizeof(G.wt));
      G.cap = 0;
    }
    G.real = nullptr;
    G.real_cap = 0;
    G.imp = nullptr;
    G.imp_cap = 0;
  }
  for (size_t s = 0; s < ns; ++s) {
    SegDev& G = segs[s];
    G.real_cap = real_capacity(spec.species[s], spec);
    G.real = cv.take<RealRec>((size_t)G.real_cap);
    G.imp_cap = impact_capacity(spec.species[s]);
    G.imp = cv.take<int>((size_t)G.imp_cap);
  }
  *total = cv.off;
  return prefix;
}
}  // namespace

std::string validate_grid(const std::vector<double>& e, int bc) {
  if (e.size() < 3) return "need at least 2 cells";
  if (e.size() - 1 > (size_t)kMaxCells) return "too many cells (max ECPIC_MAX_CELLS)";
  if (e[0] != 0.0) return "edges[0] must be 0";
  for (size_t i = 1; i < e.size(); ++i)
    if (!(e[i] > e[i - 1]) || !std::isfinite(e[i])) return "edges must be finite and strictly increasing";
  if (bc != ECPIC_DIRICHLET_RF && bc != ECPIC_PERIODIC) return "unknown boundary condition";
  return "";
}

std::string validate_tallies(const RunSpec& s) {
  if (!(s.eedf_halfwidth >= 0.0) || !std::isfinite(s.eedf_center) || !std::isfinite(s.eedf_halfwidth))
    return "bad EEDF region";
  if (!(s.eedf_dE > 0.0) || !(s.iedf_dE > 0.0)) return "tally bin widths must be positive";
  if (s.eedf_bins < 1 || s.iedf_bins < 1 || s.iad_bins < 1 || s.eedf_bins > 65536 ||
      s.iedf_bins > 65536 || s.iad_bins > 65536)
    return "tally bin counts must be 1..65536";
  return "";
}

std::string validate_spec(const RunSpec& s) {
  {
    const std::string t = validate_tallies(s);
    if (!t.empty()) return t;
  }
  std::string e = validate_grid(s.edges, s.bc);
  if (!e.empty()) return e;
  if (s.scheme < ECPIC_SCHEME_EC || s.scheme > ECPIC_SCHEME_MC2) return "unknown scheme";
  if (s.scheme >= ECPIC_SCHEME_EC2) {
    const double dx0 = s.edges[1] - s.edges[0];
    for (size_t j = 1; j + 1 < s.edges.size(); ++j)
      if (std::fabs((s.edges[j + 1] - s.edges[j]) - dx0) > 1e-9 * dx0)
        return "the EC2 and MC2 schemes need a uniform grid";
  }
  if (s.species.empty() || s.species.size() > (size_t)kMaxSpecies) return "1..4 species required";
  if (s.rb) {
    if (s.scheme != ECPIC_SCHEME_EC && s.scheme != ECPIC_SCHEME_MC)
      return "particle rebalancing needs the EC or MC scheme";
    if (s.rb_every < 0 || s.rb_target < 1 || s.rb_target > kRbMaxCell || s.rb_lo < 0 ||
        s.rb_lo > s.rb_target || s.rb_hi < s.rb_target || s.rb_m0 < 1 || s.rb_m0 > kRbMaxWeight)
      return "bad rebalancing parameters (0 <= lo <= target <= hi, target <= 4096, 1 <= m0 <= 65536)";
  }
  if (!(s.dt > 0) || !std::isfinite(s.dt)) return "dt must be positive";
  if (s.n_init.size() != s.species.size() || s.T_eV.size() != s.species.size())
    return "n_per_species/T_eV size mismatch";
  for (size_t i = 0; i < s.species.size(); ++i) {
    const auto& sp = s.species[i];
    if (!(sp.m > 0) || !(sp.w >= 0) || sp.cap < 1 || sp.cap > (long long)INT32_MAX)
      return "bad species parameters";
    if (s.n_init[i] < 0 || s.n_init[i] > sp.cap) return "initial particles exceed capacity";
    if (!(s.T_eV[i] >= 0)) return "negative temperature";
    if (sp.procs.size() > (size_t)kMaxProc) return "too many processes";
    for (const auto& p : sp.procs) {
      if (p.kind < ECPIC_ELASTIC || p.kind > ECPIC_CX) return "unknown process kind";
      if (p.sigma.size() < 2 || !(p.dE > 0) || !(p.thr >= 0)) return "bad cross-section table";
      if (p.dE != sp.procs[0].dE || p.sigma.size() != sp.procs[0].sigma.size())
        return "processes of one species must share the energy grid";
      const bool heavy = p.kind == ECPIC_ION_ELASTIC || p.kind == ECPIC_CX;
      const bool heavy0 = sp.procs[0].kind == ECPIC_ION_ELASTIC || sp.procs[0].kind == ECPIC_CX;
      if (heavy != heavy0) return "electron and ion processes mixed in one species";
      if (p.kind == ECPIC_IONIZATION &&
          (p.product < 0 || p.product >= (int)s.species.size() || p.product == (int)i))
        return "ionisation needs a product ion species";
      for (float v : p.sigma)
        if (!(v >= 0.0f) || !std::isfinite(v)) return "cross sections must be finite and >= 0";
    }
    if (!sp.procs.empty() && !(s.gas && s.mg > 0)) return "collisions need a gas";
  }
  return "";
}

void null_rate(const HostSpecies& sp, const RunSpec& s, double* nu_max, uint32_t* thr24) {
  *nu_max = 0.0;
  *thr24 = 0;
  if (sp.procs.empty() || !s.gas || !(s.ng > 0)) return;
  // per table segment: n_g * max(sigma_tot at both ends) * speed at the upper end
  const size_t n = sp.procs[0].sigma.size();
  const double dE = sp.procs[0].dE;
  double best = 0.0;
  for (size_t i = 0; i + 1 < n; ++i) {
    double a = 0.0, b = 0.0;
    for (const auto& p : sp.procs) {
      a += (double)p.sigma[i];
      b += (double)p.sigma[i + 1];
    }
    const double sig = a > b ? a : b;
    const double v = std::sqrt(2.0 * (double)(i + 1) * dE * kQe / sp.m);
    if (sig * v > best) best = sig * v;
  }
  *nu_max = s.ng * best;
  const double P = 1.0 - std::exp(-(*nu_max) * s.dt);
  double t = std::ceil(P * 16777216.0);
  if (t > 16777216.0) t = 16777216.0;
  *thr24 = (uint32_t)t;
}

size_t run_bytes(const RunSpec& s) { return layout_bytes(s); }

void fill_diag(const Diag& d, const RunSpec& spec, ecpic_diag* out) {
  const int N = d.N, ns = d.ns;
  out->step = d.st.step;
  out->time = (double)d.st.step * spec.dt;
  out->n_species = ns;
  out->n_cells = N;
  for (int s = 0; s < kMaxSpecies; ++s) {
    out->n_live[s] = s < ns ? d.n_live[s] : 0;
    out->ke[s] = s < ns ? d.st.ke[s] : 0.0;
    const unsigned long long* c = d.st.ctr[s];
    out->absorbed[s][0] = (int64_t)c[C_ABS_L];
    out->absorbed[s][1] = (int64_t)c[C_ABS_R];
    out->births[s] = (int64_t)c[C_BIRTHS];
    out->lost[s] = (int64_t)c[C_LOST];
    out->candidates[s] = (int64_t)c[C_CAND];
    out->clamps[s] = (int64_t)c[C_CLAMPS];
    for (int p = 0; p < kMaxProc; ++p) out->collisions[s][p] = (int64_t)c[C_COLL0 + p];
    out->rb_merged[s] = (int64_t)c[C_RB_MERGED];
    out->rb_split[s] = (int64_t)c[C_RB_SPLIT];
    out->rb_skipped[s] = (int64_t)c[C_RB_SKIPPED];
  }
  out->fe = d.st.fe;
  out->n_samples = d.st.n_samples;
  const double inv = d.st.n_samples > 0 ? 1.0 / (double)d.st.n_samples : 0.0;
  const size_t M = (size_t)N + 1;
  if (d.acc.size() < (size_t)acc_size(ns) * M) return;
  for (int s = 0; s < ns; ++s)
    for (size_t n = 0; n < M; ++n) {
      if (out->density) out->density[s * M + n] = d.acc[s * M + n] * inv;
      if (out->temp_x) out->temp_x[s * M + n] = d.acc[(ns + s) * M + n] * inv;
      if (out->temp_x_mom) {
        const double M0 = d.acc[(2 * ns + s) * M + n];
        double T = 0.0;
        if (M0 > 0) {
          const double a = d.acc[(3 * ns + s) * M + n] / M0, b = d.acc[(4 * ns + s) * M + n] / M0;
          T = spec.species[s].m * (b - a * a) / kQe;
        }
        out->temp_x_mom[s * M + n] = T;
      }
    }
  if (out->phi)
    for (size_t n = 0; n < M; ++n) out->phi[n] = d.acc[(size_t)(5 * ns) * M + n] * inv;
  // tallies
  out->eedf_bins = spec.eedf_bins;
  out->iedf_bins = spec.iedf_bins;
  out->iad_bins = spec.iad_bins;
  out->eedf_cell0 = d.eedf_c0;
  out->eedf_cell1 = d.eedf_c1;
  out->eedf_dE = spec.eedf_dE;
  out->iedf_dE = spec.iedf_dE;
  for (int s = 0; s < kMaxSpecies; ++s)
    out->impacts_dropped[s] = s < ns ? (int64_t)d.st.ctr[s][C_IMP_LOST] : 0;
  const size_t stride = (size_t)spec.eedf_bins + spec.iedf_bins + spec.iad_bins;
  if (d.tal.size() < (size_t)ns * stride || d.pw.size() < (size_t)ns * N) return;
  for (int s = 0; s < ns; ++s) {
    const unsigned long long* t = d.tal.data() + s * stride;
    for (int b = 0; b < spec.eedf_bins; ++b)
      if (out->eedf) out->eedf[(size_t)s * spec.eedf_bins + b] = (double)t[b];
    for (int b = 0; b < spec.iedf_bins; ++b)
      if (out->iedf) out->iedf[(size_t)s * spec.iedf_bins + b] = (double)t[spec.eedf_bins + b];
    for (int b = 0; b < spec.iad_bins; ++b)
      if (out->iad) out->iad[(size_t)s * spec.iad_bins + b] = (double)t[spec.eedf_bins + spec.iedf_bins + b];
    // J.E = q w (v^- + v^+)/2 E_i / dx_j, summed per sample, mean over samples
    const double qw = spec.species[s].q * base_weight(spec, s);
    for (int j = 0; j < N && out->power; ++j)
      out->power[(size_t)s * N + j] =
          0.5 * qw * d.pw[(size_t)s * N + j] / (spec.edges[j + 1] - spec.edges[j]) * inv;
  }
}

// ------------------------------------------------------------------ Batch
Batch::Batch(int device, cudaStream_t stream, int max_slots, int spc, int nmax)
    : device_(device), stream_(stream), max_slots_(max_slots), spc_(spc), nmax_(nmax) {
  nseg_ = max_slots_ * spc_;
  cudaSetDevice(device_);
  if (!stream_) {
    cudaStreamCreateWithFlags(&stream_, cudaStreamNonBlocking);
    own_stream_ = true;
  }
  cudaDeviceGetAttribute(&sm_count_, cudaDevAttrMultiProcessorCount, device_);
  // freed run blocks stay in the device's stream-ordered pool for the next
  // admissions instead of going back to the driver at each synchronisation
  {
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device_) == cudaSuccess) {
      uint64_t keep = UINT64_MAX;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    cudaGetLastError();
  }
  cudaMalloc(&d_runs_, sizeof(RunDev) * max_slots_);
  cudaMalloc(&d_rst_, sizeof(RunState) * max_slots_);
  cudaMalloc(&d_segs_, sizeof(SegDev) * nseg_);
  cudaMalloc(&d_sst_, sizeof(SegState) * nseg_);
  cudaMalloc(&d_hist_, sizeof(int) * (size_t)nseg_ * nmax_);
  cudaMalloc(&d_rbcnt_, sizeof(int) * (size_t)nseg_ * nmax_);
  cudaMalloc(&d_rbmode_, (size_t)nseg_ * nmax_);
  cudaMalloc(&d_rblist_, sizeof(int) * (size_t)nseg_ * nmax_);
  cudaMalloc(&d_rbnum_, sizeof(int));
  cudaMalloc(&d_wave_slots_, sizeof(int) * max_slots_);
  cudaMalloc(&d_wave_params_, sizeof(InitParams) * max_slots_);
  level_.assign(max_slots_, 0);
  h_runs_.assign(max_slots_, RunDev{});
  h_segs_.assign(nseg_, SegDev{});
  wave_sst_.assign(nseg_, SegState{});
  wave_rst_.assign(max_slots_, RunState{});
  for (int s = 0; s < nseg_; ++s) {
    h_segs_[s].run = s / spc_;
    h_segs_[s].species = s % spc_;
    h_segs_[s].hoff = s * nmax_;
  }
  cudaMemsetAsync(d_runs_, 0, sizeof(RunDev) * max_slots_, stream_);
  cudaMemsetAsync(d_rst_, 0, sizeof(RunState) * max_slots_, stream_);
  cudaMemsetAsync(d_sst_, 0, sizeof(SegState) * nseg_, stream_);
  cudaMemsetAsync(d_hist_, 0, sizeof(int) * (size_t)nseg_ * nmax_, stream_);
  cudaMemsetAsync(d_rbcnt_, 0, sizeof(int) * (size_t)nseg_ * nmax_, stream_);
  cudaMemsetAsync(d_rbmode_, 0, (size_t)nseg_ * nmax_, stream_);
  cudaMemsetAsync(d_rbnum_, 0, sizeof(int), stream_);
  cudaMemcpyAsync(d_segs_, h_segs_.data(), sizeof(SegDev) * nseg_, cudaMemcpyHostToDevice, stream_);
  slot_mem_.assign(max_slots_, nullptr);
  slot_bytes_.assign(max_slots_, 0);
  active_.assign(max_slots_, 0);
  specs_.assign(max_slots_, RunSpec{});
  cudaStreamSynchronize(stream_);
}

Batch::~Batch() {
  cudaSetDevice(device_);
  cudaStreamSynchronize(stream_);
  if (stage_ring_) {
    for (int k = 0; k < kStageSlots; ++k) cudaEventDestroy(stage_ev_[k]);
    cudaFreeHost(stage_ring_);
  }
  invalidate_graphs();
  for (int s = 0; s < max_slots_; ++s)
    if (slot_mem_[s]) cudaFree(slot_mem_[s]);
  cudaFree(d_runs_);
  cudaFree(d_rst_);
  cudaFree(d_segs_);
  cudaFree(d_sst_);
  cudaFree(d_hist_);
  cudaFree(d_rbcnt_);
  cudaFree(d_rbmode_);
  cudaFree(d_rblist_);
  cudaFree(d_rbnum_);
  cudaFree(d_wave_slots_);
  cudaFree(d_wave_params_);
  if (own_stream_) cudaStreamDestroy(stream_);
}

int Batch::check(cudaError_t e, const char* what, std::string* err) {
  if (e == cudaSuccess) return ECPIC_OK;
  if (err) *err = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? ECPIC_ERR_NOMEM : ECPIC_ERR_CUDA;
}

char* Batch::stage_slot(size_t bytes, int* slot) {
  *slot = -1;
  if (bytes > kStageBytes) return nullptr;
  if (!stage_ring_) {
    if (cudaMallocHost(&stage_ring_, kStageSlots * kStageBytes) != cudaSuccess) {
      cudaGetLastError();
      stage_ring_ = nullptr;
      return nullptr;  // the caller falls back to pageable memory
    }
    for (int k = 0; k < kStageSlots; ++k) cudaEventCreateWithFlags(&stage_ev_[k], cudaEventDisableTiming);
  }
  const int k = stage_next_;
  stage_next_ = (stage_next_ + 1) % kStageSlots;
  if (stage_used_[k]) cudaEventSynchronize(stage_ev_[k]);  // its last copy has left
  stage_used_[k] = false;
  *slot = k;
  return stage_ring_ + (size_t)k * kStageBytes;
}

void Batch::stage_done(int slot) {
  if (slot < 0) return;
  cudaEventRecord(stage_ev_[slot], stream_);
  stage_used_[slot] = true;
}

BatchView Batch::view() const {
  BatchView v;
  v.runs = d_runs_;
  v.rst = d_rst_;
  v.segs = d_segs_;
  v.sst = d_sst_;
  v.hist = d_hist_;
  v.rbcnt = d_rbcnt_;
  v.rbmode = d_rbmode_;
  v.rblist = d_rblist_;
  v.rbnum = d_rbnum_;
  v.max_slots = max_slots_;
  v.nseg = nseg_;
  v.nmax = nmax_;
  v.weighted = 0;
  for (int s = 0; s < max_slots_; ++s)
    if (active_[s] && specs_[s].rb) v.weighted = 1;
  return v;
}

void Batch::upload_run(int slot) {
  cudaMemcpyAsync(d_runs_ + slot, &h_runs_[slot], sizeof(RunDev), cudaMemcpyHostToDevice, stream_);
}

int Batch::admit(int slot, const RunSpec& spec, std::string* err, bool defer) {
  if (slot < 0 || slot >= max_slots_ || active_[slot]) {
    if (err) *err = "slot unavailable";
    return ECPIC_ERR_STATE;
  }
  // the spec was validated by its caller (ecpic_init, ecpic_engine_submit)
  const int N = (int)spec.edges.size() - 1, ns = (int)spec.species.size();
  if (N > nmax_ || ns > spc_) {
    if (err) *err = "run exceeds the batch's cell or species limits";
    return ECPIC_ERR_ARG;
  }
  cudaSetDevice(device_);
  const size_t bytes = layout_bytes(spec);
  void* mem = nullptr;
  int rc = check(cudaMallocAsync(&mem, bytes, stream_), "device allocation", err);
  if (rc) return rc;
  RunDev R{};
  size_t total = 0;
  size_t data_end = 0;
  const size_t prefix = carve_layout(spec, static_cast<char*>(mem), &R, &h_segs_[slot * spc_], spc_,
                                     &total, &data_end);
  // the host-built arrays are assembled in pinned staging memory and uploaded
  // in one asynchronous copy; the arrays that start from zero are one memset
  int ks = -1;
  char* img = stage_slot(data_end, &ks);
  std::vector<char> img_pageable;
  if (!img) {
    img_pageable.resize(data_end);
    img = img_pageable.data();
  }
  auto put = [&](const void* dev, const void* host, size_t nbytes) {
    std::memcpy(img + (static_cast<const char*>(dev) - static_cast<const char*>(mem)), host, nbytes);
  };
  if (total > bytes) {
    cudaFreeAsync(mem, stream_);
    if (err) *err = "internal: run layout exceeds its block";
    return ECPIC_ERR_CUDA;
  }
  R.active = 1;
  R.N = N;
  R.bc = spec.bc;
  R.scheme = spec.scheme;
  R.ns = ns;
  R.seg0 = slot * spc_;
  R.sample_every = spec.sample_every;
  R.rb = spec.rb ? 1 : 0;
  R.rb_every = spec.rb ? spec.rb_every : 0;
  R.rb_target = spec.rb_target;
  R.rb_lo = spec.rb_lo;
  R.rb_hi = spec.rb_hi;
  R.L = spec.edges[N];
  R.dt = spec.dt;
  R.v0 = spec.v0;
  R.freq = spec.freq;
  R.phase = spec.phase;
  R.vdc = spec.vdc;
  R.seed = spec.seed;
  R.ng = (float)(spec.gas ? spec.ng : 0.0);
  R.vth_gas = (float)(spec.gas && spec.mg > 0 ? std::sqrt(kKb * spec.Tg / spec.mg) : 0.0);
  // grid arrays
  std::vector<double> dx(N), V(N + 1);
  std::vector<float> dtdx(N), rp(N), rm(N);
  for (int j = 0; j < N; ++j) dx[j] = spec.edges[j + 1] - spec.edges[j];
  for (int n = 1; n < N; ++n) V[n] = 0.5 * (dx[n - 1] + dx[n]);
  if (spec.bc == ECPIC_PERIODIC) {
    V[0] = V[N] = 0.5 * (dx[N - 1] + dx[0]);
  } else {
    V[0] = 0.5 * dx[0];
    V[N] = 0.5 * dx[N - 1];
  }
  const double dxu = R.L / N;
  bool uniform = true;
  for (int j = 0; j < N; ++j) {
    if (std::fabs(dx[j] - dxu) > 1e-12 * dxu) uniform = false;
    dtdx[j] = (float)(spec.dt / dx[j]);
    const int jp = (j + 1 < N) ? j + 1 : (spec.bc == ECPIC_PERIODIC ? 0 : j);
    const int jm = (j > 0) ? j - 1 : (spec.bc == ECPIC_PERIODIC ? N - 1 : j);
    rp[j] = (float)(dx[j] / dx[jp]);
    rm[j] = (float)(dx[j] / dx[jm]);
  }
  R.uniform = uniform ? 1 : 0;
  R.dtdx_u = (float)(spec.dt / dxu);
  double* d_x = const_cast<double*>(R.x);
  double* d_dx = const_cast<double*>(R.dx);
  double* d_V = const_cast<double*>(R.V);
  double* d_invV = const_cast<double*>(R.invV);
  double* d_mcw = const_cast<double*>(R.mcw);
  double* d_cumV = const_cast<double*>(R.cumV);
  float* d_dtdx = const_cast<float*>(R.dtdx);
  float* d_rp = const_cast<float*>(R.rp);
  float* d_rm = const_cast<float*>(R.rm);
  R.eedf_n = spec.eedf_bins;
  R.iedf_n = spec.iedf_bins;
  R.iad_n = spec.iad_bins;
  R.tal_stride = spec.eedf_bins + spec.iedf_bins + spec.iad_bins;
  eedf_cells(spec, &R.eedf_c0, &R.eedf_c1);
  R.eedf_dEinv = (float)(1.0 / spec.eedf_dE);
  R.iedf_dEinv = (float)(1.0 / spec.iedf_dE);
  R.iad_binv = (float)(spec.iad_bins / 90.0);
  R.inv_L = 1.0 / R.L;
  put(d_x, spec.edges.data(), 8 * (N + 1));
  put(d_dx, dx.data(), 8 * N);
  put(d_V, V.data(), 8 * (N + 1));
  std::vector<double> invV(N + 1), mcw(N + 1, 0.5);
  for (int n = 0; n <= N; ++n) invV[n] = 1.0 / V[n];
  for (int n = 1; n < N; ++n) mcw[n] = dx[n] / (dx[n - 1] + dx[n]);
  if (spec.bc == ECPIC_PERIODIC) mcw[0] = mcw[N] = dx[0] / (dx[N - 1] + dx[0]);
  put(d_invV, invV.data(), 8 * (N + 1));
  put(d_mcw, mcw.data(), 8 * (N + 1));
  std::vector<double> cumV(N + 1, 0.0);
  for (int n = 1; n <= N; ++n) cumV[n] = cumV[n - 1] + V[n];
  put(d_cumV, cumV.data(), 8 * (N + 1));
  put(d_dtdx, dtdx.data(), 4 * N);
  put(d_rp, rp.data(), 4 * N);
  put(d_rm, rm.data(), 4 * N);
  // species
  for (int s = 0; s < ns; ++s) {
    const HostSpecies& hs = spec.species[s];
    SpeciesDev& D = R.sp[s];
    D.q = hs.q;
    D.m = hs.m;
    D.w = base_weight(spec, s);
    D.cw = hs.q * D.w * 2.3283064365386963e-10;  // 2^-32
    D.qm_dt = (float)(hs.q / hs.m * spec.dt);
    D.half_m_over_e = (float)(0.5 * hs.m / kQe);
    D.two_e_over_m = (float)(2.0 * kQe / hs.m);
    const double mg = spec.gas && spec.mg > 0 ? spec.mg : 1.0;
    D.two_m_over_M = (float)(2.0 * hs.m / mg);
    D.m_frac = (float)(mg / (hs.m + mg));
    D.mass_frac = (float)(hs.m / (hs.m + mg));
    double nu;
    uint32_t thr;
    null_rate(hs, spec, &nu, &thr);
    D.nu_max = (float)nu;
    D.thr24 = thr;
    D.nproc = (int)hs.procs.size();
    D.heavy = 0;
    D.ntab = hs.procs.empty() ? 2 : (int)hs.procs[0].sigma.size();
    D.dE_inv = hs.procs.empty() ? 1.0f : (float)(1.0 / hs.procs[0].dE);
    {
      double smax = 0.0;
      for (size_t i = 0; !hs.procs.empty() && i < hs.procs[0].sigma.size(); ++i) {
        double a = 0.0;
        for (const auto& hp : hs.procs) a += (double)hp.sigma[i];
        smax = a > smax ? a : smax;
      }
      D.nu_bnd = (float)((spec.gas ? spec.ng : 0.0) * smax * (1.0 + 1.0 / 65536.0));
    }
    D.np4 = (D.nproc + 3) / 4;
    for (int p = 0; p < kMaxProc; ++p) D.thr_all[p] = FLT_MAX;
    if (D.nproc > 0) {
      // node-major interleaving: one 16-byte load per node serves four processes
      const size_t nt = (size_t)D.ntab, g4 = (size_t)D.np4;
      std::vector<float> il(nt * g4 * 4, 0.0f);
      for (int p = 0; p < D.nproc; ++p)
        for (size_t i = 0; i < nt; ++i) il[(i * g4 + p / 4) * 4 + p % 4] = hs.procs[p].sigma[i];
      put(D.sig4, il.data(), 16 * nt * g4);
    }
    for (int p = 0; p < D.nproc; ++p) {
      const HostProc& hp = hs.procs[p];
      ProcDev& P = D.proc[p];
      P.kind = hp.kind;
      P.thr = (float)hp.thr;
      D.thr_all[p] = P.thr;
      P.product_species = hp.kind == ECPIC_IONIZATION ? hp.product : -1;
      P.product_seg = hp.kind == ECPIC_IONIZATION ? R.seg0 + hp.product : -1;
      if (hp.kind == ECPIC_ION_ELASTIC || hp.kind == ECPIC_CX) D.heavy = 1;
    }
  }
  // field solve: species whose q w are equal up to sign share one signed
  // integer sum of their deposits per node
  R.field_pm = 1;
  R.field_neg = 0;
  for (int s = 0; s < ns; ++s) {
    const double a = R.sp[s].q * R.sp[s].w, a0 = R.sp[0].q * R.sp[0].w;
    if (a == a0) continue;
    if (a == -a0) R.field_neg |= 1 << s;
    else R.field_pm = 0;
  }
  // particle segments
  std::vector<SegState> sst(spc_);
  for (int s = 0; s < spc_; ++s) {
    std::memset(sst.data() + s, 0, sizeof(SegState));
    if (s < ns) sst[s].n_proc = sst[s].n_alloc = spec.n_init[s];
  }
  cudaMemcpyAsync(mem, img, data_end, cudaMemcpyHostToDevice, stream_);
  stage_done(ks);
  cudaMemsetAsync(static_cast<char*>(mem) + data_end, 0, prefix - data_end, stream_);
  RunState st{};
  st.step = 0;
  st.step_end = spec.step_end;
  st.rb_level = -1;
  st.fresh = defer ? 1 : 0;
  level_[slot] = 0;
  h_runs_[slot] = R;
  if (defer) {
    // the slot's tables, states and cell arrays go up with its wave
    std::copy(sst.begin(), sst.end(), wave_sst_.begin() + (size_t)slot * spc_);
    wave_rst_[slot] = st;
  } else {
    cudaMemcpyAsync(d_segs_ + R.seg0, &h_segs_[R.seg0], sizeof(SegDev) * spc_, cudaMemcpyHostToDevice,
                    stream_);
    cudaMemcpyAsync(d_sst_ + R.seg0, sst.data(), sizeof(SegState) * spc_, cudaMemcpyHostToDevice,
                    stream_);
    // the slot's cell arrays start from zero whatever its last run left
    cudaMemsetAsync(d_hist_ + (size_t)slot * spc_ * nmax_, 0, sizeof(int) * (size_t)spc_ * nmax_,
                    stream_);
    cudaMemsetAsync(d_rbcnt_ + (size_t)slot * spc_ * nmax_, 0, sizeof(int) * (size_t)spc_ * nmax_,
                    stream_);
    cudaMemcpyAsync(d_rst_ + slot, &st, sizeof(RunState), cudaMemcpyHostToDevice, stream_);
    upload_run(slot);
  }
  slot_mem_[slot] = mem;
  slot_bytes_[slot] = bytes;
  bytes_in_use_ += bytes;
  active_[slot] = 1;
  specs_[slot] = spec;
  // particles and the field of step 0
  InitParams ip{};
  ip.quiet = spec.quiet;
  ip.rb_m0 = spec.rb ? spec.rb_m0 : 1u;
  for (int s = 0; s < ns; ++s) {
    ip.n[s] = spec.n_init[s];
    ip.sd[s] = std::sqrt(kQe * spec.T_eV[s] / spec.species[s].m);
  }
  if (defer) {
    wave_slots_.push_back(slot);
    wave_params_.push_back(ip);
    return ECPIC_OK;
  }
  launch_init(view(), slot, ip, stream_);
  refresh(slot);
  return check(cudaGetLastError(), "admit", err);
}

int Batch::admit_wave(std::string* err) {
  const int count = (int)wave_slots_.size();
  if (count == 0) return ECPIC_OK;
  cudaSetDevice(device_);
  long long nmax = 0;
  for (const InitParams& p : wave_params_)
    for (int s = 0; s < kMaxSpecies; ++s) nmax = std::max(nmax, p.n[s]);
  // the wave's run tables, segment tables and states, and zeroed cell
  // arrays, one copy per contiguous range of slots (pageable sources: each
  // copy has left them when the call returns)
  std::vector<int> sl = wave_slots_;
  std::sort(sl.begin(), sl.end());
  int rc = ECPIC_OK;
  for (size_t i = 0; i < sl.size() && !rc;) {
    size_t j = i + 1;
    while (j < sl.size() && sl[j] == sl[j - 1] + 1) ++j;
    const size_t a = (size_t)sl[i], n = (size_t)(sl[j - 1] - sl[i] + 1), sa = a * spc_, sn = n * spc_;
    rc = check(cudaMemcpyAsync(d_runs_ + a, &h_runs_[a], sizeof(RunDev) * n, cudaMemcpyHostToDevice,
                               stream_), "wave upload", err);
    if (!rc)
      rc = check(cudaMemcpyAsync(d_rst_ + a, &wave_rst_[a], sizeof(RunState) * n,
                                 cudaMemcpyHostToDevice, stream_), "wave upload", err);
    if (!rc)
      rc = check(cudaMemcpyAsync(d_segs_ + sa, &h_segs_[sa], sizeof(SegDev) * sn,
                                 cudaMemcpyHostToDevice, stream_), "wave upload", err);
    if (!rc)
      rc = check(cudaMemcpyAsync(d_sst_ + sa, &wave_sst_[sa], sizeof(SegState) * sn,
                                 cudaMemcpyHostToDevice, stream_), "wave upload", err);
    if (!rc)
      rc = check(cudaMemsetAsync(d_hist_ + sa * nmax_, 0, sizeof(int) * sn * nmax_, stream_),
                 "wave upload", err);
    if (!rc)
      rc = check(cudaMemsetAsync(d_rbcnt_ + sa * nmax_, 0, sizeof(int) * sn * nmax_, stream_),
                 "wave upload", err);
    i = j;
  }
  if (!rc)
    rc = check(cudaMemcpyAsync(d_wave_slots_, wave_slots_.data(), sizeof(int) * count,
                               cudaMemcpyHostToDevice, stream_), "wave upload", err);
  if (!rc)
    rc = check(cudaMemcpyAsync(d_wave_params_, wave_params_.data(), sizeof(InitParams) * count,
                               cudaMemcpyHostToDevice, stream_), "wave upload", err);
  wave_slots_.clear();
  wave_params_.clear();
  if (rc) return rc;
  const BatchView b = view();
  launch_init_many(b, d_wave_slots_, d_wave_params_, count, nmax, stream_);
  launch_pass(b, std::max(1, choose_grid()), MODE_REFRESH, kOnlyFresh, stream_, false);
  launch_field(b, 0, kOnlyFresh, stream_);
  return check(cudaGetLastError(), "admission wave", err);
}

void Batch::refresh(int slot) {
  const BatchView b = view();
  launch_pass(b, std::max(1, std::min(choose_grid(), sm_count_ * 2)), MODE_REFRESH, slot, stream_, false);
  launch_field(b, 0, slot, stream_);
}

int Batch::reserve(int slot, const long long* cap, std::string* err) {
  if (!slot_active(slot)) {
    if (err) *err = "no run in this slot";
    return ECPIC_ERR_STATE;
  }
  RunSpec spec = specs_[slot];
  const int ns = (int)spec.species.size();
  bool grow = false;
  for (int s = 0; s < ns; ++s)
    if (cap[s] > spec.species[s].cap) {
      if (cap[s] > (long long)INT32_MAX) {
        if (err) *err = "capacity above 2^31 - 1 particles";
        return ECPIC_ERR_ARG;
      }
      spec.species[s].cap = cap[s];
      grow = true;
    }
  if (!grow) return ECPIC_OK;
  cudaSetDevice(device_);
  const int seg0 = slot * spc_;
  // the run's sizes and current buffer set (between steps)
  std::vector<SegState> sst(spc_);
  int rc = check(cudaMemcpyAsync(sst.data(), d_sst_ + seg0, sizeof(SegState) * spc_,
                                 cudaMemcpyDeviceToHost, stream_), "read sizes", err);
  if (rc) return rc;
  rc = check(cudaStreamSynchronize(stream_), "read sizes", err);
  if (rc) return rc;
  const size_t bytes = layout_bytes(spec);
  void* mem = nullptr;
  rc = check(cudaMallocAsync(&mem, bytes, stream_), "device allocation", err);
  if (rc) return rc;  // the run keeps its present capacity
  RunDev R = h_runs_[slot];
  std::vector<SegDev> segs(h_segs_.begin() + seg0, h_segs_.begin() + seg0 + spc_);
  size_t total = 0, total_old = 0;
  const size_t prefix = carve_layout(spec, static_cast<char*>(mem), &R, segs.data(), spc_, &total);
  RunDev Rold{};
  std::vector<SegDev> old_segs(spc_);
  const size_t prefix_old = carve_layout(specs_[slot], static_cast<char*>(slot_mem_[slot]), &Rold,
                                         old_segs.data(), spc_, &total_old);
  if (prefix != prefix_old || total > bytes) {
    cudaFreeAsync(mem, stream_);
    if (err) *err = "internal: run layouts disagree";
    return ECPIC_ERR_CUDA;
  }
  // grid, field, deposit, accumulators, tallies and tables keep their offsets
  cudaMemcpyAsync(mem, slot_mem_[slot], prefix, cudaMemcpyDeviceToDevice, stream_);
  for (int s = 0; s < ns; ++s) {
    const SegDev& A = h_segs_[seg0 + s];
    SegDev& B = segs[s];
    const int c = sst[s].cur;
    const size_t n = (size_t)std::min<long long>(std::max<long long>(sst[s].n_alloc, 0), A.cap);
    if (c != 0 && c != 1) {
      cudaFreeAsync(mem, stream_);
      if (err) *err = "internal: bad buffer index";
      return ECPIC_ERR_CUDA;
    }
    if (n == 0) continue;
    cudaMemcpyAsync(B.cell[c], A.cell[c], 4 * n, cudaMemcpyDeviceToDevice, stream_);
    cudaMemcpyAsync(B.xi[c], A.xi[c], 4 * n, cudaMemcpyDeviceToDevice, stream_);
    cudaMemcpyAsync(B.vx[c], A.vx[c], 4 * n, cudaMemcpyDeviceToDevice, stream_);
    cudaMemcpyAsync(B.vy[c], A.vy[c], 4 * n, cudaMemcpyDeviceToDevice, stream_);
    cudaMemcpyAsync(B.vz[c], A.vz[c], 4 * n, cudaMemcpyDeviceToDevice, stream_);
    cudaMemcpyAsync(B.id[c], A.id[c], 8 * n, cudaMemcpyDeviceToDevice, stream_);
    if (A.wt[c] && B.wt[c]) cudaMemcpyAsync(B.wt[c], A.wt[c], 4 * n, cudaMemcpyDeviceToDevice, stream_);
  }
  // the real-collision and impact lists are empty between steps
  for (int s = 0; s < spc_; ++s) h_segs_[seg0 + s] = segs[s];
  cudaMemcpyAsync(d_segs_ + seg0, &h_segs_[seg0], sizeof(SegDev) * spc_, cudaMemcpyHostToDevice,
                  stream_);
  h_runs_[slot] = R;
  upload_run(slot);
  cudaFreeAsync(slot_mem_[slot], stream_);
  bytes_in_use_ = bytes_in_use_ - slot_bytes_[slot] + bytes;
  slot_mem_[slot] = mem;
  slot_bytes_[slot] = bytes;
  specs_[slot] = spec;
  return check(cudaGetLastError(), "reserve", err);
}

int Batch::grow_full_runs(std::string* err) {
  std::vector<SegState> sst(nseg_);
  int rc = check(cudaMemcpyAsync(sst.data(), d_sst_, sizeof(SegState) * nseg_, cudaMemcpyDeviceToHost,
                                 stream_), "read sizes", err);
  if (rc) return rc;
  rc = check(cudaStreamSynchronize(stream_), "read sizes", err);
  if (rc) return rc;
  for (int slot = 0; slot < max_slots_; ++slot) {
    if (!slot_active(slot)) continue;
    const int ns = (int)specs_[slot].species.size();
    long long cap[kMaxSpecies] = {0, 0, 0, 0};
    bool grow = false;
    for (int s = 0; s < ns; ++s) {
      const long long c = h_segs_[slot * spc_ + s].cap;
      cap[s] = c;
      if ((double)sst[slot * spc_ + s].n_alloc > grow_at_ * (double)c) {
        cap[s] = std::min<long long>((long long)INT32_MAX, 2 * c);
        grow = grow || cap[s] > c;
      }
    }
    if (!grow) continue;
    std::string e;
    rc = reserve(slot, cap, &e);
    // a failed allocation leaves the run as it was: it may still fill up and
    // then fails alone with ECPIC_ERR_CAPACITY
    if (rc && rc != ECPIC_ERR_NOMEM) {
      if (err) *err = e;
      return rc;
    }
  }
  return ECPIC_OK;
}

void Batch::release(int slot) {
  if (!slot_active(slot)) return;
  cudaSetDevice(device_);
  h_runs_[slot] = RunDev{};
  // descriptor cleared (inactive, and no pointer into the freed block left
  // behind), segments empty, block back to the pool: all stream-ordered
  // device-side writes, so retiring many runs needs no host round trips
  static_assert(offsetof(RunDev, active) == 0, "RunDev::active first");
  cudaMemsetAsync(d_runs_ + slot, 0, sizeof(RunDev), stream_);
  cudaMemsetAsync(d_sst_ + slot * spc_, 0, sizeof(SegState) * spc_, stream_);
  cudaFreeAsync(slot_mem_[slot], stream_);
  slot_mem_[slot] = nullptr;
  bytes_in_use_ -= slot_bytes_[slot];
  slot_bytes_[slot] = 0;
  active_[slot] = 0;
}

long long Batch::live_estimate() const {
  long long t = 0;
  for (int s = 0; s < max_slots_; ++s)
    if (active_[s])
      for (long long n : specs_[s].n_init) t += n;
  return t;
}

int Batch::choose_grid() const {
  if (pass_grid_override_ > 0) return pass_grid_override_;
  const int occ = pass_max_ctas_per_sm(view());
  const long long cap = (long long)occ * sm_count_;
  long long want = (live_estimate() * 5 / 4 + kPassBlock * 2 - 1) / (kPassBlock * 2);
  if (max_slots_ > 1) want = cap;  // a batch's population changes: fill the GPU
  if (want < 1) want = 1;
  return (int)std::min(cap, want);
}

void Batch::invalidate_graphs() {
  if (graph_k_) cudaGraphExecDestroy(graph_k_);
  if (graph_1_) cudaGraphExecDestroy(graph_1_);
  graph_k_ = graph_1_ = nullptr;
  // timed instances: their pending sums are kept before they go
  for (int i = 0; i < 2; ++i) {
    for (TimedGraph* tg : {&tk_[i], &t1_[i], &ts_[i]}) {
      harvest(tg, nullptr);
      drop_timed(tg);
    }
  }
  tk_next_ = t1_next_ = ts_next_ = 0;
}

void Batch::drop_timed(TimedGraph* tg) {
  if (tg->exec) cudaGraphExecDestroy(tg->exec);
  for (cudaEvent_t e : tg->ev) cudaEventDestroy(e);
  tg->exec = nullptr;
  tg->ev.clear();
  tg->ph.clear();
  tg->pending = false;
}

// Adds the phase intervals of a launched timed graph to the sums once its
// last event has completed (waits for it).
int Batch::harvest(TimedGraph* tg, std::string* err) {
  if (!tg->pending) return ECPIC_OK;
  tg->pending = false;
  int rc = check(cudaEventSynchronize(tg->ev.back()), "phase timing", err);
  if (rc) return rc;
  for (size_t i = 0; i + 1 < tg->ev.size(); ++i) {
    float ms = 0.0f;
    rc = check(cudaEventElapsedTime(&ms, tg->ev[i], tg->ev[i + 1]), "phase timing", err);
    if (rc) return rc;
    const int p = tg->ph[i];
    tsum_[p] += ms;
    tcnt_[p] += (p == 2) ? 4 : 1;  // the sort is four launches
    if (p == 0) ++tsteps_;
    if (p == 2) ++tsorts_;
  }
  return ECPIC_OK;
}

// Captures `steps` steps (and a counting sort after them when `sort`) into a
// graph.  With tg, an event-record node follows every phase: ev[0] before the
// first launch, then pass (0), collision (3), field (1) per step, sort (2).
int Batch::capture(int steps, bool sort, TimedGraph* tg, cudaGraphExec_t* out, std::string* err) {
  const BatchView b = view();
  auto mark = [&](int phase) -> int {
    cudaEvent_t e = nullptr;
    int rc = check(cudaEventCreate(&e), "phase event", err);
    if (rc) return rc;
    tg->ev.push_back(e);
    if (phase >= 0) tg->ph.push_back(phase);
    return check(cudaEventRecordWithFlags(e, stream_, cudaEventRecordExternal), "phase event", err);
  };
  cudaGraph_t graph = nullptr;
  int rc = check(cudaStreamBeginCapture(stream_, cudaStreamCaptureModeThreadLocal), "capture", err);
  if (rc) return rc;
  if (tg) rc = mark(-1);
  for (int t = 0; t < steps && rc == ECPIC_OK; ++t) {
    launch_pass(b, pass_grid_, MODE_STEP, -1, stream_, stage_field(pass_grid_));
    if (tg && (rc = mark(0))) break;
    launch_collide(b, std::min(pass_grid_, 2 * sm_count_), stream_);
    if (tg && (rc = mark(3))) break;
    launch_field(b, 1, -1, stream_);
    if (tg && (rc = mark(1))) break;
  }
  if (sort && rc == ECPIC_OK) {
    launch_sort(b, pass_grid_, stream_);
    if (tg) rc = mark(2);
  }
  const int rc_end = check(cudaStreamEndCapture(stream_, &graph), "capture end", err);
  if (rc) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (rc_end) return rc_end;
  cudaGraphExec_t exec = nullptr;
  rc = check(cudaGraphInstantiate(&exec, graph, 0), "graph instantiate", err);
  cudaGraphDestroy(graph);
  if (rc) return rc;
  if (tg) tg->exec = exec;
  else *out = exec;
  return ECPIC_OK;
}

// Launches the next of two alternating timed instances, first reading the
// events of its previous launch (the other instance keeps the GPU busy).
int Batch::launch_timed(TimedGraph* pair, int* next, std::string* err) {
  TimedGraph& tg = pair[*next];
  int rc = harvest(&tg, err);
  if (rc) return rc;
  rc = check(cudaGraphLaunch(tg.exec, stream_), "graph launch", err);
  if (rc) return rc;
  tg.pending = true;
  *next ^= 1;
  return ECPIC_OK;
}

int Batch::set_phase_timing(bool on, std::string* err) {
  if (on == timing_) return ECPIC_OK;
  if (on && !use_graphs_) {
    if (err) *err = "phase timing needs the step graphs";
    return ECPIC_ERR_STATE;
  }
  cudaSetDevice(device_);
  invalidate_graphs();
  timing_ = on;
  return ECPIC_OK;
}

int Batch::phase_times(double* ms, long long* launches, long long* steps, long long* sorts,
                       std::string* err) {
  cudaSetDevice(device_);
  for (int i = 0; i < 2; ++i) {
    int rc = harvest(&tk_[i], err);
    if (!rc) rc = harvest(&t1_[i], err);
    if (!rc) rc = harvest(&ts_[i], err);
    if (rc) return rc;
  }
  for (int i = 0; i < 4; ++i) {
    if (ms) ms[i] = tsum_[i];
    if (launches) launches[i] = tcnt_[i];
    tsum_[i] = 0.0;
    tcnt_[i] = 0;
  }
  if (steps) *steps = tsteps_;
  if (sorts) *sorts = tsorts_;
  tsteps_ = tsorts_ = 0;
  return ECPIC_OK;
}

// Staging the run's field in shared memory pays only when a pass CTA runs
// several iterations (quads per CTA >= 2 x kPassBlock).
bool Batch::stage_field(int grid) const {
  return grid > 0 && live_estimate() / 4 >= 2LL * kPassBlock * grid;
}

int Batch::ensure_graphs(std::string* err) {
  if (!use_graphs_) return ECPIC_OK;
  const int g = choose_grid();
  const bool built = timing_ ? (tk_[0].exec && tk_[1].exec && t1_[0].exec && t1_[1].exec &&
                                ts_[0].exec && ts_[1].exec)
                             : (graph_k_ && graph_1_);
  const int w = view().weighted;
  if (built && g == pass_grid_ && stage_field(g) == graph_stage_ && w == graph_weighted_)
    return ECPIC_OK;
  invalidate_graphs();
  pass_grid_ = g;
  graph_stage_ = stage_field(g);
  graph_weighted_ = w;
  int rc = ECPIC_OK;
  if (timing_) {
    for (int i = 0; i < 2 && rc == ECPIC_OK; ++i) {
      rc = capture(sort_every_, true, &tk_[i], nullptr, err);
      if (!rc) rc = capture(1, false, &t1_[i], nullptr, err);
      if (!rc) rc = capture(0, true, &ts_[i], nullptr, err);
    }
  } else {
    rc = capture(sort_every_, true, nullptr, &graph_k_, err);
    if (!rc) rc = capture(1, false, nullptr, &graph_1_, err);
  }
  if (rc) invalidate_graphs();
  return rc;
}

bool Batch::rb_due_within(int steps) const {
  for (int s = 0; s < max_slots_; ++s) {
    if (!active_[s] || !specs_[s].rb || specs_[s].rb_every <= 0) continue;
    const long long e = specs_[s].rb_every;
    const long long L = level_[s];
    const long long top = std::min(L + steps, specs_[s].step_end);
    if (top > L && (top / e) > (L / e)) return true;  // a multiple of e in (L, top]
  }
  return false;
}

void Batch::advance_levels(int steps) {
  for (int s = 0; s < max_slots_; ++s)
    if (active_[s]) level_[s] = std::min(level_[s] + steps, specs_[s].step_end);
}

void Batch::rebalance_launch() {
  launch_rebalance(view(), std::max(1, 2 * sm_count_), stream_);
}

int Batch::rebalance_now(int slot, std::string* err) {
  if (!slot_active(slot) || !specs_[slot].rb) {
    if (err) *err = "no rebalancing run in this slot (ecpic_set_rebalance before init)";
    return ECPIC_ERR_STATE;
  }
  cudaSetDevice(device_);
  const int one = 1;
  int rc = check(cudaMemcpyAsync(&d_rst_[slot].rb_force, &one, sizeof(int), cudaMemcpyHostToDevice,
                                 stream_), "rebalance flag", err);
  if (rc) return rc;
  rebalance_launch();
  rc = check(cudaStreamSynchronize(stream_), "rebalance", err);  // `one` lives until here
  if (rc) return rc;
  return check(cudaGetLastError(), "rebalance", err);
}

int Batch::get_weights(int slot, int species, uint32_t* k, long long cap, long long* n,
                       std::string* err) {
  if (!slot_active(slot) || species < 0 || species >= (int)specs_[slot].species.size() || !n ||
      !specs_[slot].rb) {
    if (err) *err = "bad slot or species, or a run without weight multipliers";
    return ECPIC_ERR_ARG;
  }
  cudaSetDevice(device_);
  int rc = check(cudaStreamSynchronize(stream_), "synchronize", err);
  if (rc) return rc;
  const int seg = slot * spc_ + species;
  SegState ss;
  cudaMemcpy(&ss, d_sst_ + seg, sizeof(SegState), cudaMemcpyDeviceToHost);
  const SegDev& G = h_segs_[seg];
  const size_t m = (size_t)ss.n_proc;
  std::vector<int32_t> c(m);
  std::vector<uint32_t> w(m);
  cudaMemcpy(c.data(), G.cell[ss.cur], 4 * m, cudaMemcpyDeviceToHost);
  rc = check(cudaMemcpy(w.data(), G.wt[ss.cur], 4 * m, cudaMemcpyDeviceToHost), "weight read", err);
  if (rc) return rc;
  long long live = 0;
  for (size_t i = 0; i < m; ++i) live += c[i] >= 0;
  *n = live;
  if (live > cap) {
    if (err) *err = "output capacity too small";
    return ECPIC_ERR_ARG;
  }
  long long q = 0;
  for (size_t i = 0; i < m; ++i)
    if (c[i] >= 0) {
      if (k) k[q] = w[i];
      ++q;
    }
  return ECPIC_OK;
}

int Batch::set_weights(int slot, int species, const uint32_t* k, long long n, std::string* err) {
  if (!slot_active(slot) || species < 0 || species >= (int)specs_[slot].species.size() ||
      !specs_[slot].rb || (n > 0 && !k)) {
    if (err) *err = "bad slot or species, or a run without weight multipliers";
    return ECPIC_ERR_ARG;
  }
  for (long long i = 0; i < n; ++i)
    if (k[i] < 1u || k[i] > kRbMaxWeight) {
      if (err) *err = "weight multipliers must lie in 1..65536";
      return ECPIC_ERR_ARG;
    }
  cudaSetDevice(device_);
  int rc = check(cudaStreamSynchronize(stream_), "synchronize", err);
  if (rc) return rc;
  const int seg = slot * spc_ + species;
  SegState ss;
  cudaMemcpy(&ss, d_sst_ + seg, sizeof(SegState), cudaMemcpyDeviceToHost);
  if (ss.n_proc != n || ss.n_dead != 0) {
    if (err) *err = "set_weights needs the particle count of the last set_particles";
    return ECPIC_ERR_ARG;
  }
  const SegDev& G = h_segs_[seg];
  rc = check(cudaMemcpy(G.wt[ss.cur], k, 4 * (size_t)n, cudaMemcpyHostToDevice), "weight write", err);
  if (rc) return rc;
  refresh(slot);
  return check(cudaGetLastError(), "set_weights", err);
}

int Batch::step(long long n, std::string* err) {
  if (n < 0) {
    if (err) *err = "negative step count";
    return ECPIC_ERR_ARG;
  }
  if (!auto_grow_) return step_chunk(n, err);
  // growth checks between chunks of whole sort cycles
  const long long chunk = std::max<long long>(sort_every_, (64 / sort_every_) * sort_every_);
  while (n > 0) {
    const long long m = std::min(n, chunk);
    int rc = step_chunk(m, err);
    if (rc) return rc;
    n -= m;
    rc = grow_full_runs(err);
    if (rc) return rc;
  }
  return ECPIC_OK;
}

int Batch::step_chunk(long long n, std::string* err) {
  cudaSetDevice(device_);
  int rc = ensure_graphs(err);
  if (rc) return rc;
  const BatchView b = view();
  if (!use_graphs_) pass_grid_ = choose_grid();
  while (n > 0) {
    // a sort cycle in which no run is due to rebalance: its graph
    if (use_graphs_ && since_sort_ == 0 && n >= sort_every_ && !rb_due_within(sort_every_)) {
      rc = timing_ ? launch_timed(tk_, &tk_next_, err)
                   : check(cudaGraphLaunch(graph_k_, stream_), "graph launch", err);
      if (rc) return rc;
      n -= sort_every_;
      advance_levels(sort_every_);
      continue;
    }
    if (use_graphs_) {
      rc = timing_ ? launch_timed(t1_, &t1_next_, err)
                   : check(cudaGraphLaunch(graph_1_, stream_), "graph launch", err);
      if (rc) return rc;
    } else {
      launch_pass(b, pass_grid_, MODE_STEP, -1, stream_, stage_field(pass_grid_));
      launch_collide(b, std::min(pass_grid_, 2 * sm_count_), stream_);
      launch_field(b, 1, -1, stream_);
    }
    --n;
    // the runs due at the new level rebalance (after its field)
    const bool due = rb_due_within(1);
    advance_levels(1);
    if (due) rebalance_launch();
    if (++since_sort_ >= sort_every_) {
      if (use_graphs_ && timing_) {
        rc = launch_timed(ts_, &ts_next_, err);
        if (rc) return rc;
      } else {
        launch_sort(b, pass_grid_, stream_);
      }
      since_sort_ = 0;
    }
  }
  return check(cudaGetLastError(), "step", err);
}

int Batch::profile_step(long long n, double* ms, long long* launches, std::string* err) {
  cudaSetDevice(device_);
  if (pass_grid_ <= 0) pass_grid_ = choose_grid();
  const BatchView b = view();
  cudaEvent_t ev[5];
  for (auto& e : ev) cudaEventCreate(&e);
  double acc[4] = {0, 0, 0, 0};
  long long cnt[4] = {0, 0, 0, 0};
  int rc = ECPIC_OK;
  // ECPIC_SYNC_PHASES=1: wait after every kernel so a device error names it
  const char* sp = std::getenv("ECPIC_SYNC_PHASES");
  const bool each = sp && sp[0] == '1';
  for (long long t = 0; t < n && rc == ECPIC_OK; ++t) {
    cudaEventRecord(ev[0], stream_);
    launch_pass(b, pass_grid_, MODE_STEP, -1, stream_, stage_field(pass_grid_));
    cudaEventRecord(ev[1], stream_);
    if (each && (rc = check(cudaEventSynchronize(ev[1]), "pass kernel", err))) break;
    launch_collide(b, std::min(pass_grid_, 2 * sm_count_), stream_);
    cudaEventRecord(ev[4], stream_);
    if (each && (rc = check(cudaEventSynchronize(ev[4]), "collision kernel", err))) break;
    launch_field(b, 1, -1, stream_);
    cudaEventRecord(ev[2], stream_);
    if (each && (rc = check(cudaEventSynchronize(ev[2]), "field kernel", err))) break;
    {
      const bool due = rb_due_within(1);
      advance_levels(1);
      if (due) rebalance_launch();  // (timed with the sort)
    }
    const bool sort = ++since_sort_ >= sort_every_;
    if (sort) {
      if (each) {
        static const char* names[4] = {"sort histogram", "sort scan", "sort scatter",
                                       "sort finalize"};
        for (int ph = 0; ph < 4 && rc == ECPIC_OK; ++ph) {
          launch_sort_phase(b, pass_grid_, ph, stream_);
          rc = check(cudaStreamSynchronize(stream_), names[ph], err);
        }
        if (rc) break;
      } else {
        launch_sort(b, pass_grid_, stream_);
      }
      since_sort_ = 0;
    }
    cudaEventRecord(ev[3], stream_);
    rc = check(cudaEventSynchronize(ev[3]), "profile step", err);
    float a = 0, x = 0, f = 0, c = 0;
    cudaEventElapsedTime(&a, ev[0], ev[1]);
    cudaEventElapsedTime(&x, ev[1], ev[4]);
    cudaEventElapsedTime(&f, ev[4], ev[2]);
    cudaEventElapsedTime(&c, ev[2], ev[3]);
    acc[0] += a;
    acc[1] += f;
    acc[3] += x;
    cnt[0] += 1;
    cnt[1] += 1;
    cnt[3] += 1;
    if (sort) {
      acc[2] += c;
      cnt[2] += 4;
    }
  }
  for (auto& e : ev) cudaEventDestroy(e);
  for (int i = 0; i < 4; ++i) {
    if (ms) ms[i] = acc[i];
    if (launches) launches[i] = cnt[i];
  }
  return rc;
}

int Batch::sort_now(std::string* err) {
  cudaSetDevice(device_);
  const int g = pass_grid_ > 0 ? pass_grid_ : choose_grid();
  launch_sort(view(), g, stream_);
  since_sort_ = 0;
  return check(cudaGetLastError(), "sort", err);
}

int Batch::autotune(long long steps, int* K_out, int* grid_out, double* ns_out, std::string* err,
                    const std::vector<int>& Ks_in) {
  cudaSetDevice(device_);
  if (steps < 1) {
    if (err) *err = "steps per trial must be positive";
    return ECPIC_ERR_ARG;
  }
  // candidates: the counting-sort cadence (8-64 steps) and the pass grid
  // (automatic = 0, one wave at full occupancy, one at half, two and four
  // waves: shorter CTAs even out the tail of the last wave)
  const int occ = pass_max_ctas_per_sm(view());
  std::vector<int> grids = {0, occ * sm_count_};
  if (occ >= 2) grids.push_back((occ / 2) * sm_count_);
  grids.push_back(2 * occ * sm_count_);
  grids.push_back(4 * occ * sm_count_);
  std::vector<int> Ks = Ks_in;
  if (Ks.empty()) Ks = {8, 16, 32, 64};
  for (int K : Ks)
    if (K < 1 || K > 4096) {
      if (err) *err = "sort cadence candidates must lie in 1..4096";
      return ECPIC_ERR_ARG;
    }
  const int K0 = sort_every_, G0 = pass_grid_override_;
  auto psteps = [&](unsigned long long* out) -> int {
    std::vector<RunState> st;
    const int rc = read_states(&st, err);
    if (rc) return rc;
    unsigned long long t = 0;
    for (int s = 0; s < max_slots_; ++s)
      if (active_[s]) t += st[s].psteps;
    *out = t;
    return ECPIC_OK;
  };
  cudaEvent_t a = nullptr, b = nullptr;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  double best = -1.0;
  int bestK = K0, bestG = G0;
  int rc = ECPIC_OK;
  // every trial holds whole sort cycles and whole energy-sample cycles of
  // the resident runs (a sample step's pass costs a few ordinary ones, so
  // trials holding different numbers of them would not compare); cadences
  // whose common multiple exceeds 8x the trial fall back to the sort cycle
  auto trial_cycle = [&](int K) -> long long {
    long long cyc = K;
    const long long cap = 8LL * std::max(steps, 2LL * K);
    for (int s = 0; s < max_slots_; ++s) {
      if (!active_[s] || specs_[s].sample_every <= 0) continue;
      const long long se = specs_[s].sample_every;
      long long a = cyc, bb = se;
      while (bb) {
        const long long t = a % bb;
        a = bb;
        bb = t;
      }
      const long long l = cyc / a * se;
      if (l > cap) return K;
      cyc = l;
    }
    return cyc;
  };
  // every candidate is tried twice, in order and then in reverse order, and
  // scored by the mean of its two trials: the discharges evolve while the
  // trials run (the cost per particle-step drifts as they grow and heat), and
  // a drift linear in time then weighs on every candidate alike
  std::vector<std::pair<int, int>> cand;
  for (int K : Ks)
    for (int g : grids) cand.emplace_back(K, g);
  const int nc = (int)cand.size();
  std::vector<double> sum(nc, 0.0);
  std::vector<int> cnt(nc, 0);
  for (int t = 0; t < 2 * nc && rc == ECPIC_OK; ++t) {
    const int i = t < nc ? t : 2 * nc - 1 - t;
    const int K = cand[i].first, g = cand[i].second;
    const long long cyc = trial_cycle(K);
    set_pass_grid(g);
    set_sort_every(K);
    const long long n = ((std::max(steps, 2LL * K) + cyc - 1) / cyc) * cyc;
    if ((rc = step(K, err))) break;  // builds the graphs, starts the cadence
    unsigned long long p0 = 0, p1 = 0;
    if ((rc = psteps(&p0))) break;
    cudaEventRecord(a, stream_);
    if ((rc = step(n, err))) break;
    cudaEventRecord(b, stream_);
    if ((rc = check(cudaEventSynchronize(b), "autotune", err))) break;
    if ((rc = psteps(&p1))) break;
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, a, b);
    if (p1 <= p0) continue;  // nothing left to step
    sum[i] += 1e6 * (double)ms / (double)(p1 - p0);
    cnt[i] += 1;
  }
  for (int i = 0; i < nc; ++i) {
    if (!cnt[i]) continue;
    const double ns = sum[i] / cnt[i];
    if (best < 0.0 || ns < best) {
      best = ns;
      bestK = cand[i].first;
      bestG = cand[i].second;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  set_pass_grid(bestG);
  set_sort_every(bestK);
  if (rc) return rc;
  if (K_out) *K_out = bestK;
  if (grid_out) *grid_out = bestG;
  if (ns_out) *ns_out = best;
  return ECPIC_OK;
}

int Batch::set_sort_every(int k) {
  if (k < 1) return ECPIC_ERR_ARG;
  sort_every_ = k;
  since_sort_ = 0;
  invalidate_graphs();
  return ECPIC_OK;
}

int Batch::sync(std::string* err) {
  cudaSetDevice(device_);
  int rc = check(cudaStreamSynchronize(stream_), "synchronize", err);
  if (rc) return rc;
  std::vector<RunState> st(max_slots_);
  rc = check(cudaMemcpy(st.data(), d_rst_, sizeof(RunState) * max_slots_, cudaMemcpyDeviceToHost),
             "status read", err);
  if (rc) return rc;
  for (int s = 0; s < max_slots_; ++s)
    if (active_[s] && st[s].status != 0) {
      if (err) *err = "device reported status " + std::to_string(st[s].status) + " in slot " +
                      std::to_string(s);
      return st[s].status;
    }
  return ECPIC_OK;
}

int Batch::slot_status(int slot) {
  cudaSetDevice(device_);
  cudaStreamSynchronize(stream_);
  RunState st;
  cudaMemcpy(&st, d_rst_ + slot, sizeof(RunState), cudaMemcpyDeviceToHost);
  return st.status;
}

int Batch::get_particles(int slot, int species, int32_t* cell, float* xi, float* vx, float* vy,
                         float* vz, uint64_t* id, long long cap, long long* n, std::string* err) {
  if (!slot_active(slot) || species < 0 || species >= (int)specs_[slot].species.size() || !n) {
    if (err) *err = "bad slot or species";
    return ECPIC_ERR_ARG;
  }
  cudaSetDevice(device_);
  int rc = check(cudaStreamSynchronize(stream_), "synchronize", err);
  if (rc) return rc;
  const int seg = slot * spc_ + species;
  SegState ss;
  cudaMemcpy(&ss, d_sst_ + seg, sizeof(SegState), cudaMemcpyDeviceToHost);
  const SegDev& G = h_segs_[seg];
  const size_t m = (size_t)ss.n_proc;
  std::vector<int32_t> c(m);
  std::vector<float> a(m), bx(m), by(m), bz(m);
  std::vector<uint64_t> ids(m);
  const int u = ss.cur;
  cudaMemcpy(c.data(), G.cell[u], 4 * m, cudaMemcpyDeviceToHost);
  cudaMemcpy(a.data(), G.xi[u], 4 * m, cudaMemcpyDeviceToHost);
  cudaMemcpy(bx.data(), G.vx[u], 4 * m, cudaMemcpyDeviceToHost);
  cudaMemcpy(by.data(), G.vy[u], 4 * m, cudaMemcpyDeviceToHost);
  cudaMemcpy(bz.data(), G.vz[u], 4 * m, cudaMemcpyDeviceToHost);
  rc = check(cudaMemcpy(ids.data(), G.id[u], 8 * m, cudaMemcpyDeviceToHost), "particle read", err);
  if (rc) return rc;
  long long live = 0;
  for (size_t i = 0; i < m; ++i) live += c[i] >= 0;
  *n = live;
  if (live > cap) {
    if (err) *err = "output capacity too small";
    return ECPIC_ERR_ARG;
  }
  long long k = 0;
  for (size_t i = 0; i < m; ++i) {
    if (c[i] < 0) continue;
    if (cell) cell[k] = c[i];
    if (xi) xi[k] = a[i];
    if (vx) vx[k] = bx[i];
    if (vy) vy[k] = by[i];
    if (vz) vz[k] = bz[i];
    if (id) id[k] = ids[i];
    ++k;
  }
  return ECPIC_OK;
}

int Batch::set_particles(int slot, int species, const int32_t* cell, const float* xi,
                         const float* vx, const float* vy, const float* vz, const uint64_t* id,
                         long long n, std::string* err) {
  if (!slot_active(slot) || species < 0 || species >= (int)specs_[slot].species.size() || n < 0) {
    if (err) *err = "bad slot or species";
    return ECPIC_ERR_ARG;
  }
  const int seg = slot * spc_ + species;
  const SegDev& G = h_segs_[seg];
  const int N = (int)specs_[slot].edges.size() - 1;
  if (n > G.cap) {
    if (err) *err = "more particles than the species capacity";
    return ECPIC_ERR_ARG;
  }
  if (n > 0 && (!cell || !xi || !vx || !vy || !vz || !id)) {
    if (err) *err = "null particle array";
    return ECPIC_ERR_ARG;
  }
  for (long long i = 0; i < n; ++i)
    if (cell[i] < 0 || cell[i] >= N || !(xi[i] >= 0.0f) || !(xi[i] < 1.0f)) {
      if (err) *err = "cell or xi out of range at index " + std::to_string(i);
      return ECPIC_ERR_ARG;
    }
  cudaSetDevice(device_);
  int rc = check(cudaStreamSynchronize(stream_), "synchronize", err);
  if (rc) return rc;
  SegState ss;
  cudaMemcpy(&ss, d_sst_ + seg, sizeof(SegState), cudaMemcpyDeviceToHost);
  const int u = ss.cur;
  const size_t m = (size_t)n;
  cudaMemcpy(G.cell[u], cell, 4 * m, cudaMemcpyHostToDevice);
  cudaMemcpy(G.xi[u], xi, 4 * m, cudaMemcpyHostToDevice);
  cudaMemcpy(G.vx[u], vx, 4 * m, cudaMemcpyHostToDevice);
  cudaMemcpy(G.vy[u], vy, 4 * m, cudaMemcpyHostToDevice);
  cudaMemcpy(G.vz[u], vz, 4 * m, cudaMemcpyHostToDevice);
  cudaMemcpy(G.id[u], id, 8 * m, cudaMemcpyHostToDevice);
  if (G.wt[u]) {
    const std::vector<uint32_t> w(m, specs_[slot].rb_m0);
    cudaMemcpy(G.wt[u], w.data(), 4 * m, cudaMemcpyHostToDevice);
  }
  ss.n_proc = ss.n_alloc = n;
  ss.n_dead = 0;
  cudaMemcpy(d_sst_ + seg, &ss, sizeof(SegState), cudaMemcpyHostToDevice);
  refresh(slot);
  return check(cudaGetLastError(), "set_particles", err);
}

int Batch::get_fields(int slot, double* phi, float* E, std::string* err) {
  if (!slot_active(slot)) {
    if (err) *err = "bad slot";
    return ECPIC_ERR_ARG;
  }
  cudaSetDevice(device_);
  int rc = check(cudaStreamSynchronize(stream_), "synchronize", err);
  if (rc) return rc;
  const RunDev& R = h_runs_[slot];
  if (phi) {
    launch_phi(view(), slot, stream_);
    rc = check(cudaStreamSynchronize(stream_), "potential", err);
    if (rc) return rc;
    cudaMemcpy(phi, R.phi, 8 * (size_t)(R.N + 1), cudaMemcpyDeviceToHost);
  }
  if (E)
    cudaMemcpy(E, R.E, 4 * (size_t)((R.scheme == ECPIC_SCHEME_MC || R.scheme == ECPIC_SCHEME_MC2) ? R.N + 1 : R.N),
               cudaMemcpyDeviceToHost);
  return check(cudaGetLastError(), "get_fields", err);
}

int Batch::diag(int slot, Diag* out, std::string* err) {
  return diag_many(std::vector<int>{slot}, std::vector<Diag*>{out}, err);
}

// Every slot's state in two copies; per run its accumulators, tallies and
// power sums, consecutive in its block, in one copy.
int Batch::diag_many(const std::vector<int>& slots, const std::vector<Diag*>& out, std::string* err) {
  for (int slot : slots)
    if (!slot_active(slot)) {
      if (err) *err = "bad slot";
      return ECPIC_ERR_ARG;
    }
  if (slots.empty()) return ECPIC_OK;
  cudaSetDevice(device_);
  int rc = check(cudaStreamSynchronize(stream_), "synchronize", err);
  if (rc) return rc;
  std::vector<RunState> st(max_slots_);
  std::vector<SegState> ss(nseg_);
  rc = check(cudaMemcpy(st.data(), d_rst_, sizeof(RunState) * max_slots_, cudaMemcpyDeviceToHost),
             "state read", err);
  if (rc) return rc;
  rc = check(cudaMemcpy(ss.data(), d_sst_, sizeof(SegState) * nseg_, cudaMemcpyDeviceToHost),
             "state read", err);
  if (rc) return rc;
  std::vector<char> buf;
  for (size_t k = 0; k < slots.size(); ++k) {
    const int slot = slots[k];
    Diag* o = out[k];
    const RunDev& R = h_runs_[slot];
    o->N = R.N;
    o->ns = R.ns;
    o->st = st[slot];
    for (int s = 0; s < R.ns; ++s) {
      const SegState& q = ss[(size_t)slot * spc_ + s];
      o->n_live[s] = q.n_proc - q.n_dead;
    }
    o->acc.resize((size_t)acc_size(R.ns) * (R.N + 1));
    o->tal.resize((size_t)R.ns * R.tal_stride);
    o->pw.resize((size_t)R.ns * R.N);
    o->eedf_c0 = R.eedf_c0;
    o->eedf_c1 = R.eedf_c1;
    const char* a0 = reinterpret_cast<const char*>(R.acc);
    const char* a1 = reinterpret_cast<const char*>(R.pw + o->pw.size());
    const char* t0 = reinterpret_cast<const char*>(R.tal);
    const char* p0 = reinterpret_cast<const char*>(R.pw);
    if (!(a0 < t0 && t0 < p0 && p0 < a1)) {
      if (err) *err = "internal: diagnostics layout";
      return ECPIC_ERR_CUDA;
    }
    buf.resize((size_t)(a1 - a0));
    rc = check(cudaMemcpy(buf.data(), a0, buf.size(), cudaMemcpyDeviceToHost), "diagnostics read", err);
    if (rc) return rc;
    std::memcpy(o->acc.data(), buf.data(), 8 * o->acc.size());
    std::memcpy(o->tal.data(), buf.data() + (t0 - a0), 8 * o->tal.size());
    std::memcpy(o->pw.data(), buf.data() + (p0 - a0), 8 * o->pw.size());
  }
  return ECPIC_OK;
}

int Batch::reset_averages(int slot, int sample_every, std::string* err) {
  if (!slot_active(slot) || sample_every < 0) {
    if (err) *err = "bad slot or sample_every";
    return ECPIC_ERR_ARG;
  }
  cudaSetDevice(device_);
  int rc = check(cudaStreamSynchronize(stream_), "synchronize", err);
  if (rc) return rc;
  RunDev& R = h_runs_[slot];
  R.sample_every = sample_every;
  specs_[slot].sample_every = sample_every;
  upload_run(slot);
  cudaMemsetAsync(R.acc, 0, 8 * (size_t)acc_size(R.ns) * (R.N + 1), stream_);
  cudaMemsetAsync(R.momd, 0, 8 * (size_t)R.ns * 2 * (R.N + 1), stream_);
  cudaMemsetAsync(R.tal, 0, 8 * (size_t)R.ns * R.tal_stride, stream_);
  cudaMemsetAsync(R.pw, 0, 8 * (size_t)R.ns * R.N, stream_);
  RunState st;
  cudaMemcpy(&st, d_rst_ + slot, sizeof(RunState), cudaMemcpyDeviceToHost);
  st.n_samples = 0;
  for (int s = 0; s < kMaxSpecies; ++s) st.ke_acc[s] = 0.0;
  cudaMemcpyAsync(d_rst_ + slot, &st, sizeof(RunState), cudaMemcpyHostToDevice, stream_);
  return check(cudaStreamSynchronize(stream_), "reset_averages", err);
}

int Batch::read_states(std::vector<RunState>* out, std::string* err) {
  cudaSetDevice(device_);
  int rc = check(cudaStreamSynchronize(stream_), "synchronize", err);
  if (rc) return rc;
  out->resize(max_slots_);
  return check(cudaMemcpy(out->data(), d_rst_, sizeof(RunState) * max_slots_,
                          cudaMemcpyDeviceToHost),
               "state read", err);
}

int Batch::set_step_end(int slot, long long step_end, std::string* err) {
  if (!slot_active(slot)) {
    if (err) *err = "bad slot";
    return ECPIC_ERR_ARG;
  }
  cudaSetDevice(device_);
  cudaStreamSynchronize(stream_);
  RunState st;
  cudaMemcpy(&st, d_rst_ + slot, sizeof(RunState), cudaMemcpyDeviceToHost);
  st.step_end = step_end;
  specs_[slot].step_end = step_end;
  level_[slot] = std::min<long long>(st.step, step_end);
  return check(cudaMemcpy(d_rst_ + slot, &st, sizeof(RunState), cudaMemcpyHostToDevice),
               "set_step_end", err);
}

}  // namespace ecpic
