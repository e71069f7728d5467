// api.cu -- the extern "C" boundary of libecpic (see include/ecpic.h).
#include <cmath>
#include <cstring>
#include <exception>
#include <memory>
#include <new>
#include <string>

#include "runtime.h"

using ecpic::Batch;
using ecpic::Diag;
using ecpic::HostProc;
using ecpic::HostSpecies;
using ecpic::RunSpec;

struct ecpic_run {
  int device = 0;
  cudaStream_t stream = nullptr;
  RunSpec spec;
  bool grid_set = false;
  std::unique_ptr<Batch> batch;
  std::string err;
  int sort_every = 16;
  bool auto_grow = false;
};

namespace {

int fail(ecpic_run* r, int code, const std::string& msg) {
  if (r) r->err = msg;
  return code;
}

template <typename F>
int guarded(ecpic_run* r, F&& f) {
  try {
    return f();
  } catch (const std::bad_alloc&) {
    return fail(r, ECPIC_ERR_NOMEM, "host allocation failed");
  } catch (const std::exception& e) {
    return fail(r, ECPIC_ERR_ARG, e.what());
  } catch (...) {
    return fail(r, ECPIC_ERR_ARG, "unknown error");
  }
}

int grid_doubling(int n_ref, double L, double L_buff, int dx_min, int dx_max, double* edges,
                  int cap) {
  // Sec. 3c: buffer of dx_min cells covering L_buff from the electrode, then
  // cells double (only where the position is a multiple of the doubled size)
  // up to dx_max; no neighbour ratio above 2; mirrored about the centre.
  if (n_ref < 2 || (n_ref % 2) != 0 || !(L > 0) || !(L_buff >= 0) || dx_min < 1 ||
      dx_max < dx_min || !edges)
    return ECPIC_ERR_ARG;
  const double ref = L / n_ref;
  const int half = n_ref / 2;
  std::vector<int> w;
  int at = 0;
  const int nbuf = (int)std::ceil(L_buff / (dx_min * ref) - 1e-9);
  while ((int)w.size() < nbuf && at < half) {
    const int c = std::min(dx_min, half - at);
    w.push_back(c);
    at += c;
  }
  int last = dx_min;
  while (at < half) {
    int c = (2 * last <= dx_max && at % (2 * last) == 0) ? 2 * last : last;
    while (at + c > half && c > dx_min) c /= 2;
    if (at + c > half) c = half - at;
    w.push_back(c);
    at += c;
    last = c;
  }
  const int n = 2 * (int)w.size();
  if (n + 1 > cap) return ECPIC_ERR_ARG;
  long long u = 0;
  edges[0] = 0.0;
  for (size_t i = 0; i < w.size(); ++i) {
    u += w[i];
    edges[i + 1] = u * ref;
  }
  for (size_t i = w.size(); i-- > 0;) {
    u += w[i];
    edges[n - i] = u * ref;
  }
  edges[n] = L;
  return n;
}

}  // namespace

extern "C" {

int ecpic_create(ecpic_run** out, int device, void* cuda_stream) {
  if (!out) return ECPIC_ERR_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    *out = nullptr;
    return ECPIC_ERR_CUDA;
  }
  ecpic_run* r = new (std::nothrow) ecpic_run;
  if (!r) return ECPIC_ERR_NOMEM;
  r->device = device;
  r->stream = static_cast<cudaStream_t>(cuda_stream);
  *out = r;
  return ECPIC_OK;
}

void ecpic_destroy(ecpic_run* r) {
  if (!r) return;
  try {
    r->batch.reset();
  } catch (...) {
  }
  delete r;
}

const char* ecpic_last_error(const ecpic_run* r) { return r ? r->err.c_str() : "null handle"; }

int ecpic_set_grid(ecpic_run* r, const double* edges, int n_edges, int bc, double v0,
                   double freq_hz, double phase_rad, double v_dc) {
  if (!r) return ECPIC_ERR_ARG;
  return guarded(r, [&]() -> int {
    if (r->batch) return fail(r, ECPIC_ERR_STATE, "grid is fixed after init");
    if (!r->spec.species.empty()) return fail(r, ECPIC_ERR_STATE, "set the grid before species");
    if (!edges || n_edges < 3) return fail(r, ECPIC_ERR_ARG, "need edges of at least 2 cells");
    std::vector<double> e(edges, edges + n_edges);
    const std::string v = ecpic::validate_grid(e, bc);
    if (!v.empty()) return fail(r, ECPIC_ERR_ARG, v);
    if (!std::isfinite(v0) || !std::isfinite(freq_hz) || !std::isfinite(phase_rad) ||
        !std::isfinite(v_dc))
      return fail(r, ECPIC_ERR_ARG, "non-finite bias parameters");
    r->spec.edges = e;
    r->spec.bc = bc;
    r->spec.v0 = v0;
    r->spec.freq = freq_hz;
    r->spec.phase = phase_rad;
    r->spec.vdc = v_dc;
    r->grid_set = true;
    return ECPIC_OK;
  });
}

int ecpic_set_scheme(ecpic_run* r, int scheme) {
  if (!r) return ECPIC_ERR_ARG;
  if (scheme < ECPIC_SCHEME_EC || scheme > ECPIC_SCHEME_MC2)
    return fail(r, ECPIC_ERR_ARG, "unknown scheme");
  if (r->batch) return fail(r, ECPIC_ERR_STATE, "scheme is fixed after init");
  r->spec.scheme = scheme;
  return ECPIC_OK;
}

int ecpic_add_species(ecpic_run* r, double q, double m, double w, int64_t capacity, int* out) {
  if (!r) return ECPIC_ERR_ARG;
  return guarded(r, [&]() -> int {
    if (!r->grid_set || r->batch) return fail(r, ECPIC_ERR_STATE, "species go after the grid, before init");
    if ((int)r->spec.species.size() >= ECPIC_MAX_SPECIES) return fail(r, ECPIC_ERR_ARG, "too many species");
    if (!(m > 0) || !(w >= 0) || !std::isfinite(q) || capacity < 1 || capacity > INT32_MAX)
      return fail(r, ECPIC_ERR_ARG, "bad species parameters");
    HostSpecies s;
    s.q = q;
    s.m = m;
    s.w = w;
    s.cap = capacity;
    r->spec.species.push_back(s);
    if (out) *out = (int)r->spec.species.size() - 1;
    return ECPIC_OK;
  });
}

int ecpic_set_gas(ecpic_run* r, double n_g, double T_g, double m_g) {
  if (!r) return ECPIC_ERR_ARG;
  if (r->batch) return fail(r, ECPIC_ERR_STATE, "gas is fixed after init");
  if (!(n_g >= 0) || !(T_g >= 0) || !(m_g > 0)) return fail(r, ECPIC_ERR_ARG, "bad gas parameters");
  r->spec.gas = true;
  r->spec.ng = n_g;
  r->spec.Tg = T_g;
  r->spec.mg = m_g;
  return ECPIC_OK;
}

int ecpic_add_process(ecpic_run* r, int species, int kind, double threshold_eV, double dE_eV,
                      int n, const float* sigma, int product_species) {
  if (!r) return ECPIC_ERR_ARG;
  return guarded(r, [&]() -> int {
    if (r->batch) return fail(r, ECPIC_ERR_STATE, "processes are fixed after init");
    if (species < 0 || species >= (int)r->spec.species.size())
      return fail(r, ECPIC_ERR_ARG, "unknown species");
    if (kind < ECPIC_ELASTIC || kind > ECPIC_CX) return fail(r, ECPIC_ERR_ARG, "unknown kind");
    if (n < 2 || !sigma || !(dE_eV > 0) || !(threshold_eV >= 0))
      return fail(r, ECPIC_ERR_ARG, "bad cross-section table");
    HostSpecies& s = r->spec.species[species];
    if ((int)s.procs.size() >= ECPIC_MAX_PROC) return fail(r, ECPIC_ERR_ARG, "too many processes");
    HostProc p;
    p.kind = kind;
    p.thr = threshold_eV;
    p.dE = dE_eV;
    p.sigma.assign(sigma, sigma + n);
    p.product = product_species;
    for (float v : p.sigma)
      if (!(v >= 0.0f) || !std::isfinite(v)) return fail(r, ECPIC_ERR_ARG, "bad cross section value");
    if (!s.procs.empty() && (s.procs[0].dE != dE_eV || (int)s.procs[0].sigma.size() != n))
      return fail(r, ECPIC_ERR_ARG, "processes of one species must share the energy grid");
    if (kind == ECPIC_IONIZATION &&
        (product_species < 0 || product_species >= (int)r->spec.species.size() ||
         product_species == species))
      return fail(r, ECPIC_ERR_ARG, "ionisation needs a product ion species");
    s.procs.push_back(std::move(p));
    return ECPIC_OK;
  });
}

int ecpic_set_tallies(ecpic_run* r, double center, double halfwidth, double eedf_dE, int eedf_bins,
                      double iedf_dE, int iedf_bins, int iad_bins) {
  if (!r) return ECPIC_ERR_ARG;
  if (r->batch) return fail(r, ECPIC_ERR_STATE, "before init");
  r->spec.eedf_center = center;
  r->spec.eedf_halfwidth = halfwidth;
  r->spec.eedf_dE = eedf_dE;
  r->spec.eedf_bins = eedf_bins;
  r->spec.iedf_dE = iedf_dE;
  r->spec.iedf_bins = iedf_bins;
  r->spec.iad_bins = iad_bins;
  const std::string v = ecpic::validate_tallies(r->spec);
  return v.empty() ? ECPIC_OK : fail(r, ECPIC_ERR_ARG, v);
}

int ecpic_set_rebalance(ecpic_run* r, int every, int target, int lo, int hi, uint32_t m0) {
  if (!r) return ECPIC_ERR_ARG;
  if (r->batch) return fail(r, ECPIC_ERR_STATE, "before init");
  if (every < 0 || target < 1 || target > ecpic::kRbMaxCell || lo < 0 || lo > target || hi < target ||
      m0 < 1u || m0 > (uint32_t)ecpic::kRbMaxWeight)
    return fail(r, ECPIC_ERR_ARG,
                "bad rebalancing parameters (0 <= lo <= target <= hi, target <= 4096, 1 <= m0 <= 65536)");
  r->spec.rb = true;
  r->spec.rb_every = every;
  r->spec.rb_target = target;
  r->spec.rb_lo = lo;
  r->spec.rb_hi = hi;
  r->spec.rb_m0 = m0;
  return ECPIC_OK;
}

int ecpic_rebalance_now(ecpic_run* r) {
  if (!r) return ECPIC_ERR_ARG;
  if (!r->batch) return fail(r, ECPIC_ERR_STATE, "init first");
  return guarded(r, [&]() -> int {
    std::string err;
    const int rc = r->batch->rebalance_now(0, &err);
    return rc ? fail(r, rc, err) : ECPIC_OK;
  });
}

int ecpic_get_weights(ecpic_run* r, int species, uint32_t* k, int64_t cap, int64_t* n) {
  if (!r || !n) return ECPIC_ERR_ARG;
  if (!r->batch) return fail(r, ECPIC_ERR_STATE, "init first");
  return guarded(r, [&]() -> int {
    std::string err;
    long long m = 0;
    const int rc = r->batch->get_weights(0, species, k, cap, &m, &err);
    *n = m;
    return rc ? fail(r, rc, err) : ECPIC_OK;
  });
}

int ecpic_set_weights(ecpic_run* r, int species, const uint32_t* k, int64_t n) {
  if (!r || n < 0) return ECPIC_ERR_ARG;
  if (!r->batch) return fail(r, ECPIC_ERR_STATE, "init first");
  return guarded(r, [&]() -> int {
    std::string err;
    const int rc = r->batch->set_weights(0, species, k, n, &err);
    return rc ? fail(r, rc, err) : ECPIC_OK;
  });
}

int ecpic_set_quiet_start(ecpic_run* r, int quiet) {
  if (!r || (quiet != 0 && quiet != 1)) return ECPIC_ERR_ARG;
  if (r->batch) return fail(r, ECPIC_ERR_STATE, "before init");
  r->spec.quiet = quiet;
  return ECPIC_OK;
}

int ecpic_init(ecpic_run* r, uint64_t seed, double dt, const int64_t* n_per_species,
               const double* T_eV) {
  if (!r) return ECPIC_ERR_ARG;
  return guarded(r, [&]() -> int {
    if (r->batch) return fail(r, ECPIC_ERR_STATE, "already initialised");
    if (!r->grid_set || r->spec.species.empty()) return fail(r, ECPIC_ERR_STATE, "grid and species first");
    if (!n_per_species || !T_eV) return fail(r, ECPIC_ERR_ARG, "null arrays");
    const size_t ns = r->spec.species.size();
    r->spec.seed = seed;
    r->spec.dt = dt;
    r->spec.n_init.assign(n_per_species, n_per_species + ns);
    r->spec.T_eV.assign(T_eV, T_eV + ns);
    const std::string v = ecpic::validate_spec(r->spec);
    if (!v.empty()) return fail(r, ECPIC_ERR_ARG, v);
    const int N = (int)r->spec.edges.size() - 1;
    std::unique_ptr<Batch> b(new Batch(r->device, r->stream, 1, (int)ns, N));
    b->set_sort_every(r->sort_every);
    b->set_auto_grow(r->auto_grow);
    std::string err;
    const int rc = b->admit(0, r->spec, &err);
    if (rc) return fail(r, rc, err);
    r->batch = std::move(b);
    return ECPIC_OK;
  });
}

int ecpic_step(ecpic_run* r, int64_t n) {
  if (!r) return ECPIC_ERR_ARG;
  if (!r->batch) return fail(r, ECPIC_ERR_STATE, "init first");
  return guarded(r, [&]() -> int {
    std::string err;
    const int rc = r->batch->step(n, &err);
    return rc ? fail(r, rc, err) : ECPIC_OK;
  });
}

int ecpic_sync(ecpic_run* r) {
  if (!r) return ECPIC_ERR_ARG;
  if (!r->batch) return fail(r, ECPIC_ERR_STATE, "init first");
  std::string err;
  const int rc = r->batch->sync(&err);
  return rc ? fail(r, rc, err) : ECPIC_OK;
}

int ecpic_reset_averages(ecpic_run* r, int sample_every) {
  if (!r) return ECPIC_ERR_ARG;
  if (!r->batch) return fail(r, ECPIC_ERR_STATE, "init first");
  std::string err;
  const int rc = r->batch->reset_averages(0, sample_every, &err);
  return rc ? fail(r, rc, err) : ECPIC_OK;
}

int ecpic_diagnostics(ecpic_run* r, ecpic_diag* out) {
  if (!r || !out) return ECPIC_ERR_ARG;
  if (!r->batch) return fail(r, ECPIC_ERR_STATE, "init first");
  return guarded(r, [&]() -> int {
    Diag d;
    std::string err;
    const int rc = r->batch->diag(0, &d, &err);
    if (rc) return fail(r, rc, err);
    ecpic::fill_diag(d, r->spec, out);
    return ECPIC_OK;
  });
}

int ecpic_get_particles(ecpic_run* r, int species, int32_t* cell, float* xi, float* vx, float* vy,
                        float* vz, uint64_t* id, int64_t cap, int64_t* n) {
  if (!r) return ECPIC_ERR_ARG;
  if (!r->batch) return fail(r, ECPIC_ERR_STATE, "init first");
  return guarded(r, [&]() -> int {
    std::string err;
    long long m = 0;
    const int rc = r->batch->get_particles(0, species, cell, xi, vx, vy, vz, id, cap, &m, &err);
    if (n) *n = m;
    return rc ? fail(r, rc, err) : ECPIC_OK;
  });
}

int ecpic_set_particles(ecpic_run* r, int species, const int32_t* cell, const float* xi,
                        const float* vx, const float* vy, const float* vz, const uint64_t* id,
                        int64_t n) {
  if (!r) return ECPIC_ERR_ARG;
  if (!r->batch) return fail(r, ECPIC_ERR_STATE, "init first");
  return guarded(r, [&]() -> int {
    std::string err;
    const int rc = r->batch->set_particles(0, species, cell, xi, vx, vy, vz, id, n, &err);
    return rc ? fail(r, rc, err) : ECPIC_OK;
  });
}

int ecpic_get_fields(ecpic_run* r, double* phi, float* E) {
  if (!r) return ECPIC_ERR_ARG;
  if (!r->batch) return fail(r, ECPIC_ERR_STATE, "init first");
  std::string err;
  const int rc = r->batch->get_fields(0, phi, E, &err);
  return rc ? fail(r, rc, err) : ECPIC_OK;
}

int ecpic_nu_max(ecpic_run* r, int species, double* nu_max, uint32_t* threshold24) {
  if (!r) return ECPIC_ERR_ARG;
  if (species < 0 || species >= (int)r->spec.species.size()) return fail(r, ECPIC_ERR_ARG, "unknown species");
  if (!r->batch) return fail(r, ECPIC_ERR_STATE, "init first");
  double nu;
  uint32_t t;
  ecpic::null_rate(r->spec.species[species], r->spec, &nu, &t);
  if (nu_max) *nu_max = nu;
  if (threshold24) *threshold24 = t;
  return ECPIC_OK;
}

int ecpic_set_sort_every(ecpic_run* r, int k) {
  if (!r) return ECPIC_ERR_ARG;
  if (k < 1) return fail(r, ECPIC_ERR_ARG, "sort cadence must be >= 1");
  r->sort_every = k;
  if (r->batch) r->batch->set_sort_every(k);
  return ECPIC_OK;
}

int ecpic_reserve(ecpic_run* r, int species, int64_t capacity) {
  if (!r) return ECPIC_ERR_ARG;
  if (!r->batch) return fail(r, ECPIC_ERR_STATE, "init first");
  if (species < 0 || species >= (int)r->spec.species.size()) return fail(r, ECPIC_ERR_ARG, "unknown species");
  if (capacity < 1) return fail(r, ECPIC_ERR_ARG, "capacity must be >= 1");
  return guarded(r, [&]() -> int {
    long long cap[ecpic::kMaxSpecies] = {0, 0, 0, 0};
    const RunSpec& cur = r->batch->spec(0);
    for (size_t s = 0; s < cur.species.size(); ++s) cap[s] = cur.species[s].cap;
    if (capacity > cap[species]) cap[species] = capacity;
    std::string err;
    const int rc = r->batch->reserve(0, cap, &err);
    if (rc) return fail(r, rc, err);
    for (size_t s = 0; s < cur.species.size(); ++s) r->spec.species[s].cap = r->batch->spec(0).species[s].cap;
    return ECPIC_OK;
  });
}

int ecpic_set_auto_grow(ecpic_run* r, int on) {
  if (!r || (on != 0 && on != 1)) return ECPIC_ERR_ARG;
  r->auto_grow = on != 0;
  if (r->batch) r->batch->set_auto_grow(r->auto_grow);
  return ECPIC_OK;
}

int ecpic_sort_now(ecpic_run* r) {
  if (!r) return ECPIC_ERR_ARG;
  if (!r->batch) return fail(r, ECPIC_ERR_STATE, "init first");
  std::string err;
  const int rc = r->batch->sort_now(&err);
  return rc ? fail(r, rc, err) : ECPIC_OK;
}

int ecpic_profile_step(ecpic_run* r, int64_t n, double* ms, int64_t* launches) {
  if (!r || n < 0) return ECPIC_ERR_ARG;
  if (!r->batch) return fail(r, ECPIC_ERR_STATE, "init first");
  std::string err;
  long long l[4] = {0, 0, 0, 0};
  const int rc = r->batch->profile_step(n, ms, l, &err);
  if (launches)
    for (int i = 0; i < 4; ++i) launches[i] = l[i];
  return rc ? fail(r, rc, err) : ECPIC_OK;
}

int ecpic_autotune(ecpic_run* r, int64_t steps_per_trial, int* sort_every, int* pass_ctas,
                   double* ns_per_particle_step) {
  if (!r || steps_per_trial < 1) return ECPIC_ERR_ARG;
  if (!r->batch) return fail(r, ECPIC_ERR_STATE, "init first");
  std::string err;
  const int rc = r->batch->autotune(steps_per_trial, sort_every, pass_ctas, ns_per_particle_step, &err);
  return rc ? fail(r, rc, err) : ECPIC_OK;
}

int ecpic_autotune_ks(ecpic_run* r, int64_t steps_per_trial, const int* ks, int n_ks, int* sort_every,
                      int* pass_ctas, double* ns_per_particle_step) {
  if (!r || steps_per_trial < 1 || n_ks < 1 || n_ks > 64 || !ks) return ECPIC_ERR_ARG;
  if (!r->batch) return fail(r, ECPIC_ERR_STATE, "init first");
  return guarded(r, [&]() -> int {
    std::string err;
    const std::vector<int> K(ks, ks + n_ks);
    const int rc = r->batch->autotune(steps_per_trial, sort_every, pass_ctas, ns_per_particle_step,
                                      &err, K);
    if (!rc && sort_every) r->sort_every = *sort_every;
    return rc ? fail(r, rc, err) : ECPIC_OK;
  });
}

int ecpic_set_phase_timing(ecpic_run* r, int on) {
  if (!r || (on != 0 && on != 1)) return ECPIC_ERR_ARG;
  if (!r->batch) return fail(r, ECPIC_ERR_STATE, "init first");
  std::string err;
  const int rc = r->batch->set_phase_timing(on == 1, &err);
  return rc ? fail(r, rc, err) : ECPIC_OK;
}

int ecpic_phase_times(ecpic_run* r, double* ms, int64_t* launches, int64_t* steps, int64_t* sorts) {
  if (!r) return ECPIC_ERR_ARG;
  if (!r->batch) return fail(r, ECPIC_ERR_STATE, "init first");
  std::string err;
  long long l[4] = {0, 0, 0, 0}, st = 0, so = 0;
  const int rc = r->batch->phase_times(ms, l, &st, &so, &err);
  if (launches)
    for (int i = 0; i < 4; ++i) launches[i] = l[i];
  if (steps) *steps = st;
  if (sorts) *sorts = so;
  return rc ? fail(r, rc, err) : ECPIC_OK;
}

int ecpic_sort_state(ecpic_run* r, int* sort_every, int* since_sort) {
  if (!r) return ECPIC_ERR_ARG;
  if (!r->batch) return fail(r, ECPIC_ERR_STATE, "init first");
  if (sort_every) *sort_every = r->batch->sort_every();
  if (since_sort) *since_sort = r->batch->since_sort();
  return ECPIC_OK;
}

int ecpic_set_pass_grid(ecpic_run* r, int ctas) {
  if (!r || ctas < 0) return ECPIC_ERR_ARG;
  if (!r->batch) return fail(r, ECPIC_ERR_STATE, "init first");
  r->batch->set_pass_grid(ctas);
  return ECPIC_OK;
}

int ecpic_doubling_grid(int n_ref, double L, double L_buff, int dx_min, int dx_max, double* edges,
                        int cap) {
  try {
    return grid_doubling(n_ref, L, L_buff, dx_min, dx_max, edges, cap);
  } catch (...) {
    return ECPIC_ERR_NOMEM;
  }
}

int ecpic_deposit_device(int N, int64_t n, const int32_t* d_cell, const float* d_xi, uint64_t* d_S,
                         void* stream) {
  if (N < 1 || N > ECPIC_MAX_CELLS || n < 0 || (n > 0 && (!d_cell || !d_xi)) || !d_S)
    return ECPIC_ERR_ARG;
  if (n == 0) return ECPIC_OK;
  ecpic::launch_deposit_device(N, n, d_cell, d_xi, reinterpret_cast<unsigned long long*>(d_S),
                               static_cast<cudaStream_t>(stream));
  return cudaGetLastError() == cudaSuccess ? ECPIC_OK : ECPIC_ERR_CUDA;
}

int ecpic_deposit_device2(int N, int bc, int64_t n, const int32_t* d_cell, const float* d_xi,
                          uint64_t* d_S, void* stream) {
  if (N < 1 || N > ECPIC_MAX_CELLS || n < 0 || (n > 0 && (!d_cell || !d_xi)) || !d_S ||
      (bc != ECPIC_DIRICHLET_RF && bc != ECPIC_PERIODIC))
    return ECPIC_ERR_ARG;
  if (n == 0) return ECPIC_OK;
  ecpic::launch_deposit2_device(N, bc == ECPIC_PERIODIC ? 1 : 0, n, d_cell, d_xi,
                                reinterpret_cast<unsigned long long*>(d_S),
                                static_cast<cudaStream_t>(stream));
  return cudaGetLastError() == cudaSuccess ? ECPIC_OK : ECPIC_ERR_CUDA;
}

int ecpic_debug_checks(int64_t* out) {
  if (!out) return ECPIC_ERR_ARG;
  unsigned long long v[4] = {0, 0, 0, 0};
  ecpic::read_checks(v);
  for (int i = 0; i < 4; ++i) out[i] = (int64_t)v[i];
  return cudaGetLastError() == cudaSuccess ? ECPIC_OK : ECPIC_ERR_CUDA;
}

int ecpic_philox_device(int64_t n, const uint32_t* d_ctr, const uint32_t* d_key, uint32_t* d_out,
                        void* stream) {
  if (n < 0 || (n > 0 && (!d_ctr || !d_key || !d_out))) return ECPIC_ERR_ARG;
  if (n == 0) return ECPIC_OK;
  ecpic::launch_philox_device(n, d_ctr, d_key, d_out, static_cast<cudaStream_t>(stream));
  return cudaGetLastError() == cudaSuccess ? ECPIC_OK : ECPIC_ERR_CUDA;
}

}  // extern "C"
