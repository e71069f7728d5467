// engine.cu -- batched and served runs behind the C ABI (ecpic_engine_*).
//
// The engine keeps runs resident in one Batch (device state of up to
// max_slots runs), admits queued requests first-fit in submission order as
// slots and the memory budget allow, advances every resident run with one
// launch per kernel phase, and retires finished runs with their diagnostics.
#include <cmath>
#include <deque>
#include <memory>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

#include "runtime.h"

using ecpic::Batch;
using ecpic::Diag;
using ecpic::RunSpec;
using ecpic::RunState;

struct ecpic_engine {
  int device = 0;
  cudaStream_t stream = nullptr;
  size_t budget = 0;
  int max_slots = 0, max_cells = 0, spc = 0;
  std::unique_ptr<Batch> batch;
  struct Request {
    uint64_t ticket;
    RunSpec spec;
    size_t bytes;
  };
  std::deque<Request> queue;
  struct Ticket {
    int state = 0;  // 0 queued, 1 resident, 2 finished, < 0 error
    int slot = -1;
    long long steps_target = 0;
    long long steps_done = 0;
    unsigned long long psteps = 0;
    Diag diag;
    RunSpec spec;  // kept for diagnostics (masses, dt)
  };
  std::unordered_map<uint64_t, Ticket> tickets;
  std::vector<uint64_t> slot_ticket;
  uint64_t next_ticket = 1;
  long long psteps_total = 0, runs_finished = 0;
  std::string err;
};

namespace {

int efail(ecpic_engine* e, int code, const std::string& msg) {
  if (e) e->err = msg;
  return code;
}

int spec_from_config(const ecpic_run_config* c, int64_t n_steps, RunSpec* s, std::string* err) {
  if (!c || !c->edges || c->n_edges < 3 || c->n_species < 1 || c->n_species > ECPIC_MAX_SPECIES ||
      n_steps < 0 || (c->n_proc > 0 && !c->procs) || c->n_proc < 0) {
    *err = "bad run configuration";
    return ECPIC_ERR_ARG;
  }
  s->edges.assign(c->edges, c->edges + c->n_edges);
  s->bc = c->bc;
  s->v0 = c->v0;
  s->freq = c->freq_hz;
  s->phase = c->phase_rad;
  s->vdc = c->v_dc;
  s->scheme = c->scheme;
  s->species.clear();
  for (int i = 0; i < c->n_species; ++i) {
    ecpic::HostSpecies h;
    h.q = c->q[i];
    h.m = c->m[i];
    h.w = c->w[i];
    h.cap = c->capacity[i];
    s->species.push_back(h);
  }
  s->gas = c->n_gas > 0 && c->m_gas > 0;
  s->ng = c->n_gas;
  s->Tg = c->T_gas;
  s->mg = c->m_gas;
  for (int p = 0; p < c->n_proc; ++p) {
    const ecpic_process_desc& d = c->procs[p];
    if (d.species < 0 || d.species >= c->n_species || d.n < 2 || !d.sigma_m2) {
      *err = "bad process description";
      return ECPIC_ERR_ARG;
    }
    ecpic::HostProc h;
    h.kind = d.kind;
    h.thr = d.threshold_eV;
    h.dE = d.dE_eV;
    h.sigma.assign(d.sigma_m2, d.sigma_m2 + d.n);
    h.product = d.product_species;
    s->species[d.species].procs.push_back(std::move(h));
  }
  s->seed = c->seed;
  s->dt = c->dt;
  s->n_init.assign(c->n_init, c->n_init + c->n_species);
  s->T_eV.assign(c->T_eV, c->T_eV + c->n_species);
  s->sample_every = c->sample_every;
  if (c->quiet_start != 0 && c->quiet_start != 1) {
    *err = "quiet_start must be 0 or 1";
    return ECPIC_ERR_ARG;
  }
  s->quiet = c->quiet_start;
  if (c->rb_m0 > 0) {  // particle rebalancing (rb_m0 = 0: off)
    s->rb = true;
    s->rb_every = c->rb_every;
    s->rb_target = c->rb_target;
    s->rb_lo = c->rb_lo;
    s->rb_hi = c->rb_hi;
    s->rb_m0 = c->rb_m0;
  }
  if (c->eedf_bins > 0) {
    s->eedf_center = c->eedf_center;
    s->eedf_halfwidth = c->eedf_halfwidth;
    s->eedf_dE = c->eedf_dE;
    s->eedf_bins = c->eedf_bins;
    s->iedf_dE = c->iedf_dE;
    s->iedf_bins = c->iedf_bins;
    s->iad_bins = c->iad_bins;
  }
  s->step_end = n_steps;
  const std::string v = ecpic::validate_spec(*s);
  if (!v.empty()) {
    *err = v;
    return ECPIC_ERR_ARG;
  }
  return ECPIC_OK;
}

template <typename F>
int eguarded(ecpic_engine* e, F&& f) {
  try {
    return f();
  } catch (const std::bad_alloc&) {
    return efail(e, ECPIC_ERR_NOMEM, "host allocation failed");
  } catch (const std::exception& ex) {
    return efail(e, ECPIC_ERR_ARG, ex.what());
  } catch (...) {
    return efail(e, ECPIC_ERR_ARG, "unknown error");
  }
}

// retire finished or failed runs; returns 0 or a CUDA-level error
int retire(ecpic_engine* e, const std::vector<RunState>& st) {
  std::string err;
  std::vector<int> done;
  std::vector<ecpic::Diag*> outs;
  for (int s = 0; s < e->max_slots; ++s) {
    const uint64_t t = e->slot_ticket[s];
    if (!t) continue;
    auto& tk = e->tickets[t];
    const RunState& r = st[s];
    tk.steps_done = r.step;
    tk.psteps = r.psteps;
    const bool failed = r.status != 0;
    if (!failed && r.step < tk.steps_target) continue;
    done.push_back(s);
    outs.push_back(&tk.diag);
  }
  int rc = e->batch->diag_many(done, outs, &err);
  if (rc) return efail(e, rc, err);
  for (int s : done) {
    const uint64_t t = e->slot_ticket[s];
    auto& tk = e->tickets[t];
    const RunState& r = st[s];
    const bool failed = r.status != 0;
    e->batch->release(s);
    e->slot_ticket[s] = 0;
    tk.slot = -1;
    tk.state = failed ? r.status : 2;
    e->psteps_total += (long long)r.psteps;
    e->runs_finished += 1;
  }
  return ECPIC_OK;
}

}  // namespace

extern "C" {

int ecpic_engine_create(ecpic_engine** out, int device, void* cuda_stream, size_t budget,
                        int max_slots, int max_cells, int species_per_run) {
  if (!out || max_slots < 1 || max_cells < 2 || max_cells > ECPIC_MAX_CELLS ||
      species_per_run < 1 || species_per_run > ECPIC_MAX_SPECIES ||
      (long long)max_slots * species_per_run > ecpic::kMaxSeg)
    return ECPIC_ERR_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return ECPIC_ERR_CUDA;
  ecpic_engine* e = new (std::nothrow) ecpic_engine;
  if (!e) return ECPIC_ERR_NOMEM;
  try {
    e->device = device;
    e->stream = static_cast<cudaStream_t>(cuda_stream);
    e->budget = budget;
    e->max_slots = max_slots;
    e->max_cells = max_cells;
    e->spc = species_per_run;
    e->batch.reset(new Batch(device, e->stream, max_slots, species_per_run, max_cells));
    e->batch->set_auto_grow(true);  // runs that grow by ionisation get room as they fill
    e->slot_ticket.assign(max_slots, 0);
  } catch (...) {
    delete e;
    return ECPIC_ERR_NOMEM;
  }
  if (cudaGetLastError() != cudaSuccess) {
    delete e;
    return ECPIC_ERR_CUDA;
  }
  *out = e;
  return ECPIC_OK;
}

void ecpic_engine_destroy(ecpic_engine* e) {
  if (!e) return;
  try {
    e->batch.reset();
  } catch (...) {
  }
  delete e;
}

const char* ecpic_engine_last_error(const ecpic_engine* e) { return e ? e->err.c_str() : "null handle"; }

int ecpic_engine_submit(ecpic_engine* e, const ecpic_run_config* cfg, int64_t n_steps,
                        uint64_t* ticket) {
  if (!e || !ticket) return ECPIC_ERR_ARG;
  return eguarded(e, [&]() -> int {
    ecpic_engine::Request rq;
    std::string err;
    int rc = spec_from_config(cfg, n_steps, &rq.spec, &err);
    if (rc) return efail(e, rc, err);
    if ((int)rq.spec.edges.size() - 1 > e->max_cells || (int)rq.spec.species.size() > e->spc)
      return efail(e, ECPIC_ERR_ARG, "run exceeds the engine's cell or species limits");
    rq.bytes = ecpic::run_bytes(rq.spec);
    if (e->budget && rq.bytes > e->budget)
      return efail(e, ECPIC_ERR_NOMEM, "run larger than the memory budget");
    rq.ticket = e->next_ticket++;
    ecpic_engine::Ticket tk;
    tk.steps_target = n_steps;
    tk.spec = rq.spec;
    e->tickets.emplace(rq.ticket, std::move(tk));
    *ticket = rq.ticket;
    e->queue.push_back(std::move(rq));
    return ECPIC_OK;
  });
}

int ecpic_engine_pump(ecpic_engine* e, int64_t max_steps, int* n_resident, int* n_queued) {
  if (!e || max_steps < 0) return ECPIC_ERR_ARG;
  return eguarded(e, [&]() -> int {
    std::string err;
    // admission: first fit in submission order
    for (auto it = e->queue.begin(); it != e->queue.end();) {
      int slot = -1;
      for (int s = 0; s < e->max_slots; ++s)
        if (!e->slot_ticket[s]) {
          slot = s;
          break;
        }
      if (slot < 0) break;
      if (e->budget && e->batch->bytes_in_use() + it->bytes > e->budget) {
        ++it;
        continue;
      }
      int rc = e->batch->admit(slot, it->spec, &err, true);
      auto& tk = e->tickets[it->ticket];
      if (rc == ECPIC_ERR_NOMEM) {
        ++it;  // device allocation failed: keep it queued
        continue;
      }
      if (rc) {
        tk.state = rc;
      } else {
        tk.state = 1;
        tk.slot = slot;
        e->slot_ticket[slot] = it->ticket;
      }
      it = e->queue.erase(it);
    }
    {
      int rc = e->batch->admit_wave(&err);
      if (rc) return efail(e, rc, err);
    }
    int resident = 0;
    for (int s = 0; s < e->max_slots; ++s) resident += e->slot_ticket[s] ? 1 : 0;
    if (resident > 0 && max_steps > 0) {
      int rc = e->batch->step(max_steps, &err);
      if (rc) return efail(e, rc, err);
    }
    std::vector<RunState> st;
    int rc = e->batch->read_states(&st, &err);
    if (rc) return efail(e, rc, err);
    rc = retire(e, st);
    if (rc) return rc;
    resident = 0;
    for (int s = 0; s < e->max_slots; ++s) resident += e->slot_ticket[s] ? 1 : 0;
    if (n_resident) *n_resident = resident;
    if (n_queued) *n_queued = (int)e->queue.size();
    return ECPIC_OK;
  });
}

int ecpic_engine_poll(ecpic_engine* e, uint64_t ticket, int* state, ecpic_diag* out,
                      int64_t* steps_done, int64_t* particle_steps) {
  if (!e || !state) return ECPIC_ERR_ARG;
  auto it = e->tickets.find(ticket);
  if (it == e->tickets.end()) return efail(e, ECPIC_ERR_ARG, "unknown ticket");
  const auto& tk = it->second;
  *state = tk.state;
  if (steps_done) *steps_done = tk.steps_done;
  if (particle_steps) *particle_steps = (int64_t)tk.psteps;
  if (out && (tk.state == 2 || tk.state < 0) && tk.diag.N > 0) ecpic::fill_diag(tk.diag, tk.spec, out);
  if (out && tk.state == 1 && e->batch->slot_active(tk.slot)) {
    // a resident run: its current diagnostics, read from the device
    ecpic::Diag d;
    std::string err;
    const int rc = e->batch->diag(tk.slot, &d, &err);
    if (rc) return efail(e, rc, err);
    ecpic::fill_diag(d, tk.spec, out);
  }
  return ECPIC_OK;
}

int ecpic_engine_release(ecpic_engine* e, uint64_t ticket) {
  if (!e) return ECPIC_ERR_ARG;
  auto it = e->tickets.find(ticket);
  if (it == e->tickets.end()) return efail(e, ECPIC_ERR_ARG, "unknown ticket");
  if (it->second.state == 0 || it->second.state == 1)
    return efail(e, ECPIC_ERR_STATE, "ticket not finished");
  e->tickets.erase(it);
  return ECPIC_OK;
}

int ecpic_engine_stats(ecpic_engine* e, int64_t* particle_steps, int64_t* runs_finished,
                       int64_t* bytes_resident) {
  if (!e) return ECPIC_ERR_ARG;
  return eguarded(e, [&]() -> int {
    long long live = 0;
    bool any = false;
    for (int s = 0; s < e->max_slots; ++s) any = any || e->slot_ticket[s] != 0;
    if (any && particle_steps) {
      std::vector<RunState> st;
      std::string err;
      const int rc = e->batch->read_states(&st, &err);
      if (rc) return efail(e, rc, err);
      for (int s = 0; s < e->max_slots; ++s)
        if (e->slot_ticket[s]) live += (long long)st[s].psteps;
    }
    if (particle_steps) *particle_steps = e->psteps_total + live;
    if (runs_finished) *runs_finished = e->runs_finished;
    if (bytes_resident) *bytes_resident = (int64_t)e->batch->bytes_in_use();
    return ECPIC_OK;
  });
}

int ecpic_engine_profile(ecpic_engine* e, int64_t n, double* ms, int64_t* launches) {
  if (!e || n < 0) return ECPIC_ERR_ARG;
  std::string err;
  long long l[4] = {0, 0, 0, 0};
  const int rc = e->batch->profile_step(n, ms, l, &err);
  if (launches)
    for (int i = 0; i < 4; ++i) launches[i] = l[i];
  return rc ? efail(e, rc, err) : ECPIC_OK;
}

int ecpic_engine_autotune(ecpic_engine* e, int64_t steps_per_trial, int* sort_every, int* pass_ctas,
                          double* ns_per_particle_step) {
  if (!e || steps_per_trial < 1) return ECPIC_ERR_ARG;
  std::string err;
  const int rc = e->batch->autotune(steps_per_trial, sort_every, pass_ctas, ns_per_particle_step, &err);
  return rc ? efail(e, rc, err) : ECPIC_OK;
}

int ecpic_engine_autotune_ks(ecpic_engine* e, int64_t steps_per_trial, const int* ks, int n_ks,
                             int* sort_every, int* pass_ctas, double* ns_per_particle_step) {
  if (!e || steps_per_trial < 1 || n_ks < 1 || n_ks > 64 || !ks) return ECPIC_ERR_ARG;
  return eguarded(e, [&]() -> int {
    std::string err;
    const std::vector<int> K(ks, ks + n_ks);
    const int rc = e->batch->autotune(steps_per_trial, sort_every, pass_ctas, ns_per_particle_step,
                                      &err, K);
    return rc ? efail(e, rc, err) : ECPIC_OK;
  });
}

int ecpic_engine_set_phase_timing(ecpic_engine* e, int on) {
  if (!e || (on != 0 && on != 1)) return ECPIC_ERR_ARG;
  std::string err;
  const int rc = e->batch->set_phase_timing(on == 1, &err);
  return rc ? efail(e, rc, err) : ECPIC_OK;
}

int ecpic_engine_phase_times(ecpic_engine* e, double* ms, int64_t* launches, int64_t* steps,
                             int64_t* sorts) {
  if (!e) return ECPIC_ERR_ARG;
  std::string err;
  long long l[4] = {0, 0, 0, 0}, st = 0, so = 0;
  const int rc = e->batch->phase_times(ms, l, &st, &so, &err);
  if (launches)
    for (int i = 0; i < 4; ++i) launches[i] = l[i];
  if (steps) *steps = st;
  if (sorts) *sorts = so;
  return rc ? efail(e, rc, err) : ECPIC_OK;
}

int ecpic_engine_sort_state(ecpic_engine* e, int* sort_every, int* since_sort) {
  if (!e) return ECPIC_ERR_ARG;
  if (sort_every) *sort_every = e->batch->sort_every();
  if (since_sort) *since_sort = e->batch->since_sort();
  return ECPIC_OK;
}

int ecpic_engine_tune(ecpic_engine* e, int pass_ctas, int sort_every) {
  if (!e || pass_ctas < 0 || sort_every < 1) return ECPIC_ERR_ARG;
  e->batch->set_pass_grid(pass_ctas);
  return e->batch->set_sort_every(sort_every);
}

}  // extern "C"
