// runtime.h -- host runtime of libecpic: a Batch owns the device state of up
// to max_slots independent runs and steps them together (one launch per
// phase for all runs, replayed from CUDA graphs).
#pragma once
#include <climits>
#include <cstdint>
#include <string>
#include <vector>

#include "kernels.h"

namespace ecpic {

struct HostProc {
  int kind = 0;
  double thr = 0, dE = 0;
  std::vector<float> sigma;
  int product = -1;
};

struct HostSpecies {
  double q = 0, m = 0, w = 0;
  long long cap = 0;
  std::vector<HostProc> procs;
};

struct RunSpec {
  std::vector<double> edges;
  int bc = ECPIC_DIRICHLET_RF;
  double v0 = 0, freq = 0, phase = 0, vdc = 0;
  int scheme = ECPIC_SCHEME_EC;
  std::vector<HostSpecies> species;
  bool gas = false;
  double ng = 0, Tg = 0, mg = 0;
  uint64_t seed = 0;
  double dt = 0;
  std::vector<long long> n_init;
  std::vector<double> T_eV;
  int sample_every = 0;
  int quiet = 0;  // loader: evenly spaced positions (quiet start)
  // tallies: EEDF region (centre < 0: L/2) and bins, impact bins
  double eedf_center = -1.0, eedf_halfwidth = 0.5e-3, eedf_dE = 0.5, iedf_dE = 2.0;
  int eedf_bins = 100, iedf_bins = 256, iad_bins = 90;
  long long step_end = LLONG_MAX;
  // particle rebalancing (weight multipliers on): every rb_every steps (0:
  // on demand only), merge above rb_hi, split below rb_lo, aim rb_target;
  // loaded particles get multiplier rb_m0 and the species base weight w / rb_m0
  bool rb = false;
  int rb_every = 0, rb_target = 0, rb_lo = 0, rb_hi = 0;
  unsigned rb_m0 = 1;
};

// base weight of a species (a particle of multiplier k weighs k times it)
inline double base_weight(const RunSpec& s, int species) {
  return s.species[species].w / (s.rb ? (double)s.rb_m0 : 1.0);
}

// argument checks of a complete run description; "" when valid
std::string validate_grid(const std::vector<double>& edges, int bc);
std::string validate_spec(const RunSpec& s);
std::string validate_tallies(const RunSpec& s);
// null-collision bound of a species (FP64, host): nu_max and the 24-bit
// candidate threshold
void null_rate(const HostSpecies& sp, const RunSpec& s, double* nu_max, uint32_t* thr24);
// bytes of device memory a run needs
size_t run_bytes(const RunSpec& s);

struct Diag {
  RunState st;
  std::vector<double> acc;
  std::vector<unsigned long long> tal;  // ns * (eedf + iedf + iad bins)
  std::vector<double> pw;               // ns * N
  int eedf_c0 = 0, eedf_c1 = -1;
  long long n_live[kMaxSpecies] = {0, 0, 0, 0};
  int N = 0, ns = 0;
};

// fill the public diagnostics record from a device snapshot
void fill_diag(const Diag& d, const RunSpec& spec, ecpic_diag* out);

class Batch {
 public:
  Batch(int device, cudaStream_t stream, int max_slots, int species_per_slot, int nmax);
  ~Batch();
  Batch(const Batch&) = delete;
  Batch& operator=(const Batch&) = delete;

  // allocate, upload, load particles (Philox), first deposit and field;
  // with defer, the loading, deposit and field wait for admit_wave(), which
  // forms them for every run admitted since in three launches
  int admit(int slot, const RunSpec& spec, std::string* err, bool defer = false);
  int admit_wave(std::string* err);
  void release(int slot);
  bool slot_active(int slot) const { return slot >= 0 && slot < max_slots_ && active_[slot]; }

  int step(long long n, std::string* err);  // async unless growth is on
  // grow species' capacities to at least cap[s] (never shrinks), keeping the
  // run's state; between steps, synchronises the stream
  int reserve(int slot, const long long* cap, std::string* err);
  // double the capacity of any species filled beyond `at` of it, checked
  // after every chunk of about 64 steps (synchronises there)
  void set_auto_grow(bool on, double at = 0.75) {
    auto_grow_ = on;
    grow_at_ = at;
  }
  int profile_step(long long n, double* ms, long long* launches, std::string* err);
  // Phase timing of the replayed steps: with it on, the step graphs carry an
  // event-record node after every kernel phase (two instances of each graph
  // alternate, so that one is read while the other runs) and every step the
  // batch advances adds its phases' device times to the sums; phase_times
  // waits for the pending graphs, returns the sums (ms and launches per phase:
  // pass, field, sort, collide; steps and sorts) and clears them.
  int set_phase_timing(bool on, std::string* err);
  int phase_times(double* ms, long long* launches, long long* steps, long long* sorts,
                  std::string* err);
  int since_sort() const { return since_sort_; }
  int sort_now(std::string* err);
  // particle rebalancing of one run now, whatever its cadence (between steps)
  int rebalance_now(int slot, std::string* err);
  // weight multipliers of a species' live particles (order of get_particles)
  int get_weights(int slot, int species, uint32_t* k, long long cap, long long* n, std::string* err);
  int set_weights(int slot, int species, const uint32_t* k, long long n, std::string* err);
  int sync(std::string* err);
  int slot_status(int slot);  // synchronises

  int get_particles(int slot, int species, int32_t* cell, float* xi, float* vx, float* vy,
                    float* vz, uint64_t* id, long long cap, long long* n, std::string* err);
  int set_particles(int slot, int species, const int32_t* cell, const float* xi, const float* vx,
                    const float* vy, const float* vz, const uint64_t* id, long long n,
                    std::string* err);
  int get_fields(int slot, double* phi, float* E, std::string* err);
  int diag(int slot, Diag* out, std::string* err);
  // several slots at once (one synchronisation, a copy per run)
  int diag_many(const std::vector<int>& slots, const std::vector<Diag*>& out, std::string* err);
  int reset_averages(int slot, int sample_every, std::string* err);
  int set_step_end(int slot, long long step_end, std::string* err);
  // synchronise and read every slot's RunState (engine scheduling)
  int read_states(std::vector<RunState>* out, std::string* err);
  int set_sort_every(int k);
  void set_pass_grid(int g) { pass_grid_override_ = g; invalidate_graphs(); }
  // measure (sort cadence, pass grid) candidates on the resident runs and
  // keep the fastest per particle-step; advances the runs (synchronises)
  // (Ks: the sort cadences tried; empty = 8, 16, 32, 64)
  int autotune(long long steps_per_trial, int* sort_every, int* pass_ctas, double* ns_per_pstep,
               std::string* err, const std::vector<int>& Ks = {});
  int pass_grid() const { return pass_grid_; }
  int sort_every() const { return sort_every_; }
  void set_use_graphs(bool on) { use_graphs_ = on; }
  long long live_estimate() const;
  cudaStream_t stream() const { return stream_; }
  int device() const { return device_; }
  size_t bytes_in_use() const { return bytes_in_use_; }
  const RunSpec& spec(int slot) const { return specs_[slot]; }

 private:
  BatchView view() const;
  void upload_run(int slot);
  void refresh(int slot);
  void invalidate_graphs();
  int ensure_graphs(std::string* err);
  int choose_grid() const;
  bool stage_field(int grid) const;
  int step_chunk(long long n, std::string* err);
  // pinned host staging for uploads: a ring of kStageSlots buffers, each
  // reused once the copy recorded after its last use has left (an event);
  // nullptr (and *slot = -1) for larger images or without pinned memory
  static constexpr int kStageSlots = 8;
  static constexpr size_t kStageBytes = (size_t)512 << 10;
  char* stage_slot(size_t bytes, int* slot);
  void stage_done(int slot);  // after the copy from the slot is enqueued
  int grow_full_runs(std::string* err);
  // host-side prediction of the runs' levels (they advance one level per step
  // up to their end), to launch the rebalancing only where a run is due; the
  // kernels check the device state themselves
  bool rb_due_within(int steps) const;
  void advance_levels(int steps);
  void rebalance_launch();
  int check(cudaError_t e, const char* what, std::string* err);
  // a step graph instance with phase events: ev[i] -> ev[i+1] is phase ph[i]
  struct TimedGraph {
    cudaGraphExec_t exec = nullptr;
    std::vector<cudaEvent_t> ev;
    std::vector<int> ph;
    bool pending = false;  // launched, its events not yet read
  };
  int capture(int steps, bool sort, TimedGraph* tg, cudaGraphExec_t* out, std::string* err);
  int launch_timed(TimedGraph* pair, int* next, std::string* err);
  int harvest(TimedGraph* tg, std::string* err);
  void drop_timed(TimedGraph* tg);

  int device_;
  cudaStream_t stream_;
  bool own_stream_ = false;
  int max_slots_, spc_, nmax_, nseg_;
  int sm_count_ = 1;
  RunDev* d_runs_ = nullptr;
  RunState* d_rst_ = nullptr;
  SegDev* d_segs_ = nullptr;
  SegState* d_sst_ = nullptr;
  int* d_hist_ = nullptr;
  int* d_rbcnt_ = nullptr;
  uint8_t* d_rbmode_ = nullptr;
  int* d_rblist_ = nullptr;
  int* d_rbnum_ = nullptr;
  std::vector<long long> level_;  // predicted level of each slot
  // runs admitted with defer, waiting for admit_wave()
  std::vector<int> wave_slots_;
  std::vector<InitParams> wave_params_;
  std::vector<SegState> wave_sst_;  // per slot x species: initial segment states
  std::vector<RunState> wave_rst_;  // per slot: initial run states
  int* d_wave_slots_ = nullptr;
  InitParams* d_wave_params_ = nullptr;
  std::vector<RunDev> h_runs_;
  std::vector<SegDev> h_segs_;
  std::vector<void*> slot_mem_;
  std::vector<size_t> slot_bytes_;
  std::vector<char> active_;
  std::vector<RunSpec> specs_;
  size_t bytes_in_use_ = 0;
  int sort_every_ = 32;
  int since_sort_ = 0;
  bool use_graphs_ = true;
  bool auto_grow_ = false;
  char* stage_ring_ = nullptr;
  cudaEvent_t stage_ev_[kStageSlots] = {};
  bool stage_used_[kStageSlots] = {};
  int stage_next_ = 0;
  double grow_at_ = 0.75;
  int pass_grid_ = 0;
  int pass_grid_override_ = 0;
  bool graph_stage_ = true;
  int graph_weighted_ = 0;  // the graphs were captured for a batch with weighted runs
  cudaGraphExec_t graph_k_ = nullptr;
  cudaGraphExec_t graph_1_ = nullptr;
  bool timing_ = false;
  // sort-cycle, single-step and sort-only graphs with phase events
  TimedGraph tk_[2], t1_[2], ts_[2];
  int tk_next_ = 0, t1_next_ = 0, ts_next_ = 0;
  double tsum_[4] = {0, 0, 0, 0};
  long long tcnt_[4] = {0, 0, 0, 0};
  long long tsteps_ = 0, tsorts_ = 0;
};

}  // namespace ecpic
