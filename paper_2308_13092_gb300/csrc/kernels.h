// kernels.h -- host-side launch wrappers of the libecpic kernels.
#pragma once
#include <cuda_runtime.h>

#include "ecpic_dev.cuh"

namespace ecpic {

constexpr int kPassBlock = 256;
constexpr int kFieldBlock = 256;
constexpr int kCollideBlock = 256;

struct BatchView {
  const RunDev* runs;   // device, max_slots
  RunState* rst;        // device, max_slots
  const SegDev* segs;   // device, nseg
  SegState* sst;        // device, nseg
  int* hist;            // device, sum of N over segments
  int* rbcnt;           // device, nseg * nmax: rebalancing output counts / cursors
  uint8_t* rbmode;      // device, nseg * nmax: rebalancing cell kind (0 keep, 1 listed, 2 skipped)
  int* rblist;          // device, nseg * nmax: the listed (segment, cell) entries
  int* rbnum;           // device: their number
  int max_slots;
  int nseg;
  int nmax;             // largest N in the batch
  int weighted;         // some resident run carries weight multipliers (rebalancing)
};

// `only` argument of the refresh pass and field: the runs admitted in the
// current wave (RunState::fresh set) instead of one slot
constexpr int kOnlyFresh = -2;

struct InitParams {
  long long n[kMaxSpecies];
  double sd[kMaxSpecies];  // sqrt(e T / m)
  int quiet;               // positions X_i = (i + 1/2) L / n instead of Philox
  unsigned rb_m0;          // weight multiplier of loaded particles (rebalancing runs)
};

size_t pass_smem_bytes(const BatchView& b);
size_t field_smem_bytes(const BatchView& b);
int pass_max_ctas_per_sm(const BatchView& b);

// stage_field: each CTA copies its run's field into shared memory first
// (pays when a CTA runs several iterations)
void launch_pass(const BatchView& b, int grid, int mode, int only, cudaStream_t s,
                 bool stage_field = true);
void launch_collide(const BatchView& b, int grid, cudaStream_t s);
void launch_field(const BatchView& b, int advance, int only, cudaStream_t s);
void launch_phi(const BatchView& b, int slot, cudaStream_t s);
void launch_sort(const BatchView& b, int grid, cudaStream_t s);
void launch_sort_phase(const BatchView& b, int grid, int phase, cudaStream_t s);
void launch_init(const BatchView& b, int slot, const InitParams& p, cudaStream_t s);
// Loads the particles of `count` runs (device arrays of slots and their
// parameters); nmax = the largest species load among them.
void launch_init_many(const BatchView& b, const int* slots, const InitParams* ps, int count,
                      long long nmax, cudaStream_t s);
// particle rebalancing of the runs due at their current level (or forced):
// counting sort by cell into the other buffer set, then per cell the merge /
// split plan, its scan, the merged/split particles written back, sizes set
void launch_rebalance(const BatchView& b, int grid, cudaStream_t s);

void launch_deposit_device(int N, long long n, const int* cell, const float* xi,
                           unsigned long long* S, cudaStream_t s);
void launch_deposit2_device(int N, int periodic, long long n, const int* cell, const float* xi,
                            unsigned long long* S, cudaStream_t s);
void read_checks(unsigned long long out[4]);
void launch_philox_device(long long n, const uint32_t* ctr, const uint32_t* key, uint32_t* out,
                          cudaStream_t s);

}  // namespace ecpic
