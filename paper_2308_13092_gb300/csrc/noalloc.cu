// noalloc.cu -- fixed-point CIC deposit (Eq. 2-3) that allocates no device
// memory: ecpic_deposit_device_noalloc.
//
// Same result as ecpic_deposit_device, reached another way: instead of
// adding each block's shared-memory sums to S with global atomics, every
// block writes its whole partial row (N+1 sums) into a fixed scratch array
// that is part of this module's image, and a second kernel adds the rows to
// S node by node in row order.  The sums are 64-bit integers, so the order
// does not change the result.
//
// Who needs this: callers that must not allocate device memory while they
// run -- a process that handed all free HBM to its own pool at start-up
// (where a cudaMalloc would fail), or a latency-bound loop in which
// cudaMalloc/cudaFree would stall it by synchronising the device.  So this
// path calls no cudaMalloc, cudaFree or allocating library routine.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/ecpic.h"

namespace {

constexpr int kNaBlock = 256;
constexpr int kNaMaxRows = 304;  // two blocks per SM on a 152-SM part
constexpr size_t kNaWords = ECPIC_NOALLOC_SCRATCH_BYTES / sizeof(unsigned long long);
constexpr int kMaxDevices = 64;

static_assert((size_t)(ECPIC_NOALLOC_MAX_CELLS + 1) <= kNaWords, "scratch must hold one row");

// Partial rows: row r = block r's sums for nodes 0..N, row-major.  Every entry
// the reduction reads is written by the same call first, so no part of it has
// to start at zero and no call clears it.
static __device__ __align__(256) unsigned long long g_na_scratch[kNaWords];

// scratch address per device, looked up at the first call on that device and
// kept for the life of the process (a device reset makes it stale: see the
// header)
std::mutex g_na_mu;
void* g_na_ptr[kMaxDevices] = {};

// Block-local deposit of a grid-stride share of the particles, written out
// as this block's row.  Lanes holding the same cell add their shares once
// (r = floor(xi * 2^32); the cell gets 2^32 - r, the next node r).
__global__ void __launch_bounds__(kNaBlock) k_na_rows(int N, long long n, const int* __restrict__ cell,
                                                      const float* __restrict__ xi,
                                                      unsigned long long* rows) {
  extern __shared__ __align__(16) unsigned char na_smem[];
  unsigned long long* acc = reinterpret_cast<unsigned long long*>(na_smem);
  for (int i = threadIdx.x; i <= N; i += kNaBlock) acc[i] = 0ull;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  for (long long base = (long long)blockIdx.x * kNaBlock + (threadIdx.x & ~31); base < n;
       base += (long long)gridDim.x * kNaBlock) {
    const long long i = base + lane;
    const int c = i < n ? cell[i] : -1;
    const bool ok = c >= 0 && c < N;
    const unsigned group = __match_any_sync(0xFFFFFFFFu, ok ? (unsigned)c : 0xFFFFFFFFu);
    if (ok) {
      const unsigned r = __float2uint_rz(xi[i] * 4294967296.0f);
      // the 32-bit shares of up to 32 lanes, summed in two 16-bit halves
      const unsigned lo = __reduce_add_sync(group, r & 0xFFFFu);
      const unsigned hi = __reduce_add_sync(group, r >> 16);
      if (lane == __ffs(group) - 1) {
        const unsigned long long sr = ((unsigned long long)hi << 16) + lo;
        const unsigned long long cnt = (unsigned long long)__popc(group);
        atomicAdd(acc + c, (cnt << 32) - sr);
        atomicAdd(acc + c + 1, sr);
      }
    }
  }
  __syncthreads();
  unsigned long long* row = rows + (size_t)blockIdx.x * (size_t)(N + 1);
  for (int i = threadIdx.x; i <= N; i += kNaBlock) row[i] = acc[i];
}

// S[i] += sum of the rows' entries i, in row order
__global__ void __launch_bounds__(kNaBlock) k_na_sum(int N, int nrows,
                                                     const unsigned long long* __restrict__ rows,
                                                     unsigned long long* S) {
  const int i = blockIdx.x * kNaBlock + threadIdx.x;
  if (i > N) return;
  unsigned long long s = 0ull;
  for (int r = 0; r < nrows; ++r) s += rows[(size_t)r * (size_t)(N + 1) + i];
  S[i] += s;
}

// The scratch address on the current device; the first call on a device
// looks it up (cudaGetSymbolAddress) with that device current.
int na_scratch(unsigned long long** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return ECPIC_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_na_mu);
  if (!g_na_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_na_scratch);
    if (e != cudaSuccess || p == nullptr) return ECPIC_ERR_CUDA;
    g_na_ptr[dev] = p;
  }
  *out = static_cast<unsigned long long*>(g_na_ptr[dev]);
  return ECPIC_OK;
}

}  // namespace

extern "C" int ecpic_deposit_device_noalloc(int N, int64_t n, const int32_t* d_cell, const float* d_xi,
                                            uint64_t* d_S, void* stream) {
  if (N < 1 || n < 0 || (n > 0 && (!d_cell || !d_xi)) || !d_S) return ECPIC_ERR_ARG;
  if (N > ECPIC_NOALLOC_MAX_CELLS) return ECPIC_ERR_CAPACITY;
  unsigned long long* rows = nullptr;
  const int rc = na_scratch(&rows);  // set-up on the first call, even when n == 0
  if (rc != ECPIC_OK) return rc;
  if (n == 0) return ECPIC_OK;
  const long long per_row = (long long)(kNaWords / (size_t)(N + 1));
  long long nrows = (n + kNaBlock - 1) / kNaBlock;
  if (nrows > kNaMaxRows) nrows = kNaMaxRows;
  if (nrows > per_row) nrows = per_row;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // one row of N + 1 sums: at most 8 x 2049 = 16,392 B (N = 2048), within the
  // 48 KiB a launch gets without an opt-in
  const size_t smem = sizeof(unsigned long long) * (size_t)(N + 1);
  k_na_rows<<<(unsigned)nrows, kNaBlock, smem, s>>>(N, (long long)n, d_cell, d_xi, rows);
  k_na_sum<<<(unsigned)((N + 1 + kNaBlock - 1) / kNaBlock), kNaBlock, 0, s>>>(
      N, (int)nrows, rows, reinterpret_cast<unsigned long long*>(d_S));
  return cudaGetLastError() == cudaSuccess ? ECPIC_OK : ECPIC_ERR_CUDA;
}
