// Sorting and scanning primitives of the setup phase (a stable least-significant-digit
// radix sort of 64-bit keys with optional int payloads, and an exclusive scan of ints,
// written here), and the symmetrised adjacency matrix S of Eq. (adjacency-matrix) built
// with them.
#include <cuda_runtime.h>

#include "common.cuh"
#include "setup_kernels.h"

namespace msp {

struct SortScratch {
  DevBuf<unsigned long long> keys_alt;
  DevBuf<int> vals_alt;
  DevBuf<int> counts;                  // radix pass: per-(digit, tile) counts, then offsets
  std::vector<DevBuf<int>> scan_levels;  // tile sums of the recursive scan, one per level
};

SortScratch* sort_scratch_create() { return new SortScratch(); }
void sort_scratch_destroy(SortScratch* s) { delete s; }

namespace {

constexpr int kThreads = 256;
// radix sort: 8-bit digits; a tile is kSortRounds rounds of kThreads consecutive keys
constexpr int kDigitBits = 8;
constexpr int kBuckets = 1 << kDigitBits;
constexpr int kSortRounds = 8;
constexpr int kSortTile = kThreads * kSortRounds;
constexpr int kSortWarps = kThreads / kWarp;
// scan: a tile is kScanItems consecutive ints per thread
constexpr int kScanItems = 8;
constexpr int kScanTile = kThreads * kScanItems;

inline int launch_status() { return launch_check(__FILE__, __LINE__); }

// counts[d * ntiles + t] = keys of tile t whose digit (at `shift`) is d
__global__ void __launch_bounds__(kThreads) radix_hist_kernel(size_t n, const unsigned long long* __restrict__ keys,
                                                             int shift, int ntiles,
                                                             int* __restrict__ counts) {
  __shared__ int hist[kBuckets];
  for (int d = threadIdx.x; d < kBuckets; d += blockDim.x) hist[d] = 0;
  __syncthreads();
  const size_t base = (size_t)blockIdx.x * kSortTile;
#pragma unroll
  for (int r = 0; r < kSortRounds; ++r) {
    const size_t k = base + (size_t)r * kThreads + threadIdx.x;
    if (k < n) atomicAdd(&hist[(int)((keys[k] >> shift) & (kBuckets - 1))], 1);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < kBuckets; d += blockDim.x)
    counts[(size_t)d * ntiles + blockIdx.x] = hist[d];
}

// Stable scatter of one tile: keys in index order (round-major, then warp, then lane) get
// consecutive places among the keys of their digit, starting at offsets[d * ntiles + tile]
// (the exclusive scan of the counts in digit-major order).
__global__ void __launch_bounds__(kThreads) radix_scatter_kernel(
    size_t n, const unsigned long long* __restrict__ keys, const int* __restrict__ vals,
    int shift, int ntiles, const int* __restrict__ offsets, unsigned long long* __restrict__ keys_out,
    int* __restrict__ vals_out) {
  __shared__ int start[kBuckets];              // next place of every digit in this tile
  __shared__ int wcount[kSortWarps][kBuckets];  // per round: keys of digit d in warp w, then
                                                // their first place
  const int lane = threadIdx.x % kWarp, w = threadIdx.x / kWarp;
  for (int d = threadIdx.x; d < kBuckets; d += blockDim.x)
    start[d] = offsets[(size_t)d * ntiles + blockIdx.x];
  const size_t base = (size_t)blockIdx.x * kSortTile;
  const unsigned lt = (1u << lane) - 1u;
  for (int r = 0; r < kSortRounds; ++r) {
    for (int q = threadIdx.x; q < kSortWarps * kBuckets; q += blockDim.x)
      (&wcount[0][0])[q] = 0;
    __syncthreads();
    const size_t k = base + (size_t)r * kThreads + threadIdx.x;
    const bool live = k < n;
    const unsigned long long key = live ? keys[k] : 0ULL;
    const int d = live ? (int)((key >> shift) & (kBuckets - 1)) : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int rank = __popc(peers & lt);
    if (live && rank == 0) wcount[w][d] = __popc(peers);
    __syncthreads();
    for (int dd = threadIdx.x; dd < kBuckets; dd += blockDim.x) {  // prefix over the warps
      int run = start[dd];
#pragma unroll
      for (int ww = 0; ww < kSortWarps; ++ww) {
        const int c = wcount[ww][dd];
        wcount[ww][dd] = run;
        run += c;
      }
      start[dd] = run;
    }
    __syncthreads();
    if (live) {
      const int pos = wcount[w][d] + rank;
      keys_out[pos] = key;
      if (vals) vals_out[pos] = vals[k];
    }
    __syncthreads();  // wcount is cleared for the next round
  }
}

__device__ __forceinline__ int block_exclusive_scan(int v, int* sh, int* total) {
  const int lane = threadIdx.x % kWarp, w = threadIdx.x / kWarp;
  int x = v;
#pragma unroll
  for (int o = 1; o < kWarp; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += t;
  }
  if (lane == kWarp - 1) sh[w] = x;
  __syncthreads();
  if (w == 0) {
    int y = lane < (int)(blockDim.x / kWarp) ? sh[lane] : 0;
#pragma unroll
    for (int o = 1; o < kWarp; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, y, o);
      if (lane >= o) y += t;
    }
    if (lane < (int)(blockDim.x / kWarp)) sh[lane] = y;
  }
  __syncthreads();
  const int before = (w > 0 ? sh[w - 1] : 0) + x - v;
  *total = sh[blockDim.x / kWarp - 1];
  __syncthreads();
  return before;
}

// exclusive scan of every tile of kScanTile ints on its own; sums[tile] = the tile's total
__global__ void __launch_bounds__(kThreads) scan_tiles_kernel(size_t n, const int* __restrict__ in,
                                                             int* __restrict__ out,
                                                             int* __restrict__ sums) {
  __shared__ int sh[kThreads / kWarp];
  const size_t base = (size_t)blockIdx.x * kScanTile + (size_t)threadIdx.x * kScanItems;
  int v[kScanItems];
  int local = 0;
#pragma unroll
  for (int q = 0; q < kScanItems; ++q) {
    v[q] = base + q < n ? in[base + q] : 0;
    local += v[q];
  }
  int total = 0;
  int run = block_exclusive_scan(local, sh, &total);
#pragma unroll
  for (int q = 0; q < kScanItems; ++q) {
    if (base + q < n) out[base + q] = run;
    run += v[q];
  }
  if (threadIdx.x == 0 && sums) sums[blockIdx.x] = total;
}

__global__ void scan_add_kernel(size_t n, const int* __restrict__ add, int* __restrict__ out) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n;
       k += (size_t)gridDim.x * blockDim.x)
    out[k] += add[k / kScanTile];
}

// exclusive scan through `level` levels of tile sums (tile sums of tile sums ...)
int scan_recursive(SortScratch* ss, size_t n, const int* in, int* out, size_t level,
                   cudaStream_t s) {
  const size_t ntiles = (n + kScanTile - 1) / kScanTile;
  if (ntiles <= 1) {
    scan_tiles_kernel<<<1, kThreads, 0, s>>>(n, in, out, nullptr);
    return launch_status();
  }
  if (ss->scan_levels.size() <= level) ss->scan_levels.resize(level + 1);
  if (ss->scan_levels[level].n < 2 * ntiles)
    MSP_TRY(ss->scan_levels[level].alloc(2 * ntiles));  // sums, then their scan
  // the pointer, not a reference into the vector: the recursion may grow the vector
  int* sums = ss->scan_levels[level].p;
  scan_tiles_kernel<<<(unsigned)ntiles, kThreads, 0, s>>>(n, in, out, sums);
  MSP_TRY(launch_status());
  MSP_TRY(scan_recursive(ss, ntiles, sums, sums + ntiles, level + 1, s));
  scan_add_kernel<<<grid_for(n, kThreads), kThreads, 0, s>>>(n, sums + ntiles, out);
  return launch_status();
}

// keys of every stored off-diagonal entry in both directions; diagonal -> ~0 (sorts last)
__global__ void adjacency_keys_kernel(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                      unsigned long long* __restrict__ keys) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    for (int p = rp[i]; p < rp[i + 1]; ++p) {
      const unsigned long long j = (unsigned)ci[p];
      if (j == (unsigned long long)i) {
        keys[2 * (size_t)p] = ~0ULL;
        keys[2 * (size_t)p + 1] = ~0ULL;
      } else {
        keys[2 * (size_t)p] = ((unsigned long long)i << 32) | j;
        keys[2 * (size_t)p + 1] = (j << 32) | (unsigned long long)i;
      }
    }
  }
}

__global__ void unique_flags_kernel(size_t m, const unsigned long long* __restrict__ keys,
                                    int* __restrict__ flags) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < m;
       k += (size_t)gridDim.x * blockDim.x)
    flags[k] = (keys[k] != ~0ULL && (k == 0 || keys[k] != keys[k - 1])) ? 1 : 0;
}

__global__ void unique_compact_kernel(size_t m, const unsigned long long* __restrict__ keys,
                                      const int* __restrict__ flags, const int* __restrict__ pos,
                                      unsigned long long* __restrict__ out) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < m;
       k += (size_t)gridDim.x * blockDim.x)
    if (flags[k]) out[pos[k]] = keys[k];
}

// row_ptr[r] = first k with (keys[k] >> 32) >= r, for sorted keys with rows < n
__global__ void rowptr_from_keys_kernel(size_t m, int n, const unsigned long long* __restrict__ keys,
                                        int* __restrict__ row_ptr) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k <= m;
       k += (size_t)gridDim.x * blockDim.x) {
    const long long prev = (k == 0) ? -1 : (long long)(keys[k - 1] >> 32);
    const long long cur = (k == m) ? (long long)n : (long long)(keys[k] >> 32);
    for (long long r = prev + 1; r <= cur; ++r) row_ptr[r] = (int)k;
  }
}

__global__ void low32_kernel(size_t m, const unsigned long long* __restrict__ keys,
                             int* __restrict__ out) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < m;
       k += (size_t)gridDim.x * blockDim.x)
    out[k] = (int)(keys[k] & 0xffffffffULL);
}

}  // namespace

// Stable LSD radix sort of keys[0..n) (bits [0, end_bit)), vals permuted alongside when
// given; the result is in keys/vals.
int sort_pairs_u64(SortScratch* ss, size_t n, unsigned long long* keys, int* vals, int end_bit,
                   cudaStream_t s) {
  if (n <= 1) return MSP_OK;
  if (n > 0x7fffffffULL || end_bit < 1 || end_bit > 64) return MSP_ERR_ARG;
  MSP_TRY(ss->keys_alt.n >= n ? MSP_OK : ss->keys_alt.alloc(n));
  if (vals) MSP_TRY(ss->vals_alt.n >= n ? MSP_OK : ss->vals_alt.alloc(n));
  const int ntiles = (int)((n + kSortTile - 1) / kSortTile);
  const size_t ncounts = (size_t)kBuckets * ntiles;
  MSP_TRY(ss->counts.n >= 2 * ncounts ? MSP_OK : ss->counts.alloc(2 * ncounts));
  int* counts = ss->counts.p;
  int* offsets = ss->counts.p + ncounts;
  unsigned long long *kin = keys, *kout = ss->keys_alt.p;
  int *vin = vals, *vout = vals ? ss->vals_alt.p : nullptr;
  for (int shift = 0; shift < end_bit; shift += kDigitBits) {
    radix_hist_kernel<<<ntiles, kThreads, 0, s>>>(n, kin, shift, ntiles, counts);
    MSP_TRY(launch_status());
    MSP_TRY(scan_recursive(ss, ncounts, counts, offsets, 0, s));
    radix_scatter_kernel<<<ntiles, kThreads, 0, s>>>(n, kin, vin, shift, ntiles, offsets, kout,
                                                     vout);
    MSP_TRY(launch_status());
    std::swap(kin, kout);
    std::swap(vin, vout);
  }
  if (kin != keys) {
    MSP_CUDA_TRY(cudaMemcpyAsync(keys, kin, n * sizeof(unsigned long long),
                                 cudaMemcpyDeviceToDevice, s));
    if (vals)
      MSP_CUDA_TRY(cudaMemcpyAsync(vals, vin, n * sizeof(int), cudaMemcpyDeviceToDevice, s));
  }
  return MSP_OK;
}

int exclusive_scan_int(SortScratch* ss, size_t n, const int* in, int* out, cudaStream_t s) {
  if (n == 0) return MSP_OK;
  if (n > 0x7fffffffULL) return MSP_ERR_ARG;
  return scan_recursive(ss, n, in, out, 0, s);
}

int unique_sorted_keys(SortScratch* ss, size_t m, unsigned long long* keys, size_t* m_out,
                       DevBuf<unsigned long long>& out, cudaStream_t s) {
  DevBuf<int> flags, pos;
  MSP_TRY(flags.alloc(m + 1));
  MSP_TRY(pos.alloc(m + 1));
  unique_flags_kernel<<<grid_for(m, kThreads), kThreads, 0, s>>>(m, keys, flags.p);
  MSP_TRY(launch_status());
  MSP_TRY(exclusive_scan_int(ss, m, flags.p, pos.p, s));
  int last_pos = 0, last_flag = 0;
  if (m > 0) {
    MSP_CUDA_TRY(cudaMemcpyAsync(&last_pos, pos.p + m - 1, sizeof(int), cudaMemcpyDeviceToHost, s));
    MSP_CUDA_TRY(cudaMemcpyAsync(&last_flag, flags.p + m - 1, sizeof(int), cudaMemcpyDeviceToHost, s));
    MSP_CUDA_TRY(cudaStreamSynchronize(s));
  }
  const size_t mu = (size_t)last_pos + last_flag;
  MSP_TRY(out.alloc(mu > 0 ? mu : 1));
  if (m > 0) {
    unique_compact_kernel<<<grid_for(m, kThreads), kThreads, 0, s>>>(m, keys, flags.p, pos.p, out.p);
    MSP_TRY(launch_status());
  }
  *m_out = mu;
  // keep the temporaries alive until the kernels that use them have run
  MSP_CUDA_TRY(cudaStreamSynchronize(s));
  return MSP_OK;
}

int rowptr_from_sorted_keys(size_t m, int n, const unsigned long long* keys, int* row_ptr,
                            cudaStream_t s) {
  rowptr_from_keys_kernel<<<grid_for(m + 1, kThreads), kThreads, 0, s>>>(m, n, keys, row_ptr);
  return launch_status();
}

int low32_of_keys(size_t m, const unsigned long long* keys, int* out, cudaStream_t s) {
  if (!m) return MSP_OK;
  low32_kernel<<<grid_for(m, kThreads), kThreads, 0, s>>>(m, keys, out);
  return launch_status();
}

int build_adjacency(SortScratch* ss, int n, const int* rp, const int* ci, int nnz,
                    DevBuf<int>& srp, DevBuf<int>& sci, int* snnz, cudaStream_t s) {
  const size_t m = 2 * (size_t)nnz;
  DevBuf<unsigned long long> keys, ukeys;
  MSP_TRY(keys.alloc(m > 0 ? m : 1));
  adjacency_keys_kernel<<<grid_for(n, kThreads), kThreads, 0, s>>>(n, rp, ci, keys.p);
  MSP_TRY(launch_status());
  MSP_TRY(sort_pairs_u64(ss, m, keys.p, nullptr, 64, s));
  size_t mu = 0;
  MSP_TRY(unique_sorted_keys(ss, m, keys.p, &mu, ukeys, s));
  MSP_TRY(srp.alloc(n + 1));
  MSP_TRY(sci.alloc(mu > 0 ? mu : 1));
  MSP_TRY(rowptr_from_sorted_keys(mu, n, ukeys.p, srp.p, s));
  MSP_TRY(low32_of_keys(mu, ukeys.p, sci.p, s));
  *snnz = (int)mu;
  MSP_CUDA_TRY(cudaStreamSynchronize(s));
  return MSP_OK;
}

}  // namespace msp
