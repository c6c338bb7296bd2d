// Sorting and scanning primitives of the setup phase (CUB radix sort and scan), and
// the symmetrised adjacency matrix S of Eq. (adjacency-matrix) built with them.
#include <cuda_runtime.h>

#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>

#include "common.cuh"
#include "setup_kernels.h"

namespace msp {

struct SortScratch {
  DevBuf<unsigned char> temp;
  DevBuf<unsigned long long> keys_alt;
  DevBuf<int> vals_alt;
};

SortScratch* sort_scratch_create() { return new SortScratch(); }
void sort_scratch_destroy(SortScratch* s) { delete s; }

namespace {

constexpr int kThreads = 256;

inline int launch_status() { return launch_check(__FILE__, __LINE__); }

int ensure_temp(SortScratch* ss, size_t bytes) {
  if (ss->temp.n >= bytes && ss->temp.p) return MSP_OK;
  return ss->temp.alloc(bytes + bytes / 4 + 256);
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

int sort_pairs_u64(SortScratch* ss, size_t n, unsigned long long* keys, int* vals, int end_bit,
                   cudaStream_t s) {
  if (n <= 1) return MSP_OK;
  MSP_TRY(ss->keys_alt.n >= n ? MSP_OK : ss->keys_alt.alloc(n));
  if (vals) MSP_TRY(ss->vals_alt.n >= n ? MSP_OK : ss->vals_alt.alloc(n));
  size_t bytes = 0;
  cub::DoubleBuffer<unsigned long long> kb(keys, ss->keys_alt.p);
  if (vals) {
    cub::DoubleBuffer<int> vb(vals, ss->vals_alt.p);
    MSP_CUDA_TRY(cub::DeviceRadixSort::SortPairs(nullptr, bytes, kb, vb, (int)n, 0, end_bit, s));
    MSP_TRY(ensure_temp(ss, bytes));
    bytes = ss->temp.n;
    MSP_CUDA_TRY(cub::DeviceRadixSort::SortPairs(ss->temp.p, bytes, kb, vb, (int)n, 0, end_bit, s));
    if (vb.Current() != vals)
      MSP_CUDA_TRY(cudaMemcpyAsync(vals, vb.Current(), n * sizeof(int), cudaMemcpyDeviceToDevice, s));
  } else {
    MSP_CUDA_TRY(cub::DeviceRadixSort::SortKeys(nullptr, bytes, kb, (int)n, 0, end_bit, s));
    MSP_TRY(ensure_temp(ss, bytes));
    bytes = ss->temp.n;
    MSP_CUDA_TRY(cub::DeviceRadixSort::SortKeys(ss->temp.p, bytes, kb, (int)n, 0, end_bit, s));
  }
  if (kb.Current() != keys)
    MSP_CUDA_TRY(cudaMemcpyAsync(keys, kb.Current(), n * sizeof(unsigned long long),
                                 cudaMemcpyDeviceToDevice, s));
  return MSP_OK;
}

int exclusive_scan_int(SortScratch* ss, size_t n, const int* in, int* out, cudaStream_t s) {
  if (n == 0) return MSP_OK;
  size_t bytes = 0;
  MSP_CUDA_TRY(cub::DeviceScan::ExclusiveSum(nullptr, bytes, in, out, (int)n, s));
  MSP_TRY(ensure_temp(ss, bytes));
  bytes = ss->temp.n;
  MSP_CUDA_TRY(cub::DeviceScan::ExclusiveSum(ss->temp.p, bytes, in, out, (int)n, s));
  return MSP_OK;
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
