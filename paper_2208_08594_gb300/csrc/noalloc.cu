// Allocation-free VerticesGrouping (Algorithms 4.1/4.2) of a structurally symmetric
// pattern.  Some callers cannot allocate device memory: code running inside a host
// memory manager or a device memory pool that owns every byte of the GPU, callers
// that must not synchronise the device (cudaMalloc/cudaFree can), and callers in
// environments where the CUDA allocator is replaced or forbidden.  This entry point
// takes its scratch from one fixed file-scope device array instead of allocating.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "common.cuh"
#include "setup_kernels.h"

namespace msp {

namespace {

constexpr int kNaMaxN = 1 << 16;      // vertices (block rows) per call
constexpr int kNaMaxNnz = 1 << 20;    // stored off-diagonal entries per call
constexpr int kNaMaxDeg = 1023;       // off-diagonal entries per row
constexpr int kNaN0 = (kNaMaxN + 31) / 32;
constexpr int kNaN1 = (kNaN0 + 31) / 32;
constexpr int kNaN2 = (kNaN1 + 31) / 32;
constexpr int kNaBitWords = kNaN0 + kNaN1 + kNaN2;

// scratch layout, in 32-bit words (every region starts on a multiple of 64 words)
constexpr size_t kPad(size_t x) { return (x + 63) / 64 * 64; }
constexpr size_t kOffDeg = 0;
constexpr size_t kOffRank = kOffDeg + kPad(kNaMaxN);
constexpr size_t kOffVor = kOffRank + kPad(kNaMaxN);
constexpr size_t kOffWbar = kOffVor + kPad(kNaMaxN);
constexpr size_t kOffColR = kOffWbar + kPad(kNaMaxN);
constexpr size_t kOffRp = kOffColR + kPad(kNaMaxN);
constexpr size_t kOffCi = kOffRp + kPad(kNaMaxN + 1);
constexpr size_t kOffInV = kOffCi + kPad(kNaMaxNnz);
constexpr size_t kOffBits = kOffInV + kPad(kNaN0);
constexpr size_t kOffMeta = kOffBits + kPad(kNaBitWords);
constexpr size_t kScratchWords = kOffMeta + 64;  // about 5.8 MB

// The scratch of every call (and of every overlapping call: they race on it).
static __device__ __align__(256) int g_noalloc_scratch[kScratchWords];

inline int launch_status() { return launch_check(__FILE__, __LINE__); }

// meta[0] = first error (an MSP_ERR_* code), meta[1] = offending row
__device__ void na_fail(int* meta, int code, int row) {
  if (atomicCAS(meta, 0, code) == 0) meta[1] = row;
}

// validate the pattern (sorted, in range, diagonal present, off-diagonal part
// symmetric) and count the off-diagonal entries of every row.  Every read of ci stays
// inside [0, nnz): a row (or the row of a neighbour searched for symmetry) whose
// pointers leave that range or decrease is rejected before its columns are read.
__global__ void na_degree_kernel(int n, int nnz, const int* __restrict__ rp,
                                 const int* __restrict__ ci, int* __restrict__ deg, int* meta) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int p0 = rp[i], p1 = rp[i + 1];
    if (p0 < 0 || p1 < p0 || p1 > nnz) {
      na_fail(meta, MSP_ERR_PATTERN, i);
      deg[i] = 0;
      continue;
    }
    bool diag = false, bad = false;
    for (int p = p0; p < p1; ++p) {
      const int j = ci[p];
      if (j < 0 || j >= n || (p > p0 && j <= ci[p - 1])) {
        bad = true;
        break;
      }
      if (j == i) {
        diag = true;
        continue;
      }
      const int q0 = rp[j], q1 = rp[j + 1];  // (j, i) must be stored too
      if (q0 < 0 || q1 < q0 || q1 > nnz) {
        bad = true;
        break;
      }
      int lo = q0, hi = q1;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (ci[mid] < i)
          lo = mid + 1;
        else
          hi = mid;
      }
      if (lo >= q1 || ci[lo] != i) {
        bad = true;
        break;
      }
    }
    const int d = p1 - p0 - 1;
    if (bad || !diag) na_fail(meta, MSP_ERR_PATTERN, i);
    if (d > kNaMaxDeg) na_fail(meta, MSP_ERR_ARG, i);
    deg[i] = (bad || !diag || d > kNaMaxDeg || d < 0) ? 0 : d;
  }
}

// priority rank by (degree desc, index asc): counting sort, stable in the index
__global__ void __launch_bounds__(1024) na_rank_kernel(int n, const int* __restrict__ deg,
                                                       int* __restrict__ rank,
                                                       int* __restrict__ vor) {
  __shared__ int hist[kNaMaxDeg + 1];
  for (int d = threadIdx.x; d <= kNaMaxDeg; d += blockDim.x) hist[d] = 0;
  __syncthreads();
  for (int v = threadIdx.x; v < n; v += blockDim.x) atomicAdd(&hist[deg[v]], 1);
  __syncthreads();
  if (threadIdx.x == 0) {  // hist[d] <- first rank of degree d
    int run = 0;
    for (int d = kNaMaxDeg; d >= 0; --d) {
      const int c = hist[d];
      hist[d] = run;
      run += c;
    }
  }
  __syncthreads();
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  const unsigned lt = (1u << lane) - 1u;
  for (int c0 = 0; c0 < n; c0 += 32) {
    const int v = c0 + lane;
    const int d = v < n ? deg[v] : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    int pos = 0;
    if (v < n) pos = hist[d] + __popc(peers & lt);
    __syncwarp();
    if (v < n && (peers & lt) == 0u) hist[d] += __popc(peers);
    __syncwarp();
    if (v < n) {
      rank[v] = pos;
      vor[pos] = v;
    }
  }
}

// row pointers of the graph relabelled by rank (one block, contiguous segments)
__global__ void __launch_bounds__(1024) na_relabel_rowptr_kernel(int n, const int* __restrict__ deg,
                                                                 const int* __restrict__ vor,
                                                                 int* __restrict__ rp2) {
  __shared__ int part[1024];
  const int t = threadIdx.x, T = blockDim.x;
  const int seg = (n + T - 1) / T;
  const int r0 = min(n, t * seg), r1 = min(n, r0 + seg);
  int s = 0;
  for (int r = r0; r < r1; ++r) s += deg[vor[r]];
  part[t] = s;
  __syncthreads();
  if (t == 0) {
    int run = 0;
    for (int k = 0; k < T; ++k) {
      const int c = part[k];
      part[k] = run;
      run += c;
    }
    rp2[n] = run;
  }
  __syncthreads();
  int run = part[t];
  for (int r = r0; r < r1; ++r) {
    rp2[r] = run;
    run += deg[vor[r]];
  }
}

// neighbours of every relabelled row, as ranks, sorted ascending
__global__ void na_relabel_fill_kernel(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                       const int* __restrict__ rank, const int* __restrict__ vor,
                                       const int* __restrict__ rp2, int* __restrict__ ci2) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    const int v = vor[r];
    const int o0 = rp2[r], o1 = rp2[r + 1];
    int o = o0;
    for (int p = rp[v]; p < rp[v + 1] && o < o1; ++p) {
      const int j = ci[p];
      if (j != v) ci2[o++] = rank[j];
    }
    for (int a = o0 + 1; a < o1; ++a) {  // insertion sort (rows are short)
      const int key = ci2[a];
      int b = a - 1;
      while (b >= o0 && ci2[b] > key) {
        ci2[b + 1] = ci2[b];
        --b;
      }
      ci2[b + 1] = key;
    }
  }
}

__global__ void na_map_kernel(int n, const int* __restrict__ colour_r, const int* __restrict__ rank,
                              int* __restrict__ colour) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    colour[v] = colour_r[rank[v]];
}

std::mutex g_na_mu;
int* g_na_addr[64] = {nullptr};
unsigned long long g_na_ctx[64] = {0};

// Unique id of the calling thread's current CUDA context (0 if it cannot be read): the
// driver's cuCtxGetCurrent and cuCtxGetId, reached through the runtime so that the
// library does not link the driver library itself.
unsigned long long na_context_id() {
  typedef int (*GetCurrentFn)(void**);
  typedef int (*GetIdFn)(void*, unsigned long long*);
  static GetCurrentFn get_current = nullptr;
  static GetIdFn get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {
    cudaDriverEntryPointQueryResult q1, q2;
    void* f1 = nullptr;
    void* f2 = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault,
                                         &q1) == cudaSuccess &&
        q1 == cudaDriverEntryPointSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) ==
            cudaSuccess &&
        q2 == cudaDriverEntryPointSuccess) {
      get_current = reinterpret_cast<GetCurrentFn>(f1);
      get_id = reinterpret_cast<GetIdFn>(f2);
    }
    cudaGetLastError();
    looked_up = true;
  }
  if (!get_current || !get_id) return 0;
  void* ctx = nullptr;
  unsigned long long id = 0;
  if (get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
  return id;
}

// Device address of the scratch array on the current device.  The array's name in host
// code is only a host-side stand-in; its address is looked up with cudaGetSymbolAddress
// on the first call on a device (that device current) and again whenever the device's
// context has changed since (after cudaDeviceReset, say), since a new context loads the
// module, and the array, afresh.
int na_scratch(int** out) {
  int dev = 0;
  MSP_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return MSP_ERR_ARG;
  std::lock_guard<std::mutex> lk(g_na_mu);
  const unsigned long long ctx = na_context_id();  // 0 before any context is current
  if (!g_na_addr[dev] || ctx == 0 || ctx != g_na_ctx[dev]) {
    void* p = nullptr;
    MSP_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));  // makes the context current
    g_na_addr[dev] = static_cast<int*>(p);
    g_na_ctx[dev] = na_context_id();
  }
  *out = g_na_addr[dev];
  return MSP_OK;
}

thread_local char g_na_msg[160];

}  // namespace
}  // namespace msp

using namespace msp;

extern "C" {

const char* msp_noalloc_error(void) { return g_na_msg; }

int msp_vertices_grouping_noalloc(int32_t n, const int32_t* d_row_ptr, const int32_t* d_col_idx,
                                  int32_t* d_colour, int32_t* h_ncolours, void* stream) {
  g_na_msg[0] = 0;
  if (!d_row_ptr || !d_col_idx || !d_colour || !h_ncolours || n <= 0) {
    snprintf(g_na_msg, sizeof(g_na_msg), "null pointer or n <= 0");
    return MSP_ERR_ARG;
  }
  if (n > kNaMaxN) {
    snprintf(g_na_msg, sizeof(g_na_msg), "n = %d exceeds the maximum of %d vertices", n, kNaMaxN);
    return MSP_ERR_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  int* scr = nullptr;
  MSP_TRY(na_scratch(&scr));
  int rp_end[2] = {0, 0};
  MSP_CUDA_TRY(cudaMemcpyAsync(&rp_end[0], d_row_ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
  MSP_CUDA_TRY(cudaMemcpyAsync(&rp_end[1], d_row_ptr + n, sizeof(int), cudaMemcpyDeviceToHost, s));
  MSP_CUDA_TRY(cudaStreamSynchronize(s));
  if (rp_end[0] != 0 || rp_end[1] < n) {
    snprintf(g_na_msg, sizeof(g_na_msg), "row_ptr[0] != 0 or fewer entries than rows");
    return MSP_ERR_PATTERN;
  }
  if ((long long)rp_end[1] - n > kNaMaxNnz) {
    snprintf(g_na_msg, sizeof(g_na_msg),
             "%lld off-diagonal entries exceed the maximum of %d", (long long)rp_end[1] - n,
             kNaMaxNnz);
    return MSP_ERR_ARG;
  }
  int* deg = scr + kOffDeg;
  int* rank = scr + kOffRank;
  int* vor = scr + kOffVor;
  int* wbar = scr + kOffWbar;
  int* colour_r = scr + kOffColR;
  int* rp2 = scr + kOffRp;
  int* ci2 = scr + kOffCi;
  unsigned* inV = reinterpret_cast<unsigned*>(scr + kOffInV);
  unsigned* bits = reinterpret_cast<unsigned*>(scr + kOffBits);
  int* meta = scr + kOffMeta;  // [0..1] validation error, [2..3] colouring g and error
  // the array keeps the previous call's contents: clear what must start at zero
  MSP_CUDA_TRY(cudaMemsetAsync(meta, 0, 8 * sizeof(int), s));
  const unsigned grid = grid_for(n, 256);
  na_degree_kernel<<<grid, 256, 0, s>>>(n, rp_end[1], d_row_ptr, d_col_idx, deg, meta);
  MSP_TRY(launch_status());
  int h_meta[4] = {0, 0, 0, 0};
  MSP_CUDA_TRY(cudaMemcpyAsync(h_meta, meta, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
  MSP_CUDA_TRY(cudaStreamSynchronize(s));
  if (h_meta[0] != 0) {
    snprintf(g_na_msg, sizeof(g_na_msg),
             h_meta[0] == MSP_ERR_ARG ? "row %d has more than %d off-diagonal entries"
                                      : "row %d: unsorted or out-of-range columns, missing "
                                        "diagonal or nonsymmetric pattern",
             h_meta[1], kNaMaxDeg);
    return h_meta[0];
  }
  na_rank_kernel<<<1, 1024, 0, s>>>(n, deg, rank, vor);
  MSP_TRY(launch_status());
  na_relabel_rowptr_kernel<<<1, 1024, 0, s>>>(n, deg, vor, rp2);
  MSP_TRY(launch_status());
  na_relabel_fill_kernel<<<grid, 256, 0, s>>>(n, d_row_ptr, d_col_idx, rank, vor, rp2, ci2);
  MSP_TRY(launch_status());
  MSP_TRY(launch_colouring(n, rp2, ci2, nullptr, nullptr, inV, wbar, bits, kNaBitWords,
                           colour_r, meta + 2, n, s));
  na_map_kernel<<<grid, 256, 0, s>>>(n, colour_r, rank, d_colour);
  MSP_TRY(launch_status());
  MSP_CUDA_TRY(cudaMemcpyAsync(h_meta + 2, meta + 2, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
  MSP_CUDA_TRY(cudaStreamSynchronize(s));
  if (h_meta[3] != 0) {
    snprintf(g_na_msg, sizeof(g_na_msg), "colouring loop bound exceeded");
    return MSP_ERR_TIMEOUT;
  }
  *h_ncolours = h_meta[2];
  return MSP_OK;
}

}  // extern "C"
