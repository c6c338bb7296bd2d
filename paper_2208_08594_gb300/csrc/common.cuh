// Shared device/host helpers of the CUDA library (not shared with the oracle).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <vector>

#include "../../include/msp.h"

namespace msp {

constexpr int kWarp = 32;

// Status carried out of internal helpers; CUDA errors map to MSP_ERR_CUDA.
struct Status {
  int code = MSP_OK;
  bool ok() const { return code == MSP_OK; }
};

#define MSP_CUDA_TRY(expr)                                                              \
  do {                                                                                  \
    cudaError_t e_ = (expr);                                                            \
    if (e_ != cudaSuccess) {                                                            \
      msp::set_last_cuda_error(e_, #expr, __FILE__, __LINE__);                          \
      return e_ == cudaErrorMemoryAllocation ? MSP_ERR_NOMEM : MSP_ERR_CUDA;            \
    }                                                                                   \
  } while (0)

#define MSP_TRY(expr)          \
  do {                         \
    int s_ = (expr);           \
    if (s_ < 0) return s_;     \
  } while (0)

void set_last_cuda_error(cudaError_t e, const char* what, const char* file, int line);

// Checks the last kernel launch and counts it (launch statistics, see Probe).
int launch_check(const char* file, int line);

// Optional per-call-site timing of kernel launches with CUDA events recorded on the
// launching stream (enabled by msp_stats_enable(2)); `bytes` is the algorithmic traffic
// of the launch.  Counting of all launches is on when the mode is >= 1.
class Probe {
 public:
  // `launches`: kernel launches the probe brackets (consecutive launches of one kernel
  // are timed as a group: an event pair per launch would cost more than a small launch)
  // `flops`: algorithmic floating-point operations of the launches (2 per FMA), where the
  // kernel's ceiling may be its arithmetic rate rather than memory
  Probe(const char* site, double bytes, cudaStream_t s, int launches = 1, double flops = 0.0);
  ~Probe();
  Probe(const Probe&) = delete;
  Probe& operator=(const Probe&) = delete;

 private:
  int site_ = -1;
  cudaEvent_t e0_ = nullptr, e1_ = nullptr;
  cudaStream_t s_ = nullptr;
  double bytes_ = 0.0;
  double flops_ = 0.0;
  int launches_ = 1;
  bool in_graph_ = false;  // recorded as event nodes of a graph being captured
};

// Net bytes of device memory the calling host thread holds through DevBuf (allocations
// minus releases); the difference across a call is that call's change of footprint.
extern thread_local long long t_dev_bytes;

// Owning device buffer (cudaMallocAsync / cudaFreeAsync would tie lifetime to a stream;
// the handle's buffers outlive any one stream, so plain cudaMalloc is used at setup).
template <typename T>
struct DevBuf {
  T* p = nullptr;
  size_t n = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept : p(o.p), n(o.n) {
    o.p = nullptr;
    o.n = 0;
  }
  DevBuf& operator=(DevBuf&& o) noexcept {
    if (this != &o) {
      release();
      p = o.p;
      n = o.n;
      o.p = nullptr;
      o.n = 0;
    }
    return *this;
  }
  ~DevBuf() { release(); }
  void release() {
    if (p) {
      cudaFree(p);
      t_dev_bytes -= (long long)(n * sizeof(T));
    }
    p = nullptr;
    n = 0;
  }
  int alloc(size_t count) {
    if (count == n && p) return MSP_OK;
    release();
    if (count == 0) return MSP_OK;
    cudaError_t e = cudaMalloc(&p, count * sizeof(T));
    if (e != cudaSuccess) {
      p = nullptr;
      set_last_cuda_error(e, "cudaMalloc", __FILE__, __LINE__);
      return e == cudaErrorMemoryAllocation ? MSP_ERR_NOMEM : MSP_ERR_CUDA;
    }
    n = count;
    t_dev_bytes += (long long)(count * sizeof(T));
    return MSP_OK;
  }
  T* get() const { return p; }
  size_t bytes() const { return n * sizeof(T); }
};

inline unsigned div_up(size_t a, size_t b) { return (unsigned)((a + b - 1) / b); }

// Grid size for grid-stride kernels: a multiple of the SM count (152 on GB300).
int sm_count();
inline unsigned grid_for(size_t work, unsigned block, unsigned per_sm = 8) {
  size_t blocks = (work + block - 1) / block;
  size_t cap = (size_t)sm_count() * per_sm;
  if (blocks > cap) blocks = cap;
  return blocks == 0 ? 1u : (unsigned)blocks;
}

// Device error flags written by kernels (first error wins).
struct DevFlags {
  int code;    // MSP_OK or an MSP_ERR_* status
  int index;   // offending row / block
  int count;   // generic counter (rounds, undecided nodes, ...)
  int pad;
};

}  // namespace msp
