// Host orchestration and the C ABI of the solver (include/msp.h).
//
// SETUP (Section 3): block-graph adjacency (Eq. adjacency-matrix), VerticesGrouping
// (Algorithms 4.1/4.2) and the colour permutation (Algorithm 4.3 step 3) once per
// pattern; per value setup the quasi-IMPES decoupling, the UA-AMG hierarchy (pairwise
// matching, Galerkin products, PGS-MC colourings, dense coarsest inverse), the stage-N
// sub-blocks and BILU(0) in colour order.  SOLVE: right-preconditioned FGMRES(m) with
// classical Gram-Schmidt and one re-orthogonalisation, the Hessenberg least squares in
// FP64 on the host, and Algorithm 3.1 as the preconditioner.  ASMSP (Section 3.2): a
// solve regenerates B iff the previous solve took more than mu iterations.
// Also here: the batched solve of the instances of a block-diagonal matrix (one FGMRES
// per instance, shared launches, a row mask for the instances that have converged), the
// pipelined value update (the copy of the next values on another stream), launch and
// per-site timing statistics, and the device-memory count of a handle.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "setup_kernels.h"

namespace msp {

namespace {
thread_local std::string g_last_error;
thread_local int t_bytes_scope_depth = 0;
}

thread_local long long t_dev_bytes = 0;

namespace {
// NVTX range over a host scope (setup phases, solves, Krylov cycles, preconditioner
// applications), visible in a timeline profiler; a no-op when no tool is attached.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
}  // namespace

void set_last_cuda_error(cudaError_t e, const char* what, const char* file, int line) {
  char buf[512];
  snprintf(buf, sizeof(buf), "%s: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
  g_last_error = buf;
}

// ---------------------------------------------------------------------------------
// launch statistics (msp_stats_*): launch counting and per-site CUDA-event timing
// ---------------------------------------------------------------------------------
namespace {
struct StatSite {
  std::string name;
  long long launches = 0;
  double ms = 0.0, bytes = 0.0, flops = 0.0;
};
struct PendingTiming {
  int site;
  cudaEvent_t e0, e1;
  bool graph_owned;  // event nodes of a captured graph: not returned to the pool
};
// a timed site inside a captured graph: its two event-record nodes
struct GraphProbe {
  int site;
  cudaEvent_t e0, e1;
  double bytes;
  int launches;
  double flops;
};
std::mutex g_stats_mu;
int g_stats_mode = 0;
long long g_launches = 0;
// while a CUDA graph is being captured on this thread, launches and probe bytes are
// tallied here instead of being counted / timed
thread_local bool t_capturing = false;
thread_local long long t_cap_launches = 0;
thread_local double t_cap_bytes = 0.0;
// stats mode 3 at capture time: every probe also becomes a pair of event-record nodes
thread_local bool t_cap_timed = false;
thread_local std::vector<GraphProbe> t_cap_probes;
std::vector<StatSite> g_sites;
std::vector<PendingTiming> g_pending;
std::vector<cudaEvent_t> g_free_events;

cudaEvent_t take_event() {
  if (!g_free_events.empty()) {
    cudaEvent_t e = g_free_events.back();
    g_free_events.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

int site_index(const char* name) {
  for (size_t k = 0; k < g_sites.size(); ++k)
    if (g_sites[k].name == name) return (int)k;
  g_sites.push_back(StatSite{name});
  return (int)g_sites.size() - 1;
}

// algorithmic bytes known only after a launch (device-side decisions) for a timed site
void stats_add_bytes(const char* site, double bytes, double flops = 0.0) {
  if (g_stats_mode < 2) return;
  std::lock_guard<std::mutex> lk(g_stats_mu);
  auto& st = g_sites[site_index(site)];
  st.bytes += bytes;
  st.flops += flops;
}

// fold finished timings into the sites (waits for the recorded events)
void resolve_pending() {
  for (auto& p : g_pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(p.e1) == cudaSuccess && cudaEventElapsedTime(&ms, p.e0, p.e1) == cudaSuccess)
      g_sites[p.site].ms += ms;
    if (!p.graph_owned) {
      g_free_events.push_back(p.e0);
      g_free_events.push_back(p.e1);
    }
  }
  g_pending.clear();
}
}  // namespace

int launch_check(const char* file, int line) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_last_cuda_error(e, "kernel launch", file, line);
    return MSP_ERR_CUDA;
  }
  if (t_capturing) {
    ++t_cap_launches;
    return MSP_OK;
  }
  if (g_stats_mode >= 1) {
    std::lock_guard<std::mutex> lk(g_stats_mu);
    ++g_launches;
  }
  return MSP_OK;
}

Probe::Probe(const char* site, double bytes, cudaStream_t s, int launches, double flops)
    : s_(s), bytes_(bytes), launches_(launches), flops_(flops) {
  if (t_capturing) {
    t_cap_bytes += bytes;
    if (!t_cap_timed) return;
    std::lock_guard<std::mutex> lk(g_stats_mu);
    e0_ = take_event();
    e1_ = take_event();
    if (!e0_ || !e1_) return;
    site_ = site_index(site);
    in_graph_ = true;
    cudaEventRecordWithFlags(e0_, s_, cudaEventRecordExternal);
    return;
  }
  if (g_stats_mode < 2) return;
  std::lock_guard<std::mutex> lk(g_stats_mu);
  e0_ = take_event();
  e1_ = take_event();
  if (!e0_ || !e1_) return;
  site_ = site_index(site);
  g_sites[site_].bytes += bytes;
  g_sites[site_].flops += flops;
  g_sites[site_].launches += launches;
  cudaEventRecord(e0_, s_);
}

Probe::~Probe() {
  if (site_ < 0) return;
  if (in_graph_) {
    cudaEventRecordWithFlags(e1_, s_, cudaEventRecordExternal);
    t_cap_probes.push_back(GraphProbe{site_, e0_, e1_, bytes_, launches_, flops_});
    return;
  }
  cudaEventRecord(e1_, s_);
  std::lock_guard<std::mutex> lk(g_stats_mu);
  g_pending.push_back(PendingTiming{site_, e0_, e1_, false});
}

int sm_count() {
  static const int cached = [] {  // thread-safe one-time initialisation
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && n > 0)
      return n;
    return 152;
  }();
  return cached;
}

namespace {

constexpr int kThreads = 256;
// Block rows with more blocks than this are walked by a warp in the level-0 block-row
// kernels (the lane-group walk of a row is a chain of dependent loads two blocks long per
// step: a well row perforating 85 layers alone would outlast a colour sweep of a million
// cells).
constexpr int kLongRowBlocks = 16;
using Clock = std::chrono::steady_clock;
double ms_since(Clock::time_point t0) {
  return std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
}

inline int launch_status() { return launch_check(__FILE__, __LINE__); }

// ---------------------------------------------------------------------------------
// small host-orchestration kernels
// ---------------------------------------------------------------------------------
__global__ void rank_keys_kernel(int n, const int* __restrict__ srp, unsigned long long* keys) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const unsigned deg = (unsigned)(srp[v + 1] - srp[v]);
    keys[v] = ((unsigned long long)(0x7fffffffu - deg) << 32) | (unsigned)v;
  }
}

__global__ void colour_keys_kernel(int n, const int* __restrict__ colour, unsigned long long* keys) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    keys[v] = ((unsigned long long)(unsigned)colour[v] << 32) | (unsigned)v;
}

__global__ void perm_keys_kernel(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                 const int* __restrict__ rowmap, const int* __restrict__ colmap,
                                 unsigned long long* __restrict__ keys, int* __restrict__ vals) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const unsigned long long r = (unsigned)rowmap[i];
    for (int p = rp[i]; p < rp[i + 1]; ++p) {
      keys[p] = (r << 32) | (unsigned)colmap[ci[p]];
      vals[p] = p;
    }
  }
}

__global__ void seg_flags_kernel(size_t m, const unsigned long long* __restrict__ keys,
                                 int* __restrict__ flags) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < m;
       k += (size_t)gridDim.x * blockDim.x)
    flags[k] = (k == 0 || keys[k] != keys[k - 1]) ? 1 : 0;
}

__global__ void seg_compact_kernel(size_t m, const unsigned long long* __restrict__ keys,
                                   const int* __restrict__ flags, const int* __restrict__ pos,
                                   unsigned long long* __restrict__ ukeys,
                                   int* __restrict__ seg_start, int nseg) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < m;
       k += (size_t)gridDim.x * blockDim.x)
    if (flags[k]) {
      ukeys[pos[k]] = keys[k];
      seg_start[pos[k]] = (int)k;
    }
  if (blockIdx.x == 0 && threadIdx.x == 0) seg_start[nseg] = (int)m;
}

__global__ void gather_double_kernel(size_t m, const int* __restrict__ src,
                                     const double* __restrict__ in, double* __restrict__ out) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < m;
       k += (size_t)gridDim.x * blockDim.x)
    out[k] = in[src[k]];
}

__global__ void compose_kernel(int n, const int* __restrict__ a1, int* __restrict__ agg) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    agg[i] = a1[agg[i]];
}

__global__ void map_kernel(int n, const int* __restrict__ m, const int* __restrict__ in,
                           int* __restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    out[i] = m[in[i]];
}

// inst_c[agg[i]] = inst_f[i]: an aggregate's members all belong to one instance (the
// matrix is block diagonal over the instances, so no pair crosses two of them)
__global__ void inst_scatter_kernel(int n, const int* __restrict__ agg,
                                    const int* __restrict__ inst_f, int* __restrict__ inst_c) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    inst_c[agg[i]] = inst_f[i];
}

__global__ void member_keys_kernel(int n, const int* __restrict__ agg, unsigned long long* keys) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    keys[i] = ((unsigned long long)(unsigned)agg[i] << 32) | (unsigned)i;
}

template <typename T>
unsigned grid1(T n) {
  return grid_for((size_t)n, kThreads);
}

// ---------------------------------------------------------------------------------
// device CSR and levels
// ---------------------------------------------------------------------------------
struct DCsr {
  int n = 0, nnz = 0;
  DevBuf<int> rp, ci;
  DevBuf<double> v;
};

// nonzeros left / right of the diagonal in the rows of every colour class (for the
// algorithmic byte counts of the sweeps)
struct ColourCounts {
  std::vector<long long> lower, upper;
};

// Slots per row of a level's ELL copy: the smallest of 8, 16, 24, 32 that leaves at most
// max(16, n / 1024) rows longer (those keep the CSR path); 0 if none does.
int ell_width(const std::vector<int>& rp, int n) {
  int hist[4] = {0, 0, 0, 0};  // rows with more than 8, 16, 24, 32 off-diagonal entries
  for (int i = 0; i < n; ++i) {
    const int len = rp[i + 1] - rp[i] - 1;
    for (int t = 0; t < 4; ++t) hist[t] += len > 8 * (t + 1);
  }
  const int allowed = std::max(16, n / 1024);
  for (int t = 0; t < 4; ++t)
    if (hist[t] <= allowed) return 8 * (t + 1);
  return 0;
}

int colour_counts(const int* d_rp, const int* d_dpos, int n, const std::vector<int>& cptr,
                  ColourCounts& cc, cudaStream_t s, int* ell_k = nullptr) {
  std::vector<int> rp(n + 1), dp(n);
  MSP_CUDA_TRY(cudaMemcpyAsync(rp.data(), d_rp, (n + 1) * sizeof(int), cudaMemcpyDeviceToHost, s));
  MSP_CUDA_TRY(cudaMemcpyAsync(dp.data(), d_dpos, n * sizeof(int), cudaMemcpyDeviceToHost, s));
  MSP_CUDA_TRY(cudaStreamSynchronize(s));
  const int g = cptr.empty() ? 0 : (int)cptr.size() - 1;
  cc.lower.assign(g, 0);
  cc.upper.assign(g, 0);
  for (int c = 0; c < g; ++c)
    for (int i = cptr[c]; i < cptr[c + 1]; ++i) {
      cc.lower[c] += dp[i] - rp[i];
      cc.upper[c] += rp[i + 1] - dp[i] - 1;
    }
  if (ell_k) *ell_k = ell_width(rp, n);
  return MSP_OK;
}

struct Level {
  DCsr A;                   // colour-ordered level matrix
  std::vector<int> cptr;    // colour classes (empty: not coloured)
  ColourCounts cc;
  DevBuf<int> perm;         // colour-ordered -> pre-colouring index
  DevBuf<int> dpos;
  DevBuf<double> rdiag;
  DevBuf<int> agg;          // -> next level index
  DevBuf<int> mptr, members;  // members of every next-level aggregate (ascending)
  int nc = 0;
  // ELL copy of the off-diagonal entries for the colour sweeps (ell_k slots per row; 0:
  // the level is swept in CSR form)
  int ell_k = 0;
  int gs_tpr = 0, rr_tpr = 0;  // lanes per row of the ELL sweep / restriction (0: default)
  DevBuf<int> ell_ci, ell_meta;
  DevBuf<double> ell_v, ell_diag;
  // FP32 copies (mixed precision)
  DevBuf<float> v32, rdiag32, ell_v32, ell_diag32;
  // work vectors (t: the start values of a PJAC-NO / PGS-NO sweep)
  DevBuf<double> b64, x64, t64;
  DevBuf<float> b32, x32, t32;
  // batched instances (levels >= 1): the instance of every row and the rows of the
  // instances still iterating
  DevBuf<int> row_inst;
  DevBuf<unsigned char> rmask;
};

}  // namespace
}  // namespace msp

struct msp_handle_s {
  msp_config cfg{};
  int nb = 0, b = 0;
  int64_t nnzb = 0;
  int device = 0;
  long long dev_bytes = 0;  // device memory the handle holds through DevBuf
  msp::SortScratch* ss = nullptr;
  msp::DevBuf<msp::DevFlags> flags;
  msp::DevFlags* h_flags = nullptr;  // pinned
  double* h_pin = nullptr;           // pinned host scratch (Hessenberg column, norms)
  // pattern (level 0)
  msp::DevBuf<int> perm0, iperm0, colour0;
  std::vector<int> cptr0;
  msp::ColourCounts cc0;
  int g0 = 0;
  msp::DevBuf<int> rp, ci, dpos, src;  // colour-ordered BSR pattern, source nonzero
  // rows with more than kLongRowBlocks blocks (the well rows), ascending: the block-row
  // kernels give each of them a warp instead of one lane group
  std::vector<int> long_h;
  msp::DevBuf<int> long_d;
  msp::DevBuf<double> vals;            // colour-ordered current values
  msp::DevBuf<double> c0;              // column 0 of every block of vals (FP64 preconditioner)
  msp::DevBuf<double> staging;         // user values before the gather
  // values copied ahead of their update (msp_stage_values_host / msp_update_values_staged)
  msp::DevBuf<double> staged;
  cudaEvent_t staged_ev = nullptr;     // the staged copy has landed
  cudaEvent_t consumed_ev = nullptr;   // the staged values have been gathered
  bool staged_pending = false;
  bool consumed_recorded = false;
  // setup products
  msp::DevBuf<double> omega, dNinv, aN, lu, uinv, cinv;
  int ncoarse = 0;
  std::vector<msp::Level> levels;
  // FP32 copies
  msp::DevBuf<float> vals32, c0_32, omega32, dNinv32, aN32, lu32, uinv32;
  // preconditioner work vectors
  msp::DevBuf<double> pr, py, px;
  msp::DevBuf<float> g32, w32, pr32, py32, px32;
  msp::DevBuf<double> ny;    // stage N: D_N^-1 g, nb * (b - 1)
  msp::DevBuf<float> ny32;
  // Krylov work
  msp::DevBuf<double> V, Z, bperm, xperm, rvec, partial, hdev, nrm, ydev;
  msp::DevBuf<int> ifl;
  // one-pass Gram-Schmidt of the single solve: triangular factor T of the stored basis
  // ((m + 2)^2, by column), the step's dot products, axpy coefficients and host-bound results
  msp::DevBuf<double> gs_T, gs_d, gs_g, gs_out;
  msp::DevBuf<double> e2e_b, e2e_x;  // staging of msp_solve_host
  // the preconditioner as a CUDA graph on fixed input/output buffers
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t graph = nullptr;
  long long graph_launches = 0;  // kernels in the graph
  double graph_bytes = 0.0;      // algorithmic bytes of one replay
  bool graph_timed = false;      // captured with event nodes around every site
  std::vector<msp::GraphProbe> graph_probes;
  msp::DevBuf<double> pg64, pw64;
  // the single solve's dot products of the basis against its newest vector u_j run inside
  // the preconditioner's graph, on a branch beside the coarse AMG levels: j is read from
  // dot_j (-1: none) and the sums land in gs_d[0..j]
  cudaStream_t side_stream = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  msp::DevBuf<int> dot_j;
  msp::DevBuf<double> partial_u;
  bool dot_launched = false, dot_branch = false;  // during one application
  int dot_j_dev = -1;  // what dot_j holds once the enqueued work has run (kDotUnknown: not known)
  // autotuned lanes per row of the ELL kernels, per (level, slots per row)
  std::map<std::pair<int, int>, std::pair<int, int>> tuned;
  // adaptive setup
  int setup_calls = 0;
  int prev_it = -1;
  bool first_solve = true;
  bool setup_valid = false;
  // independent instances of a block-diagonal matrix (msp_set_instances)
  int batch = 0;                              // number of instances, 0: none
  std::vector<int> batch_offsets;             // block-row offsets (natural order)
  msp::DevBuf<int> seg_start, seg_end, seg_inst, seg_iptr, seg_ichunks;
  int seg_n = 0;
  msp::DevBuf<int> bact, bcount, bzero;       // per instance: active, columns used, zero mask
  msp::DevBuf<double> bpart, bh, by, bn, bydev;  // chunk partials; per instance kKrylovMaxK
  double* h_bpin = nullptr;                   // pinned: bh, by, bn (3 * batch * kKrylovMaxK)
  msp::DevBuf<int> row_inst;                  // instance of every level-0 (permuted) row
  // one-pass Gram-Schmidt of the batched solve, per instance: the triangular factor
  // ((m + 2)^2), the step's dot products (2 * kKrylovMaxK), the results (kBatchOut), and a
  // mask of the instances whose column is made final at this step
  msp::DevBuf<double> gs_bT, gs_bD, gs_bout;
  msp::DevBuf<int> gs_bfin;
  double* h_bout = nullptr;                   // pinned copy of gs_bout
  msp::DevBuf<unsigned char> rmask0;          // level-0 rows of the active instances
};

namespace msp {
namespace {

void drop_graph(msp_handle h);
constexpr int kDotUnknown = -2;  // msp_handle_s::dot_j_dev when a write may not have run

int permute_pattern(msp_handle h, int n, const int* rp, const int* ci, int nnz, const int* iperm,
                    DevBuf<int>& brp, DevBuf<int>& bci, DevBuf<int>& src, cudaStream_t s);

int sync_flags(msp_handle h, cudaStream_t s) {
  MSP_CUDA_TRY(cudaMemcpyAsync(h->h_flags, h->flags.p, sizeof(DevFlags), cudaMemcpyDeviceToHost, s));
  MSP_CUDA_TRY(cudaStreamSynchronize(s));
  return h->h_flags->code;
}

int reset_flags(msp_handle h, cudaStream_t s) {
  MSP_CUDA_TRY(cudaMemsetAsync(h->flags.p, 0, sizeof(DevFlags), s));
  return MSP_OK;
}

// VerticesGrouping (Algorithms 4.1/4.2) of the symmetric graph srp/sci: colour[v] in 1..g
int vertices_grouping_gpu(msp_handle h, int n, const DevBuf<int>& srp, const DevBuf<int>& sci,
                          int snnz, DevBuf<int>& colour, int* g_out, cudaStream_t s) {
  DevBuf<unsigned long long> keys;
  DevBuf<int> vor, rank, wbar, meta, rrp, rci, rsrc, colour_r;
  DevBuf<unsigned> bitmap, inV;
  MSP_TRY(keys.alloc(n));
  MSP_TRY(vor.alloc(n));
  MSP_TRY(rank.alloc(n));
  rank_keys_kernel<<<grid1(n), kThreads, 0, s>>>(n, srp.p, keys.p);
  MSP_TRY(launch_status());
  MSP_TRY(sort_pairs_u64(h->ss, n, keys.p, nullptr, 64, s));
  MSP_TRY(low32_of_keys(n, keys.p, vor.p, s));
  MSP_TRY(launch_scatter_inverse(n, vor.p, rank.p, s));
  // relabel S by priority rank: the greedy then picks the smallest label
  MSP_TRY(permute_pattern(h, n, srp.p, sci.p, snnz, rank.p, rrp, rci, rsrc, s));
  const int n0 = (n + 31) / 32, n1 = (n0 + 31) / 32, n2 = (n1 + 31) / 32;
  const size_t words = (size_t)n0 + n1 + n2;
  MSP_TRY(inV.alloc(n0));
  MSP_TRY(wbar.alloc(n));
  MSP_TRY(bitmap.alloc(words));
  MSP_TRY(meta.alloc(2));
  MSP_TRY(colour_r.alloc(n));
  MSP_TRY(colour.alloc(n));
  MSP_CUDA_TRY(cudaMemsetAsync(meta.p, 0, 2 * sizeof(int), s));
  // two-hop lists of the relabelled graph (the second circle of every vertex as one run),
  // unless they would pass int offsets or 2 GB: then the colouring gathers the rows itself
  DevBuf<int> tcnt, tp, tl;
  DevBuf<unsigned long long> ttotal;
  MSP_TRY(tcnt.alloc(n));
  MSP_TRY(ttotal.alloc(1));
  MSP_TRY(launch_twohop_count(n, rrp.p, rci.p, tcnt.p, ttotal.p, s));
  unsigned long long htotal = 0;
  MSP_CUDA_TRY(cudaMemcpyAsync(&htotal, ttotal.p, sizeof(htotal), cudaMemcpyDeviceToHost, s));
  MSP_CUDA_TRY(cudaStreamSynchronize(s));
  const bool twohop = htotal < (1ull << 31) - 1 && htotal * sizeof(int) <= (2ull << 30);
  if (twohop) {
    MSP_TRY(tp.alloc((size_t)n + 1));
    MSP_TRY(tl.alloc(std::max<size_t>(1, (size_t)htotal)));
    MSP_TRY(exclusive_scan_int(h->ss, n, tcnt.p, tp.p, s));
    const int last = (int)htotal;
    MSP_CUDA_TRY(cudaMemcpyAsync(tp.p + n, &last, sizeof(int), cudaMemcpyHostToDevice, s));
    MSP_TRY(launch_twohop_fill(n, rrp.p, rci.p, tp.p, tl.p, s));
  }
  MSP_TRY(launch_colouring(n, rrp.p, rci.p, twohop ? tp.p : nullptr, twohop ? tl.p : nullptr,
                           inV.p, wbar.p, bitmap.p, words, colour_r.p, meta.p,
                           h->cfg.loop_limit > 0 ? h->cfg.loop_limit : n, s));
  map_kernel<<<grid1(n), kThreads, 0, s>>>(n, colour_r.p, rank.p, colour.p);  // colour[v] = colour_r[rank[v]]
  MSP_TRY(launch_status());
  int hm[2] = {0, 0};
  MSP_CUDA_TRY(cudaMemcpyAsync(hm, meta.p, sizeof(hm), cudaMemcpyDeviceToHost, s));
  MSP_CUDA_TRY(cudaStreamSynchronize(s));
  if (hm[1] != 0) return MSP_ERR_TIMEOUT;
  *g_out = hm[0];
  return MSP_OK;
}

// Greedy first-fit colouring in Jones-Plassmann priority order of the symmetric graph
// srp/sci (MSP_COLOURING_JP): colour[v] in 1..g, by parallel rounds
constexpr unsigned long long kJpSeed = 0x4A6F6E6573504CULL;
int jp_colouring_gpu(msp_handle h, int n, const int* srp, const int* sci, DevBuf<int>& colour,
                     int* g_out, cudaStream_t s) {
  DevBuf<unsigned long long> keys;
  DevBuf<int> order, rank, counters;
  MSP_TRY(keys.alloc(n));
  MSP_TRY(order.alloc(n));
  MSP_TRY(rank.alloc(n));
  MSP_TRY(counters.alloc(2));
  MSP_TRY(colour.alloc(n));
  MSP_TRY(launch_jp_keys(n, srp, kJpSeed, keys.p, order.p, s));
  MSP_TRY(sort_pairs_u64(h->ss, n, keys.p, order.p, 64, s));
  MSP_TRY(launch_scatter_inverse(n, order.p, rank.p, s));  // rank[order[k]] = k
  MSP_CUDA_TRY(cudaMemsetAsync(colour.p, 0, (size_t)n * sizeof(int), s));
  MSP_CUDA_TRY(cudaMemsetAsync(counters.p, 0, 2 * sizeof(int), s));
  // every round colours at least the first uncoloured vertex in priority order
  const long long max_rounds =
      h->cfg.loop_limit > 0 ? (long long)h->cfg.loop_limit : (long long)n + 8;
  int hc[2] = {0, 0};
  for (long long rounds = 0; hc[0] < n;) {
    if (rounds >= max_rounds) return MSP_ERR_TIMEOUT;
    const long long batch = std::min<long long>(8, max_rounds - rounds);
    for (long long r = 0; r < batch; ++r)
      MSP_TRY(launch_jp_round(n, srp, sci, rank.p, colour.p, counters.p, s));
    rounds += batch;
    MSP_CUDA_TRY(cudaMemcpyAsync(hc, counters.p, sizeof(hc), cudaMemcpyDeviceToHost, s));
    MSP_CUDA_TRY(cudaStreamSynchronize(s));
  }
  *g_out = hc[1];
  return MSP_OK;
}

// VerticesGrouping of the graph of a CSR/BSR pattern: colour[v] in 1..g, perm (colour
// order -> index), cptr (host).
int colour_graph(msp_handle h, int n, const int* rp, const int* ci, int nnz, DevBuf<int>& colour,
                 DevBuf<int>& perm, std::vector<int>& cptr, int* g_out, cudaStream_t s) {
  DevBuf<int> srp, sci;
  int snnz = 0;
  MSP_TRY(build_adjacency(h->ss, n, rp, ci, nnz, srp, sci, &snnz, s));
  int g = 0;
  if (h->cfg.colouring == MSP_COLOURING_JP)
    MSP_TRY(jp_colouring_gpu(h, n, srp.p, sci.p, colour, &g, s));
  else
    MSP_TRY(vertices_grouping_gpu(h, n, srp, sci, snnz, colour, &g, s));
  DevBuf<unsigned long long> keys;
  MSP_TRY(keys.alloc(n));
  // colour permutation: stable sort by (colour, index)
  colour_keys_kernel<<<grid1(n), kThreads, 0, s>>>(n, colour.p, keys.p);
  MSP_TRY(launch_status());
  MSP_TRY(sort_pairs_u64(h->ss, n, keys.p, nullptr, 64, s));
  MSP_TRY(perm.alloc(n));
  MSP_TRY(low32_of_keys(n, keys.p, perm.p, s));
  DevBuf<int> cp;
  MSP_TRY(cp.alloc(g + 2));
  MSP_TRY(rowptr_from_sorted_keys(n, g + 1, keys.p, cp.p, s));
  std::vector<int> hcp(g + 2);
  MSP_CUDA_TRY(cudaMemcpyAsync(hcp.data(), cp.p, (g + 2) * sizeof(int), cudaMemcpyDeviceToHost, s));
  MSP_CUDA_TRY(cudaStreamSynchronize(s));
  cptr.assign(hcp.begin() + 1, hcp.end());  // colour c (1-based) -> [hcp[c], hcp[c+1])
  *g_out = g;
  return MSP_OK;
}

// B = P A P^T for a scalar CSR matrix (rows/cols mapped by iperm), columns re-sorted;
// src[q] = nonzero of A that lands at q.
int permute_pattern(msp_handle h, int n, const int* rp, const int* ci, int nnz, const int* iperm,
                    DevBuf<int>& brp, DevBuf<int>& bci, DevBuf<int>& src, cudaStream_t s) {
  DevBuf<unsigned long long> keys;
  MSP_TRY(keys.alloc(nnz > 0 ? nnz : 1));
  MSP_TRY(src.alloc(nnz > 0 ? nnz : 1));
  perm_keys_kernel<<<grid1(n), kThreads, 0, s>>>(n, rp, ci, iperm, iperm, keys.p, src.p);
  MSP_TRY(launch_status());
  MSP_TRY(sort_pairs_u64(h->ss, nnz, keys.p, src.p, 64, s));
  MSP_TRY(brp.alloc(n + 1));
  MSP_TRY(bci.alloc(nnz > 0 ? nnz : 1));
  MSP_TRY(rowptr_from_sorted_keys(nnz, n, keys.p, brp.p, s));
  MSP_TRY(low32_of_keys(nnz, keys.p, bci.p, s));
  MSP_CUDA_TRY(cudaStreamSynchronize(s));
  return MSP_OK;
}

// A_c = P^T A P for the aggregation agg (bit-exact sums in fine-nonzero order)
int galerkin(msp_handle h, const DCsr& A, const int* agg, int nc, DCsr& C, cudaStream_t s) {
  const size_t m = A.nnz;
  DevBuf<unsigned long long> keys, ukeys;
  DevBuf<int> src, flags, pos, seg;
  MSP_TRY(keys.alloc(m));
  MSP_TRY(src.alloc(m));
  perm_keys_kernel<<<grid1(A.n), kThreads, 0, s>>>(A.n, A.rp.p, A.ci.p, agg, agg, keys.p, src.p);
  MSP_TRY(launch_status());
  MSP_TRY(sort_pairs_u64(h->ss, m, keys.p, src.p, 64, s));
  MSP_TRY(flags.alloc(m));
  MSP_TRY(pos.alloc(m));
  seg_flags_kernel<<<grid1(m), kThreads, 0, s>>>(m, keys.p, flags.p);
  MSP_TRY(launch_status());
  MSP_TRY(exclusive_scan_int(h->ss, m, flags.p, pos.p, s));
  int lp = 0, lf = 0;
  MSP_CUDA_TRY(cudaMemcpyAsync(&lp, pos.p + m - 1, sizeof(int), cudaMemcpyDeviceToHost, s));
  MSP_CUDA_TRY(cudaMemcpyAsync(&lf, flags.p + m - 1, sizeof(int), cudaMemcpyDeviceToHost, s));
  MSP_CUDA_TRY(cudaStreamSynchronize(s));
  const int nseg = lp + lf;
  MSP_TRY(ukeys.alloc(nseg));
  MSP_TRY(seg.alloc(nseg + 1));
  seg_compact_kernel<<<grid1(m), kThreads, 0, s>>>(m, keys.p, flags.p, pos.p, ukeys.p, seg.p, nseg);
  MSP_TRY(launch_status());
  C.n = nc;
  C.nnz = nseg;
  MSP_TRY(C.rp.alloc(nc + 1));
  MSP_TRY(C.ci.alloc(nseg));
  MSP_TRY(C.v.alloc(nseg));
  MSP_TRY(rowptr_from_sorted_keys(nseg, nc, ukeys.p, C.rp.p, s));
  MSP_TRY(low32_of_keys(nseg, ukeys.p, C.ci.p, s));
  MSP_TRY(launch_segment_sums(nseg, seg.p, src.p, A.v.p, C.v.p, s));
  MSP_CUDA_TRY(cudaStreamSynchronize(s));
  return MSP_OK;
}

// one pairwise matching pass (visit order splitmix64(i ^ seed)); agg in [0, *nagg)
int pairwise_pass(msp_handle h, const DCsr& A, double beta, unsigned long long seed,
                  DevBuf<int>& agg, int* nagg, cudaStream_t s) {
  const int n = A.n;
  DevBuf<int> srp, sci, tpos, partner, commit, rep, id;
  int snnz = 0;
  MSP_TRY(build_adjacency(h->ss, n, A.rp.p, A.ci.p, A.nnz, srp, sci, &snnz, s));
  DevBuf<double> sval;
  DevBuf<unsigned char> cand, state;
  DevBuf<unsigned long long> hkey;
  MSP_TRY(sval.alloc(snnz > 0 ? snnz : 1));
  MSP_TRY(cand.alloc(snnz > 0 ? snnz : 1));
  MSP_TRY(tpos.alloc(snnz > 0 ? snnz : 1));
  MSP_TRY(hkey.alloc(n));
  MSP_TRY(state.alloc(n));
  MSP_TRY(partner.alloc(n));
  MSP_TRY(commit.alloc(n));
  MSP_TRY(launch_strength(n, A.rp.p, A.ci.p, A.v.p, srp.p, sci.p, beta, sval.p, cand.p, s));
  MSP_TRY(launch_transpose_pos(n, srp.p, sci.p, tpos.p, s));
  MSP_TRY(launch_visit_keys(n, seed, hkey.p, s));
  MSP_CUDA_TRY(cudaMemsetAsync(state.p, 0, n, s));
  MSP_TRY(launch_fill_int(n, -1, partner.p, s));
  int rounds = 0;
  while (true) {
    MSP_CUDA_TRY(cudaMemsetAsync(&h->flags.p->count, 0, sizeof(int), s));
    MSP_TRY(launch_match_round(n, srp.p, sci.p, tpos.p, sval.p, cand.p, hkey.p, state.p,
                               commit.p, s));
    MSP_TRY(launch_match_apply(n, commit.p, state.p, partner.p, h->flags.p, s));
    MSP_CUDA_TRY(cudaMemcpyAsync(h->h_flags, h->flags.p, sizeof(DevFlags), cudaMemcpyDeviceToHost, s));
    MSP_CUDA_TRY(cudaStreamSynchronize(s));
    if (h->h_flags->count == 0) break;
    // at least one node decides per round, so n rounds decide every node
    if (++rounds >= (h->cfg.loop_limit > 0 ? h->cfg.loop_limit : n + 8)) return MSP_ERR_TIMEOUT;
  }
  MSP_TRY(rep.alloc(n));
  MSP_TRY(id.alloc(n));
  MSP_TRY(launch_match_reps(n, partner.p, rep.p, s));
  MSP_TRY(exclusive_scan_int(h->ss, n, rep.p, id.p, s));
  int lr = 0, li = 0;
  MSP_CUDA_TRY(cudaMemcpyAsync(&lr, rep.p + n - 1, sizeof(int), cudaMemcpyDeviceToHost, s));
  MSP_CUDA_TRY(cudaMemcpyAsync(&li, id.p + n - 1, sizeof(int), cudaMemcpyDeviceToHost, s));
  MSP_TRY(agg.alloc(n));
  MSP_TRY(launch_match_ids(n, partner.p, id.p, agg.p, s));
  MSP_CUDA_TRY(cudaStreamSynchronize(s));
  *nagg = lr + li;
  return MSP_OK;
}

// `ell`: also build the ELL copy the colour sweeps read (levels whose colour classes are
// small enough for the sweeps to be bound by load latency)
int level_extras(msp_handle h, Level& L, bool smoothed, bool ell, cudaStream_t s) {
  MSP_TRY(L.dpos.alloc(L.A.n));
  MSP_TRY(L.rdiag.alloc(L.A.n));
  MSP_TRY(launch_diag_pos(L.A.n, L.A.rp.p, L.A.ci.p, L.dpos.p, s));
  L.ell_k = 0;
  if (smoothed) {
    MSP_TRY(launch_rdiag(L.A.n, L.dpos.p, L.A.v.p, L.rdiag.p, h->flags.p, s));
    int k = 0;
    MSP_TRY(colour_counts(L.A.rp.p, L.dpos.p, L.A.n, L.cptr, L.cc, s, ell ? &k : nullptr));
    if (k > 0) {
      const size_t slots = (size_t)k * L.A.n;
      MSP_TRY(L.ell_ci.alloc(slots));
      MSP_TRY(L.ell_v.alloc(slots));
      MSP_TRY(L.ell_meta.alloc(L.A.n));
      MSP_TRY(L.ell_diag.alloc(L.A.n));
      MSP_TRY(launch_build_ell(L.A.n, k, L.A.rp.p, L.A.ci.p, L.A.v.p, L.dpos.p, L.ell_ci.p,
                               L.ell_v.p, L.ell_meta.p, L.ell_diag.p, s));
      L.ell_k = k;
    }
  }
  MSP_TRY(L.b64.alloc(L.A.n));
  MSP_TRY(L.x64.alloc(L.A.n));
  // zero from the start: with batched instances the rows of an instance that never
  // iterates are never written, and the coarsest level's dense product reads every row
  // (times exact zeros in the inverse, which must not meet a NaN bit pattern)
  MSP_CUDA_TRY(cudaMemsetAsync(L.b64.p, 0, sizeof(double) * L.A.n, s));
  MSP_CUDA_TRY(cudaMemsetAsync(L.x64.p, 0, sizeof(double) * L.A.n, s));
  const bool copies = smoothed && h->cfg.smoother != MSP_SMOOTHER_PGS_MC;
  if (copies) MSP_TRY(L.t64.alloc(L.A.n));
  if (h->cfg.precision == MSP_PRECISION_FP32) {
    MSP_TRY(L.v32.alloc(L.A.nnz));
    MSP_TRY(L.rdiag32.alloc(L.A.n));
    MSP_TRY(launch_cast_vals(L.A.nnz, L.A.v.p, L.v32.p, s));
    MSP_TRY(launch_cast_vals(L.A.n, L.rdiag.p, L.rdiag32.p, s));
    if (L.ell_k > 0) {
      MSP_TRY(L.ell_v32.alloc((size_t)L.ell_k * L.A.n));
      MSP_TRY(launch_cast_vals((size_t)L.ell_k * L.A.n, L.ell_v.p, L.ell_v32.p, s));
      MSP_TRY(L.ell_diag32.alloc(L.A.n));
      MSP_TRY(launch_cast_vals(L.A.n, L.ell_diag.p, L.ell_diag32.p, s));
    }
    MSP_TRY(L.b32.alloc(L.A.n));
    MSP_TRY(L.x32.alloc(L.A.n));
    MSP_CUDA_TRY(cudaMemsetAsync(L.b32.p, 0, sizeof(float) * L.A.n, s));
    MSP_CUDA_TRY(cudaMemsetAsync(L.x32.p, 0, sizeof(float) * L.A.n, s));
    if (copies) MSP_TRY(L.t32.alloc(L.A.n));
  }
  return MSP_OK;
}

// dense inverse of the coarsest matrix by in-place Gauss-Jordan (partial pivoting)
int coarse_inverse(msp_handle h, const DCsr& C, cudaStream_t s) {
  const int n = C.n;
  DevBuf<double> A, col;
  DevBuf<int> piv, cp;
  MSP_TRY(A.alloc((size_t)n * n));
  MSP_TRY(col.alloc(n));
  MSP_TRY(piv.alloc(n));
  MSP_TRY(cp.alloc(n));
  MSP_TRY(h->cinv.alloc((size_t)n * n));
  MSP_TRY(launch_csr_to_dense(n, C.rp.p, C.ci.p, C.v.p, A.p, s));
  // blocked: the steps of a panel of 32 columns transform the panel only, then one
  // rank-32 update applies them to the other columns (row swaps act on whole rows)
  constexpr int kPanel = 32;
  DevBuf<double> T;
  MSP_TRY(T.alloc((size_t)kPanel * n));
  for (int k0 = 0; k0 < n; k0 += kPanel) {
    const int nb = std::min(kPanel, n - k0);
    for (int k = k0; k < k0 + nb; ++k) {
      MSP_TRY(launch_gj_pivot(n, k, k0, k0 + nb, A.p, col.p, piv.p, h->flags.p, s));
      MSP_TRY(launch_gj_update(n, k, k0, nb, A.p, col.p, s));
    }
    MSP_CUDA_TRY(cudaMemcpyAsync(T.p, A.p + (size_t)k0 * n, (size_t)nb * n * sizeof(double),
                                 cudaMemcpyDeviceToDevice, s));
    MSP_TRY(launch_gj_panel_apply(n, k0, nb, A.p, T.p, s));
  }
  if (sync_flags(h, s) != MSP_OK) return h->h_flags->code;
  std::vector<int> hp(n), cols(n);
  MSP_CUDA_TRY(cudaMemcpyAsync(hp.data(), piv.p, n * sizeof(int), cudaMemcpyDeviceToHost, s));
  MSP_CUDA_TRY(cudaStreamSynchronize(s));
  for (int c = 0; c < n; ++c) cols[c] = c;
  for (int k = n - 1; k >= 0; --k)
    if (hp[k] != k) std::swap(cols[k], cols[hp[k]]);
  MSP_CUDA_TRY(cudaMemcpyAsync(cp.p, cols.data(), n * sizeof(int), cudaMemcpyHostToDevice, s));
  MSP_TRY(launch_gj_unscramble(n, cp.p, A.p, h->cinv.p, s));
  MSP_CUDA_TRY(cudaStreamSynchronize(s));
  h->ncoarse = n;
  return MSP_OK;
}

// ---------------------------------------------------------------------------------
// value setup: decoupling, AMG hierarchy, stage N, BILU(0)
// ---------------------------------------------------------------------------------
int autotune_levels(msp_handle h, cudaStream_t s);

// Batched instances: the instance of every row of the AMG levels below level 0 and their
// row masks (all rows on), so that the coarse levels too skip the instances that have left
// the active set.
int batch_level_masks(msp_handle h, cudaStream_t s) {
  if (!h->batch || !h->row_inst.p) return MSP_OK;
  const int* inst = h->row_inst.p;
  for (size_t l = 0; l + 1 < h->levels.size(); ++l) {
    Level& F = h->levels[l];
    Level& C = h->levels[l + 1];
    MSP_TRY(C.row_inst.alloc(C.A.n));
    MSP_TRY(C.rmask.alloc(C.A.n));
    inst_scatter_kernel<<<grid1(F.A.n), kThreads, 0, s>>>(F.A.n, F.agg.p, inst, C.row_inst.p);
    MSP_TRY(launch_status());
    MSP_CUDA_TRY(cudaMemsetAsync(C.rmask.p, 1, C.A.n, s));
    inst = C.row_inst.p;
  }
  MSP_CUDA_TRY(cudaStreamSynchronize(s));
  return MSP_OK;
}

int value_setup(msp_handle h, cudaStream_t s) {
  NvtxRange nvtx("msp:value_setup");
  const int nb = h->nb, b = h->b, bb = b * b, bn = b - 1;
  const size_t nnzb = (size_t)h->nnzb;
  const msp_config& cfg = h->cfg;
  h->setup_valid = false;
  drop_graph(h);
  MSP_TRY(reset_flags(h, s));
  // quasi-IMPES weights omega_i = D_i^{-T} e_0
  MSP_TRY(h->omega.alloc((size_t)nb * b));
  Probe pr_all("setup:value_total", 0.0, s);
  MSP_TRY(launch_diag_inverse(b, nb, h->dpos.p, h->vals.p, nullptr, h->omega.p, h->flags.p, s));
  if (sync_flags(h, s) != MSP_OK) return h->h_flags->code;
  // level 0: the pressure matrix A_P on the block pattern
  h->levels.clear();
  h->levels.emplace_back();
  {
    Level& L0 = h->levels[0];
    L0.A.n = nb;
    L0.A.nnz = (int)nnzb;
    MSP_TRY(L0.A.rp.alloc(nb + 1));
    MSP_TRY(L0.A.ci.alloc(nnzb));
    MSP_TRY(L0.A.v.alloc(nnzb));
    MSP_CUDA_TRY(cudaMemcpyAsync(L0.A.rp.p, h->rp.p, (nb + 1) * sizeof(int), cudaMemcpyDeviceToDevice, s));
    MSP_CUDA_TRY(cudaMemcpyAsync(L0.A.ci.p, h->ci.p, nnzb * sizeof(int), cudaMemcpyDeviceToDevice, s));
    MSP_TRY(launch_pressure_matrix(b, nb, h->rp.p, h->vals.p, h->omega.p, cfg.decoupling != 0,
                                   L0.A.v.p, s));
    L0.cptr = h->cptr0;
    MSP_TRY(L0.perm.alloc(nb));
    MSP_CUDA_TRY(cudaMemcpyAsync(L0.perm.p, h->perm0.p, nb * sizeof(int), cudaMemcpyDeviceToDevice, s));
  }
  // AMG hierarchy (Section 5: UA-AMG, pairwise matching, coarsest size coarse_max)
  for (int l = 0;; ++l) {
    const int nF = h->levels[l].A.n;
    if (nF <= cfg.coarse_max || l + 1 >= cfg.max_levels) break;
    DevBuf<int> agg;
    MSP_TRY(agg.alloc(nF));
    MSP_TRY(launch_iota(nF, agg.p, s));
    int nc = nF;
    DCsr cur;  // Galerkin matrix of the previous pass (pass >= 1)
    for (int pass = 0; pass < cfg.npass; ++pass) {
      const DCsr& A = (pass == 0) ? h->levels[l].A : cur;
      DevBuf<int> a1;
      int n1 = 0;
      const unsigned long long seed = cfg.agg_seed + (unsigned long long)(2 * l + pass);
      {
        Probe pr("setup:pairwise_matching", 0.0, s);
        MSP_TRY(pairwise_pass(h, A, cfg.beta, seed, a1, &n1, s));
      }
      compose_kernel<<<grid1(nF), kThreads, 0, s>>>(nF, a1.p, agg.p);
      MSP_TRY(launch_status());
      nc = n1;
      if (pass + 1 < cfg.npass) {
        DCsr nxt;
        Probe pr("setup:galerkin", 0.0, s);
        MSP_TRY(galerkin(h, A, a1.p, n1, nxt, s));
        cur = std::move(nxt);
      }
    }
    if ((double)nc > 0.9 * (double)nF) break;  // coarsening stalled
    DCsr Ac;
    {
      Probe pr("setup:galerkin", 0.0, s);
      MSP_TRY(galerkin(h, h->levels[l].A, agg.p, nc, Ac, s));
    }
    Level C;
    DevBuf<int> ipc;
    MSP_TRY(ipc.alloc(nc));
    const bool smoothed = nc > cfg.coarse_max && l + 2 < cfg.max_levels;
    if (smoothed && cfg.smoother == MSP_SMOOTHER_PGS_MC) {
      DevBuf<int> colour;
      int g = 0;
      {
        static const char* names[] = {"setup:colouring_l1", "setup:colouring_l2",
                                      "setup:colouring_l3", "setup:colouring_l4",
                                      "setup:colouring_l5+"};
        Probe pr(names[std::min(l, 4)], 0.0, s);
        MSP_TRY(colour_graph(h, nc, Ac.rp.p, Ac.ci.p, Ac.nnz, colour, C.perm, C.cptr, &g, s));
      }
      MSP_TRY(launch_scatter_inverse(nc, C.perm.p, ipc.p, s));
      DevBuf<int> srcmap;
      C.A.n = nc;
      C.A.nnz = Ac.nnz;
      MSP_TRY(permute_pattern(h, nc, Ac.rp.p, Ac.ci.p, Ac.nnz, ipc.p, C.A.rp, C.A.ci, srcmap, s));
      MSP_TRY(C.A.v.alloc(Ac.nnz));
      gather_double_kernel<<<grid1(Ac.nnz), kThreads, 0, s>>>(Ac.nnz, srcmap.p, Ac.v.p, C.A.v.p);
      MSP_TRY(launch_status());
      MSP_CUDA_TRY(cudaStreamSynchronize(s));
    } else {
      MSP_TRY(C.perm.alloc(nc));
      MSP_TRY(launch_iota(nc, C.perm.p, s));
      MSP_TRY(launch_iota(nc, ipc.p, s));
      C.A = std::move(Ac);
      if (smoothed) C.cptr = {0, nc};  // PJAC-NO / PGS-NO: natural order, one class
    }
    Level& F = h->levels[l];
    MSP_TRY(F.agg.alloc(nF));
    map_kernel<<<grid1(nF), kThreads, 0, s>>>(nF, ipc.p, agg.p, F.agg.p);
    MSP_TRY(launch_status());
    F.nc = nc;
    // members of every coarse aggregate, ascending (restriction order)
    {
      DevBuf<unsigned long long> keys;
      MSP_TRY(keys.alloc(nF));
      member_keys_kernel<<<grid1(nF), kThreads, 0, s>>>(nF, F.agg.p, keys.p);
      MSP_TRY(launch_status());
      MSP_TRY(sort_pairs_u64(h->ss, nF, keys.p, nullptr, 64, s));
      MSP_TRY(F.members.alloc(nF));
      MSP_TRY(F.mptr.alloc(nc + 1));
      MSP_TRY(low32_of_keys(nF, keys.p, F.members.p, s));
      MSP_TRY(rowptr_from_sorted_keys(nF, nc, keys.p, F.mptr.p, s));
      MSP_CUDA_TRY(cudaStreamSynchronize(s));
    }
    h->levels.push_back(std::move(C));
  }
  if (h->levels.back().A.n > cfg.coarse_hard_max) return MSP_ERR_ARG;
  for (size_t l = 0; l < h->levels.size(); ++l)
    MSP_TRY(level_extras(h, h->levels[l], l + 1 < h->levels.size(), true, s));
  if (sync_flags(h, s) != MSP_OK) return h->h_flags->code;
  {
    Probe pr("setup:coarse_inverse", 0.0, s);
    MSP_TRY(coarse_inverse(h, h->levels.back().A, s));
  }
  // stage N: concentration sub-blocks and the inverses of their diagonal blocks
  if (bn > 0) {
    MSP_TRY(h->aN.alloc(nnzb * bn * bn));
    MSP_TRY(h->dNinv.alloc((size_t)nb * bn * bn));
    MSP_TRY(launch_extract_N(b, nnzb, h->vals.p, h->aN.p, s));
    MSP_TRY(launch_diagN_inverse(b, nb, h->dpos.p, h->vals.p, h->dNinv.p, h->flags.p, s));
    // the sweeps read D_N,i^-1 A_ij (the row's diagonal inverse applied once here, not in
    // every sweep); a singular diagonal sub-block stops the setup at the flag check below
    MSP_TRY(launch_scale_N_rows(b, nb, h->rp.p, h->dpos.p, h->dNinv.p, h->aN.p, s));
  }
  // stage R: BILU(0) in colour order
  Probe pr_bilu("setup:bilu_factor", 0.0, s);
  MSP_TRY(h->lu.alloc(nnzb * bb));
  MSP_TRY(h->uinv.alloc((size_t)nb * bb));
  MSP_CUDA_TRY(cudaMemcpyAsync(h->lu.p, h->vals.p, nnzb * bb * sizeof(double),
                               cudaMemcpyDeviceToDevice, s));
  for (int c = 0; c < h->g0; ++c)
    MSP_TRY(launch_bilu_factor(b, h->cptr0[c], h->cptr0[c + 1], h->rp.p, h->ci.p, h->dpos.p,
                               h->lu.p, h->uinv.p, h->flags.p, s));
  if (sync_flags(h, s) != MSP_OK) return h->h_flags->code;
  if (cfg.precision == MSP_PRECISION_FP32) {
    MSP_TRY(h->omega32.alloc((size_t)nb * b));
    MSP_TRY(launch_cast_vals((size_t)nb * b, h->omega.p, h->omega32.p, s));
    if (bn > 0) {
      MSP_TRY(h->aN32.alloc(nnzb * bn * bn));
      MSP_TRY(h->dNinv32.alloc((size_t)nb * bn * bn));
      MSP_TRY(launch_cast_vals(nnzb * bn * bn, h->aN.p, h->aN32.p, s));
      MSP_TRY(launch_cast_vals((size_t)nb * bn * bn, h->dNinv.p, h->dNinv32.p, s));
    }
    MSP_TRY(h->lu32.alloc(nnzb * bb));
    MSP_TRY(h->uinv32.alloc((size_t)nb * bb));
    MSP_TRY(launch_cast_vals(nnzb * bb, h->lu.p, h->lu32.p, s));
    MSP_TRY(launch_cast_vals((size_t)nb * bb, h->uinv.p, h->uinv32.p, s));
  }
  MSP_CUDA_TRY(cudaStreamSynchronize(s));
  h->setup_calls++;
  MSP_TRY(batch_level_masks(h, s));
  if (cfg.autotune) MSP_TRY(autotune_levels(h, s));
  h->setup_valid = true;
  return MSP_OK;
}

// ---------------------------------------------------------------------------------
// preconditioner application (Algorithm 3.1), value type T
// ---------------------------------------------------------------------------------
template <typename T>
struct PView {
  const T *vals, *c0, *omega, *aN, *dNinv, *lu, *uinv;
  // per level: values, 1/diagonal, ELL values, diagonal
  std::vector<const T*> lv, lrd, lev, led;
  std::vector<T*> lb, lx, lt;
  T *r, *y, *x;
  T* ny;  // stage N: D_N^-1 g
  // level-0 rows to skip (instances of a batch that left the active set), or nullptr
  const unsigned char* m0 = nullptr;
  // the same per AMG level (lm[0] = m0), or nullptrs
  std::vector<const unsigned char*> lm;
};

PView<double> view64(msp_handle h) {
  PView<double> p;
  p.vals = h->vals.p;
  p.c0 = h->c0.p;
  p.omega = h->cfg.decoupling ? h->omega.p : nullptr;
  p.aN = h->aN.p;
  p.dNinv = h->dNinv.p;
  p.lu = h->lu.p;
  p.uinv = h->uinv.p;
  for (auto& L : h->levels) {
    p.lv.push_back(L.A.v.p);
    p.lrd.push_back(L.rdiag.p);
    p.lev.push_back(L.ell_v.p);
    p.led.push_back(L.ell_diag.p);
    p.lb.push_back(L.b64.p);
    p.lx.push_back(L.x64.p);
    p.lt.push_back(L.t64.p);
  }
  p.r = h->pr.p;
  p.y = h->py.p;
  p.x = h->px.p;
  p.ny = h->ny.p;
  p.m0 = h->batch ? h->rmask0.p : nullptr;
  for (size_t l = 0; l < h->levels.size(); ++l)
    p.lm.push_back(l == 0 ? p.m0 : (h->batch && h->levels[l].rmask.p ? h->levels[l].rmask.p : nullptr));
  return p;
}

PView<float> view32(msp_handle h) {
  PView<float> p;
  p.vals = h->vals32.p;
  p.c0 = h->c0_32.p;
  p.omega = h->cfg.decoupling ? h->omega32.p : nullptr;
  p.aN = h->aN32.p;
  p.dNinv = h->dNinv32.p;
  p.lu = h->lu32.p;
  p.uinv = h->uinv32.p;
  for (auto& L : h->levels) {
    p.lv.push_back(L.v32.p);
    p.lrd.push_back(L.rdiag32.p);
    p.lev.push_back(L.ell_v32.p);
    p.led.push_back(L.ell_diag32.p);
    p.lb.push_back(L.b32.p);
    p.lx.push_back(L.x32.p);
    p.lt.push_back(L.t32.p);
  }
  p.r = h->pr32.p;
  p.y = h->py32.p;
  p.x = h->px32.p;
  p.ny = h->ny32.p;
  p.m0 = h->batch ? h->rmask0.p : nullptr;
  for (size_t l = 0; l < h->levels.size(); ++l)
    p.lm.push_back(l == 0 ? p.m0 : (h->batch && h->levels[l].rmask.p ? h->levels[l].rmask.p : nullptr));
  return p;
}

// algorithmic bytes of one colour sweep launch over rows [r0, r1) reading `entries`
// nonzeros of `eb` bytes each (value + column index) plus `rowb` bytes per row
// The tile autotuner (msp_config.autotune): for every AMG level swept over its ELL copy,
// time a full colour sweep and the residual restriction with 2, 4 and 8 lanes per row
// (those with at most 8 slots per lane) on the level's own matrix, with CUDA events on the
// solver stream (best of three), and keep the fastest.  A choice is made once per (level,
// slots per row) and kept for the handle's life, so later SETUPs round the same way.  The
// level's work vectors are zeroed before and after.
template <typename T>
int autotune_levels_t(msp_handle h, const PView<T>& P, cudaStream_t s) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  MSP_CUDA_TRY(cudaEventCreate(&e0));
  MSP_CUDA_TRY(cudaEventCreate(&e1));
  int st = MSP_OK;
  auto time_it = [&](auto&& launch, float* best) -> int {
    *best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
      cudaEventRecord(e0, s);
      MSP_TRY(launch());
      cudaEventRecord(e1, s);
      MSP_CUDA_TRY(cudaEventSynchronize(e1));
      float ms = 0.0f;
      MSP_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
      if (rep > 0 && ms < *best) *best = ms;  // the first run warms the caches
    }
    return MSP_OK;
  };
  for (size_t l = 0; l + 1 < h->levels.size() && st == MSP_OK; ++l) {
    Level& L = h->levels[l];
    if (L.ell_k <= 0 || L.cptr.size() < 2) continue;
    const auto key = std::make_pair((int)l, L.ell_k);
    auto it = h->tuned.find(key);
    if (it != h->tuned.end()) {
      L.gs_tpr = it->second.first;
      L.rr_tpr = it->second.second;
      continue;
    }
    const int n = L.A.n, g = (int)L.cptr.size() - 1;
    int best_gs = ell_default_tpr(L.ell_k), best_rr = best_gs;
    float t_gs = 1e30f, t_rr = 1e30f;
    for (int tpr : {2, 4, 8}) {
      if (!ell_tpr_ok(L.ell_k, tpr)) continue;
      MSP_CUDA_TRY(cudaMemsetAsync(P.lx[l], 0, sizeof(T) * n, s));
      MSP_CUDA_TRY(cudaMemsetAsync(P.lb[l], 0, sizeof(T) * n, s));
      float t = 0.0f;
      st = time_it([&]() -> int {
        for (int c = 0; c < g; ++c)
          MSP_TRY(launch_ell_gs_colour<T>(L.ell_k, L.cptr[c], L.cptr[c + 1], L.ell_ci.p,
                                          P.lev[l], L.ell_meta.p, L.A.rp.p, L.A.ci.p, P.lv[l],
                                          L.dpos.p, P.lrd[l], P.lb[l], P.lx[l], false, s,
                                          nullptr, false, tpr));
        return MSP_OK;
      }, &t);
      if (st != MSP_OK) break;
      if (t < t_gs) {
        t_gs = t;
        best_gs = tpr;
      }
      st = time_it([&]() -> int {
        return launch_ell_residual_restrict<T>(L.ell_k, L.nc, L.mptr.p, L.members.p, L.ell_ci.p,
                                               P.lev[l], L.ell_meta.p, P.led[l], L.A.rp.p,
                                               L.A.ci.p, P.lv[l], P.lb[l], P.lx[l],
                                               P.lb[l + 1], s, nullptr, tpr);
      }, &t);
      if (st != MSP_OK) break;
      if (t < t_rr) {
        t_rr = t;
        best_rr = tpr;
      }
    }
    cudaMemsetAsync(P.lx[l], 0, sizeof(T) * n, s);
    cudaMemsetAsync(P.lb[l], 0, sizeof(T) * n, s);
    cudaMemsetAsync(P.lb[l + 1], 0, sizeof(T) * h->levels[l + 1].A.n, s);
    if (st != MSP_OK) break;
    L.gs_tpr = best_gs;
    L.rr_tpr = best_rr;
    h->tuned[key] = {best_gs, best_rr};
  }
  cudaStreamSynchronize(s);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return st;
}

int autotune_levels(msp_handle h, cudaStream_t s) {
  if (h->cfg.precision == MSP_PRECISION_FP32) return autotune_levels_t<float>(h, view32(h), s);
  return autotune_levels_t<double>(h, view64(h), s);
}

inline double sweep_bytes(int r0, int r1, long long entries, double eb, double rowb) {
  return (double)entries * eb + (double)(r1 - r0) * rowb;
}

// timing-site name "<prefix><level>" (levels past 6 share "<prefix>7+"); the strings live
// as long as the process
const char* level_site(const char* prefix, int l) {
  static std::mutex mu;
  static std::map<std::string, std::unique_ptr<std::string>> names;
  const std::string key = prefix + (l < 7 ? std::to_string(l) : std::string("7+"));
  std::lock_guard<std::mutex> lk(mu);
  auto& p = names[key];
  if (!p) p = std::make_unique<std::string>(key);
  return p->c_str();
}

// The dot products u_k . u_j, k <= j, of the single solve's step j (j = *dot_j; nothing when
// -1) into gs_d[0..j]; *dot_j then moves on to j + 1, so consecutive steps need no write.
// They need only the basis, so they run while the preconditioner is applied to u_j: on a
// branch of the captured graph that starts at the first coarse AMG level (whose
// latency-bound sweeps leave most of the GPU idle) — on small systems, whose every launch is
// latency-bound, at the start of the application — and joins at its end; in order on s
// when no graph is being captured.
int basis_dot(msp_handle h, cudaStream_t s, bool branch) {
  if (h->dot_launched) return MSP_OK;
  h->dot_launched = true;
  cudaStream_t d = s;
  if (branch && t_capturing) {
    if (!h->side_stream)
      MSP_CUDA_TRY(cudaStreamCreateWithFlags(&h->side_stream, cudaStreamNonBlocking));
    if (!h->ev_fork) MSP_CUDA_TRY(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
    if (!h->ev_join) MSP_CUDA_TRY(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
    MSP_CUDA_TRY(cudaEventRecord(h->ev_fork, s));
    MSP_CUDA_TRY(cudaStreamWaitEvent(h->side_stream, h->ev_fork, 0));
    d = h->side_stream;
    h->dot_branch = true;
  }
  const size_t n = (size_t)h->nb * h->b;
  // two blocks per SM (half the reduction grid): fast enough to end within the coarse
  // levels, and leaving most of each SM's registers to the sweeps it runs beside (measured
  // on the 1.12M-row system: 166.5 ms per solve, against 178.7 with one block per SM and
  // 171.3 with four)
  const int nbk = std::min(krylov_blocks(), sm_count() * 2);
  {
    Probe pr("krylov_basis_dot", 0.0, d);  // bytes are counted by the caller (j is known there)
    MSP_TRY(launch_multi_dot1(n, h->V.p, n, 0, nullptr, h->partial_u.p, kKrylovMaxK, nbk, d,
                              h->dot_j.p));
    // also moves dot_j on to the next step's index
    MSP_TRY(launch_reduce_partials_strided(0, nbk, kKrylovMaxK, h->partial_u.p, h->gs_d.p, d,
                                           h->dot_j.p));
  }
  if (d != s) MSP_CUDA_TRY(cudaEventRecord(h->ev_join, d));
  return MSP_OK;
}

template <typename T>
int vcycle(msp_handle h, const PView<T>& P, int l, cudaStream_t s) {
  Level& L = h->levels[l];
  const int n = L.A.n;
  const double sT = sizeof(T);

  if (l + 1 == (int)h->levels.size()) {
    Probe pr("coarse_gemv", (double)n * n * 8.0 + 2.0 * n * sT, s);
    return launch_dense_gemv<T>(n, h->cinv.p, P.lb[l], P.lx[l], s);
  }
  const int g = (int)L.cptr.size() - 1;
  const int avg_row = L.A.nnz / std::max(1, n);
  // ELL copy for the full sweeps and for small colour classes (latency-bound); the CSR
  // form for the lower-triangle sweep of a large class (bandwidth-bound: ELL would also
  // read the slots right of the diagonal)
  auto use_ell = [&](int c, bool lower_only) {
    return L.ell_k > 0 && !(lower_only && L.cptr[c + 1] - L.cptr[c] > 16384);
  };
  // classes of the coarse levels small enough to run beside the previous colour's launch:
  // launched as its programmatic dependents, they load their slots while it runs
  auto overlap = [&](int c) { return l >= 1 && L.cptr[c + 1] - L.cptr[c] <= 262144; };
  auto sweep = [&](int c, bool lower_only) {
    if (use_ell(c, lower_only))
      return launch_ell_gs_colour<T>(L.ell_k, L.cptr[c], L.cptr[c + 1], L.ell_ci.p, P.lev[l],
                                     L.ell_meta.p, L.A.rp.p, L.A.ci.p, P.lv[l], L.dpos.p,
                                     P.lrd[l], P.lb[l], P.lx[l], lower_only, s, P.lm[l],
                                     overlap(c), L.gs_tpr);
    return launch_csr_gs_colour<T>(L.cptr[c], L.cptr[c + 1], L.A.rp.p, L.A.ci.p, P.lv[l],
                                   L.dpos.p, P.lrd[l], P.lb[l], P.lx[l], lower_only, avg_row, s,
                                   P.lm[l]);
  };
  // one smoothing phase: its colour launches in order, timed in runs of one kernel
  struct SweepLaunch {
    int c;
    bool lower_only;
  };
  auto phase = [&](const std::vector<SweepLaunch>& order, bool pre) -> int {
    size_t k = 0;
    while (k < order.size()) {
      const bool ell = use_ell(order[k].c, order[k].lower_only);
      size_t e = k;
      double bytes = 0.0;
      int launches = 0;
      for (; e < order.size() && use_ell(order[e].c, order[e].lower_only) == ell; ++e) {
        const int c = order[e].c;
        bytes += sweep_bytes(L.cptr[c], L.cptr[c + 1],
                             L.cc.lower[c] + (order[e].lower_only ? 0 : L.cc.upper[c]), sT + 4,
                             3 * sT + 12);
        launches += L.cptr[c + 1] > L.cptr[c];
      }
      const char* site = ell ? (pre ? "amg_gs_pre_l" : "amg_gs_post_l")
                             : (pre ? "amg_gs_csr_pre_l" : "amg_gs_csr_post_l");
      Probe pr(level_site(site, l), bytes, s, launches);
      for (; k < e; ++k) MSP_TRY(sweep(order[k].c, order[k].lower_only));
    }
    return MSP_OK;
  };
  // PJAC-NO / PGS-NO (Section 5.1.1): every sweep reads the values from its start (a copy)
  const bool natural = h->cfg.smoother != MSP_SMOOTHER_PGS_MC;
  auto natural_sweep = [&](bool forward, bool from_zero) -> int {
    if (from_zero) MSP_CUDA_TRY(cudaMemsetAsync(P.lx[l], 0, n * sizeof(T), s));
    MSP_CUDA_TRY(cudaMemcpyAsync(P.lt[l], P.lx[l], n * sizeof(T), cudaMemcpyDeviceToDevice, s));
    const double bytes = (double)L.A.nnz * (sT + 4) + (double)n * (4 * sT + 12);
    if (h->cfg.smoother == MSP_SMOOTHER_PJAC) {
      Probe pr(level_site("amg_pjac_l", l), bytes, s);
      return launch_jacobi_sweep<T>(n, L.A.rp.p, L.A.ci.p, P.lv[l], L.dpos.p, P.lrd[l], P.lb[l],
                                    P.lt[l], P.lx[l], s);
    }
    Probe pr(level_site("amg_pgs_no_l", l), bytes, s);
    return launch_pgs_no_sweep<T>(n, L.A.rp.p, L.A.ci.p, P.lv[l], L.dpos.p, P.lrd[l], P.lb[l],
                                  P.lt[l], P.lx[l], forward, s);
  };
  if (l == 1) MSP_TRY(basis_dot(h, s, true));
  if (h->cfg.pre_sweeps <= 0) MSP_CUDA_TRY(cudaMemsetAsync(P.lx[l], 0, n * sizeof(T), s));
  if (natural) {
    for (int sw = 0; sw < h->cfg.pre_sweeps; ++sw) MSP_TRY(natural_sweep(true, sw == 0));
  } else {
    std::vector<SweepLaunch> order;
    for (int sw = 0; sw < h->cfg.pre_sweeps; ++sw)
      for (int c = 0; c < g; ++c) order.push_back({c, sw == 0});
    MSP_TRY(phase(order, true));
  }
  {
    const double bytes =
        (double)L.A.nnz * (sT + 4) + (double)n * (3 * sT + 12) + (double)L.nc * (sT + 4);
    if (L.ell_k > 0) {
      Probe pr(level_site("amg_residual_restrict_l", l), bytes, s);
      MSP_TRY(launch_ell_residual_restrict<T>(L.ell_k, L.nc, L.mptr.p, L.members.p, L.ell_ci.p,
                                              P.lev[l], L.ell_meta.p, P.led[l], L.A.rp.p,
                                              L.A.ci.p, P.lv[l], P.lb[l], P.lx[l], P.lb[l + 1],
                                              s, P.lm[l + 1], L.rr_tpr));
    } else {
      Probe pr(level_site("amg_residual_restrict_csr_l", l), bytes, s);
      MSP_TRY(launch_csr_residual_restrict<T>(L.nc, L.mptr.p, L.members.p, L.A.rp.p,
                                              L.A.ci.p, P.lv[l], P.lb[l], P.lx[l], P.lb[l + 1],
                                              avg_row, s, P.lm[l + 1]));
    }
  }
  MSP_TRY(vcycle<T>(h, P, l + 1, s));
  {
    Probe pr("amg_prolong", (double)n * (3 * sT + 4), s);
    MSP_TRY(launch_prolong_add<T>(n, L.agg.p, P.lx[l + 1], P.lx[l], s, P.lm[l]));
  }
  if (natural) {
    for (int sw = 0; sw < h->cfg.post_sweeps; ++sw) MSP_TRY(natural_sweep(false, false));
  } else {
    std::vector<SweepLaunch> order;
    for (int sw = 0; sw < h->cfg.post_sweeps; ++sw)
      for (int c = g - 1; c >= 0; --c) order.push_back({c, false});
    MSP_TRY(phase(order, false));
  }
  return MSP_OK;
}

// the long rows of level-0 rows [r0, r1) (a contiguous piece of the ascending list)
inline LongRows long_rows(msp_handle h, int r0, int r1) {
  LongRows lr;
  lr.thr = kLongRowBlocks;
  const auto lo = std::lower_bound(h->long_h.begin(), h->long_h.end(), r0);
  const auto hi = std::lower_bound(h->long_h.begin(), h->long_h.end(), r1);
  lr.n = (int)(hi - lo);
  lr.rows = lr.n ? h->long_d.p + (lo - h->long_h.begin()) : nullptr;
  return lr;
}

template <typename T>
int stage_N(msp_handle h, const PView<T>& P, const T* g, T* w, cudaStream_t s) {
  const int b = h->b;
  if (h->cfg.bgs_sweeps <= 0) {
    MSP_CUDA_TRY(cudaMemsetAsync(w, 0, (size_t)h->nb * b * sizeof(T), s));
    return MSP_OK;
  }
  const double sT = sizeof(T), bn = b - 1;
  // FP64 flops are recorded: the FP64 FMA rate can bind these kernels, the FP32 one cannot
  {
    Probe pr("stageN_scale", (double)h->nb * (bn * bn + 2 * bn) * sT, s, 1,
             sT == 8 ? 2.0 * (double)h->nb * bn * bn : 0.0);
    MSP_TRY(launch_nscale<T>(b, h->nb, P.dNinv, g, P.ny, s));
  }
  double bytes = 0.0, fmas = 0.0;
  for (int sw = 0; sw < h->cfg.bgs_sweeps; ++sw)
    for (int c = 0; c < h->g0; ++c) {
      const long long used = h->cc0.lower[c] + (sw == 0 ? 0 : h->cc0.upper[c]);
      bytes += sweep_bytes(h->cptr0[c], h->cptr0[c + 1], used, bn * bn * sT + 4,
                           (2 * bn + 1) * sT + 12);
      fmas += (double)used * bn * bn;
    }
  Probe pr("stageN_bgs_sweep", bytes, s, h->cfg.bgs_sweeps * h->g0, sT == 8 ? 2.0 * fmas : 0.0);
  for (int sw = 0; sw < h->cfg.bgs_sweeps; ++sw)
    for (int c = 0; c < h->g0; ++c)
      MSP_TRY(launch_bgs_colour<T>(b, h->cptr0[c], h->cptr0[c + 1], h->rp.p, h->ci.p, h->dpos.p,
                                   P.aN, P.ny, w, sw == 0, sw == 0, s, P.m0,
                                   long_rows(h, h->cptr0[c], h->cptr0[c + 1])));
  return MSP_OK;
}

// FMAs of a BSR product over all blocks
inline double bsr_fmas(msp_handle h) { return (double)h->nnzb * h->b * h->b; }

// algorithmic bytes of a BSR row sweep over all block rows (values, columns, row
// pointers, the input vector once, `vecs` further vectors of nb*b values)
inline double bsr_bytes(msp_handle h, double sT, double vecs) {
  const double b = h->b;
  return (double)h->nnzb * (b * b * sT + 4) + (double)(h->nb + 1) * 4 +
         (double)h->nb * b * sT * (1 + vecs);
}

template <typename T>
int stage_P(msp_handle h, const PView<T>& P, const T* g, T* w, T* r, cudaStream_t s) {
  // r != nullptr: leave in r the residual g - A w of the corrected w (stage R's input),
  // as (g - A w_before) - A Pi_P e instead of a second pass over the whole matrix
  const double sT = sizeof(T), b = h->b;
  {
    Probe pr("stageP_residual_restrict", bsr_bytes(h, sT, r ? 3 : 2) + (double)h->nb * sT, s,
             1, sT == 8 ? 2.0 * (bsr_fmas(h) + (double)h->nb * b) : 0.0);
    MSP_TRY(launch_bsr_restrict_p<T>(h->b, h->nb, h->rp.p, h->ci.p, P.vals, w, g, P.omega,
                                     P.lb[0], r, s, P.m0, long_rows(h, 0, h->nb)));
  }
  MSP_TRY(vcycle<T>(h, P, 0, s));
  if (!r) {
    Probe pr("stageP_prolong", (double)h->nb * 3 * sT, s);
    return launch_prolong_p<T>(h->b, h->nb, P.lx[0], w, s);
  }
  Probe pr("stageP_correct_residual",
           (double)h->nnzb * (b * sT + 4) + (double)(h->nb + 1) * 4 +
               (double)h->nb * sT * (1 + 2 * b + 2), s, 1,
           sT == 8 ? 2.0 * (double)h->nnzb * b : 0.0);
  return launch_bsr_col0_update<T>(h->b, h->nb, h->rp.p, h->ci.p, P.c0, P.lx[0], r, w, s, P.m0,
                                   long_rows(h, 0, h->nb));
}

template <typename T>
int stage_R(msp_handle h, const PView<T>& P, const T* r, T* w, cudaStream_t s) {
  const int b = h->b;
  const double sT = sizeof(T), bb = (double)b * b;
  double fwd = 0.0, bwd = 0.0, ffwd = 0.0, fbwd = 0.0;
  for (int c = 0; c < h->g0; ++c) {
    fwd += sweep_bytes(h->cptr0[c], h->cptr0[c + 1], h->cc0.lower[c], bb * sT + 4,
                       3.0 * b * sT + 12);
    bwd += sweep_bytes(h->cptr0[c], h->cptr0[c + 1], h->cc0.upper[c], bb * sT + 4,
                       (5.0 * b + bb) * sT + 12);
    ffwd += 2.0 * (double)h->cc0.lower[c] * bb;
    fbwd += 2.0 * ((double)h->cc0.upper[c] + (h->cptr0[c + 1] - h->cptr0[c])) * bb;
  }
  if (sT != 8) ffwd = fbwd = 0.0;
  {
    Probe pr("stageR_bilu_fwd", fwd, s, h->g0, ffwd);
    for (int c = 0; c < h->g0; ++c)
      MSP_TRY(launch_bilu_fwd<T>(b, h->cptr0[c], h->cptr0[c + 1], h->rp.p, h->ci.p, h->dpos.p,
                                 P.lu, r, P.y, s, P.m0,
                                 long_rows(h, h->cptr0[c], h->cptr0[c + 1])));
  }
  Probe pr("stageR_bilu_bwd", bwd, s, h->g0, fbwd);
  for (int c = h->g0 - 1; c >= 0; --c)
    MSP_TRY(launch_bilu_bwd<T>(b, h->cptr0[c], h->cptr0[c + 1], h->rp.p, h->ci.p, h->dpos.p,
                               P.lu, P.uinv, P.y, P.x, w, s, P.m0,
                               long_rows(h, h->cptr0[c], h->cptr0[c + 1])));
  return MSP_OK;
}

template <typename T>
int apply_precond_body(msp_handle h, const PView<T>& P, const T* g, T* w, cudaStream_t s);

// systems of at most this many unknowns start the basis dot products with the application
constexpr size_t kBasisDotEarly = size_t(1) << 18;

// w = B g (colour-ordered vectors of nb*b values of type T), with the single solve's basis
// dot products for the step in dot_j on a branch: from the start of the application on
// small systems, beside the coarse levels on larger ones, at the end (in order) when the
// preconditioner has no coarse levels
template <typename T>
int apply_precond_t(msp_handle h, const PView<T>& P, const T* g, T* w, cudaStream_t s) {
  h->dot_launched = false;
  h->dot_branch = false;
  int st = MSP_OK;
  if ((size_t)h->nb * h->b <= kBasisDotEarly) st = basis_dot(h, s, true);
  if (st == MSP_OK) st = apply_precond_body<T>(h, P, g, w, s);
  if (st == MSP_OK) st = basis_dot(h, s, false);
  if (h->dot_branch) {
    h->dot_branch = false;
    const cudaError_t e = cudaStreamWaitEvent(s, h->ev_join, 0);
    if (st == MSP_OK && e != cudaSuccess) {
      set_last_cuda_error(e, "cudaStreamWaitEvent", __FILE__, __LINE__);
      st = MSP_ERR_CUDA;
    }
  }
  return st;
}

template <typename T>
int apply_precond_body(msp_handle h, const PView<T>& P, const T* g, T* w, cudaStream_t s) {
  const size_t n = (size_t)h->nb * h->b;
  switch (h->cfg.precond) {
    case MSP_PREC_NONE:
      MSP_CUDA_TRY(cudaMemcpyAsync(w, g, n * sizeof(T), cudaMemcpyDeviceToDevice, s));
      return MSP_OK;
    case MSP_PREC_N_ONLY:
      if (h->b < 2) {
        MSP_CUDA_TRY(cudaMemsetAsync(w, 0, n * sizeof(T), s));
        return MSP_OK;
      }
      return stage_N<T>(h, P, g, w, s);
    case MSP_PREC_P_ONLY:
      MSP_CUDA_TRY(cudaMemsetAsync(w, 0, n * sizeof(T), s));
      return stage_P<T>(h, P, g, w, nullptr, s);
    case MSP_PREC_R_ONLY:
      MSP_CUDA_TRY(cudaMemsetAsync(w, 0, n * sizeof(T), s));
      return stage_R<T>(h, P, g, w, s);
    default:
      break;
  }
  // Algorithm 3.1 with w = 0: r = g; w += Pi_N B_N Pi_N^T r
  if (h->b >= 2)
    MSP_TRY(stage_N<T>(h, P, g, w, s));
  else
    MSP_CUDA_TRY(cudaMemsetAsync(w, 0, n * sizeof(T), s));
  // r = g - A w; w += Pi_P B_P Pi_P^T r  (residual fused into the restriction); the
  // residual r = g - A w of stage R comes out of the same stage
  MSP_TRY(stage_P<T>(h, P, g, w, P.r, s));
  // w += R r
  return stage_R<T>(h, P, P.r, w, s);
}

void release_graph_probes(std::vector<GraphProbe>& probes) {
  if (probes.empty()) return;
  std::lock_guard<std::mutex> lk(g_stats_mu);
  resolve_pending();  // no pending timing may still name these events
  for (auto& gp : probes) {
    g_free_events.push_back(gp.e0);
    g_free_events.push_back(gp.e1);
  }
  probes.clear();
}

void drop_graph(msp_handle h) {
  if (h->graph) cudaGraphExecDestroy(h->graph);
  h->graph = nullptr;
  release_graph_probes(h->graph_probes);
  h->graph_timed = false;
}

// Capture Algorithm 3.1 on the fixed buffers (pg -> pw) into a CUDA graph; it stays
// valid until the next value setup (update_values keeps every buffer in place).
int capture_graph(msp_handle h) {
  drop_graph(h);
  if (!h->cap_stream) MSP_CUDA_TRY(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
  const bool fp32 = h->cfg.precision == MSP_PRECISION_FP32;
  cudaGraph_t g = nullptr;
  MSP_CUDA_TRY(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
  t_capturing = true;
  t_cap_launches = 0;
  t_cap_bytes = 0.0;
  t_cap_timed = g_stats_mode == 3;
  t_cap_probes.clear();
  const int st = fp32 ? apply_precond_t<float>(h, view32(h), h->g32.p, h->w32.p, h->cap_stream)
                      : apply_precond_t<double>(h, view64(h), h->pg64.p, h->pw64.p, h->cap_stream);
  t_capturing = false;
  std::vector<GraphProbe> probes;
  probes.swap(t_cap_probes);
  const cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
  if (st != MSP_OK || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    release_graph_probes(probes);
    if (st != MSP_OK) return st;
    set_last_cuda_error(e, "cudaStreamEndCapture", __FILE__, __LINE__);
    return MSP_ERR_CUDA;
  }
  const cudaError_t ei = cudaGraphInstantiate(&h->graph, g, 0);
  cudaGraphDestroy(g);
  if (ei != cudaSuccess) {
    h->graph = nullptr;
    release_graph_probes(probes);
    set_last_cuda_error(ei, "cudaGraphInstantiate", __FILE__, __LINE__);
    return MSP_ERR_CUDA;
  }
  h->graph_launches = t_cap_launches;
  h->graph_bytes = t_cap_bytes;
  h->graph_timed = t_cap_timed;
  h->graph_probes = std::move(probes);
  return MSP_OK;
}

// w = B g on FP64 colour-ordered vectors, in the configured precision.  Replays the
// captured graph, except while every launch is timed (stats mode 2).
int apply_precond_run(msp_handle h, const double* g, double* w, cudaStream_t s);

// dot_j >= 0 (the single solve's step j, g = u_j): the application also leaves the dot
// products u_k . u_j, k <= j, in gs_d[0..j].  The device index is written only when it does
// not already hold dot_j (in a cycle, only at its first step).
int apply_precond(msp_handle h, const double* g, double* w, cudaStream_t s, int dot_j = -1) {
  if (dot_j < -1 || dot_j + 1 > kKrylovMaxK) return MSP_ERR_ARG;
  if (h->dot_j_dev != dot_j) {
    h->dot_j_dev = kDotUnknown;
    MSP_TRY(launch_set_int(h->dot_j.p, dot_j, s));
  }
  h->dot_j_dev = kDotUnknown;
  MSP_TRY(apply_precond_run(h, g, w, s));
  h->dot_j_dev = dot_j >= 0 ? dot_j + 1 : -1;
  return MSP_OK;
}

int apply_precond_run(msp_handle h, const double* g, double* w, cudaStream_t s) {
  NvtxRange nvtx("msp:precond");
  const size_t n = (size_t)h->nb * h->b;
  const bool fp32 = h->cfg.precision == MSP_PRECISION_FP32;
  if (g_stats_mode == 2) {
    if (fp32) {
      MSP_TRY(launch_cast_d2f(n, g, h->g32.p, s));
      MSP_TRY(apply_precond_t<float>(h, view32(h), h->g32.p, h->w32.p, s));
      return launch_cast_f2d(n, h->w32.p, w, s);
    }
    return apply_precond_t<double>(h, view64(h), g, w, s);
  }
  // stats mode 3 replays a graph with event nodes around every site; other modes a plain one
  if (h->graph && h->graph_timed != (g_stats_mode == 3)) drop_graph(h);
  if (!h->graph) MSP_TRY(capture_graph(h));
  if (fp32)
    MSP_TRY(launch_cast_d2f(n, g, h->g32.p, s));
  else
    MSP_CUDA_TRY(cudaMemcpyAsync(h->pg64.p, g, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  if (h->graph_timed) {  // this replay re-records the events of the previous one
    std::lock_guard<std::mutex> lk(g_stats_mu);
    resolve_pending();
  }
  {
    Probe pr("precond_graph", h->graph_bytes, s);  // timed in stats mode 3
    MSP_CUDA_TRY(cudaGraphLaunch(h->graph, s));
  }
  if (g_stats_mode >= 1) {
    std::lock_guard<std::mutex> lk(g_stats_mu);
    g_launches += h->graph_launches;
    for (const auto& gp : h->graph_probes) {
      g_sites[gp.site].launches += gp.launches;
      g_sites[gp.site].bytes += gp.bytes;
      g_sites[gp.site].flops += gp.flops;
      g_pending.push_back(PendingTiming{gp.site, gp.e0, gp.e1, true});
    }
  }
  if (fp32) return launch_cast_f2d(n, h->w32.p, w, s);
  MSP_CUDA_TRY(cudaMemcpyAsync(w, h->pw64.p, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  return MSP_OK;
}

int alloc_work(msp_handle h) {
  const size_t n = (size_t)h->nb * h->b;
  const int m = h->cfg.restart;
  MSP_TRY(h->pr.alloc(n));
  MSP_TRY(h->py.alloc(n));
  MSP_TRY(h->px.alloc(n));
  MSP_TRY(h->pg64.alloc(n));
  MSP_TRY(h->pw64.alloc(n));
  const size_t nN = (size_t)h->nb * std::max(1, h->b - 1);
  if (h->cfg.precision == MSP_PRECISION_FP64) {
    MSP_TRY(h->c0.alloc((size_t)h->nnzb * h->b));
    MSP_TRY(h->ny.alloc(nN));
  }
  if (h->cfg.precision == MSP_PRECISION_FP32) {
    MSP_TRY(h->c0_32.alloc((size_t)h->nnzb * h->b));
    MSP_TRY(h->g32.alloc(n));
    MSP_TRY(h->w32.alloc(n));
    MSP_TRY(h->pr32.alloc(n));
    MSP_TRY(h->py32.alloc(n));
    MSP_TRY(h->px32.alloc(n));
    MSP_TRY(h->ny32.alloc(nN));
    MSP_TRY(h->vals32.alloc((size_t)h->nnzb * h->b * h->b));
  }
  MSP_TRY(h->V.alloc((size_t)(m + 1) * n));
  MSP_TRY(h->Z.alloc((size_t)m * n));
  MSP_TRY(h->bperm.alloc(n));
  MSP_TRY(h->xperm.alloc(n));
  MSP_TRY(h->rvec.alloc(n));
  MSP_TRY(h->partial.alloc((size_t)krylov_blocks() * 2 * kKrylovMaxK));
  MSP_TRY(h->partial_u.alloc((size_t)krylov_blocks() * kKrylovMaxK));
  MSP_TRY(h->dot_j.alloc(1));
  MSP_CUDA_TRY(cudaMemset(h->dot_j.p, 0xff, sizeof(int)));  // -1
  h->dot_j_dev = -1;
  MSP_TRY(h->gs_T.alloc((size_t)(m + 2) * (m + 2)));
  MSP_TRY(h->gs_d.alloc(2 * kKrylovMaxK));
  MSP_TRY(h->gs_g.alloc(kKrylovMaxK));
  MSP_TRY(h->gs_out.alloc(160));
  MSP_TRY(h->hdev.alloc(72));
  MSP_TRY(h->nrm.alloc(72));
  MSP_TRY(h->ydev.alloc(72));
  MSP_TRY(h->ifl.alloc(4));
  return MSP_OK;
}

// ||x||_2 of a device vector (deterministic reduction), synchronous
int norm2(msp_handle h, const double* x, size_t n, double* out, cudaStream_t s) {
  const int nbk = krylov_blocks();
  MSP_TRY(launch_norm2_partial(n, x, h->partial.p, nbk, s));
  MSP_TRY(launch_reduce_partials(1, nbk, h->partial.p, h->nrm.p, false, s));
  MSP_CUDA_TRY(cudaMemcpyAsync(h->h_pin, h->nrm.p, sizeof(double), cudaMemcpyDeviceToHost, s));
  MSP_CUDA_TRY(cudaStreamSynchronize(s));
  *out = std::sqrt(h->h_pin[0]);
  return MSP_OK;
}

int refresh_values(msp_handle h, const double* d_user_values, cudaStream_t s) {
  const int bb = h->b * h->b;
  MSP_TRY(launch_gather_values((size_t)h->nnzb, bb, h->src.p, d_user_values, h->vals.p, s));
  if (h->cfg.precision == MSP_PRECISION_FP32) {
    MSP_TRY(launch_cast_vals((size_t)h->nnzb * bb, h->vals.p, h->vals32.p, s));
    return launch_extract_col0<float>(h->nnzb, h->b, h->vals32.p, h->c0_32.p, s);
  }
  return launch_extract_col0<double>(h->nnzb, h->b, h->vals.p, h->c0.p, s);
}

// ---------------------------------------------------------------------------------
// FGMRES(m) on colour-ordered vectors (x0 = 0)
// ---------------------------------------------------------------------------------
int fgmres(msp_handle h, double tol, int* iters, double* relres, double* relres_est,
           cudaStream_t s) {
  NvtxRange nvtx("msp:fgmres");
  const size_t n = (size_t)h->nb * h->b;
  const int m = h->cfg.restart;
  const int nbk = krylov_blocks();
  const double* bvec = h->bperm.p;
  double* x = h->xperm.p;
  double* V = h->V.p;
  double* Z = h->Z.p;
  *iters = 0;
  *relres = 0.0;
  *relres_est = 0.0;
  double bnorm = 0.0;
  MSP_TRY(norm2(h, bvec, n, &bnorm, s));
  if (!std::isfinite(bnorm)) return MSP_ERR_NONFINITE;
  MSP_CUDA_TRY(cudaMemsetAsync(x, 0, n * sizeof(double), s));
  if (bnorm == 0.0) return MSP_OK;
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), sv(m + 1), y(m);
  int it = 0, status = MSP_NOT_CONVERGED;
  double est = 1.0;
  while (true) {
    MSP_TRY(launch_bsr_spmv<double>(h->b, h->nb, h->rp.p, h->ci.p, h->vals.p, x, bvec, h->rvec.p,
                                    true, s, nullptr,
                                    long_rows(h, 0, h->nb)));
    double beta = 0.0;
    MSP_TRY(norm2(h, h->rvec.p, n, &beta, s));
    if (!std::isfinite(beta)) return MSP_ERR_NONFINITE;
    if (beta / bnorm <= tol) {
      est = beta / bnorm;
      status = MSP_OK;
      break;
    }
    if (it >= h->cfg.max_it) break;
    MSP_TRY(launch_scale(n, h->rvec.p, 1.0 / beta, V, s));
    std::fill(sv.begin(), sv.end(), 0.0);
    int j_used = 0;
    bool breakdown = false;
    // One-pass classical Gram-Schmidt with the reorthogonalisation carried by a triangular
    // factor (reading D17).  The stored basis u_0..u_j is orthogonalised once; the
    // orthonormal Arnoldi basis is Q = U T^-1, T upper triangular, whose column k (c_k above
    // the diagonal, nu_k on it) is the projection of u_k on the earlier q's and the norm of
    // the rest: the second pass of CGS2, applied to coefficients instead of vectors.  Step
    // j reads the basis twice: one pass of dot products against u_j and against the new
    // vector w = A z_j (which gives column j of T and h = Q^T w), one update w <- w - U g
    // with g = T^-1 h.  Then A z_j = Q h + |w'| u_{j+1}, so column j of the Hessenberg
    // matrix is final once column j + 1 of T is known: h + |w'| c_{j+1} above the
    // diagonal, |w'| nu_{j+1} below it.  It is made final at the next step, or at once
    // (one more pass of dot products, no preconditioner) when the provisional estimate
    // (c_{j+1} = 0, nu_{j+1} = 1) says the tolerance is met, at MaxIt and at the end of
    // the cycle.  Convergence is decided on final columns only.
    std::vector<double> Hraw((size_t)(m + 1) * m, 0.0), hprov(m + 1), col(m + 1);
    const int ldt = m + 2;
    double* T = h->gs_T.p;
    double* out = h->gs_out.p;
    double* hp = h->h_pin;  // host copy of out[0..147]
    double hn_prev = 0.0;   // |w'| of the pending column
    int committed = 0;      // columns 0..committed-1 are final and rotated
    // rotate final column k (Hraw) into H and update the least-squares right-hand side
    auto commit = [&](int k) {
      for (int i = 0; i <= k + 1; ++i) H[(size_t)i * m + k] = Hraw[(size_t)i * m + k];
      for (int i = 0; i < k; ++i) {
        const double a = H[(size_t)i * m + k], c = H[(size_t)(i + 1) * m + k];
        H[(size_t)i * m + k] = cs[i] * a + sn[i] * c;
        H[(size_t)(i + 1) * m + k] = -sn[i] * a + cs[i] * c;
      }
      const double a = H[(size_t)k * m + k], c = H[(size_t)(k + 1) * m + k];
      const double rho = std::sqrt(a * a + c * c);
      if (rho == 0.0) {
        cs[k] = 1.0;
        sn[k] = 0.0;
      } else {
        cs[k] = a / rho;
        sn[k] = c / rho;
      }
      H[(size_t)k * m + k] = rho;
      H[(size_t)(k + 1) * m + k] = 0.0;
      sv[k + 1] = -sn[k] * sv[k];
      sv[k] = cs[k] * sv[k];
      committed = k + 1;
    };
    // residual estimate of column k taken with c_{k+1} = 0, nu_{k+1} = 1 (rotations 0..k-1
    // are final), without changing the committed state
    auto provisional_estimate = [&](int k, double hn) {
      for (int i = 0; i <= k; ++i) col[i] = hprov[i];
      col[k + 1] = hn;
      for (int i = 0; i < k; ++i) {
        const double a = col[i], c = col[i + 1];
        col[i] = cs[i] * a + sn[i] * c;
        col[i + 1] = -sn[i] * a + cs[i] * c;
      }
      const double a = col[k], c = col[k + 1];
      const double rho = std::sqrt(a * a + c * c);
      const double snk = rho == 0.0 ? 0.0 : c / rho;
      return std::fabs(snk * sv[k]) / bnorm;
    };
    auto fetch_out = [&]() -> int {
      MSP_CUDA_TRY(cudaMemcpyAsync(hp, out, 148 * sizeof(double), cudaMemcpyDeviceToHost, s));
      MSP_CUDA_TRY(cudaMemcpyAsync(hp + 150, h->nrm.p + 1, sizeof(double),
                                   cudaMemcpyDeviceToHost, s));
      MSP_CUDA_TRY(cudaStreamSynchronize(s));
      return MSP_OK;
    };
    for (int j = 0; j < m; ++j) {
      double* vj = V + (size_t)j * n;
      double* zj = Z + (size_t)j * n;
      double* w = V + (size_t)(j + 1) * n;
      MSP_TRY(apply_precond(h, vj, zj, s, j));  // also gs_d[0..j] = u_k . u_j
      stats_add_bytes("krylov_basis_dot", (j + 2.0) * n * 8.0, 2.0 * (j + 1) * n);
      {
        Probe pr("krylov_spmv", bsr_bytes(h, 8.0, 1), s, 1, 2.0 * bsr_fmas(h));
        MSP_TRY(launch_bsr_spmv<double>(h->b, h->nb, h->rp.p, h->ci.p, h->vals.p, zj, nullptr, w,
                                        false, s, nullptr,
                                        long_rows(h, 0, h->nb)));
      }
      ++it;
      const int K = j + 2;  // u_0 .. u_j and w
      {
        Probe pr("krylov_multi_dot", (double)(K + 1) * n * 8.0, s, 1, 2.0 * K * n);
        MSP_TRY(launch_multi_dot1(n, V, n, K, w, h->partial.p, kKrylovMaxK, nbk, s));
      }
      MSP_TRY(launch_reduce_partials_strided(K, nbk, kKrylovMaxK, h->partial.p, h->gs_d.p + K,
                                             s));
      MSP_TRY(launch_dcgs_coef(j, h->gs_d.p, T, ldt, h->gs_g.p, out, s));
      {
        Probe pr("krylov_multi_axpy", (double)(K + 1) * n * 8.0, s, 1, 2.0 * K * n);
        MSP_TRY(launch_multi_axpy_norm(n, V, n, j + 1, h->gs_g.p, w, h->partial.p, nbk, s));
      }
      MSP_TRY(launch_reduce_partials(1, nbk, h->partial.p, h->nrm.p, false, s));
      MSP_TRY(launch_normalize(n, w, h->nrm.p, w, h->nrm.p + 1, s));
      MSP_TRY(fetch_out());
      const double hn = hp[150];
      if (!std::isfinite(hn) || !std::isfinite(hp[145])) return MSP_ERR_NONFINITE;
      if (hp[147] != 0.0) {
        // u_j lies in the span of the earlier vectors: the Krylov space is invariant, and
        // the pending column j - 1 ends the cycle with a zero subdiagonal
        if (j == 0) return MSP_ERR_NONFINITE;  // u_0 = r / |r| cannot be degenerate
        for (int i = 0; i < j; ++i) Hraw[(size_t)i * m + (j - 1)] += hn_prev * hp[72 + i];
        Hraw[(size_t)j * m + (j - 1)] = 0.0;
        commit(j - 1);
        j_used = j;
        breakdown = true;
        est = std::fabs(sv[j]) / bnorm;
        break;
      }
      if (j == 0) {
        sv[0] = beta * hp[144];  // r = beta u_0 = beta nu_0 q_0
      } else if (committed < j) {  // column j - 1 becomes final
        for (int i = 0; i < j; ++i) Hraw[(size_t)i * m + (j - 1)] += hn_prev * hp[72 + i];
        Hraw[(size_t)j * m + (j - 1)] = hn_prev * hp[144];
        commit(j - 1);
      }
      for (int i = 0; i <= j; ++i) hprov[i] = hp[i];
      for (int i = 0; i <= j; ++i) Hraw[(size_t)i * m + j] = hp[i];
      hn_prev = hn;
      j_used = j + 1;
      if (hn == 0.0) {  // exact breakdown: w lies in the span of the basis
        Hraw[(size_t)(j + 1) * m + j] = 0.0;
        commit(j);
        est = std::fabs(sv[j + 1]) / bnorm;
        breakdown = true;
        break;
      }
      const bool last = (j == m - 1) || it >= h->cfg.max_it;
      est = provisional_estimate(j, hn);
      if (!std::isfinite(est)) return MSP_ERR_NONFINITE;
      if (last || est <= tol * (1.0 + 1e-6)) {
        // column j final now: column j + 1 of T from the dot products of u_{j+1}
        {
          Probe pr("krylov_finalize_dot", (double)(j + 2) * n * 8.0, s, 1, 2.0 * (j + 2) * n);
          MSP_TRY(launch_multi_dot1(n, V, n, j + 2, w, h->partial.p, kKrylovMaxK, nbk, s));
        }
        MSP_TRY(launch_reduce_partials(j + 2, nbk, h->partial.p, h->gs_d.p, false, s));
        MSP_TRY(launch_dcgs_finalize(j + 1, h->gs_d.p, T, ldt, out, s));
        MSP_TRY(fetch_out());
        if (!std::isfinite(hp[145])) return MSP_ERR_NONFINITE;
        for (int i = 0; i <= j; ++i) Hraw[(size_t)i * m + j] += hn * hp[72 + i];
        Hraw[(size_t)(j + 1) * m + j] = hn * hp[144];  // 0 if u_{j+1} is degenerate
        commit(j);
        est = std::fabs(sv[j + 1]) / bnorm;
        if (!std::isfinite(est)) return MSP_ERR_NONFINITE;
        if (hp[147] != 0.0) breakdown = true;
        if (est <= tol || last || breakdown) break;
      }
    }
    for (int i = j_used - 1; i >= 0; --i) {
      double t = sv[i];
      for (int k = i + 1; k < j_used; ++k) t -= H[(size_t)i * m + k] * y[k];
      y[i] = H[(size_t)i * m + i] != 0.0 ? t / H[(size_t)i * m + i] : 0.0;
    }
    MSP_CUDA_TRY(cudaMemcpyAsync(h->ydev.p, y.data(), j_used * sizeof(double), cudaMemcpyHostToDevice, s));
    MSP_TRY(launch_update_x(n, Z, n, j_used, h->ydev.p, x, s));
    MSP_CUDA_TRY(cudaStreamSynchronize(s));
    if (breakdown) {
      MSP_TRY(launch_bsr_spmv<double>(h->b, h->nb, h->rp.p, h->ci.p, h->vals.p, x, bvec,
                                      h->rvec.p, true, s, nullptr,
                                      long_rows(h, 0, h->nb)));
      double rr = 0.0;
      MSP_TRY(norm2(h, h->rvec.p, n, &rr, s));
      rr /= bnorm;
      if (!(rr <= tol)) {
        *iters = it;
        *relres = rr;
        *relres_est = est;
        return MSP_ERR_BREAKDOWN;
      }
    }
  }
  MSP_TRY(launch_bsr_spmv<double>(h->b, h->nb, h->rp.p, h->ci.p, h->vals.p, x, bvec, h->rvec.p,
                                  true, s, nullptr,
                                  long_rows(h, 0, h->nb)));
  double rr = 0.0;
  MSP_TRY(norm2(h, h->rvec.p, n, &rr, s));
  *relres = rr / bnorm;
  *relres_est = est;
  *iters = it;
  return status;
}

// Chunks of the batched Krylov kernels: level-0 colour classes hold the rows of every
// instance in increasing original index, i.e. instance by instance, so the vector splits
// into (colour, instance) segments, cut into chunks of at most kSegChunk elements.
constexpr int kSegChunk = 8192;
constexpr int kBatchOut = 160;  // per-instance results of a Gram-Schmidt step (see dcgs_coef_kernel)

SegChunks seg_chunks(msp_handle h) {
  SegChunks sc;
  sc.n = h->seg_n;
  sc.start = h->seg_start.p;
  sc.end = h->seg_end.p;
  sc.inst = h->seg_inst.p;
  sc.iptr = h->seg_iptr.p;
  sc.ichunks = h->seg_ichunks.p;
  return sc;
}

// Right-preconditioned FGMRES(m) run for every instance at once: one preconditioner
// application and one SpMV per step serve all instances (the matrix and the preconditioner
// are block diagonal); inner products, norms, Hessenberg matrices, rotations, convergence
// and restarts are per instance.  Each step uses classical Gram-Schmidt with a second pass
// (always taken).  An instance that converges or stops leaves the active set: the Krylov
// kernels, the SpMV and the level-0 kernels of the preconditioner skip its rows (a row
// mask), so a straggling instance no longer costs the others' bandwidth there; its part
// of the next basis vector is set to zero, so what the coarse AMG levels still compute for
// it stays finite (the dense coarsest solve multiplies every instance's entries, zeros
// included, into every row).
int fgmres_batched(msp_handle h, double tol, std::vector<int>& its, std::vector<double>& relres,
                   std::vector<double>& relest, std::vector<int>& status, cudaStream_t s) {
  NvtxRange nvtx("msp:fgmres_batched");
  const int B = h->batch, m = h->cfg.restart;
  const size_t n = (size_t)h->nb * h->b;
  const int KM = kKrylovMaxK;
  const SegChunks sc = seg_chunks(h);
  const double* bvec = h->bperm.p;
  double* x = h->xperm.p;
  double* V = h->V.p;
  double* Z = h->Z.p;
  double* nb2 = h->h_bpin + (size_t)2 * B * KM;  // squared norms
  its.assign(B, 0);
  relres.assign(B, 0.0);
  relest.assign(B, 0.0);
  status.assign(B, MSP_NOT_CONVERGED);
  std::vector<int> act(B, 1), done(B, 0), stop(B, 0), jused(B, 0), brk(B, 0);
  auto upload_act = [&](const std::vector<int>& a) -> int {
    MSP_CUDA_TRY(cudaMemcpyAsync(h->bact.p, a.data(), B * sizeof(int), cudaMemcpyHostToDevice, s));
    MSP_TRY(launch_expand_mask(h->nb, h->row_inst.p, h->bact.p, h->rmask0.p, s));
    for (size_t l = 1; l < h->levels.size(); ++l) {
      Level& L = h->levels[l];
      if (L.rmask.p) MSP_TRY(launch_expand_mask(L.A.n, L.row_inst.p, h->bact.p, L.rmask.p, s));
    }
    // the host vector may change before the copy runs: wait for it
    MSP_CUDA_TRY(cudaStreamSynchronize(s));
    return MSP_OK;
  };
  // zero the part of v that belongs to the instances with z[i] != 0
  auto zero_parts = [&](const std::vector<int>& z, double* v) -> int {
    MSP_CUDA_TRY(cudaMemcpyAsync(h->bzero.p, z.data(), B * sizeof(int), cudaMemcpyHostToDevice, s));
    MSP_TRY(launch_seg_zero(sc, h->bzero.p, v, s));
    MSP_CUDA_TRY(cudaStreamSynchronize(s));
    return MSP_OK;
  };
  // per-instance squared norms of a vector into nb2[i * KM]
  auto seg_norms = [&](const double* v) -> int {
    MSP_TRY(launch_seg_multi_dot(sc, h->bact.p, v, n, 1, v, h->bpart.p, s));
    MSP_TRY(launch_seg_reduce(sc, B, 1, h->bact.p, h->bpart.p, h->bn.p, 0, s));
    MSP_CUDA_TRY(cudaMemcpyAsync(nb2, h->bn.p, (size_t)B * KM * sizeof(double),
                                 cudaMemcpyDeviceToHost, s));
    MSP_CUDA_TRY(cudaStreamSynchronize(s));
    return MSP_OK;
  };
  MSP_TRY(upload_act(act));
  MSP_TRY(seg_norms(bvec));
  std::vector<double> bnorm(B);
  for (int i = 0; i < B; ++i) {
    bnorm[i] = std::sqrt(nb2[(size_t)i * KM]);
    if (!std::isfinite(bnorm[i])) {
      status[i] = MSP_ERR_NONFINITE;
      done[i] = 1;
    } else if (bnorm[i] == 0.0) {
      status[i] = MSP_OK;
      done[i] = 1;
    }
  }
  MSP_CUDA_TRY(cudaMemsetAsync(x, 0, n * sizeof(double), s));
  std::vector<std::vector<double>> H(B), cs(B), sn(B), sv(B);
  for (int i = 0; i < B; ++i) {
    H[i].assign((size_t)(m + 1) * m, 0.0);
    cs[i].assign(m, 0.0);
    sn[i].assign(m, 0.0);
    sv[i].assign(m + 1, 0.0);
  }
  std::vector<double> est(B, 1.0), ybuf((size_t)B * KM, 0.0);
  std::vector<std::vector<double>> Hraw(B, std::vector<double>((size_t)(m + 1) * m, 0.0));
  std::vector<int> committed(B, 0);
  std::vector<double> hn_prev(B, 0.0), beta0(B, 0.0);
  std::vector<int> cnt(B, 0);
  while (true) {
    for (int i = 0; i < B; ++i) act[i] = !done[i];
    MSP_TRY(upload_act(act));
    MSP_TRY(launch_bsr_spmv<double>(h->b, h->nb, h->rp.p, h->ci.p, h->vals.p, x, bvec, h->rvec.p,
                                    true, s, h->rmask0.p,
                                    long_rows(h, 0, h->nb)));
    MSP_TRY(seg_norms(h->rvec.p));
    int ncycle = 0;
    for (int i = 0; i < B; ++i) {
      if (done[i]) continue;
      const double beta = std::sqrt(nb2[(size_t)i * KM]);
      if (!std::isfinite(beta)) {
        status[i] = MSP_ERR_NONFINITE;
        done[i] = 1;
      } else if (beta / bnorm[i] <= tol) {
        est[i] = beta / bnorm[i];
        status[i] = MSP_OK;
        done[i] = 1;
      } else if (brk[i]) {
        status[i] = MSP_ERR_BREAKDOWN;
        relest[i] = est[i];
        done[i] = 1;
      } else if (its[i] >= h->cfg.max_it) {
        done[i] = 1;
      } else {
        std::fill(sv[i].begin(), sv[i].end(), 0.0);
        sv[i][0] = beta;
        ++ncycle;
      }
      act[i] = !done[i];
      stop[i] = 0;
      jused[i] = 0;
    }
    if (ncycle == 0) break;
    MSP_TRY(upload_act(act));
    MSP_TRY(launch_seg_normalize(sc, h->bact.p, h->rvec.p, h->bn.p, V, s));
    MSP_TRY(zero_parts(done, V));  // the instances outside this cycle start from zero
    // one-pass Gram-Schmidt per instance, as in the single solve (reading D17): the basis
    // is orthogonalised once, the second pass is carried by each instance's triangular
    // factor T_i, and column j of H_i becomes final once column j + 1 of T_i is known
    const int m2 = m + 2;
    for (int i = 0; i < B; ++i) {
      if (!act[i]) continue;
      std::fill(Hraw[i].begin(), Hraw[i].end(), 0.0);
      committed[i] = 0;
      hn_prev[i] = 0.0;
      beta0[i] = sv[i][0];
    }
    // rotate final column k of instance i into H_i, update its least-squares right side
    auto commit = [&](int i, int k) {
      std::vector<double>& Hi = H[i];
      const std::vector<double>& Ri = Hraw[i];
      for (int r = 0; r <= k + 1; ++r) Hi[(size_t)r * m + k] = Ri[(size_t)r * m + k];
      for (int r = 0; r < k; ++r) {
        const double a = Hi[(size_t)r * m + k], c = Hi[(size_t)(r + 1) * m + k];
        Hi[(size_t)r * m + k] = cs[i][r] * a + sn[i][r] * c;
        Hi[(size_t)(r + 1) * m + k] = -sn[i][r] * a + cs[i][r] * c;
      }
      const double a = Hi[(size_t)k * m + k], c = Hi[(size_t)(k + 1) * m + k];
      const double rho = std::sqrt(a * a + c * c);
      if (rho == 0.0) {
        cs[i][k] = 1.0;
        sn[i][k] = 0.0;
      } else {
        cs[i][k] = a / rho;
        sn[i][k] = c / rho;
      }
      Hi[(size_t)k * m + k] = rho;
      Hi[(size_t)(k + 1) * m + k] = 0.0;
      sv[i][k + 1] = -sn[i][k] * sv[i][k];
      sv[i][k] = cs[i][k] * sv[i][k];
      committed[i] = k + 1;
    };
    auto provisional = [&](int i, int k, const double* h, double hn) {
      std::vector<double> col(k + 2);
      for (int r = 0; r <= k; ++r) col[r] = h[r];
      col[k + 1] = hn;
      for (int r = 0; r < k; ++r) {
        const double a = col[r], c = col[r + 1];
        col[r] = cs[i][r] * a + sn[i][r] * c;
        col[r + 1] = -sn[i][r] * a + cs[i][r] * c;
      }
      const double rho = std::sqrt(col[k] * col[k] + col[k + 1] * col[k + 1]);
      return std::fabs((rho == 0.0 ? 0.0 : col[k + 1] / rho) * sv[i][k]) / bnorm[i];
    };
    bool any = true;
    for (int j = 0; j < m && any; ++j) {
      double* vj = V + (size_t)j * n;
      double* zj = Z + (size_t)j * n;
      double* w = V + (size_t)(j + 1) * n;
      MSP_TRY(apply_precond(h, vj, zj, s));
      {
        Probe pr("batch_spmv", bsr_bytes(h, 8.0, 1), s);
        MSP_TRY(launch_bsr_spmv<double>(h->b, h->nb, h->rp.p, h->ci.p, h->vals.p, zj, nullptr, w,
                                        false, s, h->rmask0.p,
                                        long_rows(h, 0, h->nb)));
      }
      const int K = j + 2;
      {
        Probe pr("batch_multi_dot", (double)K * n * 8.0, s);
        MSP_TRY(launch_seg_multi_dot2(sc, h->bact.p, V, n, K, vj, w, h->bpart.p, s));
      }
      MSP_TRY(launch_seg_reduce_strided(sc, B, 2 * K, h->bact.p, h->bpart.p, 2 * KM,
                                        h->gs_bD.p, 2 * KM, s));
      MSP_TRY(launch_dcgs_coef_batch(B, j, h->bact.p, h->gs_bD.p, 2 * KM, h->gs_bT.p, m2 * m2, m2,
                                     h->by.p, KM, h->gs_bout.p, kBatchOut, s));
      {
        Probe pr("batch_multi_axpy", (double)(K + 1) * n * 8.0, s);
        MSP_TRY(launch_seg_multi_axpy_norm(sc, h->bact.p, V, n, j + 1, h->by.p, w, h->bpart.p, s));
      }
      MSP_TRY(launch_seg_reduce(sc, B, 1, h->bact.p, h->bpart.p, h->bn.p, 0, s));
      MSP_TRY(launch_seg_normalize(sc, h->bact.p, w, h->bn.p, w, s));
      MSP_CUDA_TRY(cudaMemcpyAsync(h->h_bout, h->gs_bout.p, (size_t)B * kBatchOut * sizeof(double),
                                   cudaMemcpyDeviceToHost, s));
      MSP_CUDA_TRY(cudaMemcpyAsync(nb2, h->bn.p, (size_t)B * KM * sizeof(double),
                                   cudaMemcpyDeviceToHost, s));
      MSP_CUDA_TRY(cudaStreamSynchronize(s));
      bool changed = false;
      any = false;
      std::vector<int> left(B, 0), fin(B, 0);
      std::vector<double> hn_now(B, 0.0);
      bool any_fin = false;
      auto leave = [&](int i) {
        act[i] = 0;
        left[i] = 1;
        changed = true;
      };
      for (int i = 0; i < B; ++i) {
        if (!act[i]) continue;
        ++its[i];
        const double* o = h->h_bout + (size_t)i * kBatchOut;
        const double hn = std::sqrt(nb2[(size_t)i * KM]);
        hn_now[i] = hn;
        if (!std::isfinite(hn) || !std::isfinite(o[145])) {
          status[i] = MSP_ERR_NONFINITE;
          done[i] = 1;
          jused[i] = 0;
          leave(i);
          continue;
        }
        std::vector<double>& Ri = Hraw[i];
        if (o[147] != 0.0) {  // u_j lies in the span of the earlier vectors: breakdown
          if (j == 0) {
            status[i] = MSP_ERR_NONFINITE;
            done[i] = 1;
            jused[i] = 0;
          } else {
            for (int k = 0; k < j; ++k) Ri[(size_t)k * m + (j - 1)] += hn_prev[i] * o[72 + k];
            Ri[(size_t)j * m + (j - 1)] = 0.0;
            commit(i, j - 1);
            jused[i] = j;
            est[i] = std::fabs(sv[i][j]) / bnorm[i];
            brk[i] = 1;
          }
          leave(i);
          continue;
        }
        if (j == 0) {
          sv[i][0] = beta0[i] * o[144];
        } else if (committed[i] < j) {
          for (int k = 0; k < j; ++k) Ri[(size_t)k * m + (j - 1)] += hn_prev[i] * o[72 + k];
          Ri[(size_t)j * m + (j - 1)] = hn_prev[i] * o[144];
          commit(i, j - 1);
        }
        for (int k = 0; k <= j; ++k) Ri[(size_t)k * m + j] = o[k];
        hn_prev[i] = hn;
        jused[i] = j + 1;
        if (hn == 0.0) {  // exact breakdown
          Ri[(size_t)(j + 1) * m + j] = 0.0;
          commit(i, j);
          est[i] = std::fabs(sv[i][j + 1]) / bnorm[i];
          brk[i] = 1;
          leave(i);
          continue;
        }
        const bool last = (j == m - 1) || its[i] >= h->cfg.max_it;
        est[i] = provisional(i, j, o, hn);
        if (!std::isfinite(est[i])) {
          status[i] = MSP_ERR_NONFINITE;
          done[i] = 1;
          jused[i] = 0;
          leave(i);
          continue;
        }
        if (last || est[i] <= tol * (1.0 + 1e-6)) {
          fin[i] = 1;
          any_fin = true;
        } else {
          any = true;
        }
      }
      if (any_fin) {  // make column j final for those instances (no preconditioner)
        MSP_CUDA_TRY(cudaMemcpyAsync(h->gs_bfin.p, fin.data(), B * sizeof(int),
                                     cudaMemcpyHostToDevice, s));
        {
          Probe pr("batch_finalize_dot", (double)(j + 2) * n * 8.0, s);
          MSP_TRY(launch_seg_multi_dot(sc, h->gs_bfin.p, V, n, j + 2, w, h->bpart.p, s));
        }
        MSP_TRY(launch_seg_reduce(sc, B, j + 2, h->gs_bfin.p, h->bpart.p, h->bh.p, 0, s));
        MSP_TRY(launch_dcgs_finalize_batch(B, j + 1, h->gs_bfin.p, h->bh.p, KM, h->gs_bT.p,
                                           m2 * m2, m2, h->gs_bout.p, kBatchOut, s));
        MSP_CUDA_TRY(cudaMemcpyAsync(h->h_bout, h->gs_bout.p,
                                     (size_t)B * kBatchOut * sizeof(double),
                                     cudaMemcpyDeviceToHost, s));
        MSP_CUDA_TRY(cudaStreamSynchronize(s));  // fin is read by the copy above
        for (int i = 0; i < B; ++i) {
          if (!fin[i]) continue;
          const double* o = h->h_bout + (size_t)i * kBatchOut;
          std::vector<double>& Ri = Hraw[i];
          const double hn = hn_now[i];
          for (int k = 0; k <= j; ++k) Ri[(size_t)k * m + j] += hn * o[72 + k];
          Ri[(size_t)(j + 1) * m + j] = hn * o[144];
          commit(i, j);
          est[i] = std::fabs(sv[i][j + 1]) / bnorm[i];
          if (o[147] != 0.0) brk[i] = 1;
          const bool last = (j == m - 1) || its[i] >= h->cfg.max_it;
          if (!std::isfinite(est[i])) {
            status[i] = MSP_ERR_NONFINITE;
            done[i] = 1;
            jused[i] = 0;
            leave(i);
          } else if (est[i] <= tol || last || brk[i]) {
            leave(i);
          } else {
            any = true;
          }
        }
      }
      if (changed && any) {
        MSP_TRY(upload_act(act));
        MSP_TRY(zero_parts(left, w));  // the next preconditioner input of those instances
      }
    }
    // x_i += Z y_i with y_i = H_i^{-1} s_i
    std::fill(ybuf.begin(), ybuf.end(), 0.0);
    for (int i = 0; i < B; ++i) {
      cnt[i] = jused[i];
      const int J = jused[i];
      for (int r = J - 1; r >= 0; --r) {
        double t = sv[i][r];
        for (int k = r + 1; k < J; ++k) t -= H[i][(size_t)r * m + k] * ybuf[(size_t)i * KM + k];
        const double d = H[i][(size_t)r * m + r];
        ybuf[(size_t)i * KM + r] = d != 0.0 ? t / d : 0.0;
      }
    }
    MSP_CUDA_TRY(cudaMemcpyAsync(h->bydev.p, ybuf.data(), (size_t)B * KM * sizeof(double),
                                 cudaMemcpyHostToDevice, s));
    MSP_CUDA_TRY(cudaMemcpyAsync(h->bcount.p, cnt.data(), B * sizeof(int), cudaMemcpyHostToDevice, s));
    MSP_TRY(launch_seg_update_x(sc, h->bcount.p, Z, n, h->bydev.p, x, s));
    MSP_CUDA_TRY(cudaStreamSynchronize(s));
  }
  // true residuals
  for (int i = 0; i < B; ++i) act[i] = bnorm[i] > 0.0 && std::isfinite(bnorm[i]);
  MSP_TRY(upload_act(act));
  MSP_TRY(launch_bsr_spmv<double>(h->b, h->nb, h->rp.p, h->ci.p, h->vals.p, x, bvec, h->rvec.p,
                                  true, s, h->rmask0.p,
                                  long_rows(h, 0, h->nb)));
  MSP_TRY(seg_norms(h->rvec.p));
  for (int i = 0; i < B; ++i) {
    if (act[i]) relres[i] = std::sqrt(nb2[(size_t)i * KM]) / bnorm[i];
    if (status[i] != MSP_ERR_BREAKDOWN) relest[i] = est[i];
    if (bnorm[i] == 0.0) relest[i] = 0.0;
  }
  return MSP_OK;
}

int pattern_setup(msp_handle h, const int32_t* d_rp, const int32_t* d_ci, cudaStream_t s) {
  NvtxRange nvtx("msp:pattern_setup");
  const int nb = h->nb;
  const size_t nnzb = (size_t)h->nnzb;
  DevBuf<int> urp, uci, udpos;
  MSP_TRY(urp.alloc(nb + 1));
  MSP_TRY(uci.alloc(nnzb));
  MSP_TRY(udpos.alloc(nb));
  MSP_CUDA_TRY(cudaMemcpyAsync(urp.p, d_rp, (nb + 1) * sizeof(int), cudaMemcpyDeviceToDevice, s));
  MSP_CUDA_TRY(cudaMemcpyAsync(uci.p, d_ci, nnzb * sizeof(int), cudaMemcpyDeviceToDevice, s));
  int hr[2] = {0, 0};
  MSP_CUDA_TRY(cudaMemcpyAsync(&hr[0], urp.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  MSP_CUDA_TRY(cudaMemcpyAsync(&hr[1], urp.p + nb, sizeof(int), cudaMemcpyDeviceToHost, s));
  MSP_CUDA_TRY(cudaStreamSynchronize(s));
  if (hr[0] != 0 || (int64_t)hr[1] != h->nnzb) return MSP_ERR_PATTERN;
  MSP_TRY(reset_flags(h, s));
  MSP_TRY(launch_check_pattern(nb, (int)nnzb, urp.p, uci.p, udpos.p, h->flags.p, s));
  if (sync_flags(h, s) != MSP_OK) return h->h_flags->code;
  // colouring of the block graph (Algorithms 4.1/4.2) and the colour permutation
  MSP_TRY(colour_graph(h, nb, urp.p, uci.p, (int)nnzb, h->colour0, h->perm0, h->cptr0, &h->g0, s));
  MSP_TRY(h->iperm0.alloc(nb));
  MSP_TRY(launch_scatter_inverse(nb, h->perm0.p, h->iperm0.p, s));
  MSP_TRY(permute_pattern(h, nb, urp.p, uci.p, (int)nnzb, h->iperm0.p, h->rp, h->ci, h->src, s));
  MSP_TRY(h->dpos.alloc(nb));
  MSP_TRY(launch_diag_pos(nb, h->rp.p, h->ci.p, h->dpos.p, s));
  MSP_TRY(colour_counts(h->rp.p, h->dpos.p, nb, h->cptr0, h->cc0, s));
  // rows longer than kLongRowBlocks blocks, in the colour order
  {
    std::vector<int> hrp(nb + 1);
    MSP_CUDA_TRY(cudaMemcpyAsync(hrp.data(), h->rp.p, (nb + 1) * sizeof(int),
                                 cudaMemcpyDeviceToHost, s));
    MSP_CUDA_TRY(cudaStreamSynchronize(s));
    h->long_h.clear();
    for (int i = 0; i < nb; ++i)
      if (hrp[i + 1] - hrp[i] > kLongRowBlocks) h->long_h.push_back(i);
    h->long_d.release();
    if (!h->long_h.empty()) {
      MSP_TRY(h->long_d.alloc(h->long_h.size()));
      MSP_CUDA_TRY(cudaMemcpyAsync(h->long_d.p, h->long_h.data(), h->long_h.size() * sizeof(int),
                                   cudaMemcpyHostToDevice, s));
    }
  }
  MSP_CUDA_TRY(cudaStreamSynchronize(s));
  return MSP_OK;
}

// Adds the change of the calling thread's DevBuf footprint during a public call to the
// handle's own count (the outermost call only: entry points call one another).
struct DevBytesScope {
  msp_handle h;
  long long t0;
  bool outer;
  explicit DevBytesScope(msp_handle hh)
      : h(hh), t0(t_dev_bytes), outer(t_bytes_scope_depth++ == 0) {}
  ~DevBytesScope() {
    --t_bytes_scope_depth;
    if (outer && h) h->dev_bytes += t_dev_bytes - t0;
  }
  DevBytesScope(const DevBytesScope&) = delete;
  DevBytesScope& operator=(const DevBytesScope&) = delete;
};

void destroy(msp_handle h) {
  if (!h) return;
  drop_graph(h);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->side_stream) cudaStreamDestroy(h->side_stream);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  if (h->h_flags) cudaFreeHost(h->h_flags);
  if (h->h_pin) cudaFreeHost(h->h_pin);
  if (h->h_bpin) cudaFreeHost(h->h_bpin);
  if (h->h_bout) cudaFreeHost(h->h_bout);
  if (h->staged_ev) cudaEventDestroy(h->staged_ev);
  if (h->consumed_ev) cudaEventDestroy(h->consumed_ev);
  if (h->ss) sort_scratch_destroy(h->ss);
  delete h;
}

bool config_ok(const msp_config& c, int b) {
  return c.mu >= 0 && c.restart >= 1 && c.restart <= 64 && c.max_it >= 0 && c.coarse_max >= 1 &&
         c.npass >= 1 && c.npass <= 4 && c.pre_sweeps >= 0 && c.post_sweeps >= 0 &&
         c.bgs_sweeps >= 0 && c.bilu_order == 0 && c.precond >= 0 && c.precond <= 4 &&
         c.max_levels >= 1 && c.beta >= 0.0 && c.coarse_hard_max >= 1 &&
         (c.precision == MSP_PRECISION_FP64 || c.precision == MSP_PRECISION_FP32) &&
         (c.colouring == MSP_COLOURING_ALG41 || c.colouring == MSP_COLOURING_JP) &&
         c.smoother >= MSP_SMOOTHER_PGS_MC && c.smoother <= MSP_SMOOTHER_PGS_NO &&
         c.loop_limit >= 0 && (c.autotune == 0 || c.autotune == 1) && b >= 1 &&
         b <= 8;
}

}  // namespace
}  // namespace msp

using namespace msp;

extern "C" {

int msp_config_default(msp_config* c) {
  if (!c) return MSP_ERR_ARG;
  c->mu = 20;
  c->restart = 30;
  c->max_it = 1000;
  c->coarse_max = 10000;
  c->npass = 2;
  c->pre_sweeps = 1;
  c->post_sweeps = 1;
  c->bgs_sweeps = 6;
  c->decoupling = 1;
  c->bilu_order = 0;
  c->precond = MSP_PREC_MSP;
  c->max_levels = 20;
  c->beta = 0.25;
  c->agg_seed = 0x2208085940ULL;
  c->coarse_hard_max = 20000;
  c->precision = MSP_PRECISION_FP64;
  c->colouring = MSP_COLOURING_ALG41;
  c->smoother = MSP_SMOOTHER_PGS_MC;
  c->loop_limit = 0;
  c->autotune = 0;
  return MSP_OK;
}

const char* msp_status_string(int st) {
  switch (st) {
    case MSP_OK: return "ok";
    case MSP_NOT_CONVERGED: return "not converged (MaxIt reached)";
    case MSP_ERR_ARG: return "invalid argument";
    case MSP_ERR_PATTERN: return "invalid BSR pattern (unsorted/out-of-range columns or missing diagonal)";
    case MSP_ERR_SINGULAR_BLOCK: return "singular diagonal block, pivot or coarsest matrix";
    case MSP_ERR_NONFINITE: return "non-finite value";
    case MSP_ERR_BREAKDOWN: return "Krylov breakdown";
    case MSP_ERR_NOMEM: return "out of device memory";
    case MSP_ERR_TIMEOUT: return "a bounded device loop exceeded its limit";
    case MSP_ERR_CUDA: return "CUDA error";
    default: return "unknown status";
  }
}

// Last CUDA error text of this thread (diagnostics; not part of the stable ABI).
const char* msp_last_error(void) { return g_last_error.c_str(); }

int msp_setup(msp_handle* out, const msp_config* cfg, int32_t nb, int32_t b,
              const int32_t* d_row_ptr, const int32_t* d_col_idx, const double* d_values,
              int64_t nnzb, void* stream) {
  if (!out) return MSP_ERR_ARG;
  *out = nullptr;
  if (!cfg || nb <= 0 || b < 1 || b > 8 || nnzb < nb || nnzb > 0x7fffffffLL || !d_row_ptr ||
      !d_col_idx || !d_values || !config_ok(*cfg, b))
    return MSP_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  msp_handle h = nullptr;
  const long long bytes0 = t_dev_bytes;
  try {
    h = new msp_handle_s();
    h->cfg = *cfg;
    h->nb = nb;
    h->b = b;
    h->nnzb = nnzb;
    cudaGetDevice(&h->device);
    h->ss = sort_scratch_create();
    int st = h->flags.alloc(1);
    if (st == MSP_OK && cudaMallocHost(&h->h_flags, sizeof(DevFlags)) != cudaSuccess) st = MSP_ERR_NOMEM;
    if (st == MSP_OK && cudaMallocHost(&h->h_pin, 256 * sizeof(double)) != cudaSuccess) st = MSP_ERR_NOMEM;
    if (st == MSP_OK) {
      auto t0 = Clock::now();
      st = pattern_setup(h, d_row_ptr, d_col_idx, s);
      if (st == MSP_OK) st = h->vals.alloc((size_t)nnzb * b * b);
      if (st == MSP_OK) st = alloc_work(h);
      if (st == MSP_OK) st = reset_flags(h, s);
      if (st == MSP_OK) st = launch_check_finite_vals((size_t)nnzb * b * b, d_values, h->flags.p, s);
      if (st == MSP_OK && sync_flags(h, s) != MSP_OK) st = h->h_flags->code;
      if (st == MSP_OK) st = refresh_values(h, d_values, s);
      if (st == MSP_OK) st = value_setup(h, s);
      (void)t0;
    }
    if (st != MSP_OK) {
      destroy(h);
      return st;
    }
  } catch (const std::bad_alloc&) {
    destroy(h);
    return MSP_ERR_NOMEM;
  } catch (...) {
    destroy(h);
    return MSP_ERR_CUDA;
  }
  h->dev_bytes = t_dev_bytes - bytes0;
  *out = h;
  return MSP_OK;
}

int msp_update_values(msp_handle h, const double* d_values, void* stream) {
  if (!h || !d_values) return MSP_ERR_ARG;
  DevBytesScope bytes_scope(h);
  cudaStream_t s = (cudaStream_t)stream;
  try {
    MSP_TRY(reset_flags(h, s));
    MSP_TRY(launch_check_finite_vals((size_t)h->nnzb * h->b * h->b, d_values, h->flags.p, s));
    if (sync_flags(h, s) != MSP_OK) return h->h_flags->code;
    return refresh_values(h, d_values, s);
  } catch (...) {
    return MSP_ERR_NOMEM;
  }
}

int msp_update_values_host(msp_handle h, const double* h_values, void* stream) {
  if (!h || !h_values) return MSP_ERR_ARG;
  DevBytesScope bytes_scope(h);
  cudaStream_t s = (cudaStream_t)stream;
  const size_t cnt = (size_t)h->nnzb * h->b * h->b;
  if (!h->staging.p) MSP_TRY(h->staging.alloc(cnt));
  MSP_CUDA_TRY(cudaMemcpyAsync(h->staging.p, h_values, cnt * sizeof(double),
                               cudaMemcpyHostToDevice, s));
  return msp_update_values(h, h->staging.p, stream);
}

int msp_stage_values_host(msp_handle h, const double* h_values, void* stream) {
  if (!h || !h_values) return MSP_ERR_ARG;
  DevBytesScope bytes_scope(h);
  cudaStream_t s = (cudaStream_t)stream;
  const size_t cnt = (size_t)h->nnzb * h->b * h->b;
  if (!h->staged.p) MSP_TRY(h->staged.alloc(cnt));
  if (!h->staged_ev) MSP_CUDA_TRY(cudaEventCreateWithFlags(&h->staged_ev, cudaEventDisableTiming));
  if (!h->consumed_ev)
    MSP_CUDA_TRY(cudaEventCreateWithFlags(&h->consumed_ev, cudaEventDisableTiming));
  // the buffer is free again once the previous staged values have been gathered
  if (h->consumed_recorded) MSP_CUDA_TRY(cudaStreamWaitEvent(s, h->consumed_ev, 0));
  MSP_CUDA_TRY(cudaMemcpyAsync(h->staged.p, h_values, cnt * sizeof(double),
                               cudaMemcpyHostToDevice, s));
  MSP_CUDA_TRY(cudaEventRecord(h->staged_ev, s));
  h->staged_pending = true;
  return MSP_OK;
}

int msp_update_values_staged(msp_handle h, void* stream) {
  if (!h || !h->staged_pending) return MSP_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  MSP_CUDA_TRY(cudaStreamWaitEvent(s, h->staged_ev, 0));
  const int st = msp_update_values(h, h->staged.p, stream);
  MSP_CUDA_TRY(cudaEventRecord(h->consumed_ev, s));
  h->consumed_recorded = true;
  h->staged_pending = false;
  return st;
}

int msp_solve(msp_handle h, const double* d_b, double* d_x, double rel_tol,
              msp_solve_info* info, void* stream) {
  if (!h || !d_b || !d_x || !(rel_tol > 0.0)) return MSP_ERR_ARG;
  DevBytesScope bytes_scope(h);
  cudaStream_t s = (cudaStream_t)stream;
  if (h->batch) MSP_CUDA_TRY(cudaMemsetAsync(h->rmask0.p, 1, h->nb, s));  // every row
  msp_solve_info local{};
  msp_solve_info* inf = info ? info : &local;
  std::memset(inf, 0, sizeof(*inf));
  try {
    const size_t n = (size_t)h->nb * h->b;
    MSP_CUDA_TRY(cudaMemsetAsync(h->ifl.p, 0, sizeof(int), s));
    MSP_TRY(launch_check_finite(n, d_b, h->ifl.p, s));
    int bad = 0;
    MSP_CUDA_TRY(cudaMemcpyAsync(&bad, h->ifl.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    MSP_CUDA_TRY(cudaStreamSynchronize(s));
    if (bad) {
      inf->status = MSP_ERR_NONFINITE;
      return MSP_ERR_NONFINITE;
    }
    // adaptive setup (Section 3.2)
    auto ts = Clock::now();
    if (!h->first_solve && (h->prev_it > h->cfg.mu || !h->setup_valid)) {
      const int st = value_setup(h, s);
      if (st != MSP_OK) {
        inf->status = st;
        return st;
      }
      inf->setup_performed = 1;
    } else if (h->first_solve) {
      inf->setup_performed = 1;  // generated by msp_setup (iota = 1)
    }
    inf->t_setup_ms = ms_since(ts);
    h->first_solve = false;
    auto t0 = Clock::now();
    MSP_TRY(launch_gather_blocks(h->nb, h->b, h->perm0.p, d_b, h->bperm.p, s));
    int it = 0;
    double rr = 0.0, est = 0.0;
    const int st = fgmres(h, rel_tol, &it, &rr, &est, s);
    if (st >= 0 || st == MSP_ERR_BREAKDOWN)
      MSP_TRY(launch_scatter_blocks(h->nb, h->b, h->perm0.p, h->xperm.p, d_x, s));
    MSP_CUDA_TRY(cudaStreamSynchronize(s));
    h->prev_it = it;
    inf->status = st;
    inf->iterations = it;
    inf->setup_calls = h->setup_calls;
    inf->levels = (int)h->levels.size();
    inf->colours_l0 = h->g0;
    inf->rel_residual = rr;
    inf->rel_residual_est = est;
    inf->t_solve_ms = ms_since(t0);
    return st;
  } catch (...) {
    inf->status = MSP_ERR_NOMEM;
    return MSP_ERR_NOMEM;
  }
}

int msp_solve_host(msp_handle h, const double* h_b, double* h_x, double rel_tol,
                   msp_solve_info* info, void* stream) {
  if (!h || !h_b || !h_x) return MSP_ERR_ARG;
  DevBytesScope bytes_scope(h);
  cudaStream_t s = (cudaStream_t)stream;
  const size_t n = (size_t)h->nb * h->b, bytes = n * sizeof(double);
  if (!h->e2e_b.p) MSP_TRY(h->e2e_b.alloc(n));
  if (!h->e2e_x.p) MSP_TRY(h->e2e_x.alloc(n));
  MSP_CUDA_TRY(cudaMemcpyAsync(h->e2e_b.p, h_b, bytes, cudaMemcpyHostToDevice, s));
  const int st = msp_solve(h, h->e2e_b.p, h->e2e_x.p, rel_tol, info, stream);
  if (st < 0 && st != MSP_ERR_BREAKDOWN) return st;
  MSP_CUDA_TRY(cudaMemcpyAsync(h_x, h->e2e_x.p, bytes, cudaMemcpyDeviceToHost, s));
  MSP_CUDA_TRY(cudaStreamSynchronize(s));
  return st;
}

int msp_free(msp_handle h) {
  destroy(h);
  return MSP_OK;
}

int msp_apply_precond(msp_handle h, const double* d_g, double* d_w, void* stream) {
  if (!h || !d_g || !d_w) return MSP_ERR_ARG;
  DevBytesScope bytes_scope(h);
  cudaStream_t s = (cudaStream_t)stream;
  if (h->batch) MSP_CUDA_TRY(cudaMemsetAsync(h->rmask0.p, 1, h->nb, s));  // every row
  try {
    MSP_TRY(launch_gather_blocks(h->nb, h->b, h->perm0.p, d_g, h->bperm.p, s));
    MSP_TRY(apply_precond(h, h->bperm.p, h->xperm.p, s));
    MSP_TRY(launch_scatter_blocks(h->nb, h->b, h->perm0.p, h->xperm.p, d_w, s));
    MSP_CUDA_TRY(cudaStreamSynchronize(s));
    return MSP_OK;
  } catch (...) {
    return MSP_ERR_NOMEM;
  }
}

int msp_spmv(msp_handle h, const double* d_x, double* d_y, void* stream) {
  if (!h || !d_x || !d_y) return MSP_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  MSP_TRY(launch_gather_blocks(h->nb, h->b, h->perm0.p, d_x, h->bperm.p, s));
  {
    Probe pr("api_spmv", bsr_bytes(h, 8.0, 1), s);
    MSP_TRY(launch_bsr_spmv<double>(h->b, h->nb, h->rp.p, h->ci.p, h->vals.p, h->bperm.p,
                                    nullptr, h->xperm.p, false, s, nullptr,
                                    long_rows(h, 0, h->nb)));
  }
  MSP_TRY(launch_scatter_blocks(h->nb, h->b, h->perm0.p, h->xperm.p, d_y, s));
  MSP_CUDA_TRY(cudaStreamSynchronize(s));
  return MSP_OK;
}

int msp_stats_enable(int mode) {
  if (mode < 0 || mode > 3) return MSP_ERR_ARG;
  std::lock_guard<std::mutex> lk(g_stats_mu);
  g_stats_mode = mode;
  return MSP_OK;
}

int msp_stats_reset(void) {
  std::lock_guard<std::mutex> lk(g_stats_mu);
  resolve_pending();
  // names stay (captured graphs keep their site indices); the counters restart
  for (auto& st : g_sites) st = StatSite{st.name};
  g_launches = 0;
  return MSP_OK;
}

long long msp_stats_launches(void) {
  std::lock_guard<std::mutex> lk(g_stats_mu);
  return g_launches;
}

int msp_stats_count(void) {
  std::lock_guard<std::mutex> lk(g_stats_mu);
  resolve_pending();
  return (int)g_sites.size();
}

int msp_stats_get(int index, char* name, int name_len, long long* launches, double* total_ms,
                  double* bytes, double* flops) {
  std::lock_guard<std::mutex> lk(g_stats_mu);
  resolve_pending();
  if (index < 0 || index >= (int)g_sites.size()) return MSP_ERR_ARG;
  const StatSite& st = g_sites[index];
  if (name && name_len > 0) {
    std::strncpy(name, st.name.c_str(), name_len - 1);
    name[name_len - 1] = 0;
  }
  if (launches) *launches = st.launches;
  if (total_ms) *total_ms = st.ms;
  if (bytes) *bytes = st.bytes;
  if (flops) *flops = st.flops;
  return MSP_OK;
}

int msp_set_instances(msp_handle h, int32_t count, const int32_t* h_row_offsets) {
  if (!h || count < 1 || !h_row_offsets || h_row_offsets[0] != 0 || h_row_offsets[count] != h->nb)
    return MSP_ERR_ARG;
  for (int i = 0; i < count; ++i)
    if (h_row_offsets[i + 1] <= h_row_offsets[i]) return MSP_ERR_ARG;
  DevBytesScope bytes_scope(h);
  cudaStream_t s = nullptr;
  try {
    const int nb = h->nb, b = h->b;
    DevBuf<int> off;
    MSP_TRY(off.alloc((size_t)count + 1));
    MSP_CUDA_TRY(cudaMemcpy(off.p, h_row_offsets, sizeof(int) * ((size_t)count + 1),
                            cudaMemcpyHostToDevice));
    MSP_TRY(reset_flags(h, s));
    MSP_TRY(launch_check_block_diagonal(nb, h->rp.p, h->ci.p, h->perm0.p, count, off.p,
                                        h->flags.p, s));
    if (sync_flags(h, s) != MSP_OK) return h->h_flags->code;
    // (colour, instance) segments of the colour-ordered rows, cut into chunks
    std::vector<int> perm(nb);
    MSP_CUDA_TRY(cudaMemcpy(perm.data(), h->perm0.p, sizeof(int) * (size_t)nb,
                            cudaMemcpyDeviceToHost));
    std::vector<int> cstart, cend, cinst;
    const std::vector<int> offs(h_row_offsets, h_row_offsets + count + 1);
    auto inst_of = [&](int r) {
      return (int)(std::upper_bound(offs.begin(), offs.end(), r) - offs.begin()) - 1;
    };
    for (size_t c = 0; c + 1 < h->cptr0.size(); ++c) {
      int p = h->cptr0[c];
      const int p1 = h->cptr0[c + 1];
      while (p < p1) {
        const int inst = inst_of(perm[p]);
        int q = p + 1;
        while (q < p1 && inst_of(perm[q]) == inst) ++q;
        if (q < p1 && inst_of(perm[q]) < inst) return MSP_ERR_PATTERN;  // not instance-major
        for (long long e = (long long)p * b; e < (long long)q * b; e += kSegChunk) {
          cstart.push_back((int)e);
          cend.push_back((int)std::min<long long>(e + kSegChunk, (long long)q * b));
          cinst.push_back(inst);
        }
        p = q;
      }
    }
    const int nchunks = (int)cstart.size();
    std::vector<int> iptr(count + 1, 0), ichunks(nchunks);
    for (int c = 0; c < nchunks; ++c) ++iptr[cinst[c] + 1];
    for (int i = 0; i < count; ++i) iptr[i + 1] += iptr[i];
    {
      std::vector<int> fill(iptr.begin(), iptr.end() - 1);
      for (int c = 0; c < nchunks; ++c) ichunks[fill[cinst[c]]++] = c;
    }
    MSP_TRY(h->seg_start.alloc(nchunks));
    MSP_TRY(h->seg_end.alloc(nchunks));
    MSP_TRY(h->seg_inst.alloc(nchunks));
    MSP_TRY(h->seg_iptr.alloc((size_t)count + 1));
    MSP_TRY(h->seg_ichunks.alloc(nchunks));
    MSP_CUDA_TRY(cudaMemcpy(h->seg_start.p, cstart.data(), sizeof(int) * nchunks, cudaMemcpyHostToDevice));
    MSP_CUDA_TRY(cudaMemcpy(h->seg_end.p, cend.data(), sizeof(int) * nchunks, cudaMemcpyHostToDevice));
    MSP_CUDA_TRY(cudaMemcpy(h->seg_inst.p, cinst.data(), sizeof(int) * nchunks, cudaMemcpyHostToDevice));
    MSP_CUDA_TRY(cudaMemcpy(h->seg_iptr.p, iptr.data(), sizeof(int) * (count + 1), cudaMemcpyHostToDevice));
    MSP_CUDA_TRY(cudaMemcpy(h->seg_ichunks.p, ichunks.data(), sizeof(int) * nchunks, cudaMemcpyHostToDevice));
    const size_t per = (size_t)count * kKrylovMaxK;
    MSP_TRY(h->bpart.alloc((size_t)nchunks * 2 * kKrylovMaxK));
    {
      const int m2 = h->cfg.restart + 2;
      MSP_TRY(h->gs_bT.alloc((size_t)count * m2 * m2));
      MSP_TRY(h->gs_bD.alloc((size_t)count * 2 * kKrylovMaxK));
      MSP_TRY(h->gs_bout.alloc((size_t)count * kBatchOut));
      MSP_TRY(h->gs_bfin.alloc(count));
      if (h->h_bout) cudaFreeHost(h->h_bout);
      h->h_bout = nullptr;
      MSP_CUDA_TRY(cudaMallocHost(&h->h_bout, (size_t)count * kBatchOut * sizeof(double)));
    }
    MSP_TRY(h->bh.alloc(per));
    MSP_TRY(h->by.alloc(per));
    MSP_TRY(h->bn.alloc(per));
    MSP_TRY(h->bydev.alloc(per));
    MSP_TRY(h->bact.alloc(count));
    MSP_TRY(h->bcount.alloc(count));
    MSP_TRY(h->bzero.alloc(count));
    if (h->h_bpin) cudaFreeHost(h->h_bpin);
    h->h_bpin = nullptr;
    MSP_CUDA_TRY(cudaMallocHost(&h->h_bpin, 3 * per * sizeof(double)));
    std::vector<int> rinst(nb);
    for (int p = 0; p < nb; ++p) rinst[p] = inst_of(perm[p]);
    MSP_TRY(h->row_inst.alloc(nb));
    MSP_TRY(h->rmask0.alloc(nb));
    MSP_CUDA_TRY(cudaMemcpy(h->row_inst.p, rinst.data(), sizeof(int) * (size_t)nb,
                            cudaMemcpyHostToDevice));
    MSP_CUDA_TRY(cudaMemset(h->rmask0.p, 1, nb));
    drop_graph(h);  // the preconditioner graph is captured again with the row masks
    h->seg_n = nchunks;
    h->batch = count;
    MSP_TRY(batch_level_masks(h, s));
    h->batch_offsets = offs;
    return MSP_OK;
  } catch (...) {
    return MSP_ERR_NOMEM;
  }
}

int msp_solve_batch(msp_handle h, const double* d_b, double* d_x, double rel_tol,
                    msp_solve_info* h_infos, void* stream) {
  if (!h || !d_b || !d_x || !(rel_tol > 0.0) || h->batch < 1) return MSP_ERR_ARG;
  if (h->cfg.restart >= kKrylovMaxK) return MSP_ERR_ARG;
  DevBytesScope bytes_scope(h);
  cudaStream_t s = (cudaStream_t)stream;
  const int B = h->batch;
  try {
    const size_t n = (size_t)h->nb * h->b;
    MSP_CUDA_TRY(cudaMemsetAsync(h->ifl.p, 0, sizeof(int), s));
    MSP_TRY(launch_check_finite(n, d_b, h->ifl.p, s));
    int bad = 0;
    MSP_CUDA_TRY(cudaMemcpyAsync(&bad, h->ifl.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    MSP_CUDA_TRY(cudaStreamSynchronize(s));
    if (bad) return MSP_ERR_NONFINITE;
    // adaptive setup (Section 3.2) on the largest iteration count of the previous batch
    auto ts = Clock::now();
    int setup = 0;
    if (!h->first_solve && (h->prev_it > h->cfg.mu || !h->setup_valid)) {
      MSP_TRY(value_setup(h, s));
      setup = 1;
    } else if (h->first_solve) {
      setup = 1;
    }
    const double t_setup = ms_since(ts);
    h->first_solve = false;
    auto t0 = Clock::now();
    MSP_TRY(launch_gather_blocks(h->nb, h->b, h->perm0.p, d_b, h->bperm.p, s));
    std::vector<int> its, status;
    std::vector<double> rr, est;
    MSP_TRY(fgmres_batched(h, rel_tol, its, rr, est, status, s));
    MSP_TRY(launch_scatter_blocks(h->nb, h->b, h->perm0.p, h->xperm.p, d_x, s));
    MSP_CUDA_TRY(cudaStreamSynchronize(s));
    const double t_solve = ms_since(t0);
    int worst = MSP_OK, maxit = 0;
    for (int i = 0; i < B; ++i) {
      maxit = std::max(maxit, its[i]);
      if (status[i] < 0 && worst >= 0) worst = status[i];
      else if (status[i] == MSP_NOT_CONVERGED && worst == MSP_OK) worst = MSP_NOT_CONVERGED;
      if (h_infos) {
        msp_solve_info& f = h_infos[i];
        std::memset(&f, 0, sizeof(f));
        f.status = status[i];
        f.iterations = its[i];
        f.setup_performed = setup;
        f.setup_calls = h->setup_calls;
        f.levels = (int)h->levels.size();
        f.colours_l0 = h->g0;
        f.rel_residual = rr[i];
        f.rel_residual_est = est[i];
        f.t_setup_ms = t_setup;
        f.t_solve_ms = t_solve;
      }
    }
    h->prev_it = maxit;
    return worst;
  } catch (...) {
    return MSP_ERR_NOMEM;
  }
}

int msp_device_bytes(msp_handle h, int64_t* bytes) {
  if (!h || !bytes) return MSP_ERR_ARG;
  *bytes = h->dev_bytes;
  return MSP_OK;
}

int msp_num_levels(msp_handle h) { return h ? (int)h->levels.size() : MSP_ERR_ARG; }

int msp_level_info(msp_handle h, int level, int32_t* n, int32_t* nnz, int32_t* ncolours) {
  if (!h || level < 0 || level >= (int)h->levels.size()) return MSP_ERR_ARG;
  const Level& L = h->levels[level];
  if (n) *n = L.A.n;
  if (nnz) *nnz = L.A.nnz;
  if (ncolours) *ncolours = L.cptr.empty() ? 0 : (int)L.cptr.size() - 1;
  return MSP_OK;
}

int msp_level_tiles(msp_handle h, int level, int32_t* ell_slots, int32_t* sweep_lanes,
                    int32_t* restrict_lanes) {
  if (!h || level < 0 || level >= (int)h->levels.size()) return MSP_ERR_ARG;
  const Level& L = h->levels[level];
  if (ell_slots) *ell_slots = L.ell_k;
  const int def = L.ell_k > 0 ? ell_default_tpr(L.ell_k) : 0;
  if (sweep_lanes) *sweep_lanes = L.gs_tpr ? L.gs_tpr : def;
  if (restrict_lanes) *restrict_lanes = L.rr_tpr ? L.rr_tpr : def;
  return MSP_OK;
}

int msp_level_get(msp_handle h, int level, int32_t* h_perm, int32_t* h_cptr, int32_t* h_agg,
                  int32_t* h_row_ptr, int32_t* h_col_idx, double* h_values) {
  if (!h || level < 0 || level >= (int)h->levels.size()) return MSP_ERR_ARG;
  const Level& L = h->levels[level];
  const int n = L.A.n;
  if (h_perm) MSP_CUDA_TRY(cudaMemcpy(h_perm, L.perm.p, n * sizeof(int), cudaMemcpyDeviceToHost));
  if (h_cptr && !L.cptr.empty()) std::copy(L.cptr.begin(), L.cptr.end(), h_cptr);
  if (h_agg) {
    if (L.agg.p)
      MSP_CUDA_TRY(cudaMemcpy(h_agg, L.agg.p, n * sizeof(int), cudaMemcpyDeviceToHost));
    else
      std::fill(h_agg, h_agg + n, -1);
  }
  if (h_row_ptr)
    MSP_CUDA_TRY(cudaMemcpy(h_row_ptr, L.A.rp.p, (n + 1) * sizeof(int), cudaMemcpyDeviceToHost));
  if (h_col_idx)
    MSP_CUDA_TRY(cudaMemcpy(h_col_idx, L.A.ci.p, L.A.nnz * sizeof(int), cudaMemcpyDeviceToHost));
  if (h_values)
    MSP_CUDA_TRY(cudaMemcpy(h_values, L.A.v.p, L.A.nnz * sizeof(double), cudaMemcpyDeviceToHost));
  return MSP_OK;
}

int msp_colour0(msp_handle h, int32_t* h_colour) {
  if (!h || !h_colour) return MSP_ERR_ARG;
  MSP_CUDA_TRY(cudaMemcpy(h_colour, h->colour0.p, h->nb * sizeof(int), cudaMemcpyDeviceToHost));
  return h->g0;
}

}  // extern "C"
