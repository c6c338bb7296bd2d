// Elimination of the well unknowns by the Schur complement of A_WW in the Jacobian with
// implicit wells (Eq. Jacobian-system, Section 2.2.4: reservoir rows R first, the well
// rows W last):
//   A_S = A_RR - A_RW A_WW^{-1} A_WR,   g_S = g_R - A_RW A_WW^{-1} g_W,
//   x_R = A_S^{-1} g_S,                 x_W = A_WW^{-1} (g_W - A_WR x_R).
// Layout accepted: every reservoir row couples to at most one well (one A_RW block), and
// well rows couple to no other well, so A_WW is block diagonal and each A_WW^{-1} is the
// inverse of one b x b block.  Row c of A_S holds the columns of row c of A_RR and, when c
// is perforated by well w, the columns of row w of A_WR; within the block of (c, j):
//   t = A_cw A_ww^{-1},  A_S[c, j] = A_RR[c, j] - t A_wj  (each b x b product summed over
//   k = 0..b-1 in order, every product and sum rounded separately).
// This translation unit is compiled with -fmad=false so that those sums are reproducible
// bit for bit by any implementation that forms them in the same order.
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "setup_kernels.h"

struct msp_wells_s {
  int nb = 0, b = 0, nw = 0, nr = 0;
  long long nnzb = 0;  // blocks of the full matrix
  long long nnzs = 0;  // blocks of A_S
  int nperf = 0;       // perforated reservoir rows
  int wnnz = 0;        // blocks of the well rows
  msp::SortScratch* ss = nullptr;
  msp::DevBuf<msp::DevFlags> flags;
  msp::DevFlags* h_flags = nullptr;
  msp::DevBuf<int> dpos;          // diagonal block of every row of the full matrix
  msp::DevBuf<int> well_of;       // reservoir row -> well, or -1
  msp::DevBuf<int> cw_pos;        // reservoir row -> its A_RW block in the full matrix
  msp::DevBuf<int> perf_of;       // reservoir row -> slot in acw, or -1
  msp::DevBuf<int> perf_row;      // slot -> reservoir row
  msp::DevBuf<int> srp, sci;      // pattern of A_S (nr + 1, nnzs)
  msp::DevBuf<int> s_orig, s_wc;  // per A_S block: its A_RR block and A_WR block, or -1
  msp::DevBuf<int> wrp, wci;      // the well rows (rows nr.. of the full matrix), rebased
  msp::DevBuf<double> sv;         // values of A_S
  msp::DevBuf<double> winv;       // nw blocks A_ww^{-1}
  msp::DevBuf<double> acw;        // nperf blocks A_cw
  msp::DevBuf<double> wv;         // values of the well rows
  msp::DevBuf<double> omega;      // scratch of the block inverse (first rows)
  // wells with one unknown each (msp_wells_setup_scalar): the identity-padded full matrix
  // the elimination above works on, rebuilt from the compact arrays at every value update
  bool scalar = false;
  msp::DevBuf<int> c_rp;          // the cell rows' row pointers as given (nr + 1)
  msp::DevBuf<int> p_rp;          // padded row pointers (nb + 1)
  msp::DevBuf<int> c_perf;        // cell row -> its perforation index, or -1
  msp::DevBuf<int> w_ptr;         // perforations of every well (nw + 1)
  msp::DevBuf<double> p_vals;     // padded values (nnzb * b * b)
};

namespace msp {
namespace {

constexpr int kThreads = 256;

inline int launch_status() { return launch_check(__FILE__, __LINE__); }

__device__ void raise_flag_w(DevFlags* f, int code, int index) {
  if (atomicCAS(&f->code, MSP_OK, code) == MSP_OK) f->index = index;
}

// Per row: the layout checks, well_of / cw_pos of the reservoir rows, the slots of the
// perforated rows and the candidate count of every row of A_S (own columns < nr plus, for
// a perforated row, the columns < nr of its well's row).
__global__ void wells_scan_kernel(int nb, int nr, const int* __restrict__ rp,
                                  const int* __restrict__ ci, int* __restrict__ well_of,
                                  int* __restrict__ cw_pos, int* __restrict__ perf_of,
                                  int* __restrict__ perf_row, int* __restrict__ cnt,
                                  DevFlags* flags) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += gridDim.x * blockDim.x) {
    const int p0 = rp[i], p1 = rp[i + 1];
    if (i >= nr) {
      for (int p = p0; p < p1; ++p)
        if (ci[p] >= nr && ci[p] != i) raise_flag_w(flags, MSP_ERR_ARG, i);  // well-well
      continue;
    }
    int w = -1, pos = -1, own = 0;
    for (int p = p0; p < p1; ++p) {
      const int j = ci[p];
      if (j < nr) {
        ++own;
      } else if (w >= 0) {
        raise_flag_w(flags, MSP_ERR_ARG, i);  // a second well on one cell
      } else {
        w = j - nr;
        pos = p;
      }
    }
    int extra = 0;
    if (w >= 0) {
      for (int p = rp[nr + w]; p < rp[nr + w + 1]; ++p) extra += ci[p] < nr;
      const int k = atomicAdd(&flags->count, 1);  // slot order is irrelevant to the values
      perf_of[i] = k;
      perf_row[k] = i;
    } else {
      perf_of[i] = -1;
    }
    well_of[i] = w;
    cw_pos[i] = pos;
    cnt[i] = own + extra;
  }
}

// Candidate keys (c << 32 | j) of row c of A_S, at off[c] ...
__global__ void wells_keys_kernel(int nr, const int* __restrict__ rp, const int* __restrict__ ci,
                                  const int* __restrict__ well_of, const int* __restrict__ off,
                                  unsigned long long* __restrict__ keys) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nr; c += gridDim.x * blockDim.x) {
    size_t q = (size_t)off[c];
    const unsigned long long hi = (unsigned long long)c << 32;
    for (int p = rp[c]; p < rp[c + 1]; ++p)
      if (ci[p] < nr) keys[q++] = hi | (unsigned)ci[p];
    const int w = well_of[c];
    if (w >= 0)
      for (int p = rp[nr + w]; p < rp[nr + w + 1]; ++p)
        if (ci[p] < nr) keys[q++] = hi | (unsigned)ci[p];
  }
}

// Per block (c, j) of A_S: the A_RR block (c, j) and the A_WR block (w, j) of the
// perforating well, or -1, by a merge of the sorted rows.
__global__ void wells_sources_kernel(int nr, const int* __restrict__ srp,
                                     const int* __restrict__ sci, const int* __restrict__ rp,
                                     const int* __restrict__ ci, const int* __restrict__ well_of,
                                     int* __restrict__ s_orig, int* __restrict__ s_wc) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nr; c += gridDim.x * blockDim.x) {
    int pa = rp[c];
    const int pa1 = rp[c + 1];
    const int w = well_of[c];
    int pw = w >= 0 ? rp[nr + w] : 0;
    const int pw1 = w >= 0 ? rp[nr + w + 1] : 0;
    for (int q = srp[c]; q < srp[c + 1]; ++q) {
      const int j = sci[q];
      while (pa < pa1 && ci[pa] < j) ++pa;
      while (pw < pw1 && ci[pw] < j) ++pw;
      s_orig[q] = (pa < pa1 && ci[pa] == j) ? pa : -1;
      s_wc[q] = (pw < pw1 && ci[pw] == j) ? pw : -1;
    }
  }
}

// out[q] = A_RR block of q (zero where A_RR has none), element-wise
__global__ void wells_gather_kernel(size_t nnzs, int bb, const int* __restrict__ s_orig,
                                    const double* __restrict__ v, double* __restrict__ out) {
  const size_t total = nnzs * bb;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const size_t q = t / bb;
    const int src = s_orig[q];
    out[t] = src >= 0 ? v[(size_t)src * bb + t % bb] : 0.0;
  }
}

// acw[k] = the A_RW block of the perforated row perf_row[k]
__global__ void wells_acw_kernel(int nperf, int bb, const int* __restrict__ perf_row,
                                 const int* __restrict__ cw_pos, const double* __restrict__ v,
                                 double* __restrict__ acw) {
  const size_t total = (size_t)nperf * bb;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(t / bb);
    acw[t] = v[(size_t)cw_pos[perf_row[k]] * bb + t % bb];
  }
}

// A_S[c, j] -= (A_cw A_ww^{-1}) A_wj on the blocks with an A_WR source: one warp per
// perforated row, lanes over its blocks.
template <int B>
__global__ void wells_correct_kernel(int nperf, const int* __restrict__ perf_row,
                                     const int* __restrict__ well_of, const int* __restrict__ srp,
                                     const int* __restrict__ s_wc, const double* __restrict__ acw,
                                     const double* __restrict__ winv,
                                     const double* __restrict__ v, double* __restrict__ sv) {
  constexpr int BB = B * B;
  const int lane = threadIdx.x % kWarp;
  const int warps = gridDim.x * (blockDim.x / kWarp);
  for (int k = blockIdx.x * (blockDim.x / kWarp) + threadIdx.x / kWarp; k < nperf; k += warps) {
    const int c = perf_row[k];
    const double* a = acw + (size_t)k * BB;
    const double* wi = winv + (size_t)well_of[c] * BB;
    double t[BB];
#pragma unroll
    for (int r = 0; r < B; ++r)
#pragma unroll
      for (int cc = 0; cc < B; ++cc) {
        double acc = 0.0;
#pragma unroll
        for (int kk = 0; kk < B; ++kk) acc = __dadd_rn(acc, __dmul_rn(a[r * B + kk], wi[kk * B + cc]));
        t[r * B + cc] = acc;
      }
    for (int q = srp[c] + lane; q < srp[c + 1]; q += kWarp) {
      const int src = s_wc[q];
      if (src < 0) continue;
      const double* awc = v + (size_t)src * BB;
      double* out = sv + (size_t)q * BB;
#pragma unroll
      for (int r = 0; r < B; ++r)
#pragma unroll
        for (int cc = 0; cc < B; ++cc) {
          double acc = 0.0;
#pragma unroll
          for (int kk = 0; kk < B; ++kk)
            acc = __dadd_rn(acc, __dmul_rn(t[r * B + kk], awc[kk * B + cc]));
          out[r * B + cc] = __dsub_rn(out[r * B + cc], acc);
        }
    }
  }
}

// gs = g_R - A_RW A_WW^{-1} g_W, one thread per reservoir unknown (c, r)
template <int B>
__global__ void wells_reduce_rhs_kernel(int nr, const int* __restrict__ well_of,
                                        const int* __restrict__ perf_of,
                                        const double* __restrict__ acw,
                                        const double* __restrict__ winv,
                                        const double* __restrict__ g, double* __restrict__ gs) {
  constexpr int BB = B * B;
  const size_t total = (size_t)nr * B;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(t / B), r = (int)(t % B);
    const int w = well_of[c];
    if (w < 0) {
      gs[t] = g[t];
      continue;
    }
    const double* wi = winv + (size_t)w * BB;
    const double* gw = g + (size_t)(nr + w) * B;
    double y[B];
#pragma unroll
    for (int i = 0; i < B; ++i) {
      double acc = 0.0;
#pragma unroll
      for (int k = 0; k < B; ++k) acc = __dadd_rn(acc, __dmul_rn(wi[i * B + k], gw[k]));
      y[i] = acc;
    }
    const double* a = acw + (size_t)perf_of[c] * BB + r * B;
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < B; ++k) acc = __dadd_rn(acc, __dmul_rn(a[k], y[k]));
    gs[t] = __dsub_rn(g[t], acc);
  }
}

// x_W = A_WW^{-1} (g_W - A_WR x_R), one thread per well, blocks in row order
template <int B>
__global__ void wells_recover_kernel(int nw, int nr, const int* __restrict__ wrp,
                                     const int* __restrict__ wci, const double* __restrict__ wv,
                                     const double* __restrict__ winv,
                                     const double* __restrict__ g, const double* __restrict__ xs,
                                     double* __restrict__ x) {
  constexpr int BB = B * B;
  for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < nw; w += gridDim.x * blockDim.x) {
    const int row = nr + w;
    double r[B];
#pragma unroll
    for (int i = 0; i < B; ++i) r[i] = g[(size_t)row * B + i];
    for (int p = wrp[w]; p < wrp[w + 1]; ++p) {
      const int c = wci[p];
      if (c == row) continue;
      const double* a = wv + (size_t)p * BB;
      const double* xc = xs + (size_t)c * B;
#pragma unroll
      for (int i = 0; i < B; ++i) {
        double acc = 0.0;
#pragma unroll
        for (int k = 0; k < B; ++k) acc = __dadd_rn(acc, __dmul_rn(a[i * B + k], xc[k]));
        r[i] = __dsub_rn(r[i], acc);
      }
    }
    const double* wi = winv + (size_t)w * BB;
#pragma unroll
    for (int i = 0; i < B; ++i) {
      double acc = 0.0;
#pragma unroll
      for (int k = 0; k < B; ++k) acc = __dadd_rn(acc, __dmul_rn(wi[i * B + k], r[k]));
      x[(size_t)row * B + i] = acc;
    }
  }
}

__global__ void wells_rebase_kernel(int n, const int* __restrict__ in, int base,
                                    int* __restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    out[i] = in[i] - base;
}

// ---- wells with one unknown each: the padded layout -------------------------------
// A well of Eq. Jacobian-system has one unknown (its bottom-hole pressure) and one
// equation.  Padded to a b x b block row with identity rows/columns 1..b-1 (zero
// right-hand side there), A_RW becomes column 0 of a block, A_WR row 0 and A_WW the (0, 0)
// entry of an otherwise identity block; the padded unknowns then decouple exactly, and
// eliminating the padded blocks gives the Schur complement of the scalar A_WW.

// per perforation k of well w: cell row -> (well, perforation); rejects cells out of
// range, a cell perforated twice, and cells not ascending within a well
__global__ void pad_map_kernel(int nw, int nr, const int* __restrict__ wptr,
                               const int* __restrict__ cells, int* __restrict__ perf_of_cell,
                               DevFlags* flags) {
  for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < nw; w += gridDim.x * blockDim.x) {
    for (int k = wptr[w]; k < wptr[w + 1]; ++k) {
      const int c = cells[k];
      if (c < 0 || c >= nr || (k > wptr[w] && c <= cells[k - 1])) {
        raise_flag_w(flags, MSP_ERR_ARG, w);
        break;
      }
      if (atomicCAS(perf_of_cell + c, -1, k) != -1) raise_flag_w(flags, MSP_ERR_ARG, w);
    }
  }
}

// blocks of every padded row: a cell row keeps its blocks plus one for its well, a well
// row has one block per perforation plus its diagonal
__global__ void pad_count_kernel(int nr, int nw, const int* __restrict__ rp,
                                 const int* __restrict__ perf_of_cell,
                                 const int* __restrict__ wptr, int* __restrict__ cnt) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nr + nw; i += gridDim.x * blockDim.x)
    cnt[i] = i < nr ? rp[i + 1] - rp[i] + (perf_of_cell[i] >= 0)
                    : wptr[i - nr + 1] - wptr[i - nr] + 1;
}

// padded columns (pattern only)
__global__ void pad_pattern_kernel(int nr, int nw, const int* __restrict__ rp,
                                   const int* __restrict__ ci, const int* __restrict__ perf_of_cell,
                                   const int* __restrict__ wptr, const int* __restrict__ cells,
                                   const int* __restrict__ prp, int* __restrict__ pci) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nr + nw; i += gridDim.x * blockDim.x) {
    int q = prp[i];
    if (i < nr) {
      for (int p = rp[i]; p < rp[i + 1]; ++p) pci[q++] = ci[p];
      const int k = perf_of_cell[i];
      if (k >= 0) {  // the well's column comes after every cell column
        int w = 0;
        while (wptr[w + 1] <= k) ++w;
        pci[q] = nr + w;
      }
    } else {
      const int w = i - nr;
      for (int k = wptr[w]; k < wptr[w + 1]; ++k) pci[q++] = cells[k];
      pci[q] = i;
    }
  }
}

// padded values, one thread per padded block
template <int B>
__global__ void pad_values_kernel(int nr, int nw, const int* __restrict__ rp,
                                  const int* __restrict__ perf_of_cell,
                                  const int* __restrict__ wptr, const int* __restrict__ prp,
                                  const double* __restrict__ v, const double* __restrict__ arw,
                                  const double* __restrict__ awr, const double* __restrict__ aww,
                                  double* __restrict__ pv) {
  constexpr int BB = B * B;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nr + nw; i += gridDim.x * blockDim.x) {
    double* out = pv + (size_t)prp[i] * BB;
    if (i < nr) {
      const int n = rp[i + 1] - rp[i];
      const double* in = v + (size_t)rp[i] * BB;
      for (int e = 0; e < n * BB; ++e) out[e] = in[e];
      const int k = perf_of_cell[i];
      if (k >= 0) {  // A_RW: column 0
        double* blk = out + (size_t)n * BB;
        for (int e = 0; e < BB; ++e) blk[e] = 0.0;
        for (int r = 0; r < B; ++r) blk[r * B] = arw[(size_t)k * B + r];
      }
    } else {
      const int w = i - nr;
      const int k0 = wptr[w], k1 = wptr[w + 1];
      for (int k = k0; k < k1; ++k) {  // A_WR: row 0
        double* blk = out + (size_t)(k - k0) * BB;
        for (int e = 0; e < BB; ++e) blk[e] = 0.0;
        for (int c = 0; c < B; ++c) blk[c] = awr[(size_t)k * B + c];
      }
      double* d = out + (size_t)(k1 - k0) * BB;  // A_WW and the identity padding
      for (int e = 0; e < BB; ++e) d[e] = (e % (B + 1) == 0) ? 1.0 : 0.0;
      d[0] = aww[w];
    }
  }
}

// g = [g_R; g_W padded with zeros]
__global__ void pad_rhs_kernel(int nr, int nw, int b, const double* __restrict__ gr,
                               const double* __restrict__ gw, double* __restrict__ g) {
  const size_t nrb = (size_t)nr * b, total = nrb + (size_t)nw * b;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    if (e < nrb) {
      g[e] = gr[e];
    } else {
      const size_t q = e - nrb;
      g[e] = (q % b == 0) ? gw[q / b] : 0.0;
    }
  }
}

// x_R = x[0 .. nr*b), x_W[w] = x[(nr + w) * b]
__global__ void unpad_kernel(int nr, int nw, int b, const double* __restrict__ x,
                             double* __restrict__ xr, double* __restrict__ xw) {
  const size_t nrb = (size_t)nr * b;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < nrb + nw;
       e += (size_t)gridDim.x * blockDim.x) {
    if (e < nrb) {
      if (xr) xr[e] = x[e];
    } else if (xw) {
      xw[e - nrb] = x[nrb + (e - nrb) * b];
    }
  }
}

#define MSP_WB_SWITCH(b, ...)                              \
  switch (b) {                                             \
    case 1: { constexpr int B_ = 1; __VA_ARGS__; } break;  \
    case 2: { constexpr int B_ = 2; __VA_ARGS__; } break;  \
    case 3: { constexpr int B_ = 3; __VA_ARGS__; } break;  \
    case 4: { constexpr int B_ = 4; __VA_ARGS__; } break;  \
    case 5: { constexpr int B_ = 5; __VA_ARGS__; } break;  \
    case 6: { constexpr int B_ = 6; __VA_ARGS__; } break;  \
    case 7: { constexpr int B_ = 7; __VA_ARGS__; } break;  \
    case 8: { constexpr int B_ = 8; __VA_ARGS__; } break;  \
    default: return MSP_ERR_ARG;                           \
  }

int sync_wflags(msp_wells_s* W, cudaStream_t s) {
  MSP_CUDA_TRY(cudaMemcpyAsync(W->h_flags, W->flags.p, sizeof(DevFlags), cudaMemcpyDeviceToHost, s));
  MSP_CUDA_TRY(cudaStreamSynchronize(s));
  return MSP_OK;
}

// Values of A_S, A_WW^{-1}, the A_RW blocks and the well rows from the full matrix's
// values v (device, same pattern as at setup).
int wells_values(msp_wells_s* W, const double* v, cudaStream_t s) {
  const int b = W->b, bb = b * b;
  MSP_CUDA_TRY(cudaMemsetAsync(W->flags.p, 0, sizeof(DevFlags), s));
  MSP_TRY(launch_check_finite_vals((size_t)W->nnzb * bb, v, W->flags.p, s));
  MSP_TRY(launch_diag_inverse(b, W->nw, W->dpos.p + W->nr, v, W->winv.p, W->omega.p,
                              W->flags.p, s));
  MSP_TRY(sync_wflags(W, s));
  if (W->h_flags->code != MSP_OK) return W->h_flags->code;
  const size_t total = (size_t)W->nnzs * bb;
  wells_gather_kernel<<<grid_for(total, kThreads), kThreads, 0, s>>>((size_t)W->nnzs, bb,
                                                                     W->s_orig.p, v, W->sv.p);
  MSP_TRY(launch_status());
  if (W->nperf > 0) {
    wells_acw_kernel<<<grid_for((size_t)W->nperf * bb, kThreads), kThreads, 0, s>>>(
        W->nperf, bb, W->perf_row.p, W->cw_pos.p, v, W->acw.p);
    MSP_TRY(launch_status());
    const unsigned grid = std::max(1u, std::min(grid_for((size_t)W->nperf * kWarp, kThreads),
                                                (unsigned)((W->nperf + 7) / 8)));
    MSP_WB_SWITCH(b, wells_correct_kernel<B_><<<grid, kThreads, 0, s>>>(
                         W->nperf, W->perf_row.p, W->well_of.p, W->srp.p, W->s_wc.p, W->acw.p,
                         W->winv.p, v, W->sv.p));
    MSP_TRY(launch_status());
  }
  // the well rows are the last rows, so their blocks are contiguous in the full matrix
  MSP_CUDA_TRY(cudaMemcpyAsync(W->wv.p, v + (size_t)(W->nnzb - W->wnnz) * bb,
                               (size_t)W->wnnz * bb * sizeof(double), cudaMemcpyDeviceToDevice,
                               s));
  return MSP_OK;
}

int wells_build(msp_wells_s* W, const int* rp, const int* ci, const double* v, cudaStream_t s) {
  const int nb = W->nb, nr = W->nr;
  if (!W->flags.p) MSP_TRY(W->flags.alloc(1));
  if (!W->h_flags) MSP_CUDA_TRY(cudaMallocHost(&W->h_flags, sizeof(DevFlags)));
  MSP_CUDA_TRY(cudaMemsetAsync(W->flags.p, 0, sizeof(DevFlags), s));
  MSP_TRY(W->dpos.alloc(nb));
  // reads ci only inside [0, nnzb), so a bad row_ptr is reported, never followed
  MSP_TRY(launch_check_pattern(nb, (int)W->nnzb, rp, ci, W->dpos.p, W->flags.p, s));
  MSP_TRY(sync_wflags(W, s));
  if (W->h_flags->code != MSP_OK) return W->h_flags->code;
  int rp_nb = 0, rp_nr = 0;
  MSP_CUDA_TRY(cudaMemcpyAsync(&rp_nb, rp + nb, sizeof(int), cudaMemcpyDeviceToHost, s));
  MSP_CUDA_TRY(cudaMemcpyAsync(&rp_nr, rp + nr, sizeof(int), cudaMemcpyDeviceToHost, s));
  MSP_CUDA_TRY(cudaStreamSynchronize(s));
  if ((long long)rp_nb != W->nnzb) return MSP_ERR_ARG;
  W->wnnz = rp_nb - rp_nr;

  MSP_TRY(W->well_of.alloc(nr));
  MSP_TRY(W->cw_pos.alloc(nr));
  MSP_TRY(W->perf_of.alloc(nr));
  MSP_TRY(W->perf_row.alloc(nr));
  DevBuf<int> cnt, off;
  MSP_TRY(cnt.alloc((size_t)nr + 1));
  MSP_TRY(off.alloc((size_t)nr + 1));
  MSP_CUDA_TRY(cudaMemsetAsync(cnt.p, 0, sizeof(int) * ((size_t)nr + 1), s));
  wells_scan_kernel<<<grid_for(nb, kThreads), kThreads, 0, s>>>(
      nb, nr, rp, ci, W->well_of.p, W->cw_pos.p, W->perf_of.p, W->perf_row.p, cnt.p, W->flags.p);
  MSP_TRY(launch_status());
  MSP_TRY(sync_wflags(W, s));
  if (W->h_flags->code != MSP_OK) return W->h_flags->code;
  W->nperf = W->h_flags->count;

  // pattern of A_S: candidate keys, sorted, unique
  MSP_TRY(exclusive_scan_int(W->ss, (size_t)nr + 1, cnt.p, off.p, s));
  int m = 0;
  MSP_CUDA_TRY(cudaMemcpyAsync(&m, off.p + nr, sizeof(int), cudaMemcpyDeviceToHost, s));
  MSP_CUDA_TRY(cudaStreamSynchronize(s));
  if (m < 0) return MSP_ERR_ARG;  // more candidate blocks than int32 indexes
  DevBuf<unsigned long long> keys, ukeys;
  MSP_TRY(keys.alloc(m > 0 ? (size_t)m : 1));
  wells_keys_kernel<<<grid_for(nr, kThreads), kThreads, 0, s>>>(nr, rp, ci, W->well_of.p, off.p,
                                                                keys.p);
  MSP_TRY(launch_status());
  int row_bits = 1;
  while (row_bits < 31 && (1 << row_bits) <= nr) ++row_bits;
  MSP_TRY(sort_pairs_u64(W->ss, (size_t)m, keys.p, nullptr, 32 + row_bits, s));
  size_t mu = 0;
  MSP_TRY(unique_sorted_keys(W->ss, (size_t)m, keys.p, &mu, ukeys, s));
  if (mu > 0x7fffffffULL) return MSP_ERR_ARG;
  W->nnzs = (long long)mu;
  MSP_TRY(W->srp.alloc((size_t)nr + 1));
  MSP_TRY(W->sci.alloc(mu));
  MSP_TRY(rowptr_from_sorted_keys(mu, nr, ukeys.p, W->srp.p, s));
  MSP_TRY(low32_of_keys(mu, ukeys.p, W->sci.p, s));
  MSP_TRY(W->s_orig.alloc(mu));
  MSP_TRY(W->s_wc.alloc(mu));
  wells_sources_kernel<<<grid_for(nr, kThreads), kThreads, 0, s>>>(
      nr, W->srp.p, W->sci.p, rp, ci, W->well_of.p, W->s_orig.p, W->s_wc.p);
  MSP_TRY(launch_status());

  // the well rows, rebased to start at 0
  MSP_TRY(W->wrp.alloc((size_t)W->nw + 1));
  MSP_TRY(W->wci.alloc(W->wnnz > 0 ? (size_t)W->wnnz : 1));
  wells_rebase_kernel<<<grid_for(W->nw + 1, kThreads), kThreads, 0, s>>>(W->nw + 1, rp + nr,
                                                                         rp_nr, W->wrp.p);
  MSP_TRY(launch_status());
  if (W->wnnz > 0)
    MSP_CUDA_TRY(cudaMemcpyAsync(W->wci.p, ci + rp_nr, sizeof(int) * (size_t)W->wnnz,
                                 cudaMemcpyDeviceToDevice, s));

  const int bb = W->b * W->b;
  MSP_TRY(W->sv.alloc(mu * bb));
  MSP_TRY(W->winv.alloc((size_t)W->nw * bb));
  MSP_TRY(W->omega.alloc((size_t)W->nw * W->b));
  MSP_TRY(W->acw.alloc(W->nperf > 0 ? (size_t)W->nperf * bb : 1));
  MSP_TRY(W->wv.alloc(W->wnnz > 0 ? (size_t)W->wnnz * bb : 1));
  MSP_TRY(wells_values(W, v, s));
  // keep the temporaries alive until the kernels that read them have run
  MSP_CUDA_TRY(cudaStreamSynchronize(s));
  return MSP_OK;
}

void destroy_wells(msp_wells_s* W) {
  if (!W) return;
  if (W->ss) sort_scratch_destroy(W->ss);
  if (W->h_flags) cudaFreeHost(W->h_flags);
  delete W;
}

}  // namespace
}  // namespace msp

using namespace msp;

extern "C" {

int msp_wells_setup(msp_wells* out, int32_t nb, int32_t b, int32_t nw, const int32_t* d_row_ptr,
                    const int32_t* d_col_idx, const double* d_values, int64_t nnzb,
                    void* stream) {
  if (!out) return MSP_ERR_ARG;
  *out = nullptr;
  if (nb <= 1 || b < 1 || b > 8 || nw < 1 || nw >= nb || nnzb < nb || nnzb > 0x7fffffffLL ||
      !d_row_ptr || !d_col_idx || !d_values)
    return MSP_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  msp_wells_s* W = nullptr;
  try {
    W = new msp_wells_s();
    W->nb = nb;
    W->b = b;
    W->nw = nw;
    W->nr = nb - nw;
    W->nnzb = nnzb;
    W->ss = sort_scratch_create();
    const int st = W->ss ? wells_build(W, d_row_ptr, d_col_idx, d_values, s) : MSP_ERR_NOMEM;
    if (st != MSP_OK) {
      cudaStreamSynchronize(s);
      destroy_wells(W);
      return st;
    }
  } catch (...) {
    destroy_wells(W);
    return MSP_ERR_NOMEM;
  }
  *out = W;
  return MSP_OK;
}

int msp_wells_reduced(msp_wells W, int32_t* nr, int64_t* nnzb, const int32_t** d_row_ptr,
                      const int32_t** d_col_idx, const double** d_values) {
  if (!W) return MSP_ERR_ARG;
  if (nr) *nr = W->nr;
  if (nnzb) *nnzb = W->nnzs;
  if (d_row_ptr) *d_row_ptr = W->srp.p;
  if (d_col_idx) *d_col_idx = W->sci.p;
  if (d_values) *d_values = W->sv.p;
  return MSP_OK;
}

int msp_wells_update_values(msp_wells W, const double* d_values, void* stream) {
  if (!W || !d_values) return MSP_ERR_ARG;
  try {
    return wells_values(W, d_values, (cudaStream_t)stream);
  } catch (...) {
    return MSP_ERR_NOMEM;
  }
}

int msp_wells_reduce_rhs(msp_wells W, const double* d_g, double* d_gs, void* stream) {
  if (!W || !d_g || !d_gs || d_g == d_gs) return MSP_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t total = (size_t)W->nr * W->b;
  MSP_WB_SWITCH(W->b, wells_reduce_rhs_kernel<B_><<<grid_for(total, kThreads), kThreads, 0, s>>>(
                          W->nr, W->well_of.p, W->perf_of.p, W->acw.p, W->winv.p, d_g, d_gs));
  return launch_status();
}

int msp_wells_recover(msp_wells W, const double* d_g, const double* d_xs, double* d_x,
                      void* stream) {
  if (!W || !d_g || !d_xs || !d_x || d_x == d_g) return MSP_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (d_x != d_xs)
    MSP_CUDA_TRY(cudaMemcpyAsync(d_x, d_xs, sizeof(double) * (size_t)W->nr * W->b,
                                 cudaMemcpyDeviceToDevice, s));
  MSP_WB_SWITCH(W->b, wells_recover_kernel<B_><<<grid_for(W->nw, 64), 64, 0, s>>>(
                          W->nw, W->nr, W->wrp.p, W->wci.p, W->wv.p, W->winv.p, d_g, d_xs, d_x));
  return launch_status();
}

int msp_wells_free(msp_wells W) {
  if (W) {
    cudaDeviceSynchronize();
    destroy_wells(W);
  }
  return MSP_OK;
}

// ---- wells with one unknown each ----------------------------------------------------
int msp_wells_setup_scalar(msp_wells* out, int32_t nr, int32_t b, int32_t nw,
                           const int32_t* d_row_ptr, const int32_t* d_col_idx,
                           const double* d_values, int64_t nnzb, const int32_t* d_well_ptr,
                           const int32_t* d_well_cells, const double* d_arw, const double* d_awr,
                           const double* d_aww, void* stream) {
  if (!out) return MSP_ERR_ARG;
  *out = nullptr;
  if (nr < 1 || b < 1 || b > 8 || nw < 1 || nnzb < nr || nnzb > 0x3fffffffLL || !d_row_ptr ||
      !d_col_idx || !d_values || !d_well_ptr || !d_aww)
    return MSP_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  msp_wells_s* W = nullptr;
  try {
    // the perforation ranges, checked on the host before anything reads them
    std::vector<int> wp(nw + 1);
    MSP_CUDA_TRY(cudaMemcpyAsync(wp.data(), d_well_ptr, sizeof(int) * (nw + 1),
                                 cudaMemcpyDeviceToHost, s));
    int rp_ends[2] = {0, 0};
    MSP_CUDA_TRY(cudaMemcpyAsync(&rp_ends[0], d_row_ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
    MSP_CUDA_TRY(cudaMemcpyAsync(&rp_ends[1], d_row_ptr + nr, sizeof(int), cudaMemcpyDeviceToHost,
                                 s));
    MSP_CUDA_TRY(cudaStreamSynchronize(s));
    if (rp_ends[0] != 0 || (int64_t)rp_ends[1] != nnzb) return MSP_ERR_PATTERN;
    if (wp[0] != 0) return MSP_ERR_ARG;
    for (int w = 0; w < nw; ++w)
      if (wp[w + 1] < wp[w]) return MSP_ERR_ARG;
    const int nperf = wp[nw];
    if (nperf > nr || (nperf > 0 && (!d_well_cells || !d_arw || !d_awr))) return MSP_ERR_ARG;
    W = new msp_wells_s();
    W->scalar = true;
    W->b = b;
    W->nw = nw;
    W->nr = nr;
    W->nb = nr + nw;
    W->nnzb = nnzb + 2LL * nperf + nw;
    W->ss = sort_scratch_create();
    int st = W->ss ? MSP_OK : MSP_ERR_NOMEM;
    auto fail = [&](int code) {
      cudaStreamSynchronize(s);
      destroy_wells(W);
      return code;
    };
    if (st != MSP_OK) return fail(st);
    // the cell matrix's own pattern first (reads its columns only inside [0, nnzb))
    st = W->flags.alloc(1);
    if (st == MSP_OK && cudaMallocHost(&W->h_flags, sizeof(DevFlags)) != cudaSuccess)
      st = MSP_ERR_NOMEM;
    if (st != MSP_OK) return fail(st);
    {
      DevBuf<int> cdpos;
      if ((st = cdpos.alloc(nr)) != MSP_OK) return fail(st);
      cudaMemsetAsync(W->flags.p, 0, sizeof(DevFlags), s);
      if ((st = launch_check_pattern(nr, (int)nnzb, d_row_ptr, d_col_idx, cdpos.p, W->flags.p, s)) !=
              MSP_OK ||
          (st = sync_wflags(W, s)) != MSP_OK)
        return fail(st);
      if (W->h_flags->code != MSP_OK) return fail(W->h_flags->code);
    }
    if ((st = W->c_rp.alloc(nr + 1)) != MSP_OK || (st = W->c_perf.alloc(nr)) != MSP_OK ||
        (st = W->w_ptr.alloc(nw + 1)) != MSP_OK || (st = W->p_rp.alloc(W->nb + 1)) != MSP_OK ||
        (st = W->p_vals.alloc((size_t)W->nnzb * b * b)) != MSP_OK)
      return fail(st);
    cudaMemcpyAsync(W->c_rp.p, d_row_ptr, sizeof(int) * (nr + 1), cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(W->w_ptr.p, d_well_ptr, sizeof(int) * (nw + 1), cudaMemcpyDeviceToDevice, s);
    if ((st = launch_fill_int(nr, -1, W->c_perf.p, s)) != MSP_OK) return fail(st);
    cudaMemsetAsync(W->flags.p, 0, sizeof(DevFlags), s);
    pad_map_kernel<<<grid_for(nw, 64), 64, 0, s>>>(nw, nr, W->w_ptr.p, d_well_cells,
                                                     W->c_perf.p, W->flags.p);
    if ((st = launch_status()) != MSP_OK || (st = sync_wflags(W, s)) != MSP_OK) return fail(st);
    if (W->h_flags->code != MSP_OK) return fail(W->h_flags->code);
    // padded pattern and values
    DevBuf<int> cnt, pci;
    if ((st = cnt.alloc(W->nb)) != MSP_OK || (st = pci.alloc((size_t)W->nnzb)) != MSP_OK)
      return fail(st);
    pad_count_kernel<<<grid_for(W->nb, kThreads), kThreads, 0, s>>>(nr, nw, W->c_rp.p,
                                                                    W->c_perf.p, W->w_ptr.p,
                                                                    cnt.p);
    if ((st = launch_status()) != MSP_OK ||
        (st = exclusive_scan_int(W->ss, (size_t)W->nb, cnt.p, W->p_rp.p, s)) != MSP_OK)
      return fail(st);
    const int total = (int)W->nnzb;
    cudaMemcpyAsync(W->p_rp.p + W->nb, &total, sizeof(int), cudaMemcpyHostToDevice, s);
    pad_pattern_kernel<<<grid_for(W->nb, kThreads), kThreads, 0, s>>>(
        nr, nw, W->c_rp.p, d_col_idx, W->c_perf.p, W->w_ptr.p, d_well_cells, W->p_rp.p, pci.p);
    if ((st = launch_status()) != MSP_OK) return fail(st);
    MSP_WB_SWITCH(b, pad_values_kernel<B_><<<grid_for(W->nb, kThreads), kThreads, 0, s>>>(
                         nr, nw, W->c_rp.p, W->c_perf.p, W->w_ptr.p, W->p_rp.p, d_values, d_arw,
                         d_awr, d_aww, W->p_vals.p));
    if ((st = launch_status()) != MSP_OK) return fail(st);
    // `total` is read by the copy above: wait before it goes out of scope
    if (cudaStreamSynchronize(s) != cudaSuccess) return fail(MSP_ERR_CUDA);
    if ((st = wells_build(W, W->p_rp.p, pci.p, W->p_vals.p, s)) != MSP_OK) return fail(st);
  } catch (...) {
    destroy_wells(W);
    return MSP_ERR_NOMEM;
  }
  *out = W;
  return MSP_OK;
}

int msp_wells_update_values_scalar(msp_wells W, const double* d_values, const double* d_arw,
                                   const double* d_awr, const double* d_aww, void* stream) {
  if (!W || !W->scalar || !d_values || !d_aww) return MSP_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  try {
    MSP_WB_SWITCH(W->b, pad_values_kernel<B_><<<grid_for(W->nb, kThreads), kThreads, 0, s>>>(
                            W->nr, W->nw, W->c_rp.p, W->c_perf.p, W->w_ptr.p, W->p_rp.p,
                            d_values, d_arw, d_awr, d_aww, W->p_vals.p));
    MSP_TRY(launch_status());
    return wells_values(W, W->p_vals.p, s);
  } catch (...) {
    return MSP_ERR_NOMEM;
  }
}

int msp_wells_pack_rhs(msp_wells W, const double* d_gr, const double* d_gw, double* d_g,
                       void* stream) {
  if (!W || !d_gr || !d_gw || !d_g) return MSP_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t total = (size_t)W->nb * W->b;
  pad_rhs_kernel<<<grid_for(total, kThreads), kThreads, 0, s>>>(W->nr, W->nw, W->b, d_gr, d_gw,
                                                                d_g);
  return launch_status();
}

int msp_wells_unpack(msp_wells W, const double* d_x, double* d_xr, double* d_xw, void* stream) {
  if (!W || !d_x || (!d_xr && !d_xw)) return MSP_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t total = (size_t)W->nr * W->b + W->nw;
  unpad_kernel<<<grid_for(total, kThreads), kThreads, 0, s>>>(W->nr, W->nw, W->b, d_x, d_xr,
                                                              d_xw);
  return launch_status();
}

}  // extern "C"
