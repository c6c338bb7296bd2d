// Setup kernels without bit-exactness requirements: pattern validation, value
// gathers, stage-N sub-blocks, BILU(0) factorisation by colour, the dense inverse of
// the coarsest AMG matrix (in-place Gauss-Jordan with partial pivoting), casts.
#include <cuda_runtime.h>

#include "common.cuh"
#include "setup_kernels.h"

namespace msp {

namespace {

constexpr int kThreads = 256;

inline int launch_status() { return launch_check(__FILE__, __LINE__); }

__device__ void raise_flag(DevFlags* f, int code, int index) {
  if (atomicCAS(&f->code, MSP_OK, code) == MSP_OK) f->index = index;
}

// Every read of ci stays inside [0, nnz): a row whose pointers leave that range or
// decrease is rejected before its columns are read (nnz = rp[nb], checked by the host).
__global__ void check_pattern_kernel(int nb, int nnz, const int* __restrict__ rp,
                                     const int* __restrict__ ci, int* __restrict__ dpos,
                                     DevFlags* flags) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += gridDim.x * blockDim.x) {
    const int p0 = rp[i], p1 = rp[i + 1];
    if (p0 < 0 || p1 < p0 || p1 > nnz) {
      dpos[i] = -2;
      raise_flag(flags, MSP_ERR_PATTERN, i);
      continue;
    }
    int d = -1;
    for (int p = p0; p < p1; ++p) {
      const int j = ci[p];
      if (j < 0 || j >= nb || (p > p0 && j <= ci[p - 1])) {
        raise_flag(flags, MSP_ERR_PATTERN, i);
        d = -2;
        break;
      }
      if (j == i) d = p;
    }
    if (d == -1) raise_flag(flags, MSP_ERR_PATTERN, i);
    dpos[i] = d;
  }
}

// instance of an original row: the last i with off[i] <= r
__device__ __forceinline__ int instance_of(int r, int B, const int* __restrict__ off) {
  int lo = 0, hi = B - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= r) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// MSP_ERR_PATTERN where a block couples two instances (rows and columns are positions of
// the permuted pattern; perm maps them to original rows)
__global__ void check_block_diagonal_kernel(int nb, const int* __restrict__ rp,
                                            const int* __restrict__ ci, const int* __restrict__ perm,
                                            int B, const int* __restrict__ off, DevFlags* flags) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += gridDim.x * blockDim.x) {
    const int inst = instance_of(perm[i], B, off);
    for (int p = rp[i]; p < rp[i + 1]; ++p)
      if (instance_of(perm[ci[p]], B, off) != inst) {
        raise_flag(flags, MSP_ERR_PATTERN, i);
        break;
      }
  }
}

__global__ void check_finite_vals_kernel(size_t n, const double* __restrict__ v, DevFlags* flags) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n;
       k += (size_t)gridDim.x * blockDim.x)
    if (!isfinite(v[k])) {
      raise_flag(flags, MSP_ERR_NONFINITE, (int)(k < 0x7fffffff ? k : 0x7fffffff));
      return;
    }
}

__global__ void gather_values_kernel(size_t nnz, int bb, const int* __restrict__ src,
                                     const double* __restrict__ in, double* __restrict__ out) {
  const size_t total = nnz * bb;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const size_t q = t / bb, k = t % bb;
    out[t] = in[(size_t)src[q] * bb + k];
  }
}

__global__ void extract_N_kernel(int b, size_t nnzb, const double* __restrict__ v,
                                 double* __restrict__ aN) {
  const int bn = b - 1;
  const size_t total = nnzb * bn * bn;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const size_t p = t / (bn * bn);
    const int rc = (int)(t % (bn * bn)), r = rc / bn, c = rc % bn;
    aN[t] = v[p * b * b + (size_t)(r + 1) * b + c + 1];
  }
}

// Stage N works with the concentration sub-blocks scaled by the inverse of their row's
// diagonal sub-block: aN[p] <- D_N,i^-1 aN[p] for the off-diagonal blocks p of row i (the
// diagonal block is left as it is and never read by the sweeps).  One thread per row.
template <int BN>
__global__ void scale_N_rows_kernel(int nb, const int* __restrict__ rp, const int* __restrict__ dpos,
                                    const double* __restrict__ dNinv, double* __restrict__ aN) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += gridDim.x * blockDim.x) {
    double D[BN * BN];
#pragma unroll
    for (int e = 0; e < BN * BN; ++e) D[e] = dNinv[(size_t)i * BN * BN + e];
    const int pd = dpos[i];
    for (int p = rp[i]; p < rp[i + 1]; ++p) {
      if (p == pd) continue;
      double* a = aN + (size_t)p * BN * BN;
      double in[BN * BN];
#pragma unroll
      for (int e = 0; e < BN * BN; ++e) in[e] = a[e];
#pragma unroll
      for (int r = 0; r < BN; ++r)
#pragma unroll
        for (int c = 0; c < BN; ++c) {
          double t = 0.0;
#pragma unroll
          for (int k = 0; k < BN; ++k) t = fma(D[r * BN + k], in[k * BN + c], t);
          a[r * BN + c] = t;
        }
    }
  }
}

__global__ void diag_pos_kernel(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                int* __restrict__ dpos) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int d = -1;
    for (int p = rp[i]; p < rp[i + 1]; ++p)
      if (ci[p] == i) {
        d = p;
        break;
      }
    dpos[i] = d;
  }
}

// Greedy first-fit colouring in Jones-Plassmann priority order (an alternative to
// Algorithms 4.1/4.2): priority keys, then rounds in which every vertex whose higher-
// priority neighbours are all coloured takes the smallest colour none of them has.  A
// vertex's colour depends only on those neighbours' final colours, so the result is the
// sequential greedy's in priority order whatever the rounds' timing (a neighbour coloured
// in the same round and not yet seen only delays a vertex to the next round).
__device__ __forceinline__ unsigned long long jp_splitmix64(unsigned long long x) {
  // SplitMix64 output function (Vigna)
  unsigned long long z = x + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// key: larger degree first, then the smaller high word of SplitMix64(v ^ seed); a stable
// sort of the keys in index order breaks the remaining ties by index
__global__ void jp_keys_kernel(int n, const int* __restrict__ srp, unsigned long long seed,
                               unsigned long long* __restrict__ key, int* __restrict__ idx) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const unsigned long long deg = (unsigned long long)(srp[v + 1] - srp[v]);
    key[v] = ((0x7FFFFFFFull - deg) << 32) | (jp_splitmix64((unsigned long long)v ^ seed) >> 32);
    idx[v] = v;
  }
}

__global__ void jp_round_kernel(int n, const int* __restrict__ srp, const int* __restrict__ sci,
                                const int* __restrict__ rank, int* colour,
                                int* __restrict__ counters) {
  int done_here = 0, gmax = 0;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    if (colour[v] != 0) continue;
    const int rv = rank[v];
    const int q0 = srp[v], q1 = srp[v + 1];
    unsigned long long used = 0;  // colours 1..64 of the higher-priority neighbours
    bool ready = true, high = false;
    for (int q = q0; q < q1; ++q) {
      const int u = sci[q];
      if (rank[u] > rv) continue;
      const int cu = *(volatile int*)(colour + u);
      if (cu == 0) {
        ready = false;
        break;
      }
      if (cu <= 64)
        used |= 1ull << (cu - 1);
      else
        high = true;
    }
    if (!ready) continue;
    int c = __ffsll(~used);  // smallest colour in 1..64 not taken (0 if all 64 are)
    if (c == 0 || high) {  // rare: a colour above 64 among the neighbours
      c = 1;
      for (bool taken = true; taken; ++c) {
        taken = false;
        for (int q = q0; q < q1 && !taken; ++q) {
          const int u = sci[q];
          taken = rank[u] < rv && *(volatile int*)(colour + u) == c;
        }
        if (!taken) break;
      }
    }
    colour[v] = c;
    ++done_here;
    gmax = max(gmax, c);
  }
  if (done_here) {
    atomicAdd(counters, done_here);
    atomicMax(counters + 1, gmax);
  }
}

// Two-hop lists of a graph for VerticesGrouping: for every vertex v the rows of its
// neighbours, concatenated in the order of v's row (the second circle of Algorithm 4.1,
// with repeats and with v's own neighbours, which the colouring filters out).
__global__ void twohop_count_kernel(int n, const int* __restrict__ srp,
                                    const int* __restrict__ sci, int* __restrict__ cnt,
                                    unsigned long long* __restrict__ total) {
  __shared__ unsigned long long part[kThreads / 32];
  unsigned long long mine = 0;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    int c = 0;
    for (int q = srp[v]; q < srp[v + 1]; ++q) {
      const int k = sci[q];
      c += srp[k + 1] - srp[k];
    }
    cnt[v] = c;
    mine += (unsigned long long)c;
  }
  for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
  if (threadIdx.x % 32 == 0) part[threadIdx.x / 32] = mine;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) t += part[w];
    atomicAdd(total, t);
  }
}

__global__ void twohop_fill_kernel(int n, const int* __restrict__ srp, const int* __restrict__ sci,
                                   const int* __restrict__ tp, int* __restrict__ tl) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    int pos = tp[v];
    for (int q = srp[v]; q < srp[v + 1]; ++q) {
      const int k = sci[q];
      for (int e = srp[k]; e < srp[k + 1]; ++e) tl[pos++] = sci[e];
    }
  }
}

// ELL copy of the off-diagonal entries of a CSR level matrix for the colour sweeps and the
// restriction: slot k of row i at i*K + k, in the row's CSR order; unused slots hold (i, 0);
// diag[i] = a_ii.  meta[i] = number of off-diagonal entries | (entries left of the
// diagonal) << 16, or -1 for a row with more than K of them (that row keeps only its CSR
// form and every slot is unused).
__global__ void build_ell_kernel(int n, int K, const int* __restrict__ rp,
                                 const int* __restrict__ ci, const double* __restrict__ v,
                                 const int* __restrict__ dpos, int* __restrict__ ell_ci,
                                 double* __restrict__ ell_v, int* __restrict__ meta,
                                 double* __restrict__ diag) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int p0 = rp[i], p1 = rp[i + 1], pd = dpos[i];
    diag[i] = v[pd];
    const int len = p1 - p0 - 1;
    int k = 0;
    if (len <= K) {
      for (int p = p0; p < p1; ++p) {
        if (p == pd) continue;
        ell_ci[(size_t)i * K + k] = ci[p];
        ell_v[(size_t)i * K + k] = v[p];
        ++k;
      }
      meta[i] = len | ((pd - p0) << 16);
    } else {
      meta[i] = -1;
    }
    for (; k < K; ++k) {
      ell_ci[(size_t)i * K + k] = i;
      ell_v[(size_t)i * K + k] = 0.0;
    }
  }
}

__global__ void rdiag_kernel(int n, const int* __restrict__ dpos, const double* __restrict__ v,
                             double* __restrict__ rdiag, DevFlags* flags) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int d = dpos[i];
    const double a = d >= 0 ? v[d] : 0.0;
    if (!(a != 0.0)) {
      raise_flag(flags, MSP_ERR_SINGULAR_BLOCK, i);
      rdiag[i] = 0.0;
    } else {
      rdiag[i] = 1.0 / a;
    }
  }
}

template <int N>
__device__ bool small_inverse(const double* __restrict__ D, double* X) {
  double a[N][N], x[N][N];
#pragma unroll
  for (int r = 0; r < N; ++r)
#pragma unroll
    for (int c = 0; c < N; ++c) {
      a[r][c] = D[r * N + c];
      x[r][c] = (r == c) ? 1.0 : 0.0;
    }
  for (int c = 0; c < N; ++c) {
    int p = c;
    for (int r = c + 1; r < N; ++r)
      if (fabs(a[r][c]) > fabs(a[p][c])) p = r;
    if (!(a[p][c] != 0.0) || !isfinite(a[p][c])) return false;
    if (p != c) {
#pragma unroll
      for (int k = 0; k < N; ++k) {
        double t = a[p][k];
        a[p][k] = a[c][k];
        a[c][k] = t;
        t = x[p][k];
        x[p][k] = x[c][k];
        x[c][k] = t;
      }
    }
    const double inv = 1.0 / a[c][c];
#pragma unroll
    for (int k = 0; k < N; ++k) {
      a[c][k] *= inv;
      x[c][k] *= inv;
    }
    for (int r = 0; r < N; ++r) {
      if (r == c) continue;
      const double f = a[r][c];
#pragma unroll
      for (int k = 0; k < N; ++k) {
        a[r][k] -= f * a[c][k];
        x[r][k] -= f * x[c][k];
      }
    }
  }
#pragma unroll
  for (int r = 0; r < N; ++r)
#pragma unroll
    for (int c = 0; c < N; ++c) X[r * N + c] = x[r][c];
  return true;
}

// Block ILU(0) (IKJ form) of the rows of one colour: for every k < i in the pattern,
// L_ik = A_ik U_kk^-1 and A_ij -= L_ik A_kj for the later j of row i present in row k.
template <int B>
__global__ void bilu_factor_kernel(int r0, int r1, const int* __restrict__ rp,
                                   const int* __restrict__ ci, const int* __restrict__ dpos,
                                   double* __restrict__ lu, double* __restrict__ uinv,
                                   DevFlags* flags) {
  constexpr int BB = B * B;
  for (int i = r0 + blockIdx.x * blockDim.x + threadIdx.x; i < r1; i += gridDim.x * blockDim.x) {
    const int p0 = rp[i], pd = dpos[i], p1 = rp[i + 1];
    for (int p = p0; p < pd; ++p) {
      const int k = ci[p];
      double L[BB];
      const double* Ap = lu + (size_t)p * BB;
      const double* Uk = uinv + (size_t)k * BB;
#pragma unroll
      for (int r = 0; r < B; ++r)
#pragma unroll
        for (int c = 0; c < B; ++c) {
          double s = 0.0;
#pragma unroll
          for (int m = 0; m < B; ++m) s = fma(Ap[r * B + m], Uk[m * B + c], s);
          L[r * B + c] = s;
        }
#pragma unroll
      for (int t = 0; t < BB; ++t) lu[(size_t)p * BB + t] = L[t];
      const int k0 = rp[k], k1 = rp[k + 1];
      int kr = k0;
      for (int q = p + 1; q < p1; ++q) {
        const int j = ci[q];
        while (kr < k1 && ci[kr] < j) ++kr;  // both rows ascending
        if (kr >= k1) break;
        if (ci[kr] != j) continue;
        const double* Ukj = lu + (size_t)kr * BB;
        double* Aq = lu + (size_t)q * BB;
#pragma unroll
        for (int r = 0; r < B; ++r)
#pragma unroll
          for (int c = 0; c < B; ++c) {
            double s = 0.0;
#pragma unroll
            for (int m = 0; m < B; ++m) s = fma(L[r * B + m], Ukj[m * B + c], s);
            Aq[r * B + c] -= s;
          }
      }
    }
    double X[BB];
    if (!small_inverse<B>(lu + (size_t)pd * BB, X)) {
      raise_flag(flags, MSP_ERR_SINGULAR_BLOCK, i);
      continue;
    }
#pragma unroll
    for (int t = 0; t < BB; ++t) uinv[(size_t)i * BB + t] = X[t];
  }
}

__global__ void csr_to_dense_kernel(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                    const double* __restrict__ v, double* __restrict__ A) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double* row = A + (size_t)i * n;
    for (int p = rp[i]; p < rp[i + 1]; ++p) row[ci[p]] = v[p];
  }
}

// pivot search in column k (rows k..n-1, first maximum), row swap, pivot row scaling,
// and a copy of column k (after the swap) for the rank-1 update
// Gauss-Jordan step k, pivot part: partial pivoting in column k (rows k..n-1), rows k and
// the pivot row swapped over all columns, col = column k, row k scaled by 1/pivot over the
// columns [j0, j1) being transformed now (the current panel)
__global__ void gj_pivot_kernel(int n, int k, int j0, int j1, double* __restrict__ A,
                                double* __restrict__ col, int* __restrict__ piv,
                                DevFlags* flags) {
  __shared__ double sv[1024];
  __shared__ int si[1024];
  double best = -1.0;
  int bi = n;
  for (int i = k + threadIdx.x; i < n; i += blockDim.x) {
    const double a = fabs(A[(size_t)i * n + k]);
    if (a > best) {
      best = a;
      bi = i;
    }
  }
  sv[threadIdx.x] = best;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      const double a = sv[threadIdx.x + o];
      const int ia = si[threadIdx.x + o];
      if (a > sv[threadIdx.x] || (a == sv[threadIdx.x] && ia < si[threadIdx.x])) {
        sv[threadIdx.x] = a;
        si[threadIdx.x] = ia;
      }
    }
    __syncthreads();
  }
  const int p = si[0];
  if (!(sv[0] > 0.0) || p >= n) {
    if (threadIdx.x == 0) raise_flag(flags, MSP_ERR_SINGULAR_BLOCK, k);
    return;
  }
  if (threadIdx.x == 0) piv[k] = p;
  if (p != k)
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      const double t = A[(size_t)p * n + j];
      A[(size_t)p * n + j] = A[(size_t)k * n + j];
      A[(size_t)k * n + j] = t;
    }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) col[i] = A[(size_t)i * n + k];
  __syncthreads();
  const double inv = 1.0 / col[k];
  for (int j = j0 + threadIdx.x; j < j1; j += blockDim.x)
    A[(size_t)k * n + j] = (j == k) ? inv : A[(size_t)k * n + j] * inv;
}

// Gauss-Jordan step k, elimination part over the columns [j0, j0 + w): rows i != k
__global__ void gj_update_kernel(int n, int k, int j0, int w, double* __restrict__ A,
                                 const double* __restrict__ col) {
  const double* rowk = A + (size_t)k * n;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < (size_t)n * w;
       t += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / w), j = j0 + (int)(t % w);
    if (i == k) continue;
    const double f = col[i];
    double* a = A + (size_t)i * n + j;
    if (j == k)
      *a = -f * rowk[k];
    else
      *a -= f * rowk[j];
  }
}

// After the steps of a panel of columns K = [k0, k0 + nb) have transformed the panel: the
// same steps applied to every other column c at once.  They compose to
// I + sum_q (P_q - e_q) e_q^T with P the panel's columns, so
//   c[i] += sum_q P[i][q] c[k0 + q] for the rows outside K,
//   c[i]  = sum_q P[i][q] c[k0 + q] for the rows in K,
// with c[k0 + q] the values before the update (T, a copy of the rows K).  64 x 64 tiles of
// A, 4 x 4 per thread, the panel and T staged in shared memory.
constexpr int kGjPanel = 32;
__global__ void __launch_bounds__(256) gj_panel_apply_kernel(int n, int k0, int nb,
                                                             double* __restrict__ A,
                                                             const double* __restrict__ T) {
  __shared__ double sP[64][kGjPanel + 1];
  __shared__ double sT[kGjPanel][64];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int r0 = blockIdx.y * 64, c0 = blockIdx.x * 64;
  for (int t = threadIdx.x; t < 64 * kGjPanel; t += 256) {
    const int r = t / kGjPanel, q = t % kGjPanel;
    sP[r][q] = (r0 + r < n && q < nb) ? A[(size_t)(r0 + r) * n + k0 + q] : 0.0;
    const int qq = t / 64, c = t % 64;
    sT[qq][c] = (qq < nb && c0 + c < n) ? T[(size_t)qq * n + c0 + c] : 0.0;
  }
  __syncthreads();
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
  for (int q = 0; q < nb; ++q) {
    double p[4], tv[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) p[a] = sP[ty + 16 * a][q];
#pragma unroll
    for (int b = 0; b < 4; ++b) tv[b] = sT[q][tx + 16 * b];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = fma(p[a], tv[b], acc[a][b]);
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int i = r0 + ty + 16 * a;
    if (i >= n) continue;
    const bool in_k = i >= k0 && i < k0 + nb;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int j = c0 + tx + 16 * b;
      if (j >= n || (j >= k0 && j < k0 + nb)) continue;
      double* a_ij = A + (size_t)i * n + j;
      *a_ij = in_k ? acc[a][b] : *a_ij + acc[a][b];
    }
  }
}

__global__ void gj_unscramble_kernel(int n, const int* __restrict__ colperm,
                                     const double* __restrict__ A, double* __restrict__ out) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < (size_t)n * n;
       t += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / n), c = (int)(t % n);
    out[t] = A[(size_t)i * n + colperm[c]];
  }
}

__global__ void cast_vals_kernel(size_t n, const double* __restrict__ in, float* __restrict__ out) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n;
       t += (size_t)gridDim.x * blockDim.x)
    out[t] = (float)in[t];
}

__global__ void iota_kernel(int n, int* out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    out[i] = i;
}

__global__ void fill_int_kernel(size_t n, int value, int* out) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    out[i] = value;
}

__global__ void scatter_inverse_kernel(int n, const int* __restrict__ perm, int* __restrict__ iperm) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
    iperm[perm[k]] = k;
}

}  // namespace

int launch_check_pattern(int nb, int nnz, const int* rp, const int* ci, int* dpos, DevFlags* flags,
                         cudaStream_t s) {
  check_pattern_kernel<<<grid_for(nb, kThreads), kThreads, 0, s>>>(nb, nnz, rp, ci, dpos, flags);
  return launch_status();
}

int launch_check_block_diagonal(int nb, const int* rp, const int* ci, const int* perm, int B,
                                const int* off, DevFlags* flags, cudaStream_t s) {
  if (nb <= 0) return MSP_OK;
  check_block_diagonal_kernel<<<grid_for(nb, kThreads), kThreads, 0, s>>>(nb, rp, ci, perm, B,
                                                                          off, flags);
  return launch_status();
}

int launch_check_finite_vals(size_t n, const double* v, DevFlags* flags, cudaStream_t s) {
  if (!n) return MSP_OK;
  check_finite_vals_kernel<<<grid_for(n, kThreads), kThreads, 0, s>>>(n, v, flags);
  return launch_status();
}

int launch_gather_values(size_t nnz, int bb, const int* src, const double* in, double* out,
                         cudaStream_t s) {
  if (!nnz) return MSP_OK;
  gather_values_kernel<<<grid_for(nnz * bb, kThreads), kThreads, 0, s>>>(nnz, bb, src, in, out);
  return launch_status();
}

int launch_extract_N(int b, size_t nnzb, const double* v, double* aN, cudaStream_t s) {
  if (b < 2 || !nnzb) return MSP_OK;
  extract_N_kernel<<<grid_for(nnzb * (b - 1) * (b - 1), kThreads), kThreads, 0, s>>>(b, nnzb, v,
                                                                                     aN);
  return launch_status();
}

int launch_scale_N_rows(int b, int nb, const int* rp, const int* dpos, const double* dNinv,
                        double* aN, cudaStream_t s) {
  if (nb <= 0 || b < 2) return MSP_OK;
  const unsigned grid = grid_for(nb, kThreads);
  switch (b - 1) {
    case 1: scale_N_rows_kernel<1><<<grid, kThreads, 0, s>>>(nb, rp, dpos, dNinv, aN); break;
    case 2: scale_N_rows_kernel<2><<<grid, kThreads, 0, s>>>(nb, rp, dpos, dNinv, aN); break;
    case 3: scale_N_rows_kernel<3><<<grid, kThreads, 0, s>>>(nb, rp, dpos, dNinv, aN); break;
    case 4: scale_N_rows_kernel<4><<<grid, kThreads, 0, s>>>(nb, rp, dpos, dNinv, aN); break;
    case 5: scale_N_rows_kernel<5><<<grid, kThreads, 0, s>>>(nb, rp, dpos, dNinv, aN); break;
    case 6: scale_N_rows_kernel<6><<<grid, kThreads, 0, s>>>(nb, rp, dpos, dNinv, aN); break;
    case 7: scale_N_rows_kernel<7><<<grid, kThreads, 0, s>>>(nb, rp, dpos, dNinv, aN); break;
    default: return MSP_ERR_ARG;
  }
  return launch_status();
}

int launch_diag_pos(int n, const int* rp, const int* ci, int* dpos, cudaStream_t s) {
  if (n <= 0) return MSP_OK;
  diag_pos_kernel<<<grid_for(n, kThreads), kThreads, 0, s>>>(n, rp, ci, dpos);
  return launch_status();
}

int launch_jp_keys(int n, const int* srp, unsigned long long seed, unsigned long long* key,
                   int* idx, cudaStream_t s) {
  if (n <= 0) return MSP_OK;
  jp_keys_kernel<<<grid_for(n, kThreads), kThreads, 0, s>>>(n, srp, seed, key, idx);
  return launch_status();
}

int launch_jp_round(int n, const int* srp, const int* sci, const int* rank, int* colour,
                    int* counters, cudaStream_t s) {
  if (n <= 0) return MSP_OK;
  jp_round_kernel<<<grid_for(n, kThreads), kThreads, 0, s>>>(n, srp, sci, rank, colour,
                                                             counters);
  return launch_status();
}

int launch_twohop_count(int n, const int* srp, const int* sci, int* cnt, unsigned long long* total,
                        cudaStream_t s) {
  if (n <= 0) return MSP_OK;
  MSP_CUDA_TRY(cudaMemsetAsync(total, 0, sizeof(unsigned long long), s));
  twohop_count_kernel<<<grid_for(n, kThreads), kThreads, 0, s>>>(n, srp, sci, cnt, total);
  return launch_status();
}

int launch_twohop_fill(int n, const int* srp, const int* sci, const int* tp, int* tl,
                       cudaStream_t s) {
  if (n <= 0) return MSP_OK;
  twohop_fill_kernel<<<grid_for(n, kThreads), kThreads, 0, s>>>(n, srp, sci, tp, tl);
  return launch_status();
}

int launch_build_ell(int n, int K, const int* rp, const int* ci, const double* v, const int* dpos,
                     int* ell_ci, double* ell_v, int* meta, double* diag, cudaStream_t s) {
  if (n <= 0 || K <= 0) return MSP_OK;
  build_ell_kernel<<<grid_for(n, kThreads), kThreads, 0, s>>>(n, K, rp, ci, v, dpos, ell_ci,
                                                              ell_v, meta, diag);
  return launch_status();
}

int launch_rdiag(int n, const int* dpos, const double* v, double* rdiag, DevFlags* flags,
                 cudaStream_t s) {
  if (n <= 0) return MSP_OK;
  rdiag_kernel<<<grid_for(n, kThreads), kThreads, 0, s>>>(n, dpos, v, rdiag, flags);
  return launch_status();
}

int launch_bilu_factor(int b, int r0, int r1, const int* rp, const int* ci, const int* dpos,
                       double* lu, double* uinv, DevFlags* flags, cudaStream_t s) {
  if (r1 <= r0) return MSP_OK;
  const unsigned grid = grid_for(r1 - r0, 128);
  switch (b) {
#define MSP_BF_CASE(BB)                                                                   \
  case BB:                                                                                \
    bilu_factor_kernel<BB><<<grid, 128, 0, s>>>(r0, r1, rp, ci, dpos, lu, uinv, flags);   \
    break;
    MSP_BF_CASE(1)
    MSP_BF_CASE(2)
    MSP_BF_CASE(3)
    MSP_BF_CASE(4)
    MSP_BF_CASE(5)
    MSP_BF_CASE(6)
    MSP_BF_CASE(7)
    MSP_BF_CASE(8)
#undef MSP_BF_CASE
    default:
      return MSP_ERR_ARG;
  }
  return launch_status();
}

int launch_csr_to_dense(int n, const int* rp, const int* ci, const double* v, double* A,
                        cudaStream_t s) {
  if (n <= 0) return MSP_OK;
  MSP_CUDA_TRY(cudaMemsetAsync(A, 0, (size_t)n * n * sizeof(double), s));
  csr_to_dense_kernel<<<grid_for(n, kThreads), kThreads, 0, s>>>(n, rp, ci, v, A);
  return launch_status();
}

int launch_gj_pivot(int n, int k, int j0, int j1, double* A, double* col, int* piv,
                    DevFlags* flags, cudaStream_t s) {
  gj_pivot_kernel<<<1, 1024, 0, s>>>(n, k, j0, j1, A, col, piv, flags);
  return launch_status();
}

int launch_gj_update(int n, int k, int j0, int w, double* A, const double* col, cudaStream_t s) {
  gj_update_kernel<<<grid_for((size_t)n * w, kThreads), kThreads, 0, s>>>(n, k, j0, w, A, col);
  return launch_status();
}

int launch_gj_panel_apply(int n, int k0, int nb, double* A, const double* T, cudaStream_t s) {
  if (nb <= 0 || nb > kGjPanel) return MSP_ERR_ARG;
  const dim3 grid((n + 63) / 64, (n + 63) / 64);
  gj_panel_apply_kernel<<<grid, 256, 0, s>>>(n, k0, nb, A, T);
  return launch_status();
}

int launch_gj_unscramble(int n, const int* colperm, const double* A, double* out,
                         cudaStream_t s) {
  gj_unscramble_kernel<<<grid_for((size_t)n * n, kThreads), kThreads, 0, s>>>(n, colperm, A,
                                                                             out);
  return launch_status();
}

int launch_cast_vals(size_t n, const double* in, float* out, cudaStream_t s) {
  if (!n) return MSP_OK;
  cast_vals_kernel<<<grid_for(n, kThreads), kThreads, 0, s>>>(n, in, out);
  return launch_status();
}

int launch_iota(int n, int* out, cudaStream_t s) {
  if (n <= 0) return MSP_OK;
  iota_kernel<<<grid_for(n, kThreads), kThreads, 0, s>>>(n, out);
  return launch_status();
}

int launch_fill_int(size_t n, int value, int* out, cudaStream_t s) {
  if (!n) return MSP_OK;
  fill_int_kernel<<<grid_for(n, kThreads), kThreads, 0, s>>>(n, value, out);
  return launch_status();
}

int launch_scatter_inverse(int n, const int* perm, int* iperm, cudaStream_t s) {
  if (n <= 0) return MSP_OK;
  scatter_inverse_kernel<<<grid_for(n, kThreads), kThreads, 0, s>>>(n, perm, iperm);
  return launch_status();
}

}  // namespace msp
