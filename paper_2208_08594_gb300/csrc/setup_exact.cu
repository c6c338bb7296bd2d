// Setup kernels whose floating-point results decide integer outputs (aggregates, coarse
// patterns, colourings).  This translation unit is compiled with -fmad=false: every
// product and sum is rounded separately, in the order written, with IEEE division, so
// the decoupling weights, the pressure matrix, the strength of connection and the
// Galerkin sums are reproducible bit for bit by any implementation that follows the
// same definitions in the same order:
//   * Gauss-Jordan inverse with partial pivoting (first maximum |pivot| wins): pivot row
//     divided by the pivot, then row_r - a_rc * pivot_row for every other row r;
//   * A_P[i,j] = (((0 + w_0 a_0) + w_1 a_1) + ...) with a_k = A_ij[k][0] (Eq. MSP's
//     Pi_P^T A Pi_P with the quasi-IMPES restriction);
//   * s_ij = -0.5 * (a_ij + a_ji), candidates s_ij >= beta * max_k s_ik;
//   * A_c[I,J] = ((0 + a_1) + a_2) + ... over the fine nonzeros in CSR order.
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

// Gauss-Jordan inverse of an N x N row-major block held in registers/local memory.
template <int N>
__device__ bool gj_inverse(const double* __restrict__ D, int ld_row, int off, double* X) {
  double a[N][N], x[N][N];
#pragma unroll
  for (int r = 0; r < N; ++r)
#pragma unroll
    for (int c = 0; c < N; ++c) {
      a[r][c] = D[(r + off) * ld_row + c + off];
      x[r][c] = (r == c) ? 1.0 : 0.0;
    }
  for (int c = 0; c < N; ++c) {
    int p = c;
    for (int r = c + 1; r < N; ++r)
      if (fabs(a[r][c]) > fabs(a[p][c])) p = r;
    double pv = a[p][c];
    if (!(pv != 0.0) || !isfinite(pv)) return false;
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
    const double piv = a[c][c];
#pragma unroll
    for (int k = 0; k < N; ++k) {
      a[c][k] = __ddiv_rn(a[c][k], piv);
      x[c][k] = __ddiv_rn(x[c][k], piv);
    }
    for (int r = 0; r < N; ++r) {
      if (r == c) continue;
      const double f = a[r][c];
#pragma unroll
      for (int k = 0; k < N; ++k) {
        a[r][k] = __dsub_rn(a[r][k], __dmul_rn(f, a[c][k]));
        x[r][k] = __dsub_rn(x[r][k], __dmul_rn(f, x[c][k]));
      }
    }
  }
#pragma unroll
  for (int r = 0; r < N; ++r)
#pragma unroll
    for (int c = 0; c < N; ++c) X[r * N + c] = x[r][c];
  return true;
}

template <int B>
__global__ void diag_inverse_kernel(int nb, const int* __restrict__ dpos,
                                    const double* __restrict__ v, double* __restrict__ dinv,
                                    double* __restrict__ omega, DevFlags* flags) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += gridDim.x * blockDim.x) {
    const double* D = v + (size_t)dpos[i] * B * B;
    double X[B * B];
    if (!gj_inverse<B>(D, B, 0, X)) {
      raise_flag(flags, MSP_ERR_SINGULAR_BLOCK, i);
      continue;
    }
    if (dinv)
      for (int k = 0; k < B * B; ++k) dinv[(size_t)i * B * B + k] = X[k];
    for (int k = 0; k < B; ++k) omega[(size_t)i * B + k] = X[k];
  }
}

template <int B>
__global__ void diagN_inverse_kernel(int nb, const int* __restrict__ dpos,
                                     const double* __restrict__ v, double* __restrict__ dNinv,
                                     DevFlags* flags) {
  constexpr int BN = B - 1;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += gridDim.x * blockDim.x) {
    const double* D = v + (size_t)dpos[i] * B * B;
    double X[BN * BN];
    if (!gj_inverse<BN>(D, B, 1, X)) {
      raise_flag(flags, MSP_ERR_SINGULAR_BLOCK, i);
      continue;
    }
    for (int k = 0; k < BN * BN; ++k) dNinv[(size_t)i * BN * BN + k] = X[k];
  }
}

__global__ void pressure_matrix_kernel(int b, int nb, const int* __restrict__ rp,
                                       const double* __restrict__ v,
                                       const double* __restrict__ omega, bool decoupling,
                                       double* __restrict__ ap) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += gridDim.x * blockDim.x) {
    for (int p = rp[i]; p < rp[i + 1]; ++p) {
      const double* blk = v + (size_t)p * b * b;
      double s;
      if (decoupling) {
        s = 0.0;
        for (int k = 0; k < b; ++k) s = __dadd_rn(s, __dmul_rn(omega[(size_t)i * b + k], blk[k * b]));
      } else {
        s = blk[0];
      }
      ap[p] = s;
    }
  }
}

__device__ double csr_entry(const int* __restrict__ rp, const int* __restrict__ ci,
                            const double* __restrict__ v, int i, int j) {
  int lo = rp[i], hi = rp[i + 1];
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    int c = ci[mid];
    if (c < j)
      lo = mid + 1;
    else
      hi = mid;
  }
  return (lo < rp[i + 1] && ci[lo] == j) ? v[lo] : 0.0;
}

__global__ void strength_kernel(int n, const int* __restrict__ arp, const int* __restrict__ aci,
                                const double* __restrict__ av, const int* __restrict__ srp,
                                const int* __restrict__ sci, double beta,
                                double* __restrict__ sval, unsigned char* __restrict__ cand) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double smax = 0.0;
    bool any = false;
    for (int q = srp[i]; q < srp[i + 1]; ++q) {
      const int j = sci[q];
      const double t = __dadd_rn(csr_entry(arp, aci, av, i, j), csr_entry(arp, aci, av, j, i));
      const double s = __dmul_rn(-0.5, t);
      sval[q] = s;
      if (!any || s > smax) smax = s;
      any = true;
    }
    const bool ok = any && smax > 0.0;
    const double thr = __dmul_rn(beta, smax);
    for (int q = srp[i]; q < srp[i + 1]; ++q) cand[q] = (ok && sval[q] >= thr) ? 1 : 0;
  }
}

__global__ void transpose_pos_kernel(int n, const int* __restrict__ srp, const int* __restrict__ sci,
                                     int* __restrict__ tpos) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    for (int q = srp[i]; q < srp[i + 1]; ++q) {
      const int j = sci[q];
      int lo = srp[j], hi = srp[j + 1];
      while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (sci[mid] < i)
          lo = mid + 1;
        else
          hi = mid;
      }
      tpos[q] = lo;  // S is symmetric: (j, i) exists
    }
  }
}

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
  unsigned long long z = x + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

__global__ void visit_keys_kernel(int n, unsigned long long seed, unsigned long long* hkey) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    hkey[i] = splitmix64((unsigned long long)i ^ seed);
}

// k visits before i in the sequential order (ascending (hash, index))
__device__ __forceinline__ bool before(const unsigned long long* hkey, int k, int i) {
  const unsigned long long a = hkey[k], b = hkey[i];
  return a < b || (a == b && k < i);
}

// A node i that is still undecided may take its sequential decision now iff no
// undecided node visited before it can still mark i or the partner it would choose:
// i.e. no such node k has i (or the chosen j) among its candidates.  The chosen
// partner is the best undecided candidate visited after i (those visited before are
// marked by the time i is visited).  Two nodes deciding in the same round never touch
// the same node, and the earliest undecided node always decides, so the rounds
// reproduce the sequential visit-order matching exactly.
__global__ void match_round_kernel(int n, const int* __restrict__ srp, const int* __restrict__ sci,
                                   const int* __restrict__ tpos, const double* __restrict__ sval,
                                   const unsigned char* __restrict__ cand,
                                   const unsigned long long* __restrict__ hkey,
                                   const unsigned char* __restrict__ state,
                                   int* __restrict__ commit) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    commit[i] = 0;
    if (state[i]) continue;
    bool blocked = false;
    // anyone visited before i that could pick i?
    for (int q = srp[i]; q < srp[i + 1] && !blocked; ++q) {
      const int k = sci[q];
      if (!state[k] && cand[tpos[q]] && before(hkey, k, i)) blocked = true;
    }
    if (blocked) continue;
    int best = -1;
    double sb = 0.0;
    for (int q = srp[i]; q < srp[i + 1]; ++q) {
      if (!cand[q]) continue;
      const int j = sci[q];
      if (state[j] || before(hkey, j, i)) continue;
      const double sq = sval[q];
      if (best < 0 || sq > sb || (sq == sb && j < best)) {
        best = j;
        sb = sq;
      }
    }
    if (best >= 0) {
      for (int q = srp[best]; q < srp[best + 1] && !blocked; ++q) {
        const int k = sci[q];
        if (k != i && !state[k] && cand[tpos[q]] && before(hkey, k, i)) blocked = true;
      }
    }
    if (!blocked) commit[i] = best >= 0 ? best + 2 : 1;
  }
}

__global__ void match_apply_kernel(int n, const int* __restrict__ commit,
                                   unsigned char* __restrict__ state, int* __restrict__ partner,
                                   DevFlags* flags) {
  (void)flags;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int c = commit[i];
    if (c == 0) continue;
    state[i] = 1;
    if (c >= 2) {
      const int j = c - 2;
      state[j] = 1;
      partner[i] = j;
      partner[j] = i;
    } else {
      partner[i] = -1;
    }
  }
}

__global__ void count_undecided_kernel(int n, const unsigned char* __restrict__ state,
                                       DevFlags* flags) {
  int left = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    left += state[i] == 0;
  for (int o = 16; o > 0; o >>= 1) left += __shfl_xor_sync(0xffffffffu, left, o);
  if ((threadIdx.x & 31) == 0 && left) atomicAdd(&flags->count, left);
}

__global__ void match_reps_kernel(int n, const int* __restrict__ partner, int* __restrict__ rep) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int p = partner[i];
    rep[i] = (p < 0 || i < p) ? 1 : 0;
  }
}

__global__ void match_ids_kernel(int n, const int* __restrict__ partner, const int* __restrict__ id,
                                 int* __restrict__ agg) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int p = partner[i];
    agg[i] = id[(p < 0 || i < p) ? i : p];
  }
}

__global__ void segment_sums_kernel(int nseg, const int* __restrict__ seg_start,
                                    const int* __restrict__ src, const double* __restrict__ v,
                                    double* __restrict__ out) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nseg; k += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int t = seg_start[k]; t < seg_start[k + 1]; ++t) s = __dadd_rn(s, v[src[t]]);
    out[k] = s;
  }
}

// ----------------------------------------------------------------------------------
// Sequential VerticesGrouping by one warp on the graph relabelled by priority rank
// (degree desc, index asc), so that the vertex Algorithm 4.1 picks (the largest degree,
// the smallest index among equals) is simply the smallest label.  inV is a bitmap of the
// vertices in V of the current pass (test-and-clear with atomics, so the lanes can remove
// neighbours concurrently); a vertex leaves V when it is coloured or moved to Wbar, and
// the Wbar list of a pass is V of the next one.  The frontier hat W is a three-level
// bitmap, so its first set bit is the next pick.  A vertex that leaves V as a neighbour
// of W leaves the frontier at the same time (the else branch of Algorithm 4.1 would only
// move it to Wbar, where it already is); an entry found outside V when popped is still
// dropped.  With an empty frontier the pick is the
// smallest label still in V (a cursor that only moves forward).  Both bitmaps live in
// shared memory when they fit.  The second circle is read from the graph's two-hop lists
// when they are given (one contiguous run per vertex, loaded together with the
// neighbours); otherwise it is gathered from the neighbours' rows with every lane issuing
// its loads back to back (owner rows looked up in shared memory).
// ----------------------------------------------------------------------------------
struct Bitmap3 {
  unsigned* l0;
  unsigned* l1;
  unsigned* l2;
  int n0, n1, n2;
};

__device__ int bm_find_first(const Bitmap3& bm, int lane) {
  int idx2 = -1;
  for (int base = 0; base < bm.n2; base += 32) {
    const unsigned w = (base + lane < bm.n2) ? bm.l2[base + lane] : 0u;
    const unsigned m = __ballot_sync(0xffffffffu, w != 0u);
    if (m) {
      idx2 = base + __ffs(m) - 1;
      break;
    }
  }
  if (idx2 < 0) return -1;
  const int idx1 = idx2 * 32 + __ffs(bm.l2[idx2]) - 1;
  const int idx0 = idx1 * 32 + __ffs(bm.l1[idx1]) - 1;
  return idx0 * 32 + __ffs(bm.l0[idx0]) - 1;
}

__device__ void bm_clear(const Bitmap3& bm, int r) {
  const int i0 = r >> 5, i1 = r >> 10, i2 = r >> 15;
  const unsigned w0 = bm.l0[i0] & ~(1u << (r & 31));
  bm.l0[i0] = w0;
  if (w0 == 0u) {
    const unsigned w1 = bm.l1[i1] & ~(1u << (i0 & 31));
    bm.l1[i1] = w1;
    if (w1 == 0u) bm.l2[i2] &= ~(1u << (i1 & 31));
  }
}

// clear bit r where several lanes may clear bits concurrently (and nobody sets): only the
// lane that empties a word clears its bit one level up
__device__ void bm_clear_atomic(const Bitmap3& bm, int r) {
  const int i0 = r >> 5, i1 = r >> 10, i2 = r >> 15;
  const unsigned b0 = 1u << (r & 31);
  const unsigned o0 = atomicAnd(bm.l0 + i0, ~b0);
  if (o0 == b0) {
    const unsigned b1 = 1u << (i0 & 31);
    const unsigned o1 = atomicAnd(bm.l1 + i1, ~b1);
    if (o1 == b1) atomicAnd(bm.l2 + i2, ~(1u << (i1 & 31)));
  }
}

// set bit r where several lanes may set bits concurrently (and nobody clears): the summary
// bits one and two levels up are set unconditionally (each stands for a non-empty word, which
// the word now is), so no lane waits for an old value before its next entry
__device__ void bm_set(const Bitmap3& bm, int r) {
  const int i0 = r >> 5, i1 = r >> 10, i2 = r >> 15;
  atomicOr(bm.l0 + i0, 1u << (r & 31));
  atomicOr(bm.l1 + i1, 1u << (i0 & 31));
  atomicOr(bm.l2 + i2, 1u << (i1 & 31));
}

__device__ __forceinline__ bool in_v(const unsigned* inV, int v) {
  return (inV[v >> 5] >> (v & 31)) & 1u;
}

constexpr int kSecondU = 8;  // second-circle entries gathered per lane per round

// Fetch the row pointers and two-hop pointers of vertex x into L1 without waiting: the
// next picks come from the second circles just added to the frontier, so their first
// trip to memory is then an L1 hit.
__device__ __forceinline__ void prefetch_rows(const int* srp, const int* tp, int x) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(__cvta_generic_to_global(srp + x)));
  if (tp) asm volatile("prefetch.global.L1 [%0];" ::"l"(__cvta_generic_to_global(tp + x)));
}

// Warp 1 of the colouring CTA: while warp 0 processes its pick, load the two-hop
// neighbourhood of the frontier's current first vertex (the likely next pick) so warp
// 0 finds it in L1.  It only reads; the bitmap it reads is being changed by warp 0, so
// what it finds is a hint, checked for range, and a wrong guess costs nothing but the
// loads.  Its wait for a new pick is bounded and it stops when warp 0 is done.
__device__ void colouring_prefetcher(int n, const int* __restrict__ srp, const int* __restrict__ sci,
                                     const int* __restrict__ tp, const int* __restrict__ tl,
                                     const Bitmap3& bm, volatile int* hint, volatile int* done,
                                     volatile int* sink) {
  const int lane = threadIdx.x % 32;
  const volatile unsigned* l0 = bm.l0;
  const volatile unsigned* l1 = bm.l1;
  const volatile unsigned* l2 = bm.l2;
  int last = -2, acc = 0;
  const long long limit = 256LL * n + (1LL << 20);
  for (long long it = 0; it < limit; ++it) {
    if (*done) break;
    const int v = *hint;
    if (v == last) continue;
    last = v;
    // racy first set bit of the frontier
    int c = -1;
    for (int base = 0; base < bm.n2 && c < 0; base += 32) {
      const unsigned w = (base + lane < bm.n2) ? l2[base + lane] : 0u;
      const unsigned m = __ballot_sync(0xffffffffu, w != 0u);
      if (m) {
        const int i2 = base + __ffs(m) - 1;
        const unsigned w2 = l2[i2];
        if (w2) {
          const int i1 = i2 * 32 + __ffs(w2) - 1;
          const unsigned w1 = i1 < bm.n1 ? l1[i1] : 0u;
          if (w1) {
            const int i0 = i1 * 32 + __ffs(w1) - 1;
            const unsigned w0 = i0 < bm.n0 ? l0[i0] : 0u;
            if (w0) c = i0 * 32 + __ffs(w0) - 1;
          }
        }
        break;
      }
    }
    c = __shfl_sync(0xffffffffu, c, 0);
    if (c < 0 || c >= n) continue;
    if (tp) {
      const int e1 = __ldg(tp + c + 1);
      for (int e = __ldg(tp + c) + 8 * lane; e < e1; e += 256) acc += __ldg(tl + e);
      const int r1 = __ldg(srp + c + 1);
      for (int q = __ldg(srp + c) + 8 * lane; q < r1; q += 256) acc += __ldg(sci + q);
      continue;
    }
    const int q0 = __ldg(srp + c), q1 = __ldg(srp + c + 1);
    for (int q = q0 + lane; q < q1; q += 32) {
      const int k = __ldg(sci + q);
      const int kb = __ldg(srp + k), ke = __ldg(srp + k + 1);
      for (int e = kb; e < ke; e += 8) acc += __ldg(sci + e);  // one load per 32 bytes
    }
  }
  if (acc == 0x7fffffff) *sink = acc;  // keeps the loads
}

// layout flags: bit 0 = frontier bitmap in shared memory, bit 1 = inV in shared memory
__global__ void __launch_bounds__(64) colouring_kernel(int n, const int* __restrict__ srp,
                                                       const int* __restrict__ sci,
                                                       const int* __restrict__ tp,
                                                       const int* __restrict__ tl,
                                                       unsigned* ginV, int* wbar,
                                                       unsigned* gbitmap, int layout,
                                                       int* colour, int* meta, int max_passes) {
  extern __shared__ unsigned smem_bits[];
  __shared__ int s_kb[32], s_off[33];
  __shared__ volatile int s_hint, s_done, s_sink;
  const int lane = threadIdx.x % 32;
  Bitmap3 bm;
  bm.n0 = (n + 31) / 32;
  bm.n1 = (bm.n0 + 31) / 32;
  bm.n2 = (bm.n1 + 31) / 32;
  const int fw = bm.n0 + bm.n1 + bm.n2;
  unsigned* fbase = (layout & 1) ? smem_bits : gbitmap;
  unsigned* inV = (layout & 2) ? smem_bits + ((layout & 1) ? fw : 0) : ginV;
  bm.l0 = fbase;
  bm.l1 = fbase + bm.n0;
  bm.l2 = fbase + bm.n0 + bm.n1;
  if (threadIdx.x == 0) {
    s_hint = -1;
    s_done = 0;
  }
  if (threadIdx.x < 32) {
    for (int k = lane; k < fw; k += 32) fbase[k] = 0u;
    for (int k = lane; k < bm.n0; k += 32) {
      const int rem = n - 32 * k;
      inV[k] = rem >= 32 ? 0xffffffffu : ((1u << rem) - 1u);
    }
  }
  __syncthreads();
  if (threadIdx.x >= 32) {
    colouring_prefetcher(n, srp, sci, tp, tl, bm, &s_hint, &s_done, &s_sink);
    return;
  }
  int coloured = 0, g = 0;
  while (coloured < n) {
    ++g;
    if (g > n || g > max_passes) {  // every pass colours at least one vertex
      if (lane == 0) {
        meta[1] = 1;
        s_done = 1;
      }
      return;
    }
    int cursor = 0, nwbar = 0;
    // every frontier entry of this pass is a distinct vertex of V, popped once
    const long long max_picks = 2LL * (n - coloured) + 2;
    long long picks = 0;
    while (true) {
      int v = -1;
      // frontier first (hat W), dropping stale entries
      while (true) {
        if (++picks > max_picks) {
          if (lane == 0) {
            meta[1] = 1;
            s_done = 1;
          }
          return;
        }
        const int r = bm_find_first(bm, lane);
        if (r < 0) break;
        __syncwarp();
        if (lane == 0) bm_clear(bm, r);
        __syncwarp();
        if (in_v(inV, r)) {
          v = r;
          break;
        }
      }
      if (v < 0) {
        // V by label
        while (cursor < n) {
          const int r = cursor + lane;
          const bool inv = (r < n) && in_v(inV, r);
          const unsigned m = __ballot_sync(0xffffffffu, inv);
          if (m) {
            cursor += __ffs(m) - 1;
            v = cursor;
            break;
          }
          cursor += 32;
        }
        if (v < 0) break;  // V empty: the pass is over
      }
      // W = W u {v}
      if (lane == 0) {
        atomicAnd(inV + (v >> 5), ~(1u << (v & 31)));
        colour[v] = g;
        s_hint = v;  // lets the prefetcher move on to the next likely pick
      }
      ++coloured;
      const int q0 = __ldg(srp + v), q1 = __ldg(srp + v + 1);
      // with two-hop lists the whole second circle is one contiguous run: its first round
      // is loaded here, alongside the neighbours, before they leave V
      int t0 = 0, t1 = 0;
      int xs0[kSecondU];
      if (tp) {
        t0 = __ldg(tp + v);
        t1 = __ldg(tp + v + 1);
#pragma unroll
        for (int u = 0; u < kSecondU; ++u) {
          const int t = t0 + lane + 32 * u;
          xs0[u] = t < t1 ? __ldg(tl + t) : -1;
        }
      }
      // Wbar = Wbar u (S_v n V), V = V / S_v  (all chunks first)
      int kb0 = 0, kl0 = 0;  // row of this lane's neighbour in the first chunk
      for (int q = q0; q < q1; q += 32) {
        const int qq = q + lane;
        bool take = false;
        int j = -1;
        if (qq < q1) {
          j = __ldg(sci + qq);
          if (q == q0 && !tp) {
            kb0 = __ldg(srp + j);
            kl0 = __ldg(srp + j + 1) - kb0;
          }
          const unsigned bit = 1u << (j & 31);
          const unsigned was = atomicAnd(inV + (j >> 5), ~bit);
          // a vertex leaving V also leaves the frontier now, rather than being popped and
          // dropped later (same picks: the frontier's first vertex still in V).  The frontier
          // holds vertices of V only, so j's frontier bit is cleared without waiting for the
          // test above (nothing changes when j was not in V)
          bm_clear_atomic(bm, j);
          take = (was & bit) != 0u;
        }
        const unsigned m = __ballot_sync(0xffffffffu, take);
        if (take) wbar[nwbar + __popc(m & ((1u << lane) - 1u))] = j;
        nwbar += __popc(m);
      }
      __syncwarp();
      // hat W = hat W u hat S_v: undetermined vertices of the second circle
      if (tp) {
#pragma unroll
        for (int u = 0; u < kSecondU; ++u)
          if (xs0[u] >= 0 && in_v(inV, xs0[u])) {
            bm_set(bm, xs0[u]);
            prefetch_rows(srp, tp, xs0[u]);
          }
        for (int t = t0 + 32 * kSecondU; t < t1; t += 32 * kSecondU) {
          int xs[kSecondU];
#pragma unroll
          for (int u = 0; u < kSecondU; ++u) {
            const int tt = t + lane + 32 * u;
            xs[u] = tt < t1 ? __ldg(tl + tt) : -1;
          }
#pragma unroll
          for (int u = 0; u < kSecondU; ++u)
            if (xs[u] >= 0 && in_v(inV, xs[u])) {
              bm_set(bm, xs[u]);
              prefetch_rows(srp, tp, xs[u]);
            }
        }
        __syncwarp();
        continue;
      }
      for (int q = q0; q < q1; q += 32) {
        const int qq = q + lane;
        int kb = kb0, kl = kl0;
        if (q != q0) {
          kb = 0;
          kl = 0;
          if (qq < q1) {
            const int k = __ldg(sci + qq);
            kb = __ldg(srp + k);
            kl = __ldg(srp + k + 1) - kb;
          }
        } else if (qq >= q1) {
          kl = 0;
        }
        // exclusive prefix of the row lengths across the lanes of this chunk
        int off = kl;
        for (int o = 1; o < 32; o <<= 1) {
          const int t = __shfl_up_sync(0xffffffffu, off, o);
          if (lane >= o) off += t;
        }
        const int total = __shfl_sync(0xffffffffu, off, 31);
        off -= kl;
        s_kb[lane] = kb;
        s_off[lane] = off;
        if (lane == 0) s_off[32] = total;
        __syncwarp();
        const int nk = min(32, q1 - q);
        for (int t0 = 0; t0 < total; t0 += 32 * kSecondU) {
          int xs[kSecondU];
          int owner = 0;
#pragma unroll
          for (int u = 0; u < kSecondU; ++u) {
            const int t = t0 + lane + 32 * u;
            xs[u] = -1;
            if (t < total) {
              while (owner + 1 < nk && s_off[owner + 1] <= t) ++owner;
              xs[u] = __ldg(sci + s_kb[owner] + (t - s_off[owner]));
            }
          }
#pragma unroll
          for (int u = 0; u < kSecondU; ++u)
            if (xs[u] >= 0 && in_v(inV, xs[u])) bm_set(bm, xs[u]);
        }
        __syncwarp();
      }
    }
    // Wbar of this pass is V of the next one
    for (int t = lane; t < nwbar; t += 32) {
      const int j = wbar[t];
      atomicOr(inV + (j >> 5), 1u << (j & 31));
    }
    __syncwarp();
  }
  if (lane == 0) {
    meta[0] = g;
    s_done = 1;
  }
}

}  // namespace

#define MSP_NB_SWITCH(b, ...)                          \
  switch (b) {                                         \
    case 1: { constexpr int B_ = 1; __VA_ARGS__; } break; \
    case 2: { constexpr int B_ = 2; __VA_ARGS__; } break; \
    case 3: { constexpr int B_ = 3; __VA_ARGS__; } break; \
    case 4: { constexpr int B_ = 4; __VA_ARGS__; } break; \
    case 5: { constexpr int B_ = 5; __VA_ARGS__; } break; \
    case 6: { constexpr int B_ = 6; __VA_ARGS__; } break; \
    case 7: { constexpr int B_ = 7; __VA_ARGS__; } break; \
    case 8: { constexpr int B_ = 8; __VA_ARGS__; } break; \
    default: return MSP_ERR_ARG;                       \
  }

int launch_diag_inverse(int b, int nb, const int* dpos, const double* v, double* dinv,
                        double* omega, DevFlags* flags, cudaStream_t s) {
  if (nb <= 0) return MSP_OK;
  MSP_NB_SWITCH(b, diag_inverse_kernel<B_><<<grid_for(nb, kThreads), kThreads, 0, s>>>(
                       nb, dpos, v, dinv, omega, flags));
  return launch_status();
}

int launch_diagN_inverse(int b, int nb, const int* dpos, const double* v, double* dNinv,
                         DevFlags* flags, cudaStream_t s) {
  if (nb <= 0 || b < 2) return MSP_OK;
  switch (b) {
#define MSP_DN_CASE(BB)                                                              \
  case BB:                                                                           \
    diagN_inverse_kernel<BB><<<grid_for(nb, kThreads), kThreads, 0, s>>>(nb, dpos, v, \
                                                                         dNinv, flags); \
    break;
    MSP_DN_CASE(2)
    MSP_DN_CASE(3)
    MSP_DN_CASE(4)
    MSP_DN_CASE(5)
    MSP_DN_CASE(6)
    MSP_DN_CASE(7)
    MSP_DN_CASE(8)
#undef MSP_DN_CASE
    default:
      return MSP_ERR_ARG;
  }
  return launch_status();
}

int launch_pressure_matrix(int b, int nb, const int* rp, const double* v, const double* omega,
                           bool decoupling, double* ap, cudaStream_t s) {
  if (nb <= 0) return MSP_OK;
  pressure_matrix_kernel<<<grid_for(nb, kThreads), kThreads, 0, s>>>(b, nb, rp, v, omega,
                                                                     decoupling, ap);
  return launch_status();
}

int launch_strength(int n, const int* arp, const int* aci, const double* av, const int* srp,
                    const int* sci, double beta, double* sval, unsigned char* cand,
                    cudaStream_t s) {
  if (n <= 0) return MSP_OK;
  strength_kernel<<<grid_for(n, kThreads), kThreads, 0, s>>>(n, arp, aci, av, srp, sci, beta,
                                                             sval, cand);
  return launch_status();
}

int launch_transpose_pos(int n, const int* srp, const int* sci, int* tpos, cudaStream_t s) {
  if (n <= 0) return MSP_OK;
  transpose_pos_kernel<<<grid_for(n, kThreads), kThreads, 0, s>>>(n, srp, sci, tpos);
  return launch_status();
}

int launch_visit_keys(int n, unsigned long long seed, unsigned long long* hkey, cudaStream_t s) {
  if (n <= 0) return MSP_OK;
  visit_keys_kernel<<<grid_for(n, kThreads), kThreads, 0, s>>>(n, seed, hkey);
  return launch_status();
}

int launch_match_round(int n, const int* srp, const int* sci, const int* tpos,
                       const double* sval, const unsigned char* cand,
                       const unsigned long long* hkey, const unsigned char* state, int* commit,
                       cudaStream_t s) {
  if (n <= 0) return MSP_OK;
  match_round_kernel<<<grid_for(n, kThreads), kThreads, 0, s>>>(n, srp, sci, tpos, sval, cand,
                                                                hkey, state, commit);
  return launch_status();
}

int launch_match_apply(int n, const int* commit, unsigned char* state, int* partner,
                       DevFlags* flags, cudaStream_t s) {
  if (n <= 0) return MSP_OK;
  match_apply_kernel<<<grid_for(n, kThreads), kThreads, 0, s>>>(n, commit, state, partner,
                                                                flags);
  MSP_TRY(launch_status());
  count_undecided_kernel<<<grid_for(n, kThreads), kThreads, 0, s>>>(n, state, flags);
  return launch_status();
}

int launch_match_reps(int n, const int* partner, int* rep, cudaStream_t s) {
  if (n <= 0) return MSP_OK;
  match_reps_kernel<<<grid_for(n, kThreads), kThreads, 0, s>>>(n, partner, rep);
  return launch_status();
}

int launch_match_ids(int n, const int* partner, const int* id, int* agg, cudaStream_t s) {
  if (n <= 0) return MSP_OK;
  match_ids_kernel<<<grid_for(n, kThreads), kThreads, 0, s>>>(n, partner, id, agg);
  return launch_status();
}

int launch_segment_sums(int nseg, const int* seg_start, const int* src, const double* v,
                        double* out, cudaStream_t s) {
  if (nseg <= 0) return MSP_OK;
  segment_sums_kernel<<<grid_for(nseg, kThreads), kThreads, 0, s>>>(nseg, seg_start, src, v,
                                                                    out);
  return launch_status();
}

int launch_colouring(int n, const int* srp, const int* sci, const int* tp, const int* tl,
                     unsigned* inV, int* wbar, unsigned* bitmap, size_t bitmap_words,
                     int* colour, int* meta, int max_passes, cudaStream_t s) {
  if (n <= 0) return MSP_OK;
  const int n0 = (n + 31) / 32, n1 = (n0 + 31) / 32, n2 = (n1 + 31) / 32;
  const size_t fwords = (size_t)n0 + n1 + n2;
  if (fwords > bitmap_words) return MSP_ERR_ARG;
  const size_t cap = 220 * 1024;
  const size_t fbytes = fwords * sizeof(unsigned), vbytes = (size_t)n0 * sizeof(unsigned);
  int layout = 0;
  size_t smem = 0;
  if (fbytes + vbytes <= cap) {
    layout = 3;
    smem = fbytes + vbytes;
  } else if (vbytes <= cap) {
    layout = 2;  // the membership tests are the hottest accesses
    smem = vbytes;
  } else if (fbytes <= cap) {
    layout = 1;
    smem = fbytes;
  }
  if (smem > 0) {
    cudaError_t e = cudaFuncSetAttribute(colouring_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap);
    if (e != cudaSuccess) {
      layout = 0;
      smem = 0;
    }
  }
  colouring_kernel<<<1, 64, smem, s>>>(n, srp, sci, tp, tl, inV, wbar, bitmap, layout, colour,
                                       meta, max_passes);
  return launch_status();
}

}  // namespace msp
